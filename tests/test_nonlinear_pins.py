"""Pins of the oracle's nonlinear rotation-invariant bond model (§3.2, Eq. 19-26;
CPU only).

  * finite rigid motions (a 30 degree rotation) give zero force and energy,
    where the linearized model of Eq. 17 does not;
  * for small displacements the force and energy become those of the
    linearized model (Eq. 17, 47), with an O(eps) remainder;
  * the force is minus the gradient of the total energy (central differences),
    and pairwise action and reaction make the total force vanish;
  * an all-pairs brute force written with the bond strain and the unit vector
    of Eq. 19-20 (square roots), not the polynomial of Eq. 21;
  * the convolutional form of Eq. 26 with the embedded-constraint mask: every
    monomial of f in u(x) and u(x + xi) becomes a correlation of a kernel
    (C_ij, a_i = c xi_i or c, Eq. 24) with a masked field, evaluated with numpy
    FFTs, and the sum equals the direct sum;
  * the field plan for the GPU passes (12 forward and 21 inverse half spectra
    in 3D, with the pure correlations combined in spectral space) gives the
    same force.
"""
import math

import numpy as np
import pytest

from paper_2105_06055_gb300 import inputs


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _blob(shape, seed, margin=5):
    g = inputs.rng(seed)
    dim = len(shape)
    chi = inputs.box_mask(shape, (margin,) * dim, tuple(s - margin for s in shape[::-1]))
    chi[g.random(shape) < 0.08] = 0
    return chi


def _rotation(dim, angle):
    c, s = math.cos(angle), math.sin(angle)
    if dim == 2:
        return np.array([[c, -s], [s, c]])
    # rotation by angle about the axis (1, 2, 2)/3 (Rodrigues)
    k = np.array([1.0, 2.0, 2.0]) / 3.0
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + s * K + (1 - c) * K @ K


@pytest.mark.parametrize("dim", [2, 3])
def test_finite_rigid_motion_gives_zero_force(oracle, dim):
    shape = (28, 30) if dim == 2 else (16, 17, 18)
    chi = _blob(shape, 2)
    delta = 3.0
    alpha = oracle.alpha_bond(dim, 1.0, delta)
    x = np.stack(inputs.coords(shape)).astype(float)
    x0 = np.array([s / 2 for s in shape[::-1]]).reshape((dim,) + (1,) * dim)
    R = _rotation(dim, math.radians(30.0))
    t = np.array([0.7, -0.4, 0.25][:dim]).reshape((dim,) + (1,) * dim)
    u = np.einsum("ij,j...->i...", R - np.eye(dim), x - x0) + t
    L = oracle.force_nonlinear(u, chi, 1.0, delta, alpha)
    W = oracle.energy_nonlinear(u, chi, 1.0, delta, alpha)
    assert np.max(np.abs(L)) < 1e-12
    assert np.max(np.abs(W)) < 1e-24
    # the linearized model is not invariant under a finite rotation
    Llin = oracle.force_bond(u, chi, 1.0, delta, alpha)
    assert np.max(np.abs(Llin)) > 1e-2


@pytest.mark.parametrize("dim", [2, 3])
def test_small_displacement_limit_is_the_linearized_model(oracle, dim):
    shape = (24, 26) if dim == 2 else (14, 15, 16)
    chi = _blob(shape, 4)
    delta = 2.5
    alpha = oracle.alpha_bond(dim, 1.0, delta)
    u = inputs.rng(5).normal(size=(dim,) + shape)
    Llin = oracle.force_bond(u, chi, 1.0, delta, alpha)
    Wlin = oracle.energy_bond(u, chi, 1.0, delta, alpha)
    errs, werrs = [], []
    for eps in (1e-3, 1e-4):
        errs.append(_rel(oracle.force_nonlinear(eps * u, chi, 1.0, delta, alpha) / eps, Llin))
        werrs.append(_rel(oracle.energy_nonlinear(eps * u, chi, 1.0, delta, alpha) / eps ** 2, Wlin))
    assert errs[0] < 1e-2 and werrs[0] < 1e-2
    assert 7 < errs[0] / errs[1] < 13  # first order in eps
    assert 7 < werrs[0] / werrs[1] < 13


@pytest.mark.parametrize("pv", [False, True])
def test_force_is_minus_the_energy_gradient(oracle, pv):
    """E = 1/2 Σ_x W dV (R9); L(x) = -(1/dV) dE/du(x), by central differences in
    the nonlinear regime (|u| ~ 0.3 |xi|)."""
    shape = (12, 13)
    dx = 0.9
    delta = 2.2
    alpha = 0.41
    g = inputs.rng(6)
    chi = (g.random(shape) < 0.85).astype(np.uint8)
    lam = (g.random(shape) < 0.9).astype(np.uint8)
    u = 0.3 * g.normal(size=(2,) + shape)
    dV = dx * dx
    with oracle.partial_volumes(pv):
        L = oracle.force_nonlinear(u, chi, dx, delta, alpha, lam=lam)

        def E(v):
            return 0.5 * float(np.sum(oracle.energy_nonlinear(v, chi, dx, delta, alpha, lam=lam))) * dV

        h = 1e-5
        for k in g.choice(u.size, size=24, replace=False):
            e = np.zeros(u.size)
            e[k] = h
            e = e.reshape(u.shape)
            fd = -(E(u + e) - E(u - e)) / (2 * h) / dV
            assert abs(fd - L.reshape(-1)[k]) < 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("dim", [2, 3])
def test_total_force_vanishes(oracle, dim):
    shape = (20, 22) if dim == 2 else (12, 13, 14)
    chi = _blob(shape, 7, margin=4)
    g = inputs.rng(8)
    lam = (g.random(shape) < 0.9).astype(np.uint8)
    u = 0.5 * g.normal(size=(dim,) + shape)
    for pv in (False, True):
        with oracle.partial_volumes(pv):
            L = oracle.force_nonlinear(u, chi, 1.0, 3.0, 0.3, lam=lam)
        tot = L.reshape(dim, -1).sum(1)
        assert np.max(np.abs(tot)) < 1e-12 * np.abs(L).sum()


def test_matches_all_pairs_brute_force_with_bond_strain(oracle):
    """Eq. 19-20 as printed: alpha omega |xi| (s + 3/2 s^2 + 1/2 s^3) times the unit
    vector of the deformed bond, s the bond strain; minimum-image pairs."""
    shape = (9, 10)
    delta, h = 2.3, 1.0
    alpha = 0.29
    g = inputs.rng(9)
    chi = (g.random(shape) < 0.8).astype(np.uint8)
    u = 0.4 * g.normal(size=(2,) + shape)
    L = oracle.force_nonlinear(u, chi, h, delta, alpha)
    n2, n1 = shape
    ref = np.zeros_like(u)
    for a2 in range(n2):
        for a1 in range(n1):
            if not chi[a2, a1]:
                continue
            for b2 in range(n2):
                for b1 in range(n1):
                    d1 = (b1 - a1 + n1 // 2) % n1 - n1 // 2
                    d2 = (b2 - a2 + n2 // 2) % n2 - n2 // 2
                    xi = np.array([d1 * h, d2 * h])
                    r = math.hypot(*xi)
                    if r == 0 or r > delta or not chi[b2, b1]:
                        continue
                    y = xi + u[:, b2, b1] - u[:, a2, a1]
                    ry = math.hypot(*y)
                    s = (ry - r) / r
                    ref[:, a2, a1] += alpha / r * r * (s + 1.5 * s * s + 0.5 * s ** 3) * y / ry * h * h
    assert _rel(L, ref) < 1e-12


def _correlate(K, G):
    """S(x) = Σ_xi K(xi) G(x + xi) on the periodic grid (K given on the grid,
    offset xi stored at xi mod n), by FFT."""
    return np.real(np.fft.ifftn(np.conj(np.fft.fftn(K)) * np.fft.fftn(G)))


def _eq26(oracle, u, chi, lam, dx, delta, alpha):
    """Eq. 26 with the embedded-constraint weight w = chi lam: expand
    f = c(xi.eta) xi + c(xi.eta) eta + c/2 |eta|^2 xi + c/2 |eta|^2 eta in the
    values at x and x + xi and correlate each kernel with the masked fields."""
    dim = u.shape[0]
    shape = u.shape[1:]
    off, ln, vol = oracle.horizon(dim, dx, delta, weights=True)
    dV = dx ** dim
    cK = np.zeros(shape)
    aK = np.zeros((dim,) + shape)
    CK = np.zeros((dim, dim) + shape)
    for o, r, b in zip(off, ln, vol):
        idx = tuple(int(o[dim - 1 - a]) % shape[a] for a in range(dim))  # C order: last axis is x1
        xi = o[:dim] * dx
        c = alpha / r ** 3 * b * dV
        cK[idx] += c
        for i in range(dim):
            aK[(i,) + idx] += c * xi[i]
            for j in range(dim):
                CK[(i, j) + idx] += c * xi[i] * xi[j]
    w = (chi * (1 if lam is None else lam)).astype(float)
    uu = np.sum(u * u, axis=0)
    S = _correlate
    L = np.zeros_like(u)
    for i in range(dim):
        t = 0.0
        for j in range(dim):
            t = t + S(CK[i, j], w * u[j]) - S(CK[i, j], w) * u[j]                       # c (xi.eta) xi_i
            t = t + (S(aK[j], w * u[j] * u[i]) - S(aK[j], w * u[j]) * u[i]               # c (xi.eta) eta_i
                     - S(aK[j], w * u[i]) * u[j] + S(aK[j], w) * u[j] * u[i])
            t = t - S(aK[i], w * u[j]) * u[j]                                            # c/2 |eta|^2 xi_i
            t = t - S(cK, w * u[j] * u[i]) * u[j] + S(cK, w * u[j]) * u[j] * u[i]        # c/2 |eta|^2 eta_i
        t = t + 0.5 * S(aK[i], w * uu) + 0.5 * S(aK[i], w) * uu
        t = t + (0.5 * S(cK, w * uu * u[i]) - 0.5 * S(cK, w * uu) * u[i]
                 + 0.5 * S(cK, w * u[i]) * uu - 0.5 * S(cK, w) * uu * u[i])
        L[i] = w * t
    return L


@pytest.mark.parametrize("dim,pv", [(2, False), (2, True), (3, False)])
def test_convolutional_form_eq26(oracle, dim, pv):
    shape = (24, 32) if dim == 2 else (14, 16, 18)
    chi = _blob(shape, 10, margin=4)
    g = inputs.rng(11)
    lam = (g.random(shape) < 0.9).astype(np.uint8)
    u = 0.3 * g.normal(size=(dim,) + shape)
    delta = 3.0 if dim == 2 else 2.5
    alpha = oracle.alpha_bond(dim, 1.0, delta)
    with oracle.partial_volumes(pv):
        ref = oracle.force_nonlinear(u, chi, 1.0, delta, alpha, lam=lam)
        L = _eq26(oracle, u, chi, lam, 1.0, delta, alpha)
    assert _rel(L, ref) < 1e-11


def _spectral_passes(oracle, u, chi, lam, dx, delta, alpha):
    """The decomposition planned for the GPU passes, on numpy half spectra:
    forward w u_j (d), w u_i u_j (d(d+1)/2), w |u|^2 u_i (d) with w = chi lam;
    one spectral combination per component for the terms of Eq. 26 that are
    pure correlations, plus the inverse fields a_m*(w u_n) (d^2),
    c*(w u_i u_j) (d(d+1)/2), c*(w u_j) (d); the correlations with w alone are
    plan-time fields. Correlation with an even real kernel multiplies by its
    (real) spectrum, with the odd a_i by the conjugate of its (imaginary) one."""
    dim = u.shape[0]
    shape = u.shape[1:]
    off, ln, vol = oracle.horizon(dim, dx, delta, weights=True)
    dV = dx ** dim
    cK = np.zeros(shape)
    aK = np.zeros((dim,) + shape)
    CK = np.zeros((dim, dim) + shape)
    for o, r, b in zip(off, ln, vol):
        idx = tuple(int(o[dim - 1 - a]) % shape[a] for a in range(dim))
        xi = o[:dim] * dx
        c = alpha / r ** 3 * b * dV
        cK[idx] += c
        for i in range(dim):
            aK[(i,) + idx] += c * xi[i]
            for j in range(dim):
                CK[(i, j) + idx] += c * xi[i] * xi[j]
    F = np.fft.rfftn
    axes_shape = shape

    def Fi(X):
        return np.fft.irfftn(X, s=axes_shape, axes=tuple(range(dim)))

    cH = np.conj(F(cK))
    aH = [np.conj(F(aK[i])) for i in range(dim)]
    CH = [[np.conj(F(CK[i, j])) for j in range(dim)] for i in range(dim)]
    # the kernel spectra have the parities the passes rely on
    assert np.max(np.abs(cH.imag)) < 1e-12 * np.max(np.abs(cH))
    for i in range(dim):
        assert np.max(np.abs(aH[i].real)) < 1e-12 * np.max(np.abs(aH[i]))
    w = (chi * lam).astype(float)
    X = [F(w * u[j]) for j in range(dim)]
    Y = {(i, j): F(w * u[i] * u[j]) for i in range(dim) for j in range(i, dim)}

    def Yf(i, j):
        return Y[(min(i, j), max(i, j))]

    uu = np.sum(u * u, axis=0)
    Z = [F(w * uu * u[i]) for i in range(dim)]
    Yt = sum(Yf(j, j) for j in range(dim))
    assert len(X) + len(Y) + len(Z) == (12 if dim == 3 else 7)
    # inverse fields
    P = [Fi(sum(CH[i][j] * X[j] for j in range(dim)) + sum(aH[j] * Yf(j, i) for j in range(dim))
            + 0.5 * aH[i] * Yt + 0.5 * cH * Z[i]) for i in range(dim)]
    A = [[Fi(aH[m] * X[n]) for n in range(dim)] for m in range(dim)]
    B = {k: Fi(cH * v) for k, v in Y.items()}
    Cc = [Fi(cH * X[j]) for j in range(dim)]
    assert len(P) + dim * dim + len(B) + len(Cc) == (21 if dim == 3 else 11)

    def Bf(i, j):
        return B[(min(i, j), max(i, j))]

    # plan-time correlations with w alone
    Fw = F(w)
    SC = [[Fi(CH[i][j] * Fw) for j in range(dim)] for i in range(dim)]
    Sa = [Fi(aH[j] * Fw) for j in range(dim)]
    Sc = Fi(cH * Fw)
    # epilogue per node
    L = np.zeros_like(u)
    trA = sum(A[j][j] for j in range(dim))
    trB = sum(Bf(j, j) for j in range(dim))
    for i in range(dim):
        t = P[i] - sum(SC[i][j] * u[j] for j in range(dim))
        t = t - u[i] * trA - sum(A[j][i] * u[j] for j in range(dim)) + u[i] * sum(Sa[j] * u[j] for j in range(dim))
        t = t - sum(A[i][j] * u[j] for j in range(dim)) + 0.5 * Sa[i] * uu
        t = t - 0.5 * trB * u[i] - sum(Bf(i, j) * u[j] for j in range(dim))
        t = t + u[i] * sum(Cc[j] * u[j] for j in range(dim)) + 0.5 * Cc[i] * uu - 0.5 * Sc * uu * u[i]
        L[i] = w * t
    return L


@pytest.mark.parametrize("dim", [2, 3])
def test_spectral_decomposition_for_the_passes(oracle, dim):
    """12 forward and 21 inverse fields in 3D (7 and 11 in 2D) reproduce the
    direct sum; this is the field plan of the GPU passes for this model."""
    shape = (24, 32) if dim == 2 else (14, 16, 18)
    chi = _blob(shape, 12, margin=4)
    g = inputs.rng(13)
    lam = (g.random(shape) < 0.9).astype(np.uint8)
    u = 0.3 * g.normal(size=(dim,) + shape)
    delta = 3.0 if dim == 2 else 2.5
    alpha = oracle.alpha_bond(dim, 1.0, delta)
    ref = oracle.force_nonlinear(u, chi, 1.0, delta, alpha, lam=lam)
    L = _spectral_passes(oracle, u, chi, lam, 1.0, delta, alpha)
    assert _rel(L, ref) < 1e-11
