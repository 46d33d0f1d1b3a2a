"""Pins of the oracle's partial-volume quadrature (CPU only).

§4.1.1 remarks that cells near the horizon edge are only partly covered by the
ball of radius delta and that a partial-volume weight dV(|xi|) can replace the
constant dV without leaving the convolution structure. The rule used is the
linear one of Hu, Ha and Bobaru: on cubic cells of side h a bond's weight is
beta(|xi|) dV, beta = min(1, (delta + h/2 - |xi|)/h), for |xi| < delta + h/2.

What pins it, other than itself:
  * the lattice moments of the weights converge to the continuum integrals over
    the ball (closed forms), an order of magnitude closer than the constant rule
    at the same resolution; a wrong cut-off or slope leaves an O(h/delta) error;
  * the long-wave symbol of the bond operator then matches Navier-Cauchy
    elasticity closely (the constant rule misses by percents);
  * an all-pairs brute-force sum over minimum-image distances;
  * the invariants that hold for any symmetric bond weight (rigid motions,
    reciprocity, energy identity, dilatation of an isotropic stretch, the
    nu = 1/4 reduction of the state-based solid);
  * integer family counts against a lattice count.
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


def test_rule_switch_is_scoped(oracle):
    assert oracle.volume_rule() == 0
    with oracle.partial_volumes():
        assert oracle.volume_rule() == 1
    assert oracle.volume_rule() == 0
    with pytest.raises(ValueError):
        oracle.set_volume_rule(2)


@pytest.mark.parametrize("dim,delta", [(2, 3.0), (2, 2.5), (2, 4.5), (3, 3.0), (3, 2.2)])
def test_family_is_every_partly_covered_cell(oracle, dim, delta):
    """Family = lattice offsets whose distance is below delta + h/2 (h = 1 here);
    weights lie in (0, 1], equal 1 up to delta - h/2 and never grow with |xi|."""
    with oracle.partial_volumes():
        off, ln, vol = oracle.horizon(dim, 1.0, delta, weights=True)
    r = int(delta + 0.5)
    rng3 = range(-r, r + 1) if dim == 3 else [0]
    reach2 = (delta + 0.5) ** 2
    bf = sum(1 for i in range(-r, r + 1) for j in range(-r, r + 1) for k in rng3
             if 0 < i * i + j * j + k * k < reach2)
    assert len(off) == bf
    assert np.all(vol > 0) and np.all(vol <= 1)
    assert np.all(vol[ln <= delta - 0.5] == 1.0)
    order = np.argsort(ln, kind="stable")
    assert np.all(np.diff(vol[order]) <= 1e-15)
    # the constant rule's family is the subset |xi| <= delta, all weights 1
    off0, _, vol0 = oracle.horizon(dim, 1.0, delta, weights=True)
    assert np.all(vol0 == 1.0)
    assert len(off0) == int(np.sum(ln <= delta * (1 + 1e-12)))


def _moments(oracle, dim, delta):
    """(cell volume, Σ|xi|, Σ xi_1^4/|xi|^3) of the weighted lattice, h = 1,
    relative to the integrals over the ball |xi| <= delta:
    area pi d^2 / volume 4 pi d^3 / 3; ∫|xi| = 2 pi d^3 / 3 (2D), pi d^4 (3D);
    ∫ xi_1^4 / |xi|^3 = pi d^3 / 4 (2D), pi d^4 / 5 (3D)."""
    off, ln, vol = oracle.horizon(dim, 1.0, delta, weights=True)
    x1 = off[:, 0].astype(float)
    got = np.array([1.0 + vol.sum(), np.sum(vol * ln), np.sum(vol * x1 ** 4 / ln ** 3)])
    d = delta
    if dim == 2:
        exact = np.array([math.pi * d * d, 2 * math.pi * d ** 3 / 3, math.pi * d ** 3 / 4])
    else:
        exact = np.array([4 * math.pi * d ** 3 / 3, math.pi * d ** 4, math.pi * d ** 4 / 5])
    return got / exact - 1.0


@pytest.mark.parametrize("dim,m,bound", [(2, 16, 1e-3), (2, 32, 3e-4), (2, 64, 2e-4), (3, 16, 2.5e-3),
                                         (3, 24, 1.5e-3)])
def test_weighted_moments_converge_to_the_ball(oracle, dim, m, bound):
    with oracle.partial_volumes():
        err = _moments(oracle, dim, float(m))
    assert np.max(np.abs(err)) < bound, err
    # the constant rule at the same resolution misses by more than the bound
    err0 = _moments(oracle, dim, float(m))
    assert np.max(np.abs(err0)) > bound


@pytest.mark.parametrize("dim,delta,tol,tol0", [(2, 16.0, 2e-3, 3e-2), (3, 12.0, 7e-3, 3e-2)])
def test_long_wave_symbol_is_navier(oracle, dim, delta, tol, tol0):
    """M(k) -> mu |kappa|^2 I + (lam + mu) kappa kappa^T with lam = mu = 3E/8 (2D
    plane stress) or 2E/5 (3D); kappa delta ~ 0.03 makes the O(kappa^4) term
    negligible, so what is left is the quadrature error of the horizon sum."""
    E = 1.0
    n = 8192
    shape = (n,) * dim
    alpha = oracle.alpha_bond(dim, E, delta)
    lam = mu = (3.0 * E / 8.0) if dim == 2 else (2.0 * E / 5.0)
    for pv, t in ((True, tol), (False, tol0)):
        with oracle.partial_volumes(pv):
            worst = 0.0
            for kvec in ([1, 0, 0], [1, 1, 0], [2, -1, 1]):
                k = np.array(kvec[:dim], dtype=float)
                kap = 2 * math.pi * k / n
                M = oracle.symbol_bond(shape, 1.0, delta, alpha, k)
                Mn = mu * kap.dot(kap) * np.eye(dim) + (lam + mu) * np.outer(kap, kap)
                worst = max(worst, _rel(M, Mn))
        if pv:
            assert worst < t
        else:  # the constant rule misses by more than the partial-volume tolerance
            assert tol < worst < t


def test_bond_matches_all_pairs_brute_force(oracle):
    """Pure-Python all-pairs sum over minimum-image distances with the partial
    weight of each pair, node weights s, cubic cells of side 0.9."""
    shape = (10, 11)
    delta, h = 2.2, 0.9
    alpha = 0.37
    g = inputs.rng(12)
    chi = (g.random(shape) < 0.8).astype(np.uint8)
    s = 0.5 + g.random(shape)
    u = g.normal(size=(2,) + shape)
    with oracle.partial_volumes():
        L = oracle.force_bond(u, chi, h, delta, alpha, s=s)
    n2, n1 = shape
    ref = np.zeros_like(u)
    npart = 0
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
                    if r == 0 or r >= delta + h / 2 or not chi[b2, b1]:
                        continue
                    w = min(1.0, (delta + h / 2 - r) / h)
                    npart += w < 1
                    eta = u[:, b2, b1] - u[:, a2, a1]
                    ref[:, a2, a1] += s[a2, a1] * s[b2, b1] * w * alpha / r * np.outer(xi, xi) / r ** 2 @ eta * h * h
    assert npart > 0
    assert _rel(L, ref) < 1e-13
    nodes = g.choice(chi.size, size=17, replace=False)
    with oracle.partial_volumes():
        Ls = oracle.force_bond_at(u, chi, h, delta, alpha, nodes)
        Lf = oracle.force_bond(u, chi, h, delta, alpha)
    assert np.array_equal(Ls, Lf.reshape(2, -1)[:, nodes])


@pytest.mark.parametrize("dim", [2, 3])
def test_bond_invariants(oracle, dim):
    """Rigid motions give zero force, the operator is symmetric and negative,
    and Σ W dV = -<u, L u> dV (R9), all under partial volumes."""
    shape = (26, 24) if dim == 2 else (15, 14, 16)
    chi = _blob(shape, 1)
    delta = 3.0
    alpha = oracle.alpha_bond(dim, 1.0, delta)
    x = inputs.coords(shape)
    g = inputs.rng(13)
    lam = (g.random(shape) < 0.9).astype(np.uint8)
    u = g.normal(size=(dim,) + shape)
    v = g.normal(size=(dim,) + shape)
    with oracle.partial_volumes():
        t = np.stack([np.full(shape, 0.3 + 0.1 * i) for i in range(dim)])
        assert np.max(np.abs(oracle.force_bond(t, chi, 1.0, delta, alpha))) < 1e-13
        Wm = np.zeros((dim, dim))
        Wm[0, 1], Wm[1, 0] = 0.01, -0.01
        if dim == 3:
            Wm[0, 2], Wm[2, 0] = -0.02, 0.02
        rot = np.stack([sum(Wm[i, j] * x[j] for j in range(dim)) for i in range(dim)])
        assert np.max(np.abs(oracle.force_bond(rot, chi, 1.0, delta, alpha))) < 1e-13
        Lu = oracle.force_bond(u, chi, 1.0, delta, alpha)
        Lv = oracle.force_bond(v, chi, 1.0, delta, alpha)
        a, b = float(np.sum(v * Lu)), float(np.sum(u * Lv))
        assert abs(a - b) < 1e-12 * max(abs(a), 1.0)
        assert float(np.sum(u * Lu)) < 0
        W = oracle.energy_bond(u, chi, 1.0, delta, alpha, lam=lam)
        Ll = oracle.force_bond(u, chi, 1.0, delta, alpha, s=lam.astype(float))
        assert abs(W.sum() + np.sum(u * Ll)) < 1e-12 * W.sum()
    # the weights change the operator
    L0 = oracle.force_bond(u, chi, 1.0, delta, alpha)
    assert _rel(L0, Lu) > 1e-2


def test_wc_of_isotropic_stretch(oracle):
    """W of a fully bonded node under u = s0 x is 1/2 alpha s0^2 dV Σ beta |xi|,
    which is what wc_from_stretch returns under the rule (reading R10)."""
    shape = (40, 40)
    delta, s0 = 4.0, 1e-3
    alpha = oracle.alpha_bond(2, 1.0, delta)
    chi = inputs.box_mask(shape, (5, 5), (35, 35))
    x1, x2 = inputs.coords(shape)
    u = np.stack([s0 * x1, s0 * x2])
    with oracle.partial_volumes():
        W = oracle.energy_bond(u, chi, 1.0, delta, alpha)
        wc = oracle.wc_from_stretch(2, 1.0, delta, alpha, s0)
    assert abs(W[20, 20] / wc - 1.0) < 1e-12
    # Σ beta |xi| is within 1.3 % of the ball integral 2 pi delta^3 / 3 at m = 4
    assert abs(wc / (0.5 * alpha * s0 * s0 * 2 * math.pi * delta ** 3 / 3) - 1) < 0.013


def test_lps_under_partial_volumes(oracle):
    """State-based solid: dilatation of an isotropic stretch is 3 s in the
    interior (m and the dilatation sum carry the same weights), rigid motions
    give zero force, the operator is symmetric, and at nu = 1/4 it is the bond
    form with 30 mu / m0 (m0 the weighted Σ omega |xi|^2 dV)."""
    shape = (20, 20, 20)
    delta = 2.0
    chi = inputs.box_mask(shape, (4, 4, 4), (16, 16, 16))
    x = inputs.coords(shape)
    with oracle.partial_volumes():
        ka, cb, m0 = oracle.lps_constants(1.0, 0.4, 1.0, delta)
        s = 1e-3
        iso = np.stack([s * x[i] for i in range(3)])
        L, th, m = oracle.force_lps(iso, chi, 1.0, delta, ka, cb, return_aux=True)
        inner = inputs.box_mask(shape, (7, 7, 7), (13, 13, 13)).astype(bool)
        assert np.allclose(th[inner], 3 * s, rtol=1e-12)
        assert np.allclose(m[inner], m0, rtol=1e-12)
        Wm = np.array([[0, 0.01, -0.02], [-0.01, 0, 0.03], [0.02, -0.03, 0]])
        rot = np.stack([sum(Wm[i, j] * x[j] for j in range(3)) for i in range(3)])
        assert np.max(np.abs(oracle.force_lps(rot, chi, 1.0, delta, ka, cb))) < 1e-13
        g = inputs.rng(3)
        u = g.normal(size=(3,) + shape)
        v = g.normal(size=(3,) + shape)
        a = float(np.sum(v * oracle.force_lps(u, chi, 1.0, delta, ka, cb)))
        b = float(np.sum(u * oracle.force_lps(v, chi, 1.0, delta, ka, cb)))
        assert abs(a - b) < 1e-12 * abs(a)
        ka4, cb4, _ = oracle.lps_constants(1.0, 0.25, 1.0, delta)
        assert abs(ka4) < 1e-15
        assert _rel(oracle.force_lps(u, chi, 1.0, delta, ka4, cb4), oracle.force_bond(u, chi, 1.0, delta, cb4)) < 1e-13
    _, _, m00 = oracle.lps_constants(1.0, 0.4, 1.0, delta)
    assert m0 != m00


def test_damage_counts_whole_family_bonds(oracle):
    """A partly covered bond counts as one bond: the intact count of a node deep
    inside the body is the family size (36 for 2D delta = 3, h = 1), and counts
    equal a lattice brute force everywhere."""
    shape = (20, 22)
    g = inputs.rng(8)
    chi = _blob(shape, 6)
    lam = chi.copy()
    lam[g.random(shape) < 0.15] = 0
    delta = 3.0
    with oracle.partial_volumes():
        nb, beta, d = oracle.damage(chi, lam, 1.0, delta)
        off, _ = oracle.horizon(2, 1.0, delta)
        _, b_full, _ = oracle.damage(np.ones(shape, np.uint8), np.ones(shape, np.uint8), 1.0, delta)
    assert len(off) == 36 and np.all(b_full == 36)
    n2, n1 = shape
    for a2 in range(n2):
        for a1 in range(n1):
            b = k = 0
            if chi[a2, a1]:
                for i in range(-3, 4):
                    for j in range(-3, 4):
                        if not 0 < i * i + j * j < 12.25:
                            continue
                        q2, q1 = (a2 + j) % n2, (a1 + i) % n1
                        if chi[q2, q1]:
                            b += 1
                            k += int(not (lam[a2, a1] and lam[q2, q1]))
            assert beta[a2, a1] == b and nb[a2, a1] == k
