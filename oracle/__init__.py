"""FP64 CPU oracle for the FCBM-EC peridynamic operators (arXiv 2105.06055).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The GPU library never imports, links or calls it, and the two share
no code: this package computes the model constants, the horizon and every sum
on its own, from the paper.

Contents
  * ``pd_oracle.c`` (built into ``_build/liboracle.so``): the direct O(N |H|)
    neighbour sums of the one-point quadrature (Eq. 55 first line, §4.1.1) for
    the linearized bond model (Eq. 17-18, 75, 100), its strain energy density
    (Eq. 47, 102), damage counts (Eq. 12, 44, reading R11), the linearized
    state-based solid (Eq. 33-39, 92-94), the node-weight gradient of the bond
    operator, the periodic Fourier symbol (Eq. 57), and the nonlinear
    rotation-invariant bond model with its energy density (§3.2, Eq. 19-22).
  * Python drivers written step by step in the paper's order: velocity-Verlet
    with embedded constraint and energy-based bond breaking (Eq. 63, 83-84),
    FP64 conjugate gradient on the EC static residual (Eq. 89), and model
    constants (§5.1, §5.2).

Every sum takes the bond's quadrature weight from the horizon: the constant dV
of the paper's examples, or, after ``set_volume_rule(1)`` (or inside
``with partial_volumes():``), the linear partial-volume weight beta(|xi|) dV
that §4.1.1 allows in place of dV (the rule of Hu, Ha and Bobaru).

Every function here is FP64. Parity status of each function is listed in the
``PINS`` table at the bottom (the tests that hold each pin are in
``tests/test_oracle_pins.py`` and ``tests/test_partial_volume_pins.py``).
"""
from __future__ import annotations

import contextlib
import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``pd_oracle.c`` with gcc (-O2, OpenMP). Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I, D = ctypes.c_int, ctypes.c_double
            lib.or_num_threads.restype = I
            lib.or_set_threads.argtypes = [I]
            lib.or_horizon.argtypes = [I, P, D, I, P, P, P]
            lib.or_set_volume_rule.argtypes = [I]
            lib.or_volume_rule.restype = I
            lib.or_horizon.restype = I
            lib.or_force_bond.argtypes = [I, P, P, D, D, P, P, P, P]
            lib.or_energy_bond.argtypes = [I, P, P, D, D, P, P, P, P]
            lib.or_energy_bond_w.argtypes = [I, P, P, D, D, P, P, P, P]
            lib.or_force_nl.argtypes = [I, P, P, D, D, P, P, P, P]
            lib.or_energy_nl.argtypes = [I, P, P, D, D, P, P, P, P]
            lib.or_force_bond_at.argtypes = [I, P, P, D, D, P, P, P, ctypes.c_int64, P]
            lib.or_damage.argtypes = [I, P, P, D, P, P, P, P, P]
            lib.or_force_lps.argtypes = [P, P, D, D, D, P, P, P, P, P]
            lib.or_force_bond_grad_s.argtypes = [I, P, P, D, D, P, P, P, P, P]
            lib.or_symbol_bond.argtypes = [I, P, P, D, D, P, P]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _grid(shape):
    """shape is (n2, n1) in 2D or (n3, n2, n1) in 3D (C order, x1 fastest)."""
    if len(shape) == 2:
        return 2, np.array([shape[1], shape[0], 1], dtype=np.int32)
    return 3, np.array([shape[2], shape[1], shape[0]], dtype=np.int32)


def _dx(dim, dx):
    d = np.ones(3, dtype=np.float64)
    a = np.atleast_1d(np.asarray(dx, dtype=np.float64))
    d[:dim] = a[0] if a.size == 1 else a[:dim]
    return d


def num_threads() -> int:
    return _load().or_num_threads()


def set_threads(t: int) -> None:
    _load().or_set_threads(int(t))


# ----------------------------------------------------------------------------
# Model constants (§3.1, §3.3, §5.1, §5.2)
# ----------------------------------------------------------------------------

def set_volume_rule(rule: int) -> None:
    """Quadrature weight of every later call: 0 the constant dV of the paper's
    examples (§4.1.1), 1 linear partial volumes beta(|xi|) dV (reading R3)."""
    if rule not in (0, 1):
        raise ValueError("volume rule is 0 (constant) or 1 (partial volumes)")
    _load().or_set_volume_rule(int(rule))


def volume_rule() -> int:
    return int(_load().or_volume_rule())


@contextlib.contextmanager
def partial_volumes(on: bool = True):
    """Run the enclosed oracle calls under the partial-volume rule (or not)."""
    old = volume_rule()
    set_volume_rule(1 if on else 0)
    try:
        yield
    finally:
        set_volume_rule(old)


def horizon(dim: int, dx, delta: float, weights: bool = False):
    """Integer offsets o (|H| x 3) and lengths |xi| of the horizon (R1, R2);
    with ``weights`` also each bond's quadrature weight relative to dV (1, or
    beta(|xi|) under the partial-volume rule)."""
    lib = _load()
    d = _dx(dim, dx)
    reach = delta + 0.5 * d[0] if volume_rule() == 1 else delta
    cap = 1
    for a in range(dim):
        cap *= 2 * int(math.floor(reach / d[a] + 1e-9)) + 1
    off = np.zeros((cap, 3), dtype=np.int32)
    ln = np.zeros(cap, dtype=np.float64)
    vol = np.zeros(cap, dtype=np.float64)
    cnt = lib.or_horizon(dim, _p(d), float(delta), cap, _p(off), _p(ln), _p(vol))
    if weights:
        return off[:cnt].copy(), ln[:cnt].copy(), vol[:cnt].copy()
    return off[:cnt].copy(), ln[:cnt].copy()


def alpha_bond(dim: int, E: float, delta: float) -> float:
    """Bond constant for omega = 1/|xi|.

    2D plane stress: 9E/(pi delta^3) (§5.2, with nu = 1/3).
    3D: 12E/(pi delta^4) (reading R7, nu = 1/4): equate the bond energy of an
    isotropic stretch, 1/4 int alpha omega |xi|^2 s^2 dV = pi alpha delta^4 s^2/4,
    with the classical 9 kappa s^2 / 2 = 3 E s^2.
    """
    if dim == 2:
        return 9.0 * E / (math.pi * delta ** 3)
    return 12.0 * E / (math.pi * delta ** 4)


def lps_constants(E: float, nu: float, dx, delta: float):
    """(ka, cb, m0) of the linearized state-based solid (Eq. 37; reading R5).

    kappa = E / (3 (1 - 2 nu)), mu = E / (2 (1 + nu)),
    m0 = Σ_H omega |xi|^2 dV over a full horizon (Eq. 35, omega = 1/|xi|),
    ka = (3 kappa - 5 mu)/m0, cb = 30 mu/m0.
    """
    d = _dx(3, dx)
    _, ln, vol = horizon(3, d, delta, weights=True)
    dV = float(d[0] * d[1] * d[2])
    m0 = float(np.sum(vol * ln)) * dV  # omega |xi|^2 = |xi|
    kappa = E / (3.0 * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return (3.0 * kappa - 5.0 * mu) / m0, 30.0 * mu / m0, m0


def wc_from_stretch(dim: int, dx, delta: float, alpha: float, s0: float) -> float:
    """Critical energy density for a critical stretch s0 (reading R10).

    W_c is the Eq. 47 energy density of a fully bonded node under the isotropic
    stretch u = s0 x: each bond has eta = s0 xi, so eta.C.eta = alpha s0^2 |xi|
    for omega = 1/|xi|, and W_c = 1/2 alpha s0^2 dV Σ_H |xi|.
    """
    d = _dx(dim, dx)
    _, ln, vol = horizon(dim, d, delta, weights=True)
    dV = float(np.prod(d[:dim]))
    return 0.5 * alpha * s0 * s0 * dV * float(np.sum(vol * ln))


# ----------------------------------------------------------------------------
# Direct sums (C)
# ----------------------------------------------------------------------------

def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def force_bond(u, chi, dx, delta, alpha, s=None):
    """L = chi s Σ chi' s' C (u' - u) dV (Eq. 17-18, 75, 100). u: (d, *shape)."""
    chi = _u8(chi)
    dim, n = _grid(chi.shape)
    u = _f64(u)
    assert u.shape == (dim,) + chi.shape
    s = None if s is None else _f64(s)
    L = np.empty_like(u)
    _load().or_force_bond(dim, _p(n), _p(_dx(dim, dx)), float(delta), float(alpha),
                          _p(chi), _p(s), _p(u), _p(L))
    return L


def force_bond_at(u, chi, dx, delta, alpha, nodes):
    """force_bond evaluated only at the linear node indices ``nodes``; returns (d, len(nodes))."""
    chi = _u8(chi)
    dim, n = _grid(chi.shape)
    u = _f64(u)
    assert u.shape == (dim,) + chi.shape
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    L = np.empty((dim, nodes.size), dtype=np.float64)
    _load().or_force_bond_at(dim, _p(n), _p(_dx(dim, dx)), float(delta), float(alpha), _p(chi), _p(u),
                             _p(nodes), int(nodes.size), _p(L))
    return L


def energy_bond(u, chi, dx, delta, alpha, lam=None, s=None):
    """W = 1/2 chi lam Σ chi' lam' eta.C.eta dV (Eq. 47, 102); with a real node
    weight s the bond factor is (s lam)(s' lam') (reading R17)."""
    chi = _u8(chi)
    dim, n = _grid(chi.shape)
    u = _f64(u)
    W = np.empty(chi.shape, dtype=np.float64)
    if s is not None:
        w = _f64(s) * (1.0 if lam is None else _u8(lam).astype(np.float64))
        _load().or_energy_bond_w(dim, _p(n), _p(_dx(dim, dx)), float(delta), float(alpha),
                                 _p(chi), _p(np.ascontiguousarray(w)), _p(u), _p(W))
        return W
    lam = None if lam is None else _u8(lam)
    _load().or_energy_bond(dim, _p(n), _p(_dx(dim, dx)), float(delta), float(alpha),
                           _p(chi), _p(lam), _p(u), _p(W))
    return W


def force_nonlinear(u, chi, dx, delta, alpha, lam=None):
    """Nonlinear rotation-invariant bond model (§3.2, Eq. 19-22):
    L = chi lam Σ chi' lam' c/2 (|xi+eta|^2 - |xi|^2)(xi+eta) dV, c = alpha/|xi|^3."""
    chi = _u8(chi)
    dim, n = _grid(chi.shape)
    u = _f64(u)
    lam = None if lam is None else _u8(lam)
    L = np.empty_like(u)
    _load().or_force_nl(dim, _p(n), _p(_dx(dim, dx)), float(delta), float(alpha), _p(chi), _p(lam), _p(u), _p(L))
    return L


def energy_nonlinear(u, chi, dx, delta, alpha, lam=None):
    """W = chi lam Σ chi' lam' c/8 (|xi+eta|^2 - |xi|^2)^2 dV (the potential of Eq. 21)."""
    chi = _u8(chi)
    dim, n = _grid(chi.shape)
    u = _f64(u)
    lam = None if lam is None else _u8(lam)
    W = np.empty(chi.shape, dtype=np.float64)
    _load().or_energy_nl(dim, _p(n), _p(_dx(dim, dx)), float(delta), float(alpha), _p(chi), _p(lam), _p(u), _p(W))
    return W


def damage(chi, lam, dx, delta):
    """(nb, beta, d): broken in-body bonds, initial in-body bonds, damage index
    (Eq. 12 with mu = lam lam', Eq. 44; reading R11)."""
    chi = _u8(chi)
    lam = _u8(lam)
    dim, n = _grid(chi.shape)
    nb = np.empty(chi.shape, dtype=np.int32)
    beta = np.empty(chi.shape, dtype=np.int32)
    d = np.empty(chi.shape, dtype=np.float64)
    _load().or_damage(dim, _p(n), _p(_dx(dim, dx)), float(delta), _p(chi), _p(lam),
                      _p(nb), _p(beta), _p(d))
    return nb, beta, d


def force_lps(u, chi, dx, delta, ka, cb, return_aux=False):
    """Linearized state-based force with EC (Eq. 33-39, 92-94), 3D only."""
    chi = _u8(chi)
    dim, n = _grid(chi.shape)
    assert dim == 3
    u = _f64(u)
    L = np.empty_like(u)
    th = np.empty(chi.shape, dtype=np.float64)
    m = np.empty(chi.shape, dtype=np.float64)
    _load().or_force_lps(_p(n), _p(_dx(3, dx)), float(delta), float(ka), float(cb),
                         _p(chi), _p(u), _p(L), _p(th), _p(m))
    if return_aux:
        return L, th, m
    return L


def force_bond_grad_s(u, p, chi, dx, delta, alpha, s=None):
    """d(Σ p.L)/ds for the bond operator with node weight s."""
    chi = _u8(chi)
    dim, n = _grid(chi.shape)
    u = _f64(u)
    p = _f64(p)
    s = None if s is None else _f64(s)
    g = np.empty(chi.shape, dtype=np.float64)
    _load().or_force_bond_grad_s(dim, _p(n), _p(_dx(dim, dx)), float(delta), float(alpha),
                                 _p(chi), _p(s), _p(u), _p(p), _p(g))
    return g


def symbol_bond(shape, dx, delta, alpha, k):
    """M(k) with L = -M(k) u for a single periodic mode (Eq. 57, chi = 1)."""
    dim = len(shape)
    n = np.array(list(shape[::-1]) + [1] * (3 - dim), dtype=np.int32)
    kk = np.zeros(3, dtype=np.float64)
    kk[:dim] = k
    M = np.zeros(9, dtype=np.float64)
    _load().or_symbol_bond(dim, _p(n), _p(_dx(dim, dx)), float(delta), float(alpha),
                           _p(kk), _p(M))
    return M.reshape(3, 3)[:dim, :dim].copy()


# ----------------------------------------------------------------------------
# Drivers in the paper's order
# ----------------------------------------------------------------------------

def verlet_damage(u, v, lam, chi, chi_omega, b, w, dx, delta, alpha, rho, dt, wc, nsteps, s=None, b0=None):
    """Velocity-Verlet with embedded constraint and energy-based bond breaking.

    Order per step n -> n+1 (Eq. 83-84 for the kinematics, Eq. 63 and reading R8
    for the integrity index, Eq. 100-102 for L and W with lambda):
        a^n      = L(u^n, lam^n) + b
        u^{n+1}  = chi_O { u^n + dt [v^n + dt/(2 rho) a^n] } + (1 - chi_O) w
        lam^{n+1} = lam^n [ W(u^n, lam^n) <= wc ]          (irreversible)
        a^{n+1}  = L(u^{n+1}, lam^{n+1}) + b
        v^{n+1}  = chi_O { v^n + dt/(2 rho) (a^n + a^{n+1}) }
    chi_omega has shape (d, *grid); w and b have shape (d, *grid). For a
    time-varying volume constraint w may instead be a function of the step
    index giving the prescribed field at the end of that step: u^{n+1} takes
    w(n + 1) on Gamma (t = (n + 1) dt).
    With a node weight s (a spatially varying micromodulus c = c0 s^2, reading
    R17) the bond factor in L and W is (s lam)(s' lam'). b0, if given, is an
    extra body force in a^0 only (an impulse on the first step).
    Returns (u, v, lam, flips) with flips = nodes whose lam went 1 -> 0.
    """
    u = _f64(u).copy()
    v = _f64(v).copy()
    lam = _u8(lam).copy()
    co = np.asarray(chi_omega, dtype=np.float64)
    b = _f64(b)
    w_at = w if callable(w) else (lambda n, w0=_f64(w): w0)
    sw = np.ones(chi.shape) if s is None else _f64(s)

    def force_energy(u, lam):
        L = force_bond(u, chi, dx, delta, alpha, s=sw * lam.astype(np.float64))
        W = energy_bond(u, chi, dx, delta, alpha, lam=lam) if s is None else \
            energy_bond(u, chi, dx, delta, alpha, lam=lam, s=sw)
        return L, W

    L, W = force_energy(u, lam)
    flips = 0
    for n in range(nsteps):
        a0 = L + b
        if n == 0 and b0 is not None:
            a0 = a0 + _f64(b0)
        u = co * (u + dt * (v + dt / (2.0 * rho) * a0)) + (1.0 - co) * _f64(w_at(n + 1))
        new_lam = (lam.astype(bool) & (W <= wc)).astype(np.uint8)
        flips += int(np.sum(lam.astype(np.int64) - new_lam.astype(np.int64)))
        lam = new_lam
        L, W = force_energy(u, lam)
        v = co * (v + dt / (2.0 * rho) * (a0 + L + b))
    return u, v, lam, flips


def static_residual(u, chi, chi_omega, b, dx, delta, op):
    """R = chi_O (L(u) + b) (Eq. 89); ``op`` is 'bond' with alpha or 'lps' with (ka, cb)."""
    L = _apply(op, u, chi, dx, delta)
    return np.asarray(chi_omega, dtype=np.float64) * (L + _f64(b))


def _apply(op, u, chi, dx, delta):
    kind = op[0]
    if kind == "bond":
        return force_bond(u, chi, dx, delta, op[1])
    if kind == "lps":
        return force_lps(u, chi, dx, delta, op[1], op[2])
    raise ValueError(kind)


def cg_static(chi, chi_omega, b, w, dx, delta, op, rtol=1e-12, max_iter=100000):
    """FP64 conjugate gradient for the EC static problem (Eq. 85-89, §5.1).

    Unknowns are u on Omega (chi_O = 1); u = w on Gamma (reading R14/R15).
    The system chi_O (L(u) + b) = 0 with u = e + (1 - chi_O) w, e = 0 off
    Omega, is A e = r0 with A e = -chi_O L(chi_O e) (symmetric positive
    definite on Omega) and r0 = chi_O (b + L((1 - chi_O) w)); values of w on
    Omega play no part. Unpreconditioned CG from e = 0 [50].
    Returns (u, iterations, relative residual ||chi_O(L(u)+b)|| / ||chi_O b||);
    when chi_O b = 0 (a problem driven by w alone) the residual is relative to
    the right-hand side ||r0|| = ||chi_O L((1 - chi_O) w)|| instead.
    """
    co = np.asarray(chi_omega, dtype=np.float64)
    wg = (1.0 - co) * _f64(w)  # w enters on Gamma only (Eq. 87-88)
    b = _f64(b)

    def A(e):
        return -co * _apply(op, co * e, chi, dx, delta)

    r = co * (b + _apply(op, wg, chi, dx, delta))
    e = np.zeros_like(r)
    p = r.copy()
    rr = float(np.vdot(r, r))
    bn = math.sqrt(float(np.vdot(co * b, co * b)))
    if bn == 0.0:
        bn = math.sqrt(rr) if rr > 0.0 else 1.0
    it = 0
    while it < max_iter and math.sqrt(rr) > rtol * bn:
        q = A(p)
        alpha = rr / float(np.vdot(p, q))
        e += alpha * p
        r -= alpha * q
        rr_new = float(np.vdot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    u = co * e + wg
    res = static_residual(u, chi, chi_omega, b, dx, delta, op)
    return u, it, math.sqrt(float(np.vdot(res, res))) / bn


def static_mirror(chi, chi_omega, b, g, mirror, dx, delta, op, rtol=1e-12, max_iter=2000):
    """Static EC problem with mirror-based volume constraints (§5.1; the paper's
    appendix on the method is not in its text, so this follows the description
    there: each Gamma point takes its value from the local boundary value g and
    the solution at its mirror point in Omega):

        chi_O (L(u) + b) = 0 on Omega,   u = 2 g - u(mirror) on Gamma,

    with mirror of shape (d, *grid): for each component and node of Gamma the
    flat node index of its mirror point (an Omega node), -1 elsewhere. u is
    linear in its Omega values e: u = E e + h with E e = chi_O e - (1 - chi_O)
    e(mirror) and h = 2 (1 - chi_O) g, so R(e) = -A e + r0 with
    A e = -chi_O L(E e) and r0 = chi_O (L(h) + b). A is not symmetric (the
    mirror coupling is one-sided), so the system is solved by GMRES (scipy) on
    the Omega entries. Returns (u, iterations, ||R|| / ||r0||)."""
    from scipy.sparse.linalg import LinearOperator, gmres

    co = np.asarray(chi_omega, dtype=np.float64)
    mirror = np.asarray(mirror, dtype=np.int64)
    g = _f64(g)
    b = _f64(b)
    d = co.shape[0]
    N = co[0].size
    gam = (co == 0) & (np.asarray(chi)[None].astype(bool))
    if np.any(mirror[gam] < 0):
        raise ValueError("every Gamma node of the body needs a mirror node")
    comp = np.broadcast_to(np.arange(d).reshape((d,) + (1,) * (co.ndim - 1)), co.shape)
    flat_m = np.where(gam, comp * N + np.maximum(mirror, 0), 0).reshape(-1)
    if np.any(co.reshape(-1)[flat_m[gam.reshape(-1)]] == 0):
        raise ValueError("mirror nodes must lie in Omega")
    idx = np.flatnonzero(co.reshape(-1) == 1)
    gam_f = gam.reshape(-1)

    def expand(x):
        e = np.zeros(co.size)
        e[idx] = x
        u = e.copy()
        u[gam_f] = -e[flat_m[gam_f]]
        return u.reshape(co.shape)

    h = 2.0 * np.where(gam, g, 0.0)

    def A(x):
        return -(co * _apply(op, expand(x), chi, dx, delta)).reshape(-1)[idx]

    r0 = (co * (_apply(op, h, chi, dx, delta) + b)).reshape(-1)[idx]
    n0 = float(np.linalg.norm(r0))
    if n0 == 0.0:
        return h.copy(), 0, 0.0
    count = [0]

    def cb(_):
        count[0] += 1

    x, info = gmres(LinearOperator((idx.size, idx.size), matvec=A, dtype=np.float64), r0, rtol=rtol,
                    atol=0.0, restart=200, maxiter=max_iter, callback=cb, callback_type="pr_norm")
    u = expand(x) + h
    res = static_residual(u, chi, chi_omega, b, dx, delta, op)
    return u, count[0], float(np.linalg.norm(res)) / n0


# Parity status of each oracle function: the pin tests that tie it to the
# paper or to mathematics (tests/test_oracle_pins.py).
PINS = {
    "horizon": "brute-force lattice count; |H| = 28/48/80 (2D d=3,4,5), 122 (3D d=3)",
    "alpha_bond": "energy of isotropic stretch vs classical elasticity; symbol vs Navier-Cauchy",
    "force_bond": "translation/rotation null space, affine interior, symbol, reciprocity, "
                  "all-pairs brute force, dense operator spectrum",
    "force_bond_at": "all-pairs brute force at sampled nodes (3D); equals force_bond at those nodes",
    "energy_bond": "energy identity Σ W dV = -<u, L u> dV (also with a real node weight s); isotropic-stretch "
                   "closed form; all-pairs brute force with the weight s s'",
    "damage": "integer counts vs brute force; intact body d = 0",
    "force_lps": "translation/rotation null space, affine 2-delta interior, dilatation of "
                 "isotropic stretch = 3 s, nu = 1/4 reduces to bond form, reciprocity",
    "force_bond_grad_s": "central finite differences of force_bond",
    "symbol_bond": "single-mode displacement through force_bond",
    "verlet_damage": "energy conservation without damage (also with a node weight s), time reversibility, "
                     "s = 1 reduces to the unweighted driver, a first-step impulse equals an initial velocity",
    "cg_static": "FP64 residual of the returned solution",
    "force_nonlinear": "finite rigid rotations give zero force (the linearized model does not), small-"
                       "displacement limit = force_bond, -grad of the total energy, total force zero, all-pairs "
                       "brute force, the convolutional form of Eq. 26 evaluated with numpy FFTs",
    "energy_nonlinear": "small-displacement limit = energy_bond (Eq. 47); zero under finite rigid rotations",
    "static_mirror": "reproduces the affine solution of a uniaxial stretch exactly where the naive "
                     "constraint does not; residual and mirror relation; fixed point of the per-iteration "
                     "update the paper describes",
    "partial_volumes": "weighted lattice moments vs the ball integrals (closed forms), long-wave symbol vs "
                       "Navier-Cauchy, all-pairs brute force, invariants, family counts vs lattice count",
}
