"""GPU parity of the partial-volume quadrature against the FP64 oracle under the
same rule.

§4.1.1 notes that a weight dV(|xi|) in place of dV, for cells only partly
covered by the horizon, is part of the kernel C(xi) and keeps every
convolution. The plan takes the linear rule of Hu, Ha and Bobaru
(``Problem.volume_rule = 1``): bond weight beta(|xi|) dV with
beta = min(1, (delta + h/2 - |xi|)/h) for |xi| < delta + h/2, cubic cells.
Nothing else changes, so every entry point is checked here with the
tolerances of the constant-dV tests: FP64 1e-11, FP32 1e-5 (force), W 1e-4.
"""
import math

import numpy as np
import pytest
import torch

from paper_2105_06055_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
FP64_TOL = 1e-11
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def pdm():
    from paper_2105_06055_gb300 import build, pd
    build.build()
    pd.load()
    return pd


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def _plan(pdm, shape, chi, delta, fp64, dx=1.0, chi_omega=None, **kw):
    prob = pdm.Problem(shape=shape, dx=dx, delta=delta, fp64=fp64, volume_rule=1, **kw)
    return pdm.Plan(prob, _t(chi, torch.uint8), None if chi_omega is None else _t(chi_omega, torch.uint8))


@pytest.mark.parametrize("delta,dx", [(3.0, 1.0), (4.5, 1.0), (2.2, 0.9)])
@pytest.mark.parametrize("fp64", [True, False])
def test_bond_2d_force_and_energy(pdm, oracle, delta, dx, fp64):
    """Ragged body, random displacements and node weights; W of Eq. 102."""
    shape = (64, 128)
    g = inputs.rng(17)
    r = int((delta + dx / 2) / dx) + 1
    chi = inputs.box_mask(shape, (r, r), (128 - r, 64 - r))
    chi[g.random(shape) < 0.1] = 0
    u = g.normal(size=(2,) + shape)
    lam = (g.random(shape) < 0.9).astype(np.uint8)
    alpha = oracle.alpha_bond(2, 1.0, delta)
    with oracle.partial_volumes():
        ref = oracle.force_bond(u, chi, dx, delta, alpha)
        Lref = oracle.force_bond(u, chi, dx, delta, alpha, s=lam.astype(float))
        Wref = oracle.energy_bond(u, chi, dx, delta, alpha, lam=lam)
    ref0 = oracle.force_bond(u, chi, dx, delta, alpha)
    assert _rel(ref0, ref) > 1e-2  # the rule changes the operator
    dt = torch.float64 if fp64 else torch.float32
    plan = _plan(pdm, shape, chi, delta, fp64, dx=dx)
    L = plan.force(_t(u, dt)).double().cpu().numpy()
    assert _rel(L, ref) < (FP64_TOL if fp64 else FP32_TOL)
    L2, W = plan.force(_t(u, dt), s=_t(lam, dt), want_energy=True)
    assert _rel(L2.double().cpu().numpy(), Lref) < (FP64_TOL if fp64 else FP32_TOL)
    assert _rel(W.double().cpu().numpy(), Wref) < (FP64_TOL if fp64 else 1e-4)
    plan.close()


@pytest.mark.parametrize("fp64", [True, False])
def test_state_based_3d(pdm, oracle, fp64):
    """nu = 0.4 (dilatation round active): m, q and the kernels all carry the weights."""
    shape = (32, 32, 32)
    delta = 3.0
    chi = inputs.box_mask(shape, (4, 4, 4), (28, 28, 28))
    x1, x2, x3 = inputs.coords(shape)
    chi[(x1 - 15.5) ** 2 + (x2 - 15.5) ** 2 + (x3 - 15.5) ** 2 < 36] = 0
    u = inputs.sine_modes(shape, 4, 1e-3, 3, 9)
    with oracle.partial_volumes():
        ka, cb, _ = oracle.lps_constants(1.0, 0.4, 1.0, delta)
        ref = oracle.force_lps(u, chi, 1.0, delta, ka, cb)
    dt = torch.float64 if fp64 else torch.float32
    plan = _plan(pdm, shape, chi, delta, fp64, model=pdm.PD_LIN_STATE, nu=0.4)
    L = plan.force(_t(u, dt)).double().cpu().numpy()
    assert _rel(L, ref) < (FP64_TOL if fp64 else FP32_TOL)
    plan.close()


def test_bond_3d_fp64(pdm, oracle):
    shape = (16, 32, 32)
    delta = 2.6
    g = inputs.rng(23)
    chi = inputs.box_mask(shape, (4, 4, 4), (28, 28, 12))
    chi[g.random(shape) < 0.05] = 0
    u = g.normal(size=(3,) + shape)
    alpha = oracle.alpha_bond(3, 1.0, delta)
    with oracle.partial_volumes():
        ref = oracle.force_bond(u, chi, 1.0, delta, alpha)
    plan = _plan(pdm, shape, chi, delta, True)
    assert _rel(plan.force(_t(u)).cpu().numpy(), ref) < FP64_TOL
    plan.close()


def test_kernel_spectrum_and_stable_step(pdm, oracle):
    shape = (32, 64)
    delta = 3.5
    chi = inputs.box_mask(shape, (5, 5), (59, 27))
    plan = _plan(pdm, shape, chi, delta, True)
    K = plan.kernel_spectrum().cpu().numpy()
    alpha = oracle.alpha_bond(2, 1.0, delta)
    P = K[:, 0, 0]
    with oracle.partial_volumes():
        for k1, k2 in [(0, 0), (3, 0), (0, 5), (7, 29), (32, 16), (1, 31)]:
            M = oracle.symbol_bond(shape, 1.0, delta, alpha, (k1, k2))
            Kk = K[:, k2, k1]
            Mg = np.array([[P[0] - Kk[0], P[2] - Kk[2]], [P[2] - Kk[2], P[1] - Kk[1]]])
            assert np.allclose(Mg, M, rtol=1e-12, atol=1e-14)
        lmax = max(np.linalg.eigvalsh(oracle.symbol_bond(shape, 1.0, delta, alpha, (a, b))).max()
                   for a in range(0, 33) for b in range(0, 32))
    assert abs(plan.stable_dt / (2 * math.sqrt(1.0 / lmax)) - 1) < 1e-9
    plan.close()


def test_static_2d_bond_fp64(pdm, oracle):
    """Clamped face, body-force layer: the GPU solution equals the oracle's FP64 CG."""
    shape = (64, 64)
    chi = inputs.box_mask(shape, (4, 4), (60, 56))
    x1, x2 = inputs.coords(shape)
    co = chi.copy()
    co[(x1 >= 4) & (x1 < 7)] = 0
    b = np.zeros((2,) + shape)
    b[0][(x1 >= 57) & (x1 < 60) & (chi == 1)] = 1e-3 / 3
    b[1][(x1 >= 57) & (x1 < 60) & (chi == 1)] = -0.5e-3 / 3
    plan = _plan(pdm, shape, chi, 3.0, True, chi_omega=np.stack([co, co]))
    u = torch.zeros((2,) + shape, dtype=torch.float64, device=DEV)
    it, rel, st = plan.solve_static(u, _t(b), None, rtol=1e-10, max_iter=20000)
    assert st == 0 and rel <= 1e-10
    alpha = oracle.alpha_bond(2, 1.0, 3.0)
    with oracle.partial_volumes():
        uo, _, _ = oracle.cg_static(chi, np.stack([co, co]), b, np.zeros_like(b), 1.0, 3.0, ("bond", alpha),
                                    rtol=1e-13)
    assert _rel(u.cpu().numpy(), uo) < 1e-8
    plan.close()


@pytest.mark.parametrize("direct", [False, True])
def test_verlet_damage_fp64_bit_parity(pdm, oracle, direct):
    """FP64 velocity Verlet with bond breaking: the integrity field follows the
    oracle bit for bit (both energy forms), the counts of broken bonds include
    the partly covered ones as whole bonds."""
    cfg = inputs.notched_plate(n1=128, n2=64, delta=3.0, sigma=1.0)
    shape, delta = cfg["shape"], cfg["delta"]
    alpha = oracle.alpha_bond(2, 1.0, delta)
    with oracle.partial_volumes():
        wc = oracle.wc_from_stretch(2, 1.0, delta, alpha, 1e-3)
        b = cfg["b"] * (0.25 * math.sqrt(wc))
        lmax = max(np.linalg.eigvalsh(oracle.symbol_bond(shape, 1.0, delta, alpha, (k, k))).max()
                   for k in range(0, 33))
        dt = 0.5 * 2 * math.sqrt(1.0 / lmax)
        nsteps = 60
        uo, vo, lo, flo = oracle.verlet_damage(np.zeros((2,) + shape), np.zeros((2,) + shape), cfg["lam"],
                                               cfg["chi"], cfg["chi_omega"], b, cfg["w"], 1.0, delta, alpha, 1.0,
                                               dt, wc, nsteps)
        nbo, _, _ = oracle.damage(cfg["chi"], lo, 1.0, delta)
    assert flo > 0
    plan = _plan(pdm, shape, cfg["chi"], delta, True, rho=1.0, Wc=wc)
    plan.set_energy_mode(direct)
    u = torch.zeros((2,) + shape, dtype=torch.float64, device=DEV)
    v = torch.zeros_like(u)
    lam = _t(cfg["lam"], torch.uint8)
    nb = plan.step_verlet(u, v, lam, _t(b), None, dt=dt, nsteps=nsteps, count_broken=True)
    assert nb == flo
    assert np.array_equal(lam.cpu().numpy(), lo)
    assert _rel(u.cpu().numpy(), uo) < 1e-10 and _rel(v.cpu().numpy(), vo) < 1e-10
    nbg, _ = plan.damage(lam)
    assert np.array_equal(nbg.cpu().numpy(), nbo)
    plan.close()


def test_margin_and_cell_checks(pdm):
    """The family reaches delta + h/2: a body that clears delta but not the
    family's reach is refused under the rule; non-cubic cells are refused."""
    shape = (64, 64)
    delta = 3.6  # constant rule: 3 cells; partial volumes: |xi| < 4.1, 4 cells
    chi = inputs.box_mask(shape, (3, 3), (61, 61))
    p0 = pdm.Plan(pdm.Problem(shape=shape, delta=delta), _t(chi, torch.uint8))
    p0.close()
    with pytest.raises(pdm.PDError):
        pdm.Plan(pdm.Problem(shape=shape, delta=delta, volume_rule=1), _t(chi, torch.uint8))
    chi4 = inputs.box_mask(shape, (4, 4), (60, 60))
    p1 = pdm.Plan(pdm.Problem(shape=shape, delta=delta, volume_rule=1), _t(chi4, torch.uint8))
    p1.close()
    with pytest.raises(pdm.PDError):
        pdm.Plan(pdm.Problem(shape=shape, dx=(1.0, 1.1), delta=delta, volume_rule=1), _t(chi4, torch.uint8))
