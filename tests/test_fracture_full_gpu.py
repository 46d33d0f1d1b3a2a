"""The dynamic brittle-fracture workload at full size: 1024 x 512 nodes,
delta = 4, critical energy from the critical stretch s0 = 1e-3, constant
traction layers, 4000 FP32 velocity-Verlet steps with bond breaking
(Eq. 63, 83-84, 101-102).

Full-size parity:
  - FP64: the GPU path follows the FP64 oracle bit for bit in the integrity
    index, in both energy modes (the convolution form of Eq. 102 and the
    horizon sum of Eq. 47), through the first 250 steps (bonds start to break
    at about step 120);
  - FP32, energy mode 1: after 4000 steps, one more step from the run's
    state takes the oracle's decisions on every node that is not borderline;
    the final damage counts are exact integers.

Borderline (FP32, horizon-sum energy): eta = u' - u is one correctly rounded
FP32 subtraction of the stored values and each bond adds
(alpha/|xi|) (xi.eta)^2 / |xi|^2 with the projection xi.eta formed first, so a
bond term errs by at most about 4 eps32 (alpha/|xi|) |xi^.eta| |eta| and the
summation by |H| eps32 W: |W32 - W| <= 32 eps32 (S + 2 W) with
S(x) = 1/2 chi lam Σ_H chi' lam' (alpha/|xi|) |xi^.eta| |eta| (a factor of
about 4 to spare). A node is borderline when |W - Wc| is within that bound.

(The convolution form in FP32 errs globally, by about
eps32 lambda_max (rms|u|^2 + 2 |u(x)| rms|u|); in this run that exceeds Wc
after about 1000 steps, when the broken halves fly apart, which is why the
long FP32 run uses the horizon-sum energy.)"""
import math

import numpy as np
import pytest
import torch

from paper_2105_06055_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.fixture(scope="module")
def pdm():
    from paper_2105_06055_gb300 import build, pd
    build.build()
    pd.load()
    return pd


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def test_fracture_config3_full_size(pdm, oracle):
    delta = 4.0
    cfg = inputs.notched_plate(n1=1024, n2=512, delta=delta, sigma=1.0)
    shape = cfg["shape"]
    alpha = oracle.alpha_bond(2, 1.0, delta)
    assert abs(alpha - 9.0 / (64.0 * math.pi)) < 1e-15
    wc = oracle.wc_from_stretch(2, 1.0, delta, alpha, 1e-3)
    b = cfg["b"] * (0.242 * math.sqrt(wc))
    # the critical stretch goes to the library, which derives Wc itself
    plans = {fp64: pdm.Plan(pdm.Problem(shape=shape, delta=delta, rho=1.0, s0=1e-3, nu=1.0 / 3.0, fp64=fp64),
                            _t(cfg["chi"], torch.uint8)) for fp64 in (True, False)}
    for p in plans.values():
        assert abs(p.critical_energy / wc - 1.0) < 1e-14
    dt = 0.8 * plans[True].stable_dt

    # (1) FP64 GPU path against the oracle through crack initiation, both energy modes
    n0 = 250
    uo, vo, lo, flo = oracle.verlet_damage(np.zeros((2,) + shape), np.zeros((2,) + shape), cfg["lam"], cfg["chi"],
                                           cfg["chi_omega"], b, cfg["w"], 1.0, delta, alpha, 1.0, dt, wc, n0)
    assert flo > 0
    for direct in (False, True):
        plans[True].set_energy_mode(direct)
        u = torch.zeros((2,) + shape, dtype=torch.float64, device=DEV)
        v = torch.zeros_like(u)
        lam = _t(cfg["lam"], torch.uint8)
        nb = plans[True].step_verlet(u, v, lam, _t(b), None, dt=dt, nsteps=n0, count_broken=True)
        assert nb == flo
        assert np.array_equal(lam.cpu().numpy(), lo)
        assert float(np.linalg.norm(u.cpu().numpy() - uo) / np.linalg.norm(uo)) < 1e-10

    # (2) the FP32 run of 4000 steps (horizon-sum energy), broken counts every 100 steps
    plans[False].set_energy_mode(True)
    u32 = torch.zeros((2,) + shape, dtype=torch.float32, device=DEV)
    v32 = torch.zeros_like(u32)
    lam32 = _t(cfg["lam"], torch.uint8)
    b32 = _t(b, torch.float32)
    total, hist = 0, []
    for _ in range(40):
        lam_prev = lam32.clone()
        total += plans[False].step_verlet(u32, v32, lam32, b32, None, dt=dt, nsteps=100, count_broken=True)
        hist.append(total)
        assert bool(torch.all(lam32 <= lam_prev))  # irreversible
    assert hist[1] > 0 and hist[-1] > 4 * hist[1]  # the crack initiates and grows
    assert torch.isfinite(u32).all()

    # (3) one more step from the FP32 state: decisions against the oracle
    us, vs, ls = u32.double().cpu().numpy(), v32.double().cpu().numpy(), lam32.cpu().numpy()
    W = oracle.energy_bond(us, cfg["chi"], 1.0, delta, alpha, lam=ls)
    _, _, lo1, _ = oracle.verlet_damage(us, vs, ls, cfg["chi"], cfg["chi_omega"], b, cfg["w"], 1.0, delta, alpha,
                                        1.0, dt, wc, 1)
    plans[False].step_verlet(u32, v32, lam32, b32, None, dt=dt, nsteps=1)
    lg = lam32.cpu().numpy()
    off, ln = oracle.horizon(2, 1.0, delta)
    live = ((cfg["chi"] == 1) & (ls == 1)).astype(np.float64)
    S = np.zeros(shape)
    for (o1, o2, _), r in zip(off, ln):
        sh = (-int(o2), -int(o1))
        e0 = np.roll(us[0], sh, axis=(0, 1)) - us[0]
        e1 = np.roll(us[1], sh, axis=(0, 1)) - us[1]
        proj = np.abs(o1 * e0 + o2 * e1) / r
        S += np.roll(live, sh, axis=(0, 1)) * proj * np.sqrt(e0 * e0 + e1 * e1) / r
    S *= 0.5 * alpha * live
    clear = np.abs(W - wc) > 32 * np.finfo(np.float32).eps * (S + 2 * np.abs(W))
    assert np.array_equal(lg[clear], lo1[clear])
    assert np.sum(lg != lo1) <= np.sum(~clear)
    assert np.sum(~clear) < 1e-3 * np.sum(cfg["chi"])

    # (4) damage counts of the final state, exact
    nbo, _, do = oracle.damage(cfg["chi"], lg, 1.0, delta)
    nbg, dg = plans[False].damage(lam32)
    assert np.array_equal(nbg.cpu().numpy(), nbo)
    assert np.allclose(dg.double().cpu().numpy(), do, rtol=1e-6, atol=0)
    for p in plans.values():
        p.close()
