"""Failure handling on the GPU, made to happen from the host (nothing faults,
traps or hangs the GPU):

* a bounded device wait that runs out: pd_plan_inject_stall makes one block of
  the next row pass (or inverse plane pass of the FP32 CG) issue no copies, so
  its wait on the copy barrier gives up
  after the library's limit and records the time-out in the plan's status
  word; pd_solve_static must return PD_ERR_TIMEOUT and the same plan must then
  solve normally;
* non-finite values: a NaN in the body force, and a body force so large that
  the FP32 CG inner products overflow, must give PD_ERR_NONFINITE, and the
  plan must stay usable;
* the critical stretch s0 at the boundary: the plan's Wc equals the oracle's
  value of reading R10 (Wc of a fully bonded node under u = s0 x), with
  constant and partial-volume quadrature, 2D and 3D.
"""
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


def _cube(pdm, fp64):
    cfg = inputs.cube_with_cavity(n=32, radius_frac=0.2)
    prob = pdm.Problem(shape=cfg["shape"], delta=3.0, model=pdm.PD_LIN_STATE, nu=0.25, fp64=fp64)
    plan = pdm.Plan(prob, _t(cfg["chi"], torch.uint8), _t(cfg["chi_omega"], torch.uint8))
    return cfg, plan


def _solve_ok(pdm, plan, cfg, oracle):
    u = torch.zeros((3,) + cfg["shape"], dtype=torch.float64, device=DEV)
    it, rel, st = plan.solve_static(u, _t(cfg["b"]), None, rtol=1e-8, max_iter=5000)
    assert st == 0 and rel <= 1e-8
    ka, cb, _ = oracle.lps_constants(1.0, 0.25, 1.0, 3.0)
    res = oracle.static_residual(u.cpu().numpy(), cfg["chi"], cfg["chi_omega"], cfg["b"], 1.0, 3.0, ("lps", ka, cb))
    assert np.linalg.norm(res) / np.linalg.norm(cfg["chi_omega"] * cfg["b"]) <= 1.5e-8


@pytest.mark.parametrize("kind", [0, 3, 5])
def test_wait_time_out_is_reported_and_plan_stays_usable(pdm, oracle, kind):
    cfg, plan = _cube(pdm, fp64=False)
    if kind == 5:
        plan.set_plane_passes(3)  # the inverse half of the CG iteration as a plane pass
    plan.inject_stall(kind)
    u = torch.zeros((3,) + cfg["shape"], dtype=torch.float64, device=DEV)
    with pytest.raises(pdm.PDError, match="PD_ERR_TIMEOUT"):
        plan.solve_static(u, _t(cfg["b"]), None, rtol=1e-8, max_iter=5000)
    torch.cuda.synchronize()  # the context is still usable
    _solve_ok(pdm, plan, cfg, oracle)
    plan.close()


def test_nonfinite_inputs_are_reported(pdm, oracle):
    cfg, plan = _cube(pdm, fp64=False)
    u = torch.zeros((3,) + cfg["shape"], dtype=torch.float64, device=DEV)
    b = cfg["b"].copy()
    idx = np.argwhere(cfg["chi_omega"][0] == 1)[17]
    b[(0,) + tuple(idx)] = np.nan
    with pytest.raises(pdm.PDError, match="PD_ERR_NONFINITE"):
        plan.solve_static(u, _t(b), None, rtol=1e-8, max_iter=5000)
    # finite in FP64, but its square overflows the FP32 CG inner products
    u.zero_()
    with pytest.raises(pdm.PDError, match="PD_ERR_NONFINITE"):
        plan.solve_static(u, _t(cfg["b"] * 1e25), None, rtol=1e-8, max_iter=5000)
    _solve_ok(pdm, plan, cfg, oracle)
    plan.close()


@pytest.mark.parametrize("dim,delta,rule", [(2, 4.0, 0), (2, 3.0, 1), (3, 3.0, 0), (3, 2.5, 1)])
def test_critical_stretch_gives_the_oracle_wc(pdm, oracle, dim, delta, rule):
    n = 64 if dim == 2 else 32
    shape = (n,) * dim
    m = int(math.ceil(delta + 0.5)) + 1
    chi = inputs.box_mask(shape, (m,) * dim, (n - m,) * dim)
    plan = pdm.Plan(pdm.Problem(shape=shape, delta=delta, E=2.0, s0=1e-3, volume_rule=rule, fp64=True),
                    _t(chi, torch.uint8))
    with oracle.partial_volumes(rule == 1):
        wc = oracle.wc_from_stretch(dim, 1.0, delta, oracle.alpha_bond(dim, 2.0, delta), 1e-3)
    assert abs(plan.critical_energy / wc - 1.0) < 1e-14
    plan.close()
    # an explicit Wc wins over s0; s0 with the state-based model is refused
    plan = pdm.Plan(pdm.Problem(shape=shape, delta=delta, E=2.0, s0=1e-3, Wc=0.5, volume_rule=rule, fp64=True),
                    _t(chi, torch.uint8))
    assert plan.critical_energy == 0.5
    plan.close()
    if dim == 3:
        with pytest.raises(pdm.PDError, match="PD_ERR_ARG"):
            pdm.Plan(pdm.Problem(shape=shape, delta=delta, model=pdm.PD_LIN_STATE, s0=1e-3), _t(chi, torch.uint8))
