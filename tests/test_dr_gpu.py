"""Dynamic relaxation (single plan and batched specimens in one graph launch)
and the pass autotuner, against the FP64 oracle and the FP64 GPU CG path."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _t(a, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def _bond_problem(pdm, cfg, fp64):
    return pdm.Problem(shape=cfg["shape"], delta=cfg["delta"], nu=1.0 / 3.0, fp64=fp64)


@pytest.mark.parametrize("fp64", [False, True])
def test_dr_2d_matches_oracle(pdm, oracle, fp64):
    cfg = inputs.batched_specimens(count=1, seed=3, sizes=[100])[0]
    plan = pdm.Plan(_bond_problem(pdm, cfg, fp64), _t(cfg["chi"], torch.uint8), _t(cfg["chi_omega"], torch.uint8))
    u = torch.zeros((2,) + cfg["shape"], dtype=torch.float64, device=DEV)
    it, rel, st = plan.solve_dr(u, _t(cfg["b"]), None, rtol=1e-8, max_iter=300000)
    assert st == 0 and rel <= 1e-8 and it > 0
    ug = u.cpu().numpy()
    alpha = oracle.alpha_bond(2, 1.0, cfg["delta"])
    op = ("bond", alpha)
    res = oracle.static_residual(ug, cfg["chi"], cfg["chi_omega"], cfg["b"], 1.0, cfg["delta"], op)
    bn = np.linalg.norm(cfg["chi_omega"] * cfg["b"])
    assert np.linalg.norm(res) / bn <= 1.5e-8
    uo, _, relo = oracle.cg_static(cfg["chi"], cfg["chi_omega"], cfg["b"], cfg["w"], 1.0, cfg["delta"], op,
                                   rtol=1e-12)
    assert relo < 1e-11
    assert _rel(ug, uo) < 2e-6
    assert np.all(ug[:, cfg["chi_omega"][0] == 0] == 0)
    plan.close()


def test_dr_3d_state_based_matches_oracle(pdm, oracle):
    """The unfused step (state-based operator with its dilatation round)."""
    cfg = inputs.cube_with_cavity(n=32, radius_frac=0.2)
    shape = cfg["shape"]
    prob = pdm.Problem(shape=shape, delta=3.0, model=pdm.PD_LIN_STATE, nu=0.4, fp64=False)
    plan = pdm.Plan(prob, _t(cfg["chi"], torch.uint8), _t(cfg["chi_omega"], torch.uint8))
    u = torch.zeros((3,) + shape, dtype=torch.float64, device=DEV)
    it, rel, st = plan.solve_dr(u, _t(cfg["b"]), None, rtol=1e-8, max_iter=300000)
    assert st == 0 and rel <= 1e-8
    ka, cb, _ = oracle.lps_constants(1.0, 0.4, 1.0, 3.0)
    op = ("lps", ka, cb)
    uo, _, _ = oracle.cg_static(cfg["chi"], cfg["chi_omega"], cfg["b"], cfg["w"], 1.0, 3.0, op, rtol=1e-12)
    assert _rel(u.cpu().numpy(), uo) < 2e-6
    plan.close()


def test_dr_3d_bond_fused_matches_cg(pdm):
    """The fused 3D step against the FP64 GPU CG path at the same tolerance."""
    cfg = inputs.cube_with_cavity(n=64, radius_frac=0.2)
    shape = cfg["shape"]
    sols = []
    for fp64, method in ((False, "dr"), (True, "cg")):
        prob = pdm.Problem(shape=shape, delta=3.0, model=pdm.PD_LIN_BOND, fp64=fp64)
        plan = pdm.Plan(prob, _t(cfg["chi"], torch.uint8), _t(cfg["chi_omega"], torch.uint8))
        u = torch.zeros((3,) + shape, dtype=torch.float64, device=DEV)
        solve = plan.solve_dr if method == "dr" else plan.solve_static
        it, rel, st = solve(u, _t(cfg["b"]), None, rtol=1e-8, max_iter=300000)
        assert st == 0 and rel <= 1e-8
        sols.append(u.cpu().numpy())
        plan.close()
    assert _rel(sols[0], sols[1]) < 2e-6


def test_dr_budget_exhausted_terminates(pdm):
    """A step budget far too small ends the device-side loop with NOT_CONVERGED."""
    cfg = inputs.batched_specimens(count=1, seed=5, sizes=[120])[0]
    plan = pdm.Plan(_bond_problem(pdm, cfg, False), _t(cfg["chi"], torch.uint8), _t(cfg["chi_omega"], torch.uint8))
    u = torch.zeros((2,) + cfg["shape"], dtype=torch.float64, device=DEV)
    it, rel, st = plan.solve_dr(u, _t(cfg["b"]), None, rtol=1e-8, max_iter=64, raise_on_fail=False)
    assert st == -5 and 64 <= it <= 80 and 0 < rel < 10.0
    plan.close()


def _solve_batch(pdm, cfgs, rtol, tune=False):
    probs = [_bond_problem(pdm, c, False) for c in cfgs]
    batch = pdm.Batch(probs, [_t(c["chi"], torch.uint8) for c in cfgs],
                      [_t(c["chi_omega"], torch.uint8) for c in cfgs])
    if tune:
        batch.autotune()
    us = [torch.zeros((2,) + c["shape"], dtype=torch.float64, device=DEV) for c in cfgs]
    bs = [_t(c["b"]) for c in cfgs]
    its, rels, sts = batch.solve_dr(us, bs, rtol=rtol, max_iter=300000)
    return batch, us, bs, its, rels, sts


def test_dr_batched_uneven_matches_fp64_cg(pdm, oracle):
    cfgs = inputs.batched_specimens(count=8, seed=11, nmin=40, nmax=250)
    batch, us, bs, its, rels, sts = _solve_batch(pdm, cfgs, 1e-8)
    assert all(s == 0 for s in sts) and all(r <= 1e-8 for r in rels)
    assert len({c["shape"] for c in cfgs}) > 1 and len({c["delta"] for c in cfgs}) > 1
    for c, u in zip(cfgs, us):
        plan = pdm.Plan(_bond_problem(pdm, c, True), _t(c["chi"], torch.uint8), _t(c["chi_omega"], torch.uint8))
        uc = torch.zeros_like(u)
        _, relc, stc = plan.solve_static(uc, _t(c["b"]), None, rtol=1e-8, max_iter=100000)
        assert stc == 0
        assert _rel(u.cpu().numpy(), uc.cpu().numpy()) < 2e-6
        plan.close()
    # the smallest specimen also against the oracle's FP64 operator
    k = int(np.argmin([c["shape"][0] for c in cfgs]))
    c = cfgs[k]
    res = oracle.static_residual(us[k].cpu().numpy(), c["chi"], c["chi_omega"], c["b"], 1.0, c["delta"],
                                 ("bond", oracle.alpha_bond(2, 1.0, c["delta"])))
    assert np.linalg.norm(res) / np.linalg.norm(c["chi_omega"] * c["b"]) <= 1.5e-8
    # second call: cached graph, new right-hand sides in the same buffers
    for b in bs:
        b.mul_(-2.0)
    us2 = [torch.zeros_like(u) for u in us]
    its2, rels2, sts2 = batch.solve_dr(us2, bs, rtol=1e-8, max_iter=300000)
    assert all(s == 0 for s in sts2)
    for u, u2 in zip(us, us2):
        assert _rel(u2.cpu().numpy(), -2.0 * u.cpu().numpy()) < 2e-6
    batch.close()


def test_autotune_keeps_results(pdm):
    cfg = inputs.cube_with_cavity(n=64)
    shape = cfg["shape"]
    prob = pdm.Problem(shape=shape, delta=3.0, fp64=False)
    plan = pdm.Plan(prob, _t(cfg["chi"], torch.uint8))
    g = inputs.rng(2)
    u = torch.tensor(g.normal(size=(3,) + shape) * cfg["chi"], dtype=torch.float32, device=DEV)
    L0 = plan.force(u).double()
    tun = plan.autotune()
    assert tun["rows"] > 0 and tun["w_x2"] in (4, 8, 16, 32) and tun["w_last"] in (4, 8, 16, 32)
    assert tun["sched"] in (0, 1) and tun["stages"] in (1, 2)
    L1 = plan.force(u).double()
    assert float(torch.linalg.norm(L1 - L0) / torch.linalg.norm(L0)) < 2e-6
    plan.close()


def test_dr_batched_config4_full_size(pdm, oracle):
    """64 uneven specimens (sides 256..1024, delta 3..5) in one graph launch,
    each to 1e-8; two against the FP64 GPU CG path, one against the oracle's
    FP64 operator."""
    cfgs = inputs.batched_specimens(count=64, seed=0)
    batch, us, bs, its, rels, sts = _solve_batch(pdm, cfgs, 1e-8, tune=True)
    assert all(s == 0 for s in sts), sts
    assert max(rels) <= 1e-8
    assert {c["shape"][0] for c in cfgs} >= {512, 1024} and {c["delta"] for c in cfgs} == {3.0, 4.0, 5.0}
    for k in (0, 2):
        c = cfgs[k]
        plan = pdm.Plan(_bond_problem(pdm, c, True), _t(c["chi"], torch.uint8), _t(c["chi_omega"], torch.uint8))
        uc = torch.zeros_like(us[k])
        _, _, stc = plan.solve_static(uc, bs[k], None, rtol=1e-8, max_iter=100000)
        assert stc == 0
        assert float(torch.linalg.norm(uc - us[k]) / torch.linalg.norm(uc)) < 1e-6
        plan.close()
    k = next(i for i, c in enumerate(cfgs) if c["shape"][0] == 512)
    c = cfgs[k]
    res = oracle.static_residual(us[k].cpu().numpy(), c["chi"], c["chi_omega"], c["b"], 1.0, c["delta"],
                                 ("bond", oracle.alpha_bond(2, 1.0, c["delta"])))
    assert np.linalg.norm(res) / np.linalg.norm(c["chi_omega"] * c["b"]) <= 1.5e-8
    batch.close()


def test_tuning_and_mode_arguments_are_checked(pdm):
    """Bad pass configurations and energy modes are rejected with PD_ERR_ARG and
    leave the plan usable; a pinned configuration round-trips."""
    shape = (64, 64)
    chi = inputs.box_mask(shape, (4, 4), (60, 60))
    plan = pdm.Plan(pdm.Problem(shape=shape, delta=3.0), _t(chi, torch.uint8))
    for bad in [(3, 0, 0, 0, 0, 0), (0, 64, 0, 0, 0, 0), (0, 0, 6, 0, 0, 0), (0, 0, 0, 2, 0, 0),
                (0, 0, 0, 0, 3, 0), (0, 0, 0, 0, 0, -1)]:
        with pytest.raises(pdm.PDError) as ei:
            plan.set_tuning(*bad)
        assert ei.value.status == -1
    assert pdm.load().pd_plan_set_energy_mode(plan._h, 2) == -1  # modes are 0 and 1
    plan.set_tuning(8, 0, 8, 1, 1, 2)
    assert plan.tuning == {"rows": 8, "w_x2": 0, "w_last": 8, "sched": 1, "stages": 1, "stages_inv": 2}
    u = torch.tensor(inputs.sine_modes(shape, 2, 1e-3, 2, 1) * chi, dtype=torch.float32, device=DEV)
    L = plan.force(u)
    assert torch.isfinite(L).all()
    plan.close()
