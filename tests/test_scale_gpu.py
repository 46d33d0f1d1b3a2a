"""Force evaluation at 256^3 and 512^3 nodes (3D bond model, delta = 3, body =
cube minus a centred ball): the FP32 and FP64 GPU paths against the FP64
oracle's direct sum at 4096 sampled nodes, half of them within delta of the
body's surface (where the boundary field G acts) and half anywhere in the body."""
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


def _samples(chi, n, seed):
    g = inputs.rng(seed)
    body = np.flatnonzero(chi.reshape(-1))
    anywhere = g.choice(body, size=2048, replace=False)
    # near the ball's surface: random directions at radius R + [0, 3)
    c = (n - 1) / 2.0
    R = 0.25 * n
    d = g.normal(size=(8192, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = np.rint(c + d * (R + g.uniform(0, 3, size=(8192, 1)))).astype(np.int64)
    lin = (pts[:, 2] * n + pts[:, 1]) * n + pts[:, 0]
    lin = np.unique(lin[chi.reshape(-1)[lin] == 1])[:2048]
    assert lin.size > 1024
    return np.concatenate([anywhere, lin])


@pytest.mark.parametrize("n,fp64", [(256, False), (256, True), (512, False)])
def test_bond_force_large_sampled(pdm, oracle, n, fp64):
    shape = (n, n, n)
    chi = inputs.cube_with_ball_mask(n)
    # wave numbers n/32..n/16 (a deformation field; FP32 error ~ eps32 kappa, kappa ~ 10-30)
    u = inputs.separable_modes(shape, 4, n // 16, 1e-3, seed=n, dtype=np.float64 if fp64 else np.float32,
                               kmin=n // 32)
    u *= chi
    dt = torch.float64 if fp64 else torch.float32
    plan = pdm.Plan(pdm.Problem(shape=shape, delta=3.0, fp64=fp64), torch.tensor(chi, device=DEV))
    ud = torch.tensor(u, dtype=dt, device=DEV)
    L = plan.force(ud)
    nodes = _samples(chi, n, seed=n + 1)
    idx = torch.tensor(nodes, device=DEV)
    Lg = L.reshape(3, -1)[:, idx].double().cpu().numpy()
    del L, ud
    plan.close()
    alpha = oracle.alpha_bond(3, 1.0, 3.0)
    Lo = oracle.force_bond_at(u.astype(np.float64), chi, 1.0, 3.0, alpha, nodes)
    rel = float(np.linalg.norm(Lg - Lo) / np.linalg.norm(Lo))
    assert rel < (1e-11 if fp64 else 1e-5), rel


@pytest.mark.parametrize("n", [256, 512])
def test_static_solve_large(pdm, oracle, n):
    """The config-2 static solve (state-based, nu = 1/4, cube minus a centred
    ball, clamp and load layers) at 256^3 and 512^3: FP32 FFT CG with FP64
    refinement to a relative residual of 1e-8, the returned u checked with the
    oracle's FP64 state-based operator on every node (a full direct sum)."""
    cfg = inputs.cube_with_cavity(n=n)
    shape = cfg["shape"]
    prob = pdm.Problem(shape=shape, delta=3.0, model=pdm.PD_LIN_STATE, nu=0.25, fp64=False)
    plan = pdm.Plan(prob, torch.tensor(cfg["chi"], device=DEV), torch.tensor(cfg["chi_omega"], device=DEV))
    b = torch.tensor(cfg["b"], dtype=torch.float64, device=DEV)
    u = torch.zeros((3,) + shape, dtype=torch.float64, device=DEV)
    it, rel, st = plan.solve_static(u, b, None, rtol=1e-8, max_iter=100000)
    assert st == 0 and rel <= 1e-8 and it > 0
    del b
    ug = u.cpu().numpy()
    del u
    plan.close()
    torch.cuda.empty_cache()
    ka, cb, _ = oracle.lps_constants(1.0, 0.25, 1.0, 3.0)
    res = oracle.static_residual(ug, cfg["chi"], cfg["chi_omega"], cfg["b"], 1.0, 3.0, ("lps", ka, cb))
    bn = np.linalg.norm(cfg["chi_omega"] * cfg["b"])
    assert np.linalg.norm(res) / bn <= 1.5e-8
    assert np.all(ug[:, cfg["chi_omega"][0] == 0] == 0)
