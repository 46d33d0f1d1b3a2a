"""The allocation-free 2D force entry point (pd_force2d_noalloc).

It serves callers that may not call cudaMalloc and therefore cannot build a
plan; it must give the same forces as pd_plan_create + pd_force. Collected
last on purpose: it checks two calls in a row through the C ABI against the
plan path, within the FP32 force tolerance used by the other tests, and must
pass both alone in a fresh process and after the whole suite.
"""
import numpy as np
import pytest
import torch

from paper_2105_06055_gb300 import inputs

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def pdm():
    from paper_2105_06055_gb300 import build, pd
    build.build()
    pd.load()
    return pd


def _rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


def _plan_force(pdm, prob, chi, u):
    plan = pdm.Plan(prob, chi)
    L = plan.force(u)
    torch.cuda.synchronize()
    plan.close()
    return L


def test_noalloc_matches_plan_path_twice(pdm):
    dev = torch.device("cuda")
    # call 1: the 128^2 single-evaluation geometry, deformation part
    cfg = inputs.plate_2d_single_eval(n=128, margin=16, seed=0)
    prob1 = pdm.Problem(shape=cfg["shape"], delta=3.0, E=1.0, fp64=False)
    chi1 = torch.tensor(cfg["chi"], device=dev)
    u1 = torch.tensor(inputs.sine_modes(cfg["shape"], 8, 1e-3, 4, 0), dtype=torch.float32, device=dev)
    # call 2: the largest grid the fixed scratch admits, another horizon and body
    shape2 = (256, 256)
    chi2_np = inputs.box_mask(shape2, (6, 6), (250, 250))
    x1, x2 = inputs.coords(shape2)
    chi2_np[(x1 - 128) ** 2 + (x2 - 100) ** 2 < 40 ** 2] = 0
    prob2 = pdm.Problem(shape=shape2, delta=4.5, E=2.0, fp64=False)
    chi2 = torch.tensor(chi2_np, device=dev)
    u2 = torch.tensor(inputs.rng(4).normal(size=(2,) + shape2), dtype=torch.float32, device=dev)

    La = pdm.force2d_noalloc(prob1, chi1, u1)
    Lb = pdm.force2d_noalloc(prob2, chi2, u2)
    torch.cuda.synchronize()
    assert _rel(La, _plan_force(pdm, prob1, chi1, u1)) < FP32_TOL
    assert _rel(Lb, _plan_force(pdm, prob2, chi2, u2)) < FP32_TOL
    # the same call again on the first input after the larger one
    Lc = pdm.force2d_noalloc(prob1, chi1, u1)
    torch.cuda.synchronize()
    assert _rel(Lc, La) < FP32_TOL


def test_noalloc_rejects_oversize_and_bad_masks(pdm):
    dev = torch.device("cuda")
    shape = (256, 512)  # 131072 nodes > 65536
    prob = pdm.Problem(shape=shape, delta=3.0, fp64=False)
    chi = torch.tensor(inputs.box_mask(shape, (4, 4), (508, 252)), device=dev)
    u = torch.zeros((2,) + shape, dtype=torch.float32, device=dev)
    with pytest.raises(pdm.PDError, match="PD_ERR_SIZE"):
        pdm.force2d_noalloc(prob, chi, u)
    shape = (64, 64)
    prob = pdm.Problem(shape=shape, delta=3.0, fp64=False)
    chi = torch.ones(shape, dtype=torch.uint8, device=dev)  # touches the box faces
    u = torch.zeros((2,) + shape, dtype=torch.float32, device=dev)
    with pytest.raises(pdm.PDError, match="PD_ERR_ARG"):
        pdm.force2d_noalloc(prob, chi, u)
