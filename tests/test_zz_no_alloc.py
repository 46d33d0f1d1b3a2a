"""The allocation-free 2D force entry point (pd_force2d_noalloc).

It serves callers that may not call cudaMalloc and therefore cannot build a
plan. Its forces are checked against the FP64 direct-sum oracle, element by
element, with the FP32 force tolerances the other tests use: 1e-5 relative L2
on a deformation field, 4 eps32 kappa on a random field (kappa = ||chi u||
lam_max / ||L||, the conditioning of the FP32 FFT convolution). Calls that
follow one another share the library's fixed scratch array, so repeating a
call after calls on other grids and horizons must give the same bits.
Collected last on purpose; it must pass both alone in a fresh process and
after the whole suite.
"""
import numpy as np
import pytest
import torch

from paper_2105_06055_gb300 import inputs

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-5
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def pdm():
    from paper_2105_06055_gb300 import build, pd
    build.build()
    pd.load()
    return pd


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _kappa(oracle, shape, chi, u, L, dx, delta, alpha):
    lam = 0.0
    for a in range(0, shape[-1] // 2 + 1, 4):
        for b in range(0, shape[-2] // 2 + 1, 4):
            lam = max(lam, float(np.linalg.eigvalsh(oracle.symbol_bond(shape, dx, delta, alpha, (a, b))).max()))
    return float(np.linalg.norm(chi * u) * lam / np.linalg.norm(L))


def test_noalloc_matches_oracle_on_calls_in_a_row(pdm, oracle):
    dev = torch.device("cuda")
    # call 1: the 128^2 single-evaluation geometry, deformation part
    cfg = inputs.plate_2d_single_eval(n=128, margin=16, seed=0)
    u1_np = inputs.sine_modes(cfg["shape"], 8, 1e-3, 4, 0)
    prob1 = pdm.Problem(shape=cfg["shape"], delta=3.0, E=1.0, fp64=False)
    chi1 = torch.tensor(cfg["chi"], device=dev)
    u1 = torch.tensor(u1_np, dtype=torch.float32, device=dev)
    ref1 = oracle.force_bond(u1_np.astype(np.float32), cfg["chi"], 1.0, 3.0, oracle.alpha_bond(2, 1.0, 3.0))
    # call 2: the largest grid the fixed scratch admits, another horizon and body
    shape2 = (256, 256)
    chi2_np = inputs.box_mask(shape2, (6, 6), (250, 250))
    x1, x2 = inputs.coords(shape2)
    chi2_np[(x1 - 128) ** 2 + (x2 - 100) ** 2 < 40 ** 2] = 0
    u2_np = inputs.rng(4).normal(size=(2,) + shape2).astype(np.float32)
    prob2 = pdm.Problem(shape=shape2, delta=4.5, E=2.0, fp64=False)
    chi2 = torch.tensor(chi2_np, device=dev)
    u2 = torch.tensor(u2_np, device=dev)
    alpha2 = oracle.alpha_bond(2, 2.0, 4.5)
    ref2 = oracle.force_bond(u2_np, chi2_np, 1.0, 4.5, alpha2)
    kappa2 = _kappa(oracle, shape2, chi2_np, u2_np, ref2, 1.0, 4.5, alpha2)
    # call 3: a small grid with a short horizon and a non-square spacing
    shape3 = (32, 64)
    chi3_np = inputs.box_mask(shape3, (3, 3), (61, 29))
    u3_np = inputs.rng(9).normal(size=(2,) + shape3).astype(np.float32)
    prob3 = pdm.Problem(shape=shape3, dx=(1.0, 0.8), delta=2.0, E=1.0, fp64=False)
    chi3 = torch.tensor(chi3_np, device=dev)
    u3 = torch.tensor(u3_np, device=dev)

    La = pdm.force2d_noalloc(prob1, chi1, u1)
    Lb = pdm.force2d_noalloc(prob2, chi2, u2)
    torch.cuda.synchronize()
    assert _rel(La.double().cpu().numpy(), ref1) < FP32_TOL
    assert _rel(Lb.double().cpu().numpy(), ref2) < 4 * EPS32 * kappa2
    assert torch.all(La[:, chi1 == 0] == 0) and torch.all(Lb[:, chi2 == 0] == 0)
    # the same calls again, after another grid and horizon filled the scratch:
    # every value the call reads from the array is recomputed, so the bits agree
    pdm.force2d_noalloc(prob3, chi3, u3)
    Lc = pdm.force2d_noalloc(prob1, chi1, u1)
    Ld = pdm.force2d_noalloc(prob2, chi2, u2)
    torch.cuda.synchronize()
    assert torch.equal(Lc, La)
    assert torch.equal(Ld, Lb)


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
