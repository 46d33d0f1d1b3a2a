"""GPU parity of the nonlinear rotation-invariant bond model (§3.2, Eq. 19-26)
through pd_force (PD_NONLIN_BOND) against the oracle's direct sum of Eq. 21,
element by element.

Tolerances: FP64 1e-11 relative L2 (the passes are an exact reorganisation of
the same quadrature); FP32 1e-5 on deformation-dominated fields, against the
oracle on the same FP32 input. The FP32 error of this model grows with the
size of the deformation (the products u_i u_j and |u|^2 u_i are transformed),
so large rotations belong to the FP64 path; a rigid translation costs nothing
because the body mean is removed before the transforms.
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _body(shape, seed, margin):
    g = inputs.rng(seed)
    dim = len(shape)
    chi = inputs.box_mask(shape, (margin,) * dim, tuple(s - margin for s in shape[::-1]))
    x = inputs.coords(shape)
    c = [0.5 * s for s in shape[::-1]]
    r = min(shape) / 6.0
    chi[sum((x[a] - c[a]) ** 2 for a in range(dim)) < r * r] = 0  # a cavity
    chi[g.random(shape) < 0.03] = 0
    return chi


def _force(pdm, shape, chi, u, delta, fp64, dx=1.0):
    plan = pdm.Plan(pdm.Problem(shape=shape, dx=dx, delta=delta, model=pdm.PD_NONLIN_BOND, fp64=fp64),
                    torch.tensor(chi, device=DEV))
    L = plan.force(torch.tensor(u, dtype=torch.float64 if fp64 else torch.float32, device=DEV))
    torch.cuda.synchronize()
    plan.close()
    return L.double().cpu().numpy()


@pytest.mark.parametrize("shape,delta,dx", [((32, 64), 3.0, 1.0), ((64, 32), 2.5, (1.0, 1.25)),
                                            ((16, 32, 32), 2.5, 1.0), ((32, 32, 64), 3.0, 1.0)])
def test_nonlinear_force_fp64_matches_oracle(pdm, oracle, shape, delta, dx):
    dim = len(shape)
    chi = _body(shape, 3 + dim, margin=5)
    u = 0.3 * inputs.rng(5).normal(size=(dim,) + shape) + inputs.sine_modes(shape, 3, 0.5, 2, 6)
    alpha = oracle.alpha_bond(dim, 1.0, delta)
    ref = oracle.force_nonlinear(u, chi, dx, delta, alpha)
    L = _force(pdm, shape, chi, u, delta, True, dx=dx)
    assert _rel(L, ref) < 1e-11
    assert np.all(L[:, chi == 0] == 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_nonlinear_force_fp32_matches_oracle(pdm, oracle, dim):
    """Smooth deformation (strain ~ 1e-2) plus a large rigid translation."""
    shape = (64, 128) if dim == 2 else (32, 32, 64)
    chi = _body(shape, 11, margin=5)
    u = inputs.sine_modes(shape, 6, 0.2, 3, 12) + 7.5
    u = u.astype(np.float32)
    alpha = oracle.alpha_bond(dim, 1.0, 3.0)
    ref = oracle.force_nonlinear(u, chi, 1.0, 3.0, alpha)
    L = _force(pdm, shape, chi, u, 3.0, False)
    assert _rel(L, ref) < 1e-5


@pytest.mark.parametrize("dim", [2, 3])
def test_nonlinear_finite_rotation_gives_zero_force(pdm, oracle, dim):
    """A rigid motion with a 30 degree rotation: every bond keeps its length, so
    the force vanishes (to rounding, relative to the force of a deformation of
    the same displacement size); the linearized model's does not."""
    shape = (64, 64) if dim == 2 else (32, 32, 32)
    chi = _body(shape, 17, margin=4)
    x = np.stack(inputs.coords(shape))
    th = math.radians(30.0)
    R = np.eye(dim)
    R[0, 0] = R[1, 1] = math.cos(th)
    R[0, 1], R[1, 0] = -math.sin(th), math.sin(th)
    c = np.array([0.5 * s for s in shape[::-1]]).reshape((dim,) + (1,) * dim)
    u = np.einsum("ij,j...->i...", R - np.eye(dim), x - c) + 2.0
    alpha = oracle.alpha_bond(dim, 1.0, 3.0)
    L = _force(pdm, shape, chi, u, 3.0, True)
    scale = np.linalg.norm(oracle.force_nonlinear(0.05 * inputs.sine_modes(shape, 3, 1.0, 2, 8) * np.abs(u).max(),
                                                  chi, 1.0, 3.0, alpha))
    assert np.linalg.norm(L) < 1e-11 * scale
    lin = oracle.force_bond(u, chi, 1.0, 3.0, alpha)
    assert np.linalg.norm(lin) > 1e-2 * scale


def test_nonlinear_model_is_force_only(pdm):
    shape = (32, 32)
    chi = inputs.box_mask(shape, (4, 4), (28, 28))
    plan = pdm.Plan(pdm.Problem(shape=shape, delta=3.0, model=pdm.PD_NONLIN_BOND, fp64=True),
                    torch.tensor(chi, device=DEV))
    u = torch.zeros((2,) + shape, dtype=torch.float64, device=DEV)
    with pytest.raises(pdm.PDError, match="PD_ERR_ARG"):
        plan.solve_static(u, torch.zeros_like(u), None)
    with pytest.raises(pdm.PDError, match="PD_ERR_ARG"):
        plan.step_verlet(u, torch.zeros_like(u), None, torch.zeros_like(u), None, dt=0.1, nsteps=1)
    with pytest.raises(pdm.PDError, match="PD_ERR_ARG"):
        plan.force(u, want_energy=True)
    plan.close()
