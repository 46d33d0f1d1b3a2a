"""The inverse-problem workload at full size: 256^3 box, delta = 3, bond model
(alpha = 12E/(pi delta^4)), micromodulus c(x) = 1 + 0.2 g(x), loss
||u(T) - u_target||^2 after 50 velocity-Verlet steps from a Gaussian impulse,
gradient dLoss/dc through pd_force_adjoint with checkpoints every 10 steps.

The FP64 GPU gradient is checked against central finite differences of the
FP64 loss in 16 seeded smooth directions; the FP32 gradient against the FP64
one."""
import math

import numpy as np
import pytest
import torch

from paper_2105_06055_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
SHAPE = (256, 256, 256)
DELTA = 3.0
NSTEPS = 50


@pytest.fixture(scope="module")
def mods():
    from paper_2105_06055_gb300 import autograd, build, pd
    build.build()
    pd.load()
    return pd, autograd


@pytest.fixture(scope="module")
def fields():
    chi = inputs.box_mask(SHAPE, (3, 3, 3), (253, 253, 253))
    c = inputs.smooth_positive_field(SHAPE, 1)
    ct = inputs.smooth_positive_field(SHAPE, 2)
    imp = inputs.gaussian_impulse(SHAPE, 2 * DELTA, 3) * chi
    return chi, c, ct, imp


def _run(pdm, ag, fields, fp64, directions):
    chi, c, ct, imp = fields
    dt = torch.float64 if fp64 else torch.float32
    plan = pdm.Plan(pdm.Problem(shape=SHAPE, delta=DELTA, fp64=fp64, rho=1.0),
                    torch.tensor(chi, device=DEV))
    step = 0.5 * plan.stable_dt
    cd = torch.tensor(c, dtype=dt, device=DEV)
    impd = torch.tensor(imp, dtype=dt, device=DEV)
    u_target = _final_state(ag, plan, torch.tensor(ct, dtype=dt, device=DEV), impd, step)
    cc = cd.clone().requires_grad_(True)
    loss = ag.verlet_loss(plan, cc, u_target, impd, step, NSTEPS, checkpoint_every=10)
    loss.backward()
    grad = cc.grad.detach()
    out = []
    eps = 1e-5
    for k in range(directions):
        h = torch.tensor(inputs.sine_modes(SHAPE, 4, 1.0, 3, 100 + k, ncomp=1)[0], dtype=dt, device=DEV)
        with torch.no_grad():
            lp = ag.verlet_loss(plan, cd + eps * h, u_target, impd, step, NSTEPS)
            lm = ag.verlet_loss(plan, cd - eps * h, u_target, impd, step, NSTEPS)
        out.append((float((lp - lm) / (2 * eps)), float((grad * h).sum())))
    plan.close()
    return float(loss.detach()), grad.double(), out


def _final_state(ag, plan, c, imp, dt):
    _, _, uf, _ = plan.verlet_loss_grad(c, torch.zeros_like(imp), dt, NSTEPS, b0=imp, want_grad=False,
                                        want_final=True)
    return uf


def test_adjoint_config5_full_size(mods, fields):
    pdm, ag = mods
    loss64, g64, fd = _run(pdm, ag, fields, True, 16)
    assert loss64 > 0 and math.isfinite(loss64)
    for k, (f, a) in enumerate(fd):
        assert abs(f - a) <= 1e-6 * abs(a) + 1e-12 * loss64, (k, f, a)
    loss32, g32, _ = _run(pdm, ag, fields, False, 0)
    assert abs(loss32 / loss64 - 1) < 1e-3
    assert float(torch.linalg.norm(g32 - g64) / torch.linalg.norm(g64)) < 1e-3
