"""Autograd over the C ABI: PDForce and the checkpointed Verlet inverse-problem loss.

Gradients with respect to the micromodulus field c(x) are checked against
central finite differences (FP64 plan) in random smooth directions, and the
loss itself against the FP64 oracle's Verlet run.
"""
import math

import numpy as np
import pytest
import torch

from paper_2105_06055_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.fixture(scope="module")
def mods():
    from paper_2105_06055_gb300 import autograd, build, pd
    build.build()
    pd.load()
    return pd, autograd


def _setup(pdm, shape, fp64, seed=0):
    dim = len(shape)
    delta = 3.0
    chi = inputs.box_mask(shape, (4,) * dim, tuple(s - 4 for s in shape[::-1]))
    dt = torch.float64 if fp64 else torch.float32
    plan = pdm.Plan(pdm.Problem(shape=shape, delta=delta, fp64=fp64, rho=1.0), torch.tensor(chi, device=DEV))
    c = torch.tensor(inputs.smooth_positive_field(shape, seed + 1), dtype=dt, device=DEV)
    ct = torch.tensor(inputs.smooth_positive_field(shape, seed + 2), dtype=dt, device=DEV)
    imp = torch.tensor(inputs.gaussian_impulse(shape, 2 * delta, seed + 3) * chi, dtype=dt, device=DEV)
    return plan, chi, c, ct, imp


def test_pdforce_gradcheck(mods):
    pdm, ag = mods
    shape = (16, 32)
    plan, chi, _, _, _ = _setup(pdm, shape, True)
    g = inputs.rng(1)
    u = torch.tensor(g.normal(size=(2,) + shape), device=DEV, requires_grad=True)
    s = torch.tensor(0.8 + 0.4 * g.random(shape), device=DEV, requires_grad=True)
    assert torch.autograd.gradcheck(lambda uu, ss: ag.pd_force(plan, uu, ss), (u, s), eps=1e-6, atol=1e-8,
                                    rtol=1e-6, fast_mode=True)
    plan.close()


def test_verlet_loss_directional_fd(mods):
    pdm, ag = mods
    shape = (32, 32, 32)
    plan, chi, c, ct, imp = _setup(pdm, shape, True)
    dt = 0.3 * plan.stable_dt
    nsteps = 20
    with torch.no_grad():
        # target: the final state of a second micromodulus field
        u_target = _final_state(ag, plan, ct, imp, dt, nsteps)
    cc = c.clone().requires_grad_(True)
    loss = ag.verlet_loss(plan, cc, u_target, imp, dt, nsteps, checkpoint_every=5)
    loss.backward()
    grad = cc.grad.detach()
    g = inputs.rng(7)
    eps = 1e-5
    for k in range(16):
        h = torch.tensor(inputs.sine_modes(shape, 4, 1.0, 3, 100 + k, ncomp=1)[0], device=DEV)
        with torch.no_grad():
            lp = ag.verlet_loss(plan, c + eps * h, u_target, imp, dt, nsteps)
            lm = ag.verlet_loss(plan, c - eps * h, u_target, imp, dt, nsteps)
        fd = float((lp - lm) / (2 * eps))
        an = float((grad * h).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-30) + 1e-12 * abs(float(loss.detach())), (k, fd, an)
    plan.close()


def _final_state(ag, plan, c, imp, dt, nsteps):
    """u(T) from rest under the weighted force (the library's dynamics, no gradient)."""
    _, _, uf, _ = plan.verlet_loss_grad(c, torch.zeros_like(imp), dt, nsteps, b0=imp, want_grad=False,
                                        want_final=True)
    return uf


def test_verlet_loss_matches_oracle(mods, oracle):
    """The loss and one directional derivative against the FP64 oracle's own
    Verlet run (independent force sums)."""
    pdm, ag = mods
    shape = (16, 32, 32)
    plan, chi, c, ct, imp = _setup(pdm, shape, True, seed=4)
    delta = 3.0
    alpha = oracle.alpha_bond(3, 1.0, delta)
    dt = 0.3 * plan.stable_dt
    nsteps = 12

    def oracle_final(cn):
        z = np.zeros((3,) + shape)
        u, _, _, _ = oracle.verlet_damage(z, z, chi, chi, np.stack([chi] * 3), z, z, 1.0, delta, alpha, 1.0, dt,
                                          1e300, nsteps, s=np.sqrt(cn), b0=imp.cpu().numpy())
        return u

    cn, ctn = c.cpu().numpy(), ct.cpu().numpy()
    ut = oracle_final(ctn)
    u_target = torch.tensor(ut, device=DEV)

    def oracle_loss(cc):
        return float(np.sum((oracle_final(cc) - ut) ** 2))

    cc = c.clone().requires_grad_(True)
    loss = ag.verlet_loss(plan, cc, u_target, imp, dt, nsteps, checkpoint_every=4)
    loss.backward()
    assert abs(float(loss) / oracle_loss(cn) - 1) < 1e-10
    h = inputs.sine_modes(shape, 3, 1.0, 2, 9, ncomp=1)[0]
    eps = 1e-5
    fd = (oracle_loss(cn + eps * h) - oracle_loss(cn - eps * h)) / (2 * eps)
    an = float((cc.grad.cpu().numpy() * h).sum())
    assert abs(fd - an) <= 1e-6 * abs(an)
    plan.close()


def test_verlet_loss_fp32_matches_fp64(mods):
    """The FP32 path's gradient agrees with the FP64 path's on the same problem."""
    pdm, ag = mods
    shape = (64, 64, 64)
    grads = []
    for fp64 in (True, False):
        plan, chi, c, ct, imp = _setup(pdm, shape, fp64, seed=11)
        dt = 0.3 * plan.stable_dt
        with torch.no_grad():
            u_target = _final_state(ag, plan, ct, imp, dt, 30)
        cc = c.clone().requires_grad_(True)
        ag.verlet_loss(plan, cc, u_target, imp, dt, 30, checkpoint_every=10).backward()
        grads.append(cc.grad.double())
        plan.close()
    rel = float(torch.linalg.norm(grads[1] - grads[0]) / torch.linalg.norm(grads[0]))
    assert rel < 1e-3
