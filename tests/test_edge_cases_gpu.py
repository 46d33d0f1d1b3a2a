"""Edge cases of the FFT path against the oracle: an empty body, a body of one
node or of isolated nodes (no bonds inside the body), the largest supported
2D grid, non-cubic boxes with non-square spacings and a horizon that is not a
multiple of the spacing, a body that touches the required margin exactly, and
the argument errors for horizons that do not fit the grid."""
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


def _force(pdm, shape, chi, u, delta, fp64, dx=1.0, model=0, nu=0.25):
    plan = pdm.Plan(pdm.Problem(shape=shape, dx=dx, delta=delta, model=model, nu=nu, fp64=fp64),
                    torch.tensor(chi, device=DEV))
    L = plan.force(torch.tensor(u, dtype=torch.float64 if fp64 else torch.float32, device=DEV))
    torch.cuda.synchronize()
    plan.close()
    return L.double().cpu().numpy()


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("dim", [2, 3])
def test_empty_and_bondless_bodies_give_zero_force(pdm, fp64, dim):
    shape = (32, 64) if dim == 2 else (16, 16, 32)
    u = inputs.rng(3).normal(size=(dim,) + shape)
    chi = np.zeros(shape, dtype=np.uint8)
    assert np.all(_force(pdm, shape, chi, u, 3.0, fp64) == 0)
    # isolated nodes 8 apart (delta = 3) and 4 from the faces (margin 3): no bond
    # has both ends in the body
    chi[tuple(slice(4, n - 3, 8) for n in shape)] = 1
    assert chi.sum() > 1
    L = _force(pdm, shape, chi, u, 3.0, fp64)
    assert np.max(np.abs(L)) <= (1e-14 if fp64 else 1e-6) * np.max(np.abs(u))


@pytest.mark.parametrize("fp64", [True, False])
def test_largest_2d_grid_sampled(pdm, oracle, fp64):
    """2048 x 1024 nodes (the largest 2D box), delta = 5, FP32 and FP64 against the
    direct sum at sampled nodes (half of them within delta of the boundary)."""
    shape = (1024, 2048)
    chi = inputs.box_mask(shape, (6, 6), (2042, 1018))
    x1, x2 = inputs.coords(shape)
    chi[(x1 - 700) ** 2 + (x2 - 500) ** 2 < 150 ** 2] = 0
    u = inputs.sine_modes(shape, 6, 1e-3, 24, 17)
    if not fp64:
        u = u.astype(np.float32)
    L = _force(pdm, shape, chi, u, 5.0, fp64)
    g = inputs.rng(19)
    body = np.flatnonzero(chi.reshape(-1))
    edge = np.flatnonzero((chi.reshape(-1) == 1) & (np.abs(np.sqrt((x1 - 700.0) ** 2 + (x2 - 500.0) ** 2) - 152).reshape(-1) < 4))
    nodes = np.concatenate([g.choice(body, 3000, replace=False), g.choice(edge, 1000, replace=False)])
    alpha = oracle.alpha_bond(2, 1.0, 5.0)
    Lo = oracle.force_bond_at(u.astype(np.float64), chi, 1.0, 5.0, alpha, nodes)
    Lg = L.reshape(2, -1)[:, nodes]
    rel = float(np.linalg.norm(Lg - Lo) / np.linalg.norm(Lo))
    assert rel < (1e-11 if fp64 else 1e-5), rel


@pytest.mark.parametrize("fp64", [True, False])
def test_noncubic_box_anisotropic_spacing_tight_margin(pdm, oracle, fp64):
    """n = (64, 32, 16) with spacings (1, 1.25, 0.8), delta = 2.6 (not a multiple
    of any spacing): the horizon reaches (2, 2, 3) cells, and the body fills the
    box up to exactly that margin on every face."""
    shape = (16, 32, 64)
    dx = (1.0, 1.25, 0.8)
    r = (2, 2, 3)
    chi = inputs.box_mask(shape, r, (64 - r[0], 32 - r[1], 16 - r[2]))
    u = inputs.rng(23).normal(size=(3,) + shape)
    alpha = oracle.alpha_bond(3, 1.0, 2.6)
    ref = oracle.force_bond(u, chi, dx, 2.6, alpha)
    L = _force(pdm, shape, chi, u, 2.6, fp64, dx=dx)
    assert float(np.linalg.norm(L - ref) / np.linalg.norm(ref)) < (1e-11 if fp64 else 1e-5)


def test_horizon_that_does_not_fit_is_refused(pdm):
    shape = (16, 64)
    chi = np.zeros(shape, dtype=np.uint8)
    with pytest.raises(pdm.PDError, match="PD_ERR_SIZE"):
        pdm.Plan(pdm.Problem(shape=shape, delta=8.0, fp64=True), torch.tensor(chi, device=DEV))
    with pytest.raises(pdm.PDError, match="PD_ERR_SIZE"):
        pdm.Plan(pdm.Problem(shape=shape, delta=0.5, fp64=True), torch.tensor(chi, device=DEV))
    chi = inputs.box_mask(shape, (2, 2), (62, 14))  # one cell closer to the faces than delta = 3
    with pytest.raises(pdm.PDError, match="PD_ERR_ARG"):
        pdm.Plan(pdm.Problem(shape=shape, delta=3.0, fp64=True), torch.tensor(chi, device=DEV))
