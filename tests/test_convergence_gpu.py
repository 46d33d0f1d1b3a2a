"""m-convergence study (Eq. 99, §5.1) with the GPU static solver: three levels
of the same 2D body (dx = 1, 1/2, 1/4 with delta = 3 fixed, so m = 3, 6, 12),
each solution against the oracle's FP64 CG, and the Eq. 99 changes against the
oracle's."""
import numpy as np
import pytest

from paper_2105_06055_gb300 import convergence, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdm():
    from paper_2105_06055_gb300 import build, pd
    build.build()
    pd.load()
    return pd


def test_m_convergence_matches_oracle(pdm, oracle):
    delta = 3.0
    alpha = oracle.alpha_bond(2, 1.0, delta)

    def make(k):
        return inputs.plate_with_hole_level(k, n0=32, delta=delta)

    gpu_solve = convergence.gpu_level_solver(make, rtol=1e-11)
    ref = {}

    def oracle_solve(k):
        cfg = make(k)
        u, _, _ = oracle.cg_static(cfg["chi"], cfg["chi_omega"], cfg["b"], cfg["w"], cfg["dx"], delta,
                                   ("bond", alpha), rtol=1e-13)
        ref[k] = u
        return u

    def checked_gpu_solve(k):
        u = gpu_solve(k)
        uo = ref[k] if k in ref else oracle_solve(k)
        assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo)
        return u

    r_oracle = convergence.study(oracle_solve, [0, 1, 2], 2)
    r_gpu = convergence.study(checked_gpu_solve, [0, 1, 2], 2)
    for eg, eo in zip(r_gpu["errors"], r_oracle["errors"]):
        assert abs(eg - eo) <= 1e-6 * eo
    assert r_gpu["errors"][1] < r_gpu["errors"][0]
