"""m-convergence driver (Eq. 99, §5.1): host logic, and the study itself run
with the FP64 oracle's CG on a small multi-resolution body (CPU only)."""
import math

import numpy as np
import pytest

from paper_2105_06055_gb300 import convergence, inputs


def test_restriction_takes_the_coarse_nodes():
    """A field sampled at level k + 1 and restricted equals the same field
    sampled at level k (node i of level k sits at fine node 2 i)."""
    def sample(k, n0=32):
        dx = 2.0 ** -k
        x1, x2 = inputs.coords((n0 * 2 ** k,) * 2, dx)
        return np.stack([np.sin(x1 / 5.0) * np.cos(x2 / 7.0), x1 * x2])
    assert np.array_equal(convergence.restrict(sample(1), 2), sample(0))
    assert np.array_equal(convergence.restrict(sample(2), 2), sample(1))
    a, b = inputs.plate_with_hole_level(1), inputs.plate_with_hole_level(0)
    assert np.array_equal(convergence.restrict(a["chi"], 2), b["chi"])
    assert np.array_equal(convergence.restrict(a["chi_omega"], 2), b["chi_omega"])
    assert np.array_equal(convergence.restrict(a["b"], 2), b["b"])
    assert a["m"] == 2 * b["m"]


def test_eq99_and_orders():
    g = inputs.rng(1)
    fine = g.normal(size=(2, 16, 16))
    coarse = convergence.restrict(fine, 2).copy()
    assert convergence.eq99(fine, coarse, 2) == 0.0
    assert abs(convergence.eq99(fine, 0.9 * coarse, 2) - 0.1) < 1e-15
    with pytest.raises(ValueError):
        convergence.eq99(fine, coarse[:, :4], 2)
    assert convergence.orders([0.4, 0.1, 0.025]) == [2.0, 2.0]
    with pytest.raises(ValueError):
        convergence.study(lambda k: fine, [0, 2], 2)


@pytest.mark.parametrize("pv", [False, True])
def test_oracle_solutions_converge_in_m(oracle, pv):
    """Fixed horizon delta = 2, dx = 1, 1/2, 1/4, 1/8 (m = 2 ... 16): the Eq. 99
    changes shrink from level to level, faster than linearly, as §5.1 reports for
    its 3D example; also with partial volumes."""
    delta = 2.0
    alpha = oracle.alpha_bond(2, 1.0, delta)

    def solve(k):
        cfg = inputs.plate_with_hole_level(k, n0=16, delta=delta)
        with oracle.partial_volumes(pv):
            u, _, rel = oracle.cg_static(cfg["chi"], cfg["chi_omega"], cfg["b"], cfg["w"], cfg["dx"], delta,
                                         ("bond", alpha), rtol=1e-12)
        assert rel < 1e-11
        return u

    r = convergence.study(solve, [0, 1, 2, 3], 2)
    e = r["errors"]
    assert e[0] > e[1] > e[2]
    assert all(o > 1.0 for o in r["orders"]), r
    assert e[2] < 0.02
