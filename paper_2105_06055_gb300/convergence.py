"""m-convergence of a static solution (§5.1, Eq. 99).

The same body, fixed in physical units, is solved on grids of spacing dx,
dx/2, dx/4, ... with the horizon delta fixed, so m = delta/dx doubles from one
level to the next. Eq. 99 measures the change between two successive levels on
the coarser grid's nodes:

    e_k = |U_{k+1} - U_k|_2 / |U_{k+1}|_2,   U_{k+1} restricted to level k's nodes,

with U all displacement components at all nodes. The observed order between
two pairs of levels is log2(e_k / e_{k+1}) (the paper finds a superlinear rate
for its 3D example, Fig. 10).

Host logic only: each level is solved by ``Plan.solve_static`` (the library's
CG with FP64 refinement); this module restricts, compares and reports.
"""
from __future__ import annotations

import math
from typing import Callable, Dict, List, Sequence

import numpy as np


def restrict(u_fine: np.ndarray, dim: int) -> np.ndarray:
    """Values of a field of level k + 1 at the nodes of level k: node i of the
    coarse grid sits at x = i dx = (2 i)(dx / 2), every second fine node along
    each axis (component axis first, then the dim spatial axes)."""
    lead = u_fine.ndim - dim
    return u_fine[(slice(None),) * lead + (slice(None, None, 2),) * dim]


def eq99(u_new: np.ndarray, u_old: np.ndarray, dim: int) -> float:
    """Relative change of Eq. 99 between a solution and the one on the grid of
    twice the spacing, on the coarser grid's nodes."""
    r = restrict(u_new, dim)
    if r.shape != u_old.shape:
        raise ValueError(f"level shapes do not nest: {u_new.shape} restricted to {r.shape}, coarse {u_old.shape}")
    den = float(np.linalg.norm(r))
    if den == 0.0:
        raise ValueError("the finer solution is zero on the coarse nodes")
    return float(np.linalg.norm(r - u_old)) / den


def orders(errors: Sequence[float]) -> List[float]:
    """Observed orders log2(e_k / e_{k+1}) of successive Eq. 99 changes."""
    return [math.log2(a / b) for a, b in zip(errors[:-1], errors[1:])]


def study(solve_level: Callable[[int], np.ndarray], levels: Sequence[int], dim: int) -> Dict[str, list]:
    """Solve each level (``solve_level(k)`` returns the displacement field of
    level k, component axis first) and report the Eq. 99 changes between
    successive levels and the observed orders."""
    levels = list(levels)
    if any(b != a + 1 for a, b in zip(levels[:-1], levels[1:])):
        raise ValueError("levels must be consecutive (each halves dx)")
    sols = [np.asarray(solve_level(k), dtype=np.float64) for k in levels]
    errs = [eq99(sols[i + 1], sols[i], dim) for i in range(len(sols) - 1)]
    return {"levels": levels, "errors": errs, "orders": orders(errs) if len(errs) > 1 else []}


def gpu_level_solver(make_level: Callable[[int], dict], E: float = 1.0, rtol: float = 1e-10, fp64: bool = True,
                     max_iter: int = 50000, volume_rule: int = 0):
    """solve_level(k) for ``study``: builds level k from ``make_level(k)`` (a dict
    with shape, dx, delta, chi, chi_omega, b, w; e.g.
    ``inputs.plate_with_hole_level``) and solves it on the GPU with the bond
    model to ``rtol``."""
    import torch

    from . import pd

    def solve(k):
        cfg = make_level(k)
        dev = torch.device("cuda")
        prob = pd.Problem(shape=cfg["shape"], dx=cfg["dx"], delta=cfg["delta"], E=E, fp64=fp64,
                          volume_rule=volume_rule)
        plan = pd.Plan(prob, torch.tensor(cfg["chi"], device=dev), torch.tensor(cfg["chi_omega"], device=dev))
        try:
            u = torch.zeros(cfg["b"].shape, dtype=torch.float64, device=dev)
            w = torch.tensor(cfg["w"], dtype=torch.float64, device=dev)
            plan.solve_static(u, torch.tensor(cfg["b"], dtype=torch.float64, device=dev), w, rtol=rtol,
                              max_iter=max_iter)
            return u.cpu().numpy()
        finally:
            plan.close()

    return solve
