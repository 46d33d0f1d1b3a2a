"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds geometry and random fields only: characteristic functions
(chi_B, chi_Omega), displacement fields, load layers and material fields. It
contains none of the method's arithmetic, imports nothing else from this
package, and serves both the GPU path (bench, tests) and the FP64 oracle.

Grid convention (Eq. 52): node (i1, i2, i3) sits at x = (i1 dx1, i2 dx2, i3 dx3);
arrays are C-ordered [i3][i2][i1] (2D: [i2][i1]), x1 fastest; vector fields
carry a leading component axis.

The paper's own geometries (the §5.1 dog-bone, whose dimensions are only in a
missing figure, and the §5.2 glass plate) and its comparison data are not
available; these recipes stand in for them.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def coords(shape, dx=1.0):
    """Node coordinates, one array per axis in x1, x2[, x3] order."""
    dim = len(shape)
    dxv = np.broadcast_to(np.asarray(dx, dtype=np.float64), (dim,))
    axes = [np.arange(shape[dim - 1 - a], dtype=np.float64) * dxv[a] for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # C order: slowest first
    return grids[::-1]  # x1, x2[, x3]


def sine_modes(shape, nmodes, amp, kmax, seed, ncomp=None):
    """Σ_m amp sin(2 pi k_m . i / n + phi_m) per component, k_m in [-kmax, kmax]^d \\ 0.

    Smooth periodic fields in grid units (phase uses node indices, so the field
    is periodic on the box whatever dx is)."""
    g = rng(seed)
    dim = len(shape)
    ncomp = dim if ncomp is None else ncomp
    idx = coords(shape, 1.0)
    out = np.zeros((ncomp,) + tuple(shape), dtype=np.float64)
    n_axes = [shape[dim - 1 - a] for a in range(dim)]
    for c in range(ncomp):
        for _ in range(nmodes):
            while True:
                k = g.integers(-kmax, kmax + 1, size=dim)
                if np.any(k != 0):
                    break
            phi = g.uniform(0.0, 2.0 * math.pi)
            ph = sum(2.0 * math.pi * k[a] * idx[a] / n_axes[a] for a in range(dim))
            out[c] += amp * np.sin(ph + phi)
    return out


def affine_field(shape, dx, scale, seed):
    """u = A x + t with A, t ~ U(-scale, scale)."""
    g = rng(seed)
    dim = len(shape)
    A = g.uniform(-scale, scale, size=(dim, dim))
    t = g.uniform(-scale, scale, size=dim)
    x = coords(shape, dx)
    u = np.zeros((dim,) + tuple(shape), dtype=np.float64)
    for i in range(dim):
        u[i] = t[i] + sum(A[i, j] * x[j] for j in range(dim))
    return u, A, t


def box_mask(shape, lo, hi):
    """uint8 mask = 1 on the index box [lo_a, hi_a) along each axis (x1 first)."""
    dim = len(shape)
    idx = coords(shape, 1.0)
    m = np.ones(shape, dtype=bool)
    for a in range(dim):
        m &= (idx[a] >= lo[a]) & (idx[a] < hi[a])
    return m.astype(np.uint8)


# ---------------------------------------------------------------------------
# Workload recipes (sizes in grid units, dx = 1)
# ---------------------------------------------------------------------------

def plate_2d_single_eval(n=128, margin=16, seed=0):
    """2D single force evaluation: n x n box, square body [margin, n - margin)^2,
    u = 8 seeded sine modes (amplitude 1e-3, |k| <= 4) + seeded affine field
    (entries of A and t ~ U(+-1e-3))."""
    shape = (n, n)
    chi = box_mask(shape, (margin, margin), (n - margin, n - margin))
    u = sine_modes(shape, 8, 1e-3, 4, seed)
    ua, _, _ = affine_field(shape, 1.0, 1e-3, seed + 1000)
    return dict(shape=shape, dx=1.0, delta=3.0, chi=chi, u=u + ua, E=1.0, nu=1.0 / 3.0)


def cube_with_cavity(n=128, delta=3.0, margin=3, radius_frac=0.25, clamp_layers=3,
                     load_layers=3, sigma=1e-3):
    """3D static case: body = [margin, n - margin)^3 minus a centred ball of
    radius radius_frac * n; clamp (chi_Omega = 0, w = 0, all components) on the
    clamp_layers node layers at the body's x1-low face; body-force layer
    b_1 = sigma / delta on the load_layers node layers at the x1-high face
    (traction as a delta-thick body-force layer, §5.2)."""
    shape = (n, n, n)
    chi = box_mask(shape, (margin,) * 3, (n - margin,) * 3)
    x1, x2, x3 = coords(shape, 1.0)
    c = (n - 1) / 2.0
    r = radius_frac * n
    ball = (x1 - c) ** 2 + (x2 - c) ** 2 + (x3 - c) ** 2 < r * r
    chi[ball] = 0
    clamp = (x1 >= margin) & (x1 < margin + clamp_layers) & (chi == 1)
    chi_om = chi.copy()
    chi_om[clamp] = 0
    b = np.zeros((3,) + shape, dtype=np.float64)
    layer = (x1 >= n - margin - load_layers) & (x1 < n - margin) & (chi == 1)
    b[0][layer] = sigma / delta
    return dict(shape=shape, dx=1.0, delta=delta, chi=chi,
                chi_omega=np.stack([chi_om] * 3), b=b, w=np.zeros_like(b))


def notched_plate(n1=1024, n2=512, delta=4.0, sigma=1.0):
    """2D dynamic fracture case: body = [delta, n1 - delta) x [delta, n2 - delta)
    (box = body grown by delta, §5.2); pre-notch = integrity lam = 0 on a
    delta-thick row band at mid-height from the body's left edge over half the
    body width (reading R12); body force b_2 = +-sigma/delta on the delta-thick
    top and bottom node layers (§5.2, reading R13). No kinematic constraint:
    chi_Omega = chi_B, w = 0."""
    shape = (n2, n1)
    m = int(round(delta))
    chi = box_mask(shape, (m, m), (n1 - m, n2 - m))
    x1, x2 = coords(shape, 1.0)
    lam = chi.copy()
    mid = n2 / 2.0
    notch = (x1 >= m) & (x1 < m + (n1 - 2 * m) // 2) & (np.abs(x2 - mid + 0.5) < delta / 2.0)
    lam[notch] = 0
    b = np.zeros((2,) + shape, dtype=np.float64)
    top = (x2 >= n2 - m - m) & (x2 < n2 - m) & (chi == 1)
    bot = (x2 >= m) & (x2 < m + m) & (chi == 1)
    b[1][top] = sigma / delta
    b[1][bot] = -sigma / delta
    return dict(shape=shape, dx=1.0, delta=delta, chi=chi, lam=lam,
                chi_omega=np.stack([chi, chi]), b=b, w=np.zeros_like(b))


def smooth_positive_field(shape, seed, nmodes=16, kmax=3, amp=0.2):
    """1 + amp * g(x), g = seeded sum of nmodes low-k modes normalised to max |g| = 1."""
    g = sine_modes(shape, nmodes, 1.0, kmax, seed, ncomp=1)[0]
    g /= max(1e-300, float(np.max(np.abs(g))))
    return 1.0 + amp * g


def gaussian_impulse(shape, width, seed, amp=1e-3):
    """Vector body force: amp * exp(-|x - x0|^2 / (2 width^2)) along a seeded
    unit direction, x0 seeded in the middle half of the box."""
    g = rng(seed)
    dim = len(shape)
    x = coords(shape, 1.0)
    n_axes = [shape[dim - 1 - a] for a in range(dim)]
    x0 = [g.uniform(0.25, 0.75) * n_axes[a] for a in range(dim)]
    d = g.normal(size=dim)
    d /= np.linalg.norm(d)
    r2 = sum((x[a] - x0[a]) ** 2 for a in range(dim))
    prof = amp * np.exp(-r2 / (2.0 * width * width))
    return np.stack([d[a] * prof for a in range(dim)])


def batched_specimens(count=64, seed=0, nmin=256, nmax=1024, sizes=None):
    """Uneven 2D static specimens: side n ~ U{nmin..nmax} padded up to the next
    power of two, delta ~ U{3,4,5}, body = box minus a delta margin minus a
    seeded ellipse (semi-axes 5-25% of the side, random angle and centre),
    clamp on the body's left delta layer, body-force layer on the right delta
    layer in a seeded direction with |sigma| in [1e-4, 1e-3]."""
    g = rng(seed)
    out = []
    for s in range(count):
        n = int(g.integers(nmin, nmax + 1)) if sizes is None else int(sizes[s])
        npad = 1 << int(math.ceil(math.log2(n)))
        delta = float(g.integers(3, 6))
        m = int(delta)
        shape = (npad, npad)
        lo, hi = m, n - m
        chi = box_mask(shape, (lo, lo), (hi, hi))
        x1, x2 = coords(shape, 1.0)
        cx, cy = g.uniform(0.35, 0.65) * n, g.uniform(0.35, 0.65) * n
        a_ax, b_ax = g.uniform(0.05, 0.25) * n, g.uniform(0.05, 0.25) * n
        th = g.uniform(0, math.pi)
        xr = (x1 - cx) * math.cos(th) + (x2 - cy) * math.sin(th)
        yr = -(x1 - cx) * math.sin(th) + (x2 - cy) * math.cos(th)
        chi[(xr / a_ax) ** 2 + (yr / b_ax) ** 2 < 1.0] = 0
        clamp = (x1 >= lo) & (x1 < lo + m) & (chi == 1)
        chi_om = chi.copy()
        chi_om[clamp] = 0
        sig = g.uniform(1e-4, 1e-3)
        ang = g.uniform(0, 2 * math.pi)
        layer = (x1 >= hi - m) & (x1 < hi) & (chi == 1)
        b = np.zeros((2,) + shape, dtype=np.float64)
        b[0][layer] = sig * math.cos(ang) / delta
        b[1][layer] = sig * math.sin(ang) / delta
        out.append(dict(shape=shape, n_body=n, dx=1.0, delta=delta, chi=chi,
                        chi_omega=np.stack([chi_om, chi_om]), b=b, w=np.zeros_like(b)))
    return out


def cube_with_ball_mask(n, margin=3, radius_frac=0.25):
    """chi of a cube [margin, n - margin)^3 minus a centred ball of radius
    radius_frac * n, built by broadcasting (cheap at 512^3)."""
    x = np.arange(n, dtype=np.float64)
    c = (n - 1) / 2.0
    inside = (x >= margin) & (x < n - margin)
    r2 = ((x[None, None, :] - c) ** 2 + (x[None, :, None] - c) ** 2) + (x[:, None, None] - c) ** 2
    chi = inside[:, None, None] & inside[None, :, None] & inside[None, None, :] & (r2 >= (radius_frac * n) ** 2)
    return chi.astype(np.uint8)


def separable_modes(shape, nterms, kmax, amp, seed, dtype=np.float32, kmin=1):
    """Smooth vector field (3, *shape): per component a sum of nterms products
    of 1D random sine waves (wave numbers kmin <= k <= kmax, random phases)
    along x1, x2, x3, scaled to amplitude amp; separable, so cheap on large grids."""
    g = rng(seed)
    n3, n2, n1 = shape
    out = np.zeros((3,) + tuple(shape), dtype=dtype)
    for c in range(3):
        for _ in range(nterms):
            f = [np.sin(2 * math.pi * g.integers(kmin, kmax + 1) * np.arange(m) / m + g.uniform(0, 2 * math.pi))
                 .astype(dtype) for m in (n1, n2, n3)]
            out[c] += (amp / nterms) * (f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :])
    return out


def plate_with_hole_level(level, n0=32, delta=3.0, hole_frac=0.125, sigma=1e-3, angle=0.3):
    """One resolution level of a 2D static body fixed in physical units, for an
    m-convergence study (§5.1, Eq. 99): box [0, n0)^2 with dx = 2^-level, so
    n = n0 2^level nodes per side and m = delta / dx = delta 2^level.

    Body: delta <= x1, x2 < n0 - delta minus a centred disk of radius
    hole_frac * n0; clamp (chi_Omega = 0, w = 0) on delta <= x1 < 2 delta;
    body-force layer b = sigma / delta (cos angle, sin angle) on
    n0 - 2 delta <= x1 < n0 - delta. Every node of level k is a node of level
    k + 1 (x = i dx), so successive levels compare on the coarser nodes."""
    dx = 2.0 ** -level
    n = int(n0 * 2 ** level)
    shape = (n, n)
    x1, x2 = coords(shape, dx)
    eps = 1e-9 * dx
    L = float(n0)
    c = L / 2.0
    inside = (x1 >= delta - eps) & (x1 < L - delta - eps) & (x2 >= delta - eps) & (x2 < L - delta - eps)
    hole = (x1 - c) ** 2 + (x2 - c) ** 2 < (hole_frac * L) ** 2
    chi = (inside & ~hole).astype(np.uint8)
    clamp = (x1 < 2 * delta - eps) & (chi == 1)
    chi_om = chi.copy()
    chi_om[clamp] = 0
    b = np.zeros((2,) + shape, dtype=np.float64)
    layer = (x1 >= L - 2 * delta - eps) & (chi == 1)
    b[0][layer] = sigma / delta * math.cos(angle)
    b[1][layer] = sigma / delta * math.sin(angle)
    return dict(shape=shape, dx=dx, delta=delta, m=delta / dx, chi=chi,
                chi_omega=np.stack([chi_om, chi_om]), b=b, w=np.zeros_like(b))
