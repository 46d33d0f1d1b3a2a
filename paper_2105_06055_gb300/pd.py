"""Python binding of the C ABI in ``include/pd.h`` (argument marshalling only).

Every computation runs in ``libpdfft.so``; this module only checks tensor
shapes, dtypes and devices, passes raw device pointers and the current CUDA
stream, and turns status codes into exceptions. There is no fallback: if the
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpdfft.so")
_lib = None

PD_LIN_BOND = 0
PD_LIN_STATE = 1
PD_NONLIN_BOND = 2

STATUS = {0: "PD_OK", -1: "PD_ERR_ARG", -2: "PD_ERR_SIZE", -3: "PD_ERR_NOMEM", -4: "PD_ERR_CUDA",
          -5: "PD_ERR_NOT_CONVERGED", -6: "PD_ERR_TIMEOUT", -7: "PD_ERR_NONFINITE"}

EXPORTS = ["pd_plan_create", "pd_plan_destroy", "pd_kernel_spectrum", "pd_force", "pd_step_verlet",
           "pd_solve_static", "pd_force_adjoint", "pd_damage", "pd_plan_workspace_bytes",
           "pd_stable_dt", "pd_plan_launch_count", "pd_status_string", "pd_last_error_detail",
           "pd_plan_profile", "pd_plan_profile_read", "pd_force2d_noalloc", "pd_plan_boundary_nodes",
           "pd_solve_dr", "pd_plan_create_batched", "pd_batch_size", "pd_batch_plan", "pd_solve_dr_batched",
           "pd_batch_destroy", "pd_plan_autotune", "pd_batch_autotune", "pd_plan_tuning",
           "pd_plan_set_energy_mode", "pd_plan_set_tuning", "pd_plan_autotune_solve", "pd_plan_critical_energy",
           "pd_plan_inject_stall", "pd_plan_set_affine_split", "pd_plan_set_plane_passes", "pd_step_verlet_ramp",
           "pd_verlet_adjoint_workspace", "pd_verlet_loss_grad", "pd_solve_mirror"]

PASS_KINDS = {0: "rows_fwd", 1: "cols_x2", 2: "last_axis", 3: "rows_inv", 4: "plane_fwd", 5: "plane_inv"}


class PDError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        lib = load()
        detail = lib.pd_last_error_detail().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")


class _Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("delta", ctypes.c_double), ("model", ctypes.c_int), ("E", ctypes.c_double),
                ("nu", ctypes.c_double), ("rho", ctypes.c_double), ("Wc", ctypes.c_double),
                ("fp64", ctypes.c_int), ("volume_rule", ctypes.c_int), ("s0", ctypes.c_double)]


def load():
    """Load ``libpdfft.so`` (built by ``paper_2105_06055_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_2105_06055_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    lib.pd_plan_create.argtypes = [ctypes.POINTER(_Problem), P, P, P, ctypes.POINTER(P)]
    lib.pd_plan_create.restype = I
    lib.pd_plan_destroy.argtypes = [P]
    lib.pd_plan_destroy.restype = None
    lib.pd_kernel_spectrum.argtypes = [P, P, P]
    lib.pd_kernel_spectrum.restype = I
    lib.pd_force.argtypes = [P, P, P, P, P, P]
    lib.pd_force.restype = I
    lib.pd_step_verlet.argtypes = [P, P, P, P, P, P, D, I, ctypes.POINTER(I64), P]
    lib.pd_step_verlet.restype = I
    lib.pd_step_verlet_ramp.argtypes = [P, P, P, P, P, P, P, D, D, I, ctypes.POINTER(I64), P]
    lib.pd_step_verlet_ramp.restype = I
    lib.pd_solve_mirror.argtypes = [P, P, P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]
    lib.pd_solve_mirror.restype = I
    lib.pd_verlet_adjoint_workspace.argtypes = [P, I, I]
    lib.pd_verlet_adjoint_workspace.restype = I64
    lib.pd_verlet_loss_grad.argtypes = [P, P, P, P, P, P, P, P, D, I, I, P, I64, ctypes.POINTER(D), P, P, P, P]
    lib.pd_verlet_loss_grad.restype = I
    lib.pd_solve_static.argtypes = [P, P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]
    lib.pd_solve_static.restype = I
    lib.pd_force_adjoint.argtypes = [P, P, P, P, P, P, P]
    lib.pd_force_adjoint.restype = I
    lib.pd_damage.argtypes = [P, P, P, P, P]
    lib.pd_damage.restype = I
    lib.pd_plan_workspace_bytes.argtypes = [P]
    lib.pd_plan_workspace_bytes.restype = I64
    lib.pd_plan_launch_count.argtypes = [P]
    lib.pd_plan_launch_count.restype = I64
    lib.pd_plan_boundary_nodes.argtypes = [P]
    lib.pd_plan_boundary_nodes.restype = I64
    lib.pd_stable_dt.argtypes = [P]
    lib.pd_stable_dt.restype = D
    lib.pd_plan_critical_energy.argtypes = [P]
    lib.pd_plan_critical_energy.restype = D
    lib.pd_plan_inject_stall.argtypes = [P, I]
    lib.pd_plan_inject_stall.restype = I
    lib.pd_plan_set_affine_split.argtypes = [P, I]
    lib.pd_plan_set_affine_split.restype = I
    lib.pd_plan_set_plane_passes.argtypes = [P, I]
    lib.pd_plan_set_plane_passes.restype = I
    lib.pd_plan_profile.argtypes = [P, I]
    lib.pd_plan_profile.restype = I
    lib.pd_plan_profile_read.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(I64)]
    lib.pd_plan_profile_read.restype = I
    lib.pd_force2d_noalloc.argtypes = [ctypes.POINTER(_Problem), P, P, P, P]
    lib.pd_force2d_noalloc.restype = I
    lib.pd_solve_dr.argtypes = [P, P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]
    lib.pd_solve_dr.restype = I
    lib.pd_plan_create_batched.argtypes = [I, ctypes.POINTER(_Problem), ctypes.POINTER(P), ctypes.POINTER(P), P,
                                           ctypes.POINTER(P)]
    lib.pd_plan_create_batched.restype = I
    lib.pd_batch_size.argtypes = [P]
    lib.pd_batch_size.restype = I
    lib.pd_batch_plan.argtypes = [P, I]
    lib.pd_batch_plan.restype = P
    lib.pd_solve_dr_batched.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), D, I,
                                        ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I), P]
    lib.pd_solve_dr_batched.restype = I
    lib.pd_batch_destroy.argtypes = [P]
    lib.pd_batch_destroy.restype = None
    lib.pd_plan_autotune.argtypes = [P, P]
    lib.pd_plan_autotune.restype = I
    lib.pd_plan_autotune_solve.argtypes = [P, P]
    lib.pd_plan_autotune_solve.restype = I
    lib.pd_batch_autotune.argtypes = [P, P]
    lib.pd_batch_autotune.restype = I
    lib.pd_plan_tuning.argtypes = [P, ctypes.POINTER(I)]
    lib.pd_plan_tuning.restype = I
    lib.pd_plan_set_tuning.argtypes = [P, ctypes.POINTER(I)]
    lib.pd_plan_set_tuning.restype = I
    lib.pd_plan_set_energy_mode.argtypes = [P, I]
    lib.pd_plan_set_energy_mode.restype = I
    lib.pd_status_string.argtypes = [I]
    lib.pd_status_string.restype = ctypes.c_char_p
    lib.pd_last_error_detail.argtypes = []
    lib.pd_last_error_detail.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st, where):
    if st != 0:
        raise PDError(st, where)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Problem:
    """Arguments of ``pd_problem`` (grid of Eq. 52, horizon, material)."""
    shape: Sequence[int]           # (n2, n1) or (n3, n2, n1), C order
    dx: float | Sequence[float] = 1.0
    delta: float = 3.0
    model: int = PD_LIN_BOND
    E: float = 1.0
    nu: float = 0.25
    rho: float = 1.0
    Wc: float = 0.0
    fp64: bool = False
    volume_rule: int = 0           # 0 constant dV (§4.1.1); 1 linear partial volumes (cubic cells)
    s0: float = 0.0                # critical stretch; the plan derives Wc from it when Wc <= 0

    def to_c(self) -> _Problem:
        p = _Problem()
        dim = len(self.shape)
        p.dim = dim
        n = list(self.shape[::-1]) + [1] * (3 - dim)
        for a in range(3):
            p.n[a] = int(n[a])
        dx = [float(self.dx)] * dim if isinstance(self.dx, (int, float)) else [float(v) for v in self.dx]
        for a in range(3):
            p.dx[a] = dx[a] if a < dim else 1.0
        p.delta = float(self.delta)
        p.model = int(self.model)
        p.E, p.nu, p.rho, p.Wc = float(self.E), float(self.nu), float(self.rho), float(self.Wc)
        p.fp64 = 1 if self.fp64 else 0
        p.volume_rule = int(self.volume_rule)
        p.s0 = float(self.s0)
        return p

    @property
    def dim(self):
        return len(self.shape)

    @property
    def dtype(self):
        return torch.float64 if self.fp64 else torch.float32


class Plan:
    """Owns a ``pd_plan``: spectra, masks and workspace on the current GPU."""

    def __init__(self, problem: Problem, chi: torch.Tensor, chi_omega: Optional[torch.Tensor] = None,
                 stream=None):
        lib = load()
        self.problem = problem
        self.shape = tuple(int(s) for s in problem.shape)
        self.dim = len(self.shape)
        self.dtype = problem.dtype
        chi = self._mask(chi, self.shape, "chi")
        if chi_omega is not None:
            chi_omega = self._mask(chi_omega, (self.dim,) + self.shape, "chi_omega")
        self._c = problem.to_c()
        h = ctypes.c_void_p()
        _check(lib.pd_plan_create(ctypes.byref(self._c), _ptr(chi), _ptr(chi_omega), _stream(stream),
                                  ctypes.byref(h)), "pd_plan_create")
        self._h = h
        self._owned = True
        self.device = chi.device

    @classmethod
    def _borrowed(cls, handle, problem: Problem, device):
        """A view of a plan owned by a Batch (closing it does nothing)."""
        self = cls.__new__(cls)
        self.problem = problem
        self.shape = tuple(int(s) for s in problem.shape)
        self.dim = len(self.shape)
        self.dtype = problem.dtype
        self._c = problem.to_c()
        self._h = ctypes.c_void_p(handle)
        self._owned = False
        self.device = device
        return self

    @staticmethod
    def _mask(t, shape, name):
        if t.dtype != torch.uint8 or not t.is_cuda or tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name}: expected a CUDA uint8 tensor of shape {tuple(shape)}")
        return t.contiguous()

    def _field(self, t, ncomp, name, dtype=None, allow_none=False):
        if t is None:
            if allow_none:
                return None
            raise ValueError(f"{name} is required")
        shape = (ncomp,) + self.shape if ncomp else self.shape
        dt = dtype or self.dtype
        if t.dtype != dt or not t.is_cuda or tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous CUDA {dt} tensor of shape {shape}, got "
                             f"{t.dtype} {tuple(t.shape)} (cuda={t.is_cuda}, contiguous={t.is_contiguous()})")
        if t.device != self.device:
            raise ValueError(f"{name}: tensor on {t.device}, the plan's buffers are on {self.device}")
        return t

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                load().pd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points -------------------------------------------------------
    def kernel_spectrum(self, stream=None) -> torch.Tensor:
        nc = 3 if self.dim == 2 else 6
        half = self.shape[-1] // 2 + 1
        out = torch.empty((nc,) + self.shape[:-1] + (half,), dtype=torch.float64, device=self.device)
        _check(load().pd_kernel_spectrum(self._h, _ptr(out), _stream(stream)), "pd_kernel_spectrum")
        return out

    def force(self, u, s=None, L=None, W=None, want_energy=False, stream=None):
        u = self._field(u, self.dim, "u")
        s = self._field(s, 0, "s", allow_none=True)
        if L is None:
            L = torch.empty_like(u)
        L = self._field(L, self.dim, "L")
        if want_energy and W is None:
            W = torch.empty(self.shape, dtype=self.dtype, device=u.device)
        W = self._field(W, 0, "W", allow_none=True)
        _check(load().pd_force(self._h, _ptr(u), _ptr(s), _ptr(L), _ptr(W), _stream(stream)), "pd_force")
        return (L, W) if W is not None else L

    def step_verlet(self, u, v, lam, b, w=None, dt=1.0, nsteps=1, count_broken=False, stream=None):
        u = self._field(u, self.dim, "u")
        v = self._field(v, self.dim, "v")
        b = self._field(b, self.dim, "b")
        w = self._field(w, self.dim, "w", allow_none=True)
        if lam is not None:
            lam = self._field(lam, 0, "lambda", dtype=torch.uint8)
        nb = ctypes.c_int64(0)
        _check(load().pd_step_verlet(self._h, _ptr(u), _ptr(v), _ptr(lam), _ptr(b), _ptr(w), float(dt),
                                     int(nsteps), ctypes.byref(nb) if count_broken else None,
                                     _stream(stream)), "pd_step_verlet")
        return int(nb.value) if count_broken else None

    def step_verlet_ramp(self, u, v, lam, b, w0, w1, t0=0.0, dt=1.0, nsteps=1, count_broken=False, stream=None):
        """pd_step_verlet_ramp: Gamma values w0 + t w1 at the end of each step."""
        u = self._field(u, self.dim, "u")
        v = self._field(v, self.dim, "v")
        b = self._field(b, self.dim, "b")
        w0 = self._field(w0, self.dim, "w0", allow_none=True)
        w1 = self._field(w1, self.dim, "w1")
        if lam is not None:
            lam = self._field(lam, 0, "lambda", dtype=torch.uint8)
        nb = ctypes.c_int64(0)
        _check(load().pd_step_verlet_ramp(self._h, _ptr(u), _ptr(v), _ptr(lam), _ptr(b), _ptr(w0), _ptr(w1),
                                          float(t0), float(dt), int(nsteps),
                                          ctypes.byref(nb) if count_broken else None, _stream(stream)),
               "pd_step_verlet_ramp")
        return int(nb.value) if count_broken else None

    def verlet_loss_grad(self, c_rel, u_target, dt, nsteps, checkpoint_every=10, lam0=None, u0=None, v0=None,
                         b=None, b0=None, want_grad=True, want_final=False, stream=None):
        """pd_verlet_loss_grad: returns (loss, grad_c or None[, u_final, lambda_final])."""
        lib = load()
        c_rel = self._field(c_rel, 0, "c_rel")
        u_target = self._field(u_target, self.dim, "u_target")
        u0 = self._field(u0, self.dim, "u0", allow_none=True)
        v0 = self._field(v0, self.dim, "v0", allow_none=True)
        b = self._field(b, self.dim, "b", allow_none=True)
        b0 = self._field(b0, self.dim, "b0", allow_none=True)
        if lam0 is not None:
            lam0 = self._field(lam0, 0, "lambda0", dtype=torch.uint8)
        nbytes = int(lib.pd_verlet_adjoint_workspace(self._h, int(nsteps), int(checkpoint_every)))
        if nbytes < 0:
            raise PDError(-1, "pd_verlet_adjoint_workspace")
        work = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        grad = torch.empty_like(c_rel) if want_grad else None
        uf = torch.empty_like(u_target) if want_final else None
        lf = torch.empty(self.shape, dtype=torch.uint8, device=self.device) if want_final else None
        loss = ctypes.c_double(0.0)
        _check(lib.pd_verlet_loss_grad(self._h, _ptr(c_rel), _ptr(lam0), _ptr(u0), _ptr(v0), _ptr(b), _ptr(b0),
                                       _ptr(u_target), float(dt), int(nsteps), int(checkpoint_every), _ptr(work),
                                       nbytes, ctypes.byref(loss), _ptr(grad), _ptr(uf), _ptr(lf),
                                       _stream(stream)), "pd_verlet_loss_grad")
        if want_final:
            return loss.value, grad, uf, lf
        return loss.value, grad

    def solve_static(self, u, b, w=None, rtol=1e-8, max_iter=20000, stream=None, raise_on_fail=True):
        u = self._field(u, self.dim, "u", dtype=torch.float64)
        b = self._field(b, self.dim, "b", dtype=torch.float64)
        w = self._field(w, self.dim, "w", dtype=torch.float64, allow_none=True)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = load().pd_solve_static(self._h, _ptr(u), _ptr(b), _ptr(w), float(rtol), int(max_iter),
                                    ctypes.byref(it), ctypes.byref(rr), _stream(stream))
        if st != 0 and (raise_on_fail or st != -5):
            raise PDError(st, "pd_solve_static")
        return int(it.value), float(rr.value), st

    def solve_mirror(self, u, b, g, mirror, rtol=1e-10, max_iter=20000, stream=None, raise_on_fail=True):
        """pd_solve_mirror: mirror-based volume constraints (FP64 plans)."""
        u = self._field(u, self.dim, "u", dtype=torch.float64)
        b = self._field(b, self.dim, "b", dtype=torch.float64, allow_none=True)
        g = self._field(g, self.dim, "g", dtype=torch.float64, allow_none=True)
        mirror = self._field(mirror, self.dim, "mirror", dtype=torch.int32)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = load().pd_solve_mirror(self._h, _ptr(u), _ptr(b), _ptr(g), _ptr(mirror), float(rtol), int(max_iter),
                                    ctypes.byref(it), ctypes.byref(rr), _stream(stream))
        if st != 0 and (raise_on_fail or st != -5):
            raise PDError(st, "pd_solve_mirror")
        return int(it.value), float(rr.value), st

    def solve_dr(self, u, b, w=None, rtol=1e-8, max_iter=200000, stream=None, raise_on_fail=True):
        """Adaptive dynamic relaxation with FP64 refinement (pd_solve_dr)."""
        u = self._field(u, self.dim, "u", dtype=torch.float64)
        b = self._field(b, self.dim, "b", dtype=torch.float64)
        w = self._field(w, self.dim, "w", dtype=torch.float64, allow_none=True)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = load().pd_solve_dr(self._h, _ptr(u), _ptr(b), _ptr(w), float(rtol), int(max_iter),
                                ctypes.byref(it), ctypes.byref(rr), _stream(stream))
        if st != 0 and (raise_on_fail or st != -5):
            raise PDError(st, "pd_solve_dr")
        return int(it.value), float(rr.value), st

    def autotune(self, stream=None, solve=False):
        """Pick the pass configuration by timing force evaluations, or (solve=True)
        chunks of the static solver's CG iterations."""
        if solve:
            _check(load().pd_plan_autotune_solve(self._h, _stream(stream)), "pd_plan_autotune_solve")
        else:
            _check(load().pd_plan_autotune(self._h, _stream(stream)), "pd_plan_autotune")
        return self.tuning

    def set_energy_mode(self, direct: bool):
        """W for bond breaking: False = convolution form (Eq. 102), True = horizon sum (Eq. 47)."""
        _check(load().pd_plan_set_energy_mode(self._h, 1 if direct else 0), "pd_plan_set_energy_mode")

    def set_tuning(self, rows=0, w_x2=0, w_last=0, sched=0, stages=0, stages_inv=0):
        """Pin a pass configuration (0 = built-in heuristic)."""
        arr = (ctypes.c_int * 6)(int(rows), int(w_x2), int(w_last), int(sched), int(stages), int(stages_inv))
        _check(load().pd_plan_set_tuning(self._h, arr), "pd_plan_set_tuning")

    @property
    def tuning(self):
        """{rows, w_x2, w_last, sched, stages, stages_inv} picked by autotune (0 = built-in heuristic)."""
        out = (ctypes.c_int * 6)()
        _check(load().pd_plan_tuning(self._h, out), "pd_plan_tuning")
        return {"rows": out[0], "w_x2": out[1], "w_last": out[2], "sched": out[3], "stages": out[4],
                "stages_inv": out[5]}

    def force_adjoint(self, u, gL, s=None, want_gu=True, want_gs=True, stream=None):
        u = self._field(u, self.dim, "u")
        gL = self._field(gL, self.dim, "gL")
        s = self._field(s, 0, "s", allow_none=True)
        gu = torch.empty_like(u) if want_gu else None
        gs = torch.empty(self.shape, dtype=self.dtype, device=u.device) if want_gs else None
        _check(load().pd_force_adjoint(self._h, _ptr(u), _ptr(s), _ptr(gL), _ptr(gu), _ptr(gs),
                                       _stream(stream)), "pd_force_adjoint")
        return gu, gs

    def damage(self, lam, stream=None):
        lam = self._field(lam, 0, "lambda", dtype=torch.uint8)
        nb = torch.empty(self.shape, dtype=torch.int32, device=lam.device)
        d = torch.empty(self.shape, dtype=self.dtype, device=lam.device)
        _check(load().pd_damage(self._h, _ptr(lam), _ptr(nb), _ptr(d), _stream(stream)), "pd_damage")
        return nb, d

    def profile(self, enable: bool = True, kinds=None):
        """Time the selected pass kinds (names of PASS_KINDS; all by default)."""
        mask = 0
        if enable:
            names = list(PASS_KINDS.values()) if kinds is None else list(kinds)
            for k, nm in PASS_KINDS.items():
                if nm in names:
                    mask |= 1 << k
        _check(load().pd_plan_profile(self._h, mask), "pd_plan_profile")

    def profile_read(self):
        """{pass kind: (total ms, launches)} since the last profile() call."""
        out = {}
        for k, name in PASS_KINDS.items():
            ms = ctypes.c_double(0.0)
            n = ctypes.c_int64(0)
            _check(load().pd_plan_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n)),
                   "pd_plan_profile_read")
            out[name] = (float(ms.value), int(n.value))
        return out

    @property
    def workspace_bytes(self):
        return int(load().pd_plan_workspace_bytes(self._h))

    @property
    def launch_count(self):
        return int(load().pd_plan_launch_count(self._h))

    @property
    def boundary_nodes(self):
        return int(load().pd_plan_boundary_nodes(self._h))

    def set_plane_passes(self, mask):
        """FP32 CG on 32^3 / 64^3 / 128^3 cubes: which halves of the iteration run as
        fused x1-x2 plane passes (bit 0 forward, bit 1 inverse; True = both, False =
        neither: row and column passes) (pd_plan_set_plane_passes)."""
        m = 3 if mask is True else 0 if mask is False else int(mask)
        _check(load().pd_plan_set_plane_passes(self._h, m), "pd_plan_set_plane_passes")

    def set_affine_split(self, on: bool):
        """pd_force on fields with a large affine part: transform u - a (a the
        least-squares affine fit) and add the exact force of a (pd_plan_set_affine_split)."""
        _check(load().pd_plan_set_affine_split(self._h, 1 if on else 0), "pd_plan_set_affine_split")

    def inject_stall(self, kind: int):
        """Failure-handling test hook (pd_plan_inject_stall): the next pass of
        this kind (0 forward row pass, 3 inverse row pass, 5 inverse plane pass)
        has one block whose wait runs out."""
        _check(load().pd_plan_inject_stall(self._h, int(kind)), "pd_plan_inject_stall")

    @property
    def critical_energy(self):
        return float(load().pd_plan_critical_energy(self._h))

    @property
    def stable_dt(self):
        return float(load().pd_stable_dt(self._h))


def force2d_noalloc(problem: Problem, chi: torch.Tensor, u: torch.Tensor, L: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
    """2D FP32 bond force through ``pd_force2d_noalloc``: no plan, no device
    allocation inside the library (for callers that cannot call cudaMalloc).
    The output tensor L may be passed in; otherwise it is allocated here, by the
    caller's side (torch), not by the library."""
    shape = tuple(int(s) for s in problem.shape)
    if (len(shape) != 2 or chi.dtype != torch.uint8 or tuple(chi.shape) != shape or not chi.is_cuda
            or u.dtype != torch.float32 or tuple(u.shape) != (2,) + shape or not u.is_contiguous()):
        raise ValueError("force2d_noalloc: expects a 2D uint8 chi and a contiguous float32 u of shape (2, n2, n1)")
    if L is None:
        L = torch.empty_like(u)
    c = problem.to_c()
    _check(load().pd_force2d_noalloc(ctypes.byref(c), _ptr(chi.contiguous()), _ptr(u), _ptr(L), _stream(stream)),
           "pd_force2d_noalloc")
    return L


class Batch:
    """Owns a ``pd_batch``: independent specimens solved in one graph launch."""

    def __init__(self, problems: Sequence[Problem], chis: Sequence[torch.Tensor],
                 chi_omegas: Optional[Sequence[Optional[torch.Tensor]]] = None, stream=None):
        lib = load()
        n = len(problems)
        if len(chis) != n or (chi_omegas is not None and len(chi_omegas) != n):
            raise ValueError("one problem and one mask per specimen")
        self.problems = list(problems)
        self._chis = [Plan._mask(c, tuple(p.shape), "chi") for p, c in zip(problems, chis)]
        com = [None] * n
        if chi_omegas is not None:
            com = [None if c is None else Plan._mask(c, (len(p.shape),) + tuple(p.shape), "chi_omega")
                   for p, c in zip(problems, chi_omegas)]
        cp = (_Problem * n)(*[p.to_c() for p in problems])
        chp = (ctypes.c_void_p * n)(*[c.data_ptr() for c in self._chis])
        cop = (ctypes.c_void_p * n)(*[None if c is None else c.data_ptr() for c in com])
        h = ctypes.c_void_p()
        _check(lib.pd_plan_create_batched(n, cp, chp, cop, _stream(stream), ctypes.byref(h)),
               "pd_plan_create_batched")
        self._h = h
        self.device = self._chis[0].device
        self.plans = [Plan._borrowed(lib.pd_batch_plan(h, i), problems[i], self.device) for i in range(n)]

    def __len__(self):
        return len(self.problems)

    def autotune(self, stream=None):
        _check(load().pd_batch_autotune(self._h, _stream(stream)), "pd_batch_autotune")
        return [p.tuning for p in self.plans]

    def solve_dr(self, us, bs, ws=None, rtol=1e-8, max_iter=200000, stream=None, raise_on_fail=True):
        """Solve every specimen in one graph launch; returns (steps, relres, status) lists."""
        n = len(self.plans)
        us = [pl._field(u, pl.dim, "u", dtype=torch.float64) for pl, u in zip(self.plans, us)]
        bs = [pl._field(b, pl.dim, "b", dtype=torch.float64) for pl, b in zip(self.plans, bs)]
        if ws is not None:
            ws = [pl._field(w, pl.dim, "w", dtype=torch.float64, allow_none=True) for pl, w in zip(self.plans, ws)]
        up = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
        bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
        wp = None if ws is None else (ctypes.c_void_p * n)(*[None if w is None else w.data_ptr() for w in ws])
        it = (ctypes.c_int * n)()
        rr = (ctypes.c_double * n)()
        stt = (ctypes.c_int * n)()
        st = load().pd_solve_dr_batched(self._h, up, bp, wp, float(rtol), int(max_iter), it, rr, stt,
                                        _stream(stream))
        if st != 0 and (raise_on_fail or st != -5):
            raise PDError(st, "pd_solve_dr_batched")
        return list(it), list(rr), list(stt)

    def close(self):
        if getattr(self, "_h", None):
            for p in self.plans:
                p._h = None
            load().pd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
