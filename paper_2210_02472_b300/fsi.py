"""Thin ctypes binding of libfsi's C ABI (include/fsi.h).

Argument marshalling only: every arithmetic step runs in the CUDA library.  Arrays are
torch CUDA tensors in FP64 (positions/velocities (3, N) contiguous, masses (N,)), index
lists int32 CUDA tensors, black-hole flags uint8/bool CUDA tensors.  Work is enqueued on
torch's current CUDA stream.

Importing this module loads ``libfsi.so`` and raises ImportError if it is missing: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path
from typing import Optional

import torch

_LIB_PATH = Path(__file__).resolve().parent / "libfsi.so"
if not _LIB_PATH.exists():
    raise ImportError(f"libfsi.so not built at {_LIB_PATH}; run "
                      "`python -m paper_2210_02472_b300.build` (needs nvcc)")
_lib = C.CDLL(str(_LIB_PATH))

FSI_OK = 0
FSI_ERR_ARG = -1
FSI_ERR_CUDA = -2
FSI_ERR_NONFINITE = -3
FSI_ERR_COINCIDENT = -4
FSI_ERR_TIMEOUT = -5
FSI_ERR_MAXLEVEL = -6
FSI_ERR_UNSUPPORTED = -7
FSI_ERR_NOMEM = -8
FSI_FP64 = 0
FSI_MIXED = 1

EXPORTED = ["fsi_default_params", "fsi_create", "fsi_destroy", "fsi_set_params", "fsi_reserve",
            "fsi_last_error", "fsi_sync_status", "fsi_accel", "fsi_grad", "fsi_accel_grad",
            "fsi_pn_accel", "fsi_step", "fsi_step_record", "fsi_kick_drift", "fsi_timesteps", "fsi_energy", "fsi_hhs_interval",
            "fsi_level_stats", "fsi_hhs_interval_restart", "fsi_step_sub", "fsi_profile", "fsi_profile_read", "fsi_launch_count",
            "fsi_fma_probe", "fsi_autotune", "fsi_get_tuning", "fsi_set_tuning",
            "fsi_step_vjp", "fsi_step_vjp_rec", "fsi_batch_create", "fsi_batch_destroy", "fsi_batch_step",
            "fsi_batch_set_tuning", "fsi_batch_get_tuning", "fsi_batch_inject_stall", "fsi_batch_stats",
            "fsi_work_stats", "fsi_accel_noalloc", "fsi_far_stats", "fsi_get_tuning_for", "fsi_grid_stats",
            "fsi_batch_item_stats", "fsi_timesteps_sub", "fsi_accel_part", "fsi_grad_part"]


class fsi_params(C.Structure):
    _fields_ = [("precision", C.c_int), ("eps2", C.c_double), ("eta_ff", C.c_double),
                ("eta_fb", C.c_double), ("eta_jerk", C.c_double), ("max_level", C.c_int),
                ("c", C.c_double), ("split", C.c_int), ("timeout_ns", C.c_longlong),
                ("symmetric", C.c_int), ("hhs_small_max", C.c_int), ("order_min", C.c_int),
                ("eta_grad", C.c_double), ("eta_va", C.c_double), ("wide_ctas", C.c_int),
                ("hhs_grid_max", C.c_int), ("hhs_grid_ctas", C.c_int)]


_vp, _ip, _dp = C.c_void_p, C.c_int, C.c_double
_lib.fsi_default_params.argtypes = [C.POINTER(fsi_params)]
_lib.fsi_default_params.restype = None
_lib.fsi_create.argtypes = [C.POINTER(_vp), C.POINTER(fsi_params)]
_lib.fsi_destroy.argtypes = [_vp]
_lib.fsi_set_params.argtypes = [_vp, C.POINTER(fsi_params)]
_lib.fsi_reserve.argtypes = [_vp, _ip, _ip]
_lib.fsi_last_error.restype = C.c_char_p
_lib.fsi_sync_status.argtypes = [_vp, _vp]
_lib.fsi_accel.argtypes = [_vp, _ip, _vp, _vp, _vp, _ip, _vp, _ip, _dp, _vp, _vp]
_lib.fsi_grad.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _vp, _ip, _dp, _vp, _vp]
_lib.fsi_accel_part.argtypes = [_vp, _ip, _vp, _vp, _vp, _ip, _ip, _ip, _dp, _vp, _vp]
_lib.fsi_grad_part.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _ip, _ip, _dp, _vp, _vp]
_lib.fsi_accel_grad.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _vp, _ip, _dp, _vp, _vp, _vp]
_lib.fsi_pn_accel.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _dp, _vp, _ip, _vp, _ip, _vp, _vp]
_lib.fsi_step.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _vp, _ip, _dp, _ip, _vp]
_lib.fsi_kick_drift.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _dp, _dp, _vp]
_lib.fsi_timesteps.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _vp, _vp]
_lib.fsi_timesteps_sub.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _ip, _ip, _vp, _vp]
_lib.fsi_energy.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _vp, _vp]
_lib.fsi_hhs_interval.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _dp, _vp]
_lib.fsi_level_stats.argtypes = [_vp, C.POINTER(C.c_longlong), _ip]
_lib.fsi_step_sub.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _vp, _ip, _dp, _ip, _vp]
_lib.fsi_hhs_interval_restart.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _dp, _dp, _ip,
                                          C.POINTER(_ip), C.POINTER(_dp), _vp]
_lib.fsi_profile.argtypes = [_vp, _ip]
_lib.fsi_profile_read.argtypes = [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_double)]
_lib.fsi_launch_count.restype = C.c_longlong
_lib.fsi_accel_noalloc.argtypes = [_ip, _vp, _vp, _dp, _vp, _vp]
_lib.fsi_work_stats.argtypes = [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), _ip]
_lib.fsi_far_stats.argtypes = [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), _ip, _vp]
_lib.fsi_grid_stats.argtypes = [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), _ip, _vp]
_lib.fsi_batch_item_stats.argtypes = [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), _ip]
_lib.fsi_fma_probe.argtypes = [_ip, _ip, _ip, _vp, C.POINTER(C.c_double), _vp]
_lib.fsi_autotune.argtypes = [_vp, _ip, _vp, _vp, _ip, _ip, _vp]
_lib.fsi_get_tuning.argtypes = [_vp, C.POINTER(_ip), C.POINTER(_ip)]
_lib.fsi_get_tuning_for.argtypes = [_vp, _ip, C.POINTER(_ip), C.POINTER(_ip)]
_lib.fsi_set_tuning.argtypes = [_vp, _ip, _ip]
_lib.fsi_batch_create.argtypes = [_vp, _ip, C.POINTER(C.c_longlong), _ip, C.POINTER(_vp)]
_lib.fsi_batch_destroy.argtypes = [_vp]
_lib.fsi_batch_step.argtypes = [_vp, _vp, _vp, _vp, _vp, _dp, _ip, _vp]
_lib.fsi_batch_set_tuning.argtypes = [_vp, _vp, _ip, _ip]
_lib.fsi_batch_get_tuning.argtypes = [_vp, C.POINTER(_ip), C.POINTER(_ip)]
_lib.fsi_batch_inject_stall.argtypes = [_vp, _ip]
_lib.fsi_batch_stats.argtypes = [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                 C.POINTER(_ip), _ip]
_lib.fsi_step_vjp.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _dp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.fsi_step_record.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _dp, _vp, _vp, _vp, _vp]
_lib.fsi_step_vjp_rec.argtypes = [_vp, _ip, _vp, _vp, _vp, _vp, _ip, _dp, _vp, _vp, _vp, _vp, _vp,
                                  _vp, _vp, _vp, _vp]


class FsiError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = _lib.fsi_last_error().decode(errors="replace")
        super().__init__(f"{what}: status {code} ({msg})")
        self.code = code


def _check(code: int, what: str) -> None:
    if code != FSI_OK:
        raise FsiError(code, what)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _f64(t: torch.Tensor, shape, name: str) -> int:
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA float64 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _ids(t: Optional[torch.Tensor], N: int, name: str):
    if t is None:
        return None, N
    if not (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous() and t.dim() == 1):
        raise TypeError(f"{name} must be a contiguous 1-D CUDA int32 tensor")
    return (t.data_ptr() if t.numel() else None), int(t.numel())


def _u8(t: Optional[torch.Tensor], N: int, name: str):
    if t is None:
        return None
    if t.dtype == torch.bool:
        t = t.view(torch.uint8)
    if not (t.is_cuda and t.dtype == torch.uint8 and t.is_contiguous() and t.numel() == N):
        raise TypeError(f"{name} must be a contiguous CUDA uint8/bool tensor of N entries")
    return t.data_ptr()


class Context:
    """Owns an fsi_ctx (device workspace + error word) on the current CUDA device."""

    def __init__(self, precision: str = "fp64", eps2: float = 0.0, eta_ff: float = 0.2,
                 eta_fb: float = 0.2, eta_jerk: float = 0.1, max_level: int = 40,
                 c: float = 0.0, split: int = 0, timeout_ns: int = 0, symmetric: bool = True,
                 hhs_small_max: int = 0, order_min: int = 0, eta_grad: float = 0.0,
                 eta_va: float = 0.0, wide_ctas: int = 0, hhs_grid_max: int = 0,
                 hhs_grid_ctas: int = 0):
        p = fsi_params()
        _lib.fsi_default_params(C.byref(p))
        p.precision = {"fp64": FSI_FP64, "mixed": FSI_MIXED}[precision]
        p.eps2, p.eta_ff, p.eta_fb, p.eta_jerk = eps2, eta_ff, eta_fb, eta_jerk
        p.max_level, p.c, p.split, p.timeout_ns = max_level, c, split, timeout_ns
        p.symmetric = int(bool(symmetric))
        p.hhs_small_max = int(hhs_small_max)
        p.order_min = int(order_min)
        p.eta_grad, p.eta_va = float(eta_grad), float(eta_va)
        p.wide_ctas = int(wide_ctas)
        p.hhs_grid_max = int(hhs_grid_max)
        p.hhs_grid_ctas = int(hhs_grid_ctas)
        self.params = p
        self.precision = precision
        h = _vp()
        _check(_lib.fsi_create(C.byref(h), C.byref(p)), "fsi_create")
        self.handle = h

    def set_params(self, **fields) -> None:
        """Change fields of the context's fsi_params (fsi_set_params), e.g. timeout_ns=0."""
        for k, v in fields.items():
            if not hasattr(self.params, k):
                raise AttributeError(k)
            setattr(self.params, k, v)
        _check(_lib.fsi_set_params(self.handle, C.byref(self.params)), "fsi_set_params")

    def close(self) -> None:
        if getattr(self, "handle", None):
            _lib.fsi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def fsi_reserve(ctx: Context, N: int, n: int) -> None:
    _check(_lib.fsi_reserve(ctx.handle, N, n), "fsi_reserve")


def fsi_sync_status(ctx: Context, stream=None) -> int:
    return int(_lib.fsi_sync_status(ctx.handle, _stream(stream)))


def fsi_accel(ctx: Context, pos, mass, A=None, B=None, eps2: float = 0.0, out=None, stream=None):
    N = mass.numel()
    pa, nA = _ids(A, N, "A")
    pb, nB = _ids(B, N, "B")
    if out is None:
        out = torch.empty((3, nA), dtype=torch.float64, device=pos.device)
    _check(_lib.fsi_accel(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(mass, (N,), "mass"),
                          pa, nA, pb, nB, float(eps2), _f64(out, (3, nA), "out"), _stream(stream)),
           "fsi_accel")
    return out


def fsi_grad(ctx: Context, pos, mass, accg, A=None, B=None, eps2: float = 0.0, out=None,
             stream=None):
    N = mass.numel()
    pa, nA = _ids(A, N, "A")
    pb, nB = _ids(B, N, "B")
    if out is None:
        out = torch.empty((3, nA), dtype=torch.float64, device=pos.device)
    _check(_lib.fsi_grad(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(mass, (N,), "mass"),
                         _f64(accg, (3, N), "accg"), pa, nA, pb, nB, float(eps2),
                         _f64(out, (3, nA), "out"), _stream(stream)), "fsi_grad")
    return out


def fsi_accel_part(ctx: Context, pos, mass, part: int, nparts: int, A=None, eps2: float = 0.0,
                   out=None, stream=None):
    """Share `part` of nparts of the same-set pass acc(A <- A): (3, nA) partial sums; the
    shares add up to fsi_accel(A <- A)."""
    N = mass.numel()
    pa, nA = _ids(A, N, "A")
    if out is None:
        out = torch.empty((3, nA), dtype=torch.float64, device=pos.device)
    _check(_lib.fsi_accel_part(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(mass, (N,), "mass"),
                               pa, nA, int(part), int(nparts), float(eps2),
                               _f64(out, (3, nA), "out"), _stream(stream)), "fsi_accel_part")
    return out


def fsi_grad_part(ctx: Context, pos, mass, accg, part: int, nparts: int, A=None,
                  eps2: float = 0.0, out=None, stream=None):
    """Share `part` of nparts of the same-set pass G(A <- A) with the accelerations accg
    (3, N): (3, nA) partial sums; the shares add up to fsi_grad(A <- A)."""
    N = mass.numel()
    pa, nA = _ids(A, N, "A")
    if out is None:
        out = torch.empty((3, nA), dtype=torch.float64, device=pos.device)
    _check(_lib.fsi_grad_part(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(mass, (N,), "mass"),
                              _f64(accg, (3, N), "accg"), pa, nA, int(part), int(nparts),
                              float(eps2), _f64(out, (3, nA), "out"), _stream(stream)),
           "fsi_grad_part")
    return out


def fsi_accel_grad(ctx: Context, pos, vel, mass, A=None, B=None, eps2: float = 0.0,
                   acc_out=None, grad_out=None, stream=None):
    N = mass.numel()
    pa, nA = _ids(A, N, "A")
    pb, nB = _ids(B, N, "B")
    if A is not None and B is not None and A is B:
        pb = pa
    if acc_out is None:
        acc_out = torch.empty((3, nA), dtype=torch.float64, device=pos.device)
    if grad_out is None:
        grad_out = torch.empty((3, nA), dtype=torch.float64, device=pos.device)
    pv = _f64(vel, (3, N), "vel") if vel is not None else None
    _check(_lib.fsi_accel_grad(ctx.handle, N, _f64(pos, (3, N), "pos"), pv, _f64(mass, (N,), "mass"),
                               pa, nA, pb, nB, float(eps2), _f64(acc_out, (3, nA), "acc_out"),
                               _f64(grad_out, (3, nA), "grad_out"), _stream(stream)),
           "fsi_accel_grad")
    return acc_out, grad_out


def fsi_pn_accel(ctx: Context, pos, vel, mass, is_bh, c: float, A=None, B=None, out=None,
                 stream=None):
    N = mass.numel()
    pa, nA = _ids(A, N, "A")
    pb, nB = _ids(B, N, "B")
    if out is None:
        out = torch.empty((3, nA), dtype=torch.float64, device=pos.device)
    _check(_lib.fsi_pn_accel(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(vel, (3, N), "vel"),
                             _f64(mass, (N,), "mass"), _u8(is_bh, N, "is_bh"), float(c), pa, nA,
                             pb, nB, _f64(out, (3, nA), "out"), _stream(stream)), "fsi_pn_accel")
    return out


def fsi_step(ctx: Context, pos, vel, mass, h: float, nsteps: int = 1, is_bh=None, idx=None,
             stream=None) -> None:
    """nsteps FSI cycles of step h, in place on pos/vel."""
    N = mass.numel()
    pi, n = _ids(idx, N, "idx")
    _check(_lib.fsi_step(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(vel, (3, N), "vel"),
                         _f64(mass, (N,), "mass"), _u8(is_bh, N, "is_bh"), pi, n, float(h),
                         int(nsteps), _stream(stream)), "fsi_step")


def fsi_kick_drift(ctx: Context, pos, vel, acc, c_kick: float, c_drift: float, idx=None,
                   stream=None) -> None:
    """In place: vel[:, i] += c_kick acc[:, k], then pos[:, i] += c_drift vel[:, i] for
    i = idx[k] (all particles when idx is None); acc (3, n) or None for a drift only."""
    N = pos.shape[1]
    pi, n = _ids(idx, N, "idx")
    pa = None if acc is None else _f64(acc, (3, n), "acc")
    _check(_lib.fsi_kick_drift(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(vel, (3, N), "vel"),
                               pa, pi, n, float(c_kick), float(c_drift), _stream(stream)),
           "fsi_kick_drift")


def fsi_timesteps(ctx: Context, pos, vel, mass, P=None, out=None, stream=None):
    N = mass.numel()
    pp, n = _ids(P, N, "P")
    if out is None:
        out = torch.empty((n,), dtype=torch.float64, device=pos.device)
    _check(_lib.fsi_timesteps(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(vel, (3, N), "vel"),
                              _f64(mass, (N,), "mass"), pp, n, _f64(out, (n,), "out"),
                              _stream(stream)), "fsi_timesteps")
    return out


def fsi_timesteps_sub(ctx: Context, pos, vel, mass, P, lo: int, hi: int, out=None, stream=None):
    """Time steps of the entries P[lo:hi] against the whole set P (one receiver slice)."""
    N = mass.numel()
    pp, n = _ids(P, N, "P")
    lo, hi = int(lo), int(hi)
    if out is None:
        out = torch.empty((max(hi - lo, 0),), dtype=torch.float64, device=pos.device)
    _check(_lib.fsi_timesteps_sub(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(vel, (3, N), "vel"),
                                  _f64(mass, (N,), "mass"), pp, n, lo, hi,
                                  _f64(out, (max(hi - lo, 0),), "out"), _stream(stream)),
           "fsi_timesteps_sub")
    return out


def fsi_energy(ctx: Context, pos, vel, mass, P=None, out=None, stream=None):
    """Device tensor (2,): kinetic and potential energy of the set."""
    N = mass.numel()
    pp, n = _ids(P, N, "P")
    if out is None:
        out = torch.empty((2,), dtype=torch.float64, device=pos.device)
    _check(_lib.fsi_energy(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(vel, (3, N), "vel"),
                           _f64(mass, (N,), "mass"), pp, n, _f64(out, (2,), "out"),
                           _stream(stream)), "fsi_energy")
    return out


def fsi_hhs_interval(ctx: Context, pos, vel, mass, tau: float, is_bh=None, stream=None) -> int:
    """One HHS interval in place; returns FSI_OK or FSI_ERR_MAXLEVEL (interval completed)."""
    N = mass.numel()
    code = _lib.fsi_hhs_interval(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(vel, (3, N), "vel"),
                                 _f64(mass, (N,), "mass"), _u8(is_bh, N, "is_bh"), float(tau),
                                 _stream(stream))
    if code not in (FSI_OK, FSI_ERR_MAXLEVEL):
        raise FsiError(code, "fsi_hhs_interval")
    return int(code)


def fsi_step_sub(ctx: Context, pos, vel, mass, pairs, h: float, nsteps: int = 1, idx=None,
                 stream=None) -> None:
    """nsteps FSI cycles with binary subsystems (Algorithm 1), in place; pairs: int32
    device tensor of shape (n_pairs, 2) holding global ids."""
    N = mass.numel()
    pi, n = _ids(idx, N, "idx")
    if pairs is None or pairs.numel() == 0:
        pp, npairs = None, 0
    else:
        if pairs.dtype != torch.int32 or not pairs.is_cuda or not pairs.is_contiguous():
            raise TypeError("pairs must be a contiguous int32 CUDA tensor of shape (n_pairs, 2)")
        pp, npairs = pairs.data_ptr(), pairs.numel() // 2
    _check(_lib.fsi_step_sub(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(vel, (3, N), "vel"),
                             _f64(mass, (N,), "mass"), pi, n, pp, int(npairs), float(h),
                             int(nsteps), _stream(stream)), "fsi_step_sub")


def fsi_hhs_interval_restart(ctx: Context, pos, vel, mass, tau: float, eta_restart: float,
                             max_restarts: int = 8, is_bh=None, stream=None):
    """One HHS interval with adaptive energy-error restarts, in place; returns
    (status, restarts, |dE/E| of the accepted attempt)."""
    N = mass.numel()
    k = C.c_int()
    e = C.c_double()
    code = _lib.fsi_hhs_interval_restart(ctx.handle, N, _f64(pos, (3, N), "pos"),
                                         _f64(vel, (3, N), "vel"), _f64(mass, (N,), "mass"),
                                         _u8(is_bh, N, "is_bh"), float(tau), float(eta_restart),
                                         int(max_restarts), C.byref(k), C.byref(e),
                                         _stream(stream))
    if code not in (FSI_OK, FSI_ERR_MAXLEVEL):
        raise FsiError(code, "fsi_hhs_interval_restart")
    return int(code), int(k.value), float(e.value)


def fsi_level_stats(ctx: Context, max_levels: int = 64):
    counts = (C.c_longlong * max_levels)()
    used = _lib.fsi_level_stats(ctx.handle, counts, max_levels)
    return [int(x) for x in counts[:max(used, 0)]]


def fsi_grid_stats(ctx: Context, reset: bool = False, stream=None):
    """Phase profile of the cooperative-launch HHS recursions (while fsi_profile is on):
    (ns, phases), each a list of 8 per phase kind (time steps, split (empty), inter-level
    kick, FSI pass, one-CTA recursion, gradient criteria, set-up, PN kick)."""
    ns = (C.c_longlong * 8)()
    ph = (C.c_longlong * 8)()
    _check(_lib.fsi_grid_stats(ctx.handle, ns, ph, int(bool(reset)), _stream(stream)), "fsi_grid_stats")
    return [int(x) for x in ns], [int(x) for x in ph]


def fsi_profile(ctx: Context, enable: bool = True) -> None:
    """Record an event pair around every pair-kernel launch on its launch stream."""
    _check(_lib.fsi_profile(ctx.handle, int(bool(enable))), "fsi_profile")


def fsi_profile_read(ctx: Context):
    """{kind: (launches, milliseconds)} for kinds 'acc', 'grad', 'finalize'; clears."""
    n = (C.c_longlong * 3)()
    ms = (C.c_double * 3)()
    _check(_lib.fsi_profile_read(ctx.handle, n, ms), "fsi_profile_read")
    return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(("acc", "grad", "finalize"))}


def fsi_launch_count() -> int:
    """Kernels launched by libfsi in this process."""
    return int(_lib.fsi_launch_count())


def fsi_fma_probe(fp64: int, blocks: int, iters: int, sink: torch.Tensor, stream=None) -> float:
    """Enqueue the FMA throughput probe (0: FP32, 1: FP64, 2: packed FP32x2); returns its
    nominal flop count."""
    f = C.c_double()
    _check(_lib.fsi_fma_probe(int(fp64), int(blocks), int(iters), sink.data_ptr(),
                              C.byref(f), _stream(stream)), "fsi_fma_probe")
    return f.value


def fsi_autotune(ctx: Context, pos, mass, n: int = 0, reps: int = 2, stream=None):
    """Pick the fastest pair-kernel variants on the first n particles; returns them."""
    N = mass.numel()
    n = N if n <= 0 else min(n, N)
    _check(_lib.fsi_autotune(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(mass, (N,), "mass"),
                             int(n), int(reps), _stream(stream)), "fsi_autotune")
    return fsi_get_tuning_for(ctx, n)


def fsi_get_tuning(ctx: Context):
    """(acc, grad) variants of the largest set-size class."""
    a, g = _ip(), _ip()
    _check(_lib.fsi_get_tuning(ctx.handle, C.byref(a), C.byref(g)), "fsi_get_tuning")
    return int(a.value), int(g.value)


def fsi_get_tuning_for(ctx: Context, n: int):
    """(acc, grad) variants a set of n particles runs."""
    a, g = _ip(), _ip()
    _check(_lib.fsi_get_tuning_for(ctx.handle, int(n), C.byref(a), C.byref(g)), "fsi_get_tuning_for")
    return int(a.value), int(g.value)


def fsi_set_tuning(ctx: Context, ipt_acc: int, ipt_grad: int) -> None:
    _check(_lib.fsi_set_tuning(ctx.handle, int(ipt_acc), int(ipt_grad)), "fsi_set_tuning")


def fsi_step_vjp(ctx: Context, pos0, vel0, mass, h: float, gx_out, gv_out, idx=None, gm=None,
                 stream=None):
    """Cotangents (gx_in, gv_in, gm) of one FSI cycle's input state; gm accumulates."""
    N = mass.numel()
    pi, n = _ids(idx, N, "idx")
    gx_in = torch.empty_like(gx_out)
    gv_in = torch.empty_like(gv_out)
    if gm is None:
        gm = torch.zeros_like(mass)
    _check(_lib.fsi_step_vjp(ctx.handle, N, _f64(pos0, (3, N), "pos0"), _f64(vel0, (3, N), "vel0"),
                             _f64(mass, (N,), "mass"), pi, n, float(h),
                             _f64(gx_out, (3, N), "gx_out"), _f64(gv_out, (3, N), "gv_out"),
                             _f64(gx_in, (3, N), "gx_in"), _f64(gv_in, (3, N), "gv_in"),
                             _f64(gm, (N,), "gm"), _stream(stream)), "fsi_step_vjp")
    return gx_in, gv_in, gm


def fsi_step_record(ctx: Context, pos, vel, mass, h: float, idx=None, stream=None):
    """One FSI cycle in place (as fsi_step, nsteps = 1); returns the intermediates
    (a0, a1, g1), each (3, n) in the order of idx, for fsi_step_vjp_rec."""
    N = mass.numel()
    pi, n = _ids(idx, N, "idx")
    a0 = torch.empty((3, n), dtype=torch.float64, device=pos.device)
    a1, g1 = torch.empty_like(a0), torch.empty_like(a0)
    _check(_lib.fsi_step_record(ctx.handle, N, _f64(pos, (3, N), "pos"), _f64(vel, (3, N), "vel"),
                                _f64(mass, (N,), "mass"), pi, n, float(h), _f64(a0, (3, n), "a0"),
                                _f64(a1, (3, n), "a1"), _f64(g1, (3, n), "g1"), _stream(stream)),
           "fsi_step_record")
    return a0, a1, g1


def fsi_step_vjp_rec(ctx: Context, pos0, vel0, mass, h: float, rec, gx_out, gv_out, idx=None,
                     gm=None, stream=None):
    """fsi_step_vjp with the cycle's recorded intermediates rec = (a0, a1, g1)."""
    N = mass.numel()
    pi, n = _ids(idx, N, "idx")
    a0, a1, g1 = rec
    gx_in = torch.empty_like(gx_out)
    gv_in = torch.empty_like(gv_out)
    if gm is None:
        gm = torch.zeros_like(mass)
    _check(_lib.fsi_step_vjp_rec(ctx.handle, N, _f64(pos0, (3, N), "pos0"), _f64(vel0, (3, N), "vel0"),
                                 _f64(mass, (N,), "mass"), pi, n, float(h), _f64(a0, (3, n), "a0"),
                                 _f64(a1, (3, n), "a1"), _f64(g1, (3, n), "g1"),
                                 _f64(gx_out, (3, N), "gx_out"), _f64(gv_out, (3, N), "gv_out"),
                                 _f64(gx_in, (3, N), "gx_in"), _f64(gv_in, (3, N), "gv_in"),
                                 _f64(gm, (N,), "gm"), _stream(stream)), "fsi_step_vjp_rec")
    return gx_in, gv_in, gm


class Batch:
    """A plan for FSI cycles of K independent clusters concatenated in one SoA set."""

    def __init__(self, ctx: Context, offsets, max_steps: int = 16):
        import numpy as _np
        off = _np.ascontiguousarray(_np.asarray(offsets, dtype=_np.int64))
        self.K = int(off.shape[0] - 1)
        self.ntot = int(off[-1])
        h = _vp()
        _check(_lib.fsi_batch_create(ctx.handle, self.K, off.ctypes.data_as(C.POINTER(C.c_longlong)),
                                     int(max_steps), C.byref(h)), "fsi_batch_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            _lib.fsi_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fsi_batch_create(ctx: Context, offsets, max_steps: int = 16) -> Batch:
    return Batch(ctx, offsets, max_steps)


def fsi_batch_destroy(batch: Batch) -> None:
    batch.close()


def fsi_batch_step(ctx: Context, batch: Batch, pos, vel, mass, h: float, nsteps: int = 1,
                   stream=None) -> None:
    N = batch.ntot
    _check(_lib.fsi_batch_step(ctx.handle, batch.handle, _f64(pos, (3, N), "pos"),
                               _f64(vel, (3, N), "vel"), _f64(mass, (N,), "mass"), float(h),
                               int(nsteps), _stream(stream)), "fsi_batch_step")


def fsi_batch_set_tuning(ctx: Context, batch: Batch, ipt: int, ctas_per_sm: int = 0) -> None:
    _check(_lib.fsi_batch_set_tuning(ctx.handle, batch.handle, int(ipt), int(ctas_per_sm)),
           "fsi_batch_set_tuning")


def fsi_batch_get_tuning(batch: Batch):
    a, b = _ip(), _ip()
    _check(_lib.fsi_batch_get_tuning(batch.handle, C.byref(a), C.byref(b)), "fsi_batch_get_tuning")
    return int(a.value), int(b.value)


def fsi_batch_stats(batch: Batch, reset: bool = False):
    """(wait_ns, life_ns, ctas) of the batch's launches since the last reset: the CTAs'
    summed waits for other CTAs' phases, their summed lifetimes, CTAs per launch."""
    w, l, n = C.c_longlong(), C.c_longlong(), _ip()
    _check(_lib.fsi_batch_stats(batch.handle, C.byref(w), C.byref(l), C.byref(n), int(bool(reset))),
           "fsi_batch_stats")
    return int(w.value), int(l.value), int(n.value)


def fsi_batch_item_stats(batch: Batch, reset: bool = False):
    """Busy ns and item counts of the symmetric launches' work items by kind: (own-pair sum
    items, two-block sum items, pack / apply items), each a (ns, items) pair."""
    ns = (C.c_longlong * 3)()
    it = (C.c_longlong * 3)()
    _check(_lib.fsi_batch_item_stats(batch.handle, ns, it, int(bool(reset))), "fsi_batch_item_stats")
    return [(int(ns[k]), int(it[k])) for k in range(3)]


def fsi_batch_inject_stall(batch: Batch, cluster: int) -> None:
    _check(_lib.fsi_batch_inject_stall(batch.handle, int(cluster)), "fsi_batch_inject_stall")


def fsi_work_stats(ctx: Context, reset: bool = False):
    """(acc_pairs, grad_pairs): ordered pairs evaluated by this context's pair passes."""
    a, g = C.c_longlong(), C.c_longlong()
    _check(_lib.fsi_work_stats(ctx.handle, C.byref(a), C.byref(g), int(bool(reset))), "fsi_work_stats")
    return int(a.value), int(g.value)


def fsi_far_stats(ctx: Context, reset: bool = False, stream=None):
    """(far_visits, near_visits): (warp, source sub-tile) visits of the symmetric mixed
    far-tile kernel that took the far-tile / the hi-lo separation."""
    f, n = C.c_longlong(), C.c_longlong()
    _check(_lib.fsi_far_stats(ctx.handle, C.byref(f), C.byref(n), int(bool(reset)), _stream(stream)),
           "fsi_far_stats")
    return int(f.value), int(n.value)


def fsi_accel_noalloc(pos, mass, eps2: float = 0.0, out=None, stream=None):
    """FP64 accelerations of all N particles with no context and no device allocation by
    the library (fixed 4 MiB scratch in the library; N <= 32768).  `out` (3, N) must be
    supplied by callers that cannot allocate; otherwise it is created here with torch."""
    N = mass.numel()
    if out is None and pos.is_cuda:
        out = torch.empty((3, N), dtype=torch.float64, device=pos.device)
    # the library launches on the current device: every tensor must live there
    cur = torch.cuda.current_device()
    for name, t in (("pos", pos), ("mass", mass), ("out", out)):
        if not (t is not None and t.is_cuda and t.device.index == cur):
            raise TypeError(f"{name} must be a CUDA tensor on the current device (cuda:{cur})")
    _check(_lib.fsi_accel_noalloc(N, _f64(pos, (3, N), "pos"), _f64(mass, (N,), "mass"),
                                  float(eps2), _f64(out, (3, N), "out"), _stream(stream)),
           "fsi_accel_noalloc")
    return out
