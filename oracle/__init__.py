"""Python access to the plain FP64 CPU oracle (fsi_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the benchmark's
CPU-baseline leg are the only users.  The oracle shares no code with the CUDA library
and must never sit on the product path.

Arrays are numpy FP64 in structure-of-arrays layout: positions and velocities have shape
(3, N).  Index lists are int32 global ids; None means all particles in order.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "fsi_oracle.c"
LIB = HERE / "liboracle.so"

OK = 0
ERR_ARG = -1
ERR_NOMEM = -2
ERR_COINCIDENT = -4
ERR_MAXLEVEL = -6


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc -O2 (no fast-math), OpenMP enabled."""
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", str(tmp), str(SRC), "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


class _HHSParams(C.Structure):
    _fields_ = [("eta_ff", C.c_double), ("eta_fb", C.c_double), ("eta_jerk", C.c_double),
                ("eps2", C.c_double), ("c", C.c_double),
                ("is_bh", C.POINTER(C.c_ubyte)), ("max_level", C.c_int),
                ("fixed_steps", C.POINTER(C.c_double)),
                ("eta_grad", C.c_double), ("eta_va", C.c_double)]


class _StepParams(C.Structure):
    _fields_ = [("eta_ff", C.c_double), ("eta_fb", C.c_double), ("eta_jerk", C.c_double),
                ("eta_grad", C.c_double), ("eta_va", C.c_double)]


class _ForceParams(C.Structure):
    _fields_ = [("eps2", C.c_double), ("c", C.c_double), ("is_bh", C.POINTER(C.c_ubyte))]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(LIB))
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.or_acc.argtypes = [C.c_int, dp, dp, ip, C.c_int, ip, C.c_int, C.c_double, dp]
        L.or_grad.argtypes = [C.c_int, dp, dp, dp, ip, C.c_int, ip, C.c_int, C.c_double, dp]
        L.or_accel_grad.argtypes = [C.c_int, dp, dp, ip, C.c_int, ip, C.c_int, C.c_double,
                                    dp, dp]
        L.or_pn_acc.argtypes = [C.c_int, dp, dp, dp, C.POINTER(C.c_ubyte), C.c_double,
                                ip, C.c_int, ip, C.c_int, dp]
        L.or_energy.argtypes = [C.c_int, dp, dp, dp, ip, C.c_int, C.c_double, dp, dp]
        L.or_fsi_step.argtypes = [C.c_int, dp, dp, dp, ip, C.c_int, C.c_double,
                                  C.POINTER(_ForceParams)]
        L.or_timesteps.argtypes = [C.c_int, dp, dp, dp, ip, C.c_int, C.c_double, C.c_double,
                                   C.c_double, C.c_double, dp]
        L.or_timesteps_all.argtypes = [C.c_int, dp, dp, dp, ip, C.c_int,
                                       C.POINTER(_StepParams), C.c_double, dp]
        L.or_hhs_interval.argtypes = [C.c_int, dp, dp, dp, C.c_double, C.POINTER(_HHSParams),
                                      C.POINTER(C.c_longlong)]
        L.or_hhs_interval_restart.argtypes = [C.c_int, dp, dp, dp, C.c_double,
                                              C.POINTER(_HHSParams), C.c_double, C.c_int,
                                              C.POINTER(C.c_longlong), ip, dp]
        L.or_acc_sub.argtypes = [C.c_int, dp, dp, ip, ip, C.c_int, ip, C.c_int, C.c_double, dp]
        L.or_grad_sub.argtypes = [C.c_int, dp, dp, ip, dp, ip, C.c_int, ip, C.c_int, C.c_double,
                                  dp]
        L.or_fsi_step_sub.argtypes = [C.c_int, dp, dp, dp, ip, ip, C.c_int, ip, C.c_int,
                                      C.c_double, C.c_double]
        L.or_vjp_acc.argtypes = [C.c_int, dp, dp, ip, C.c_int, C.c_double, dp, C.c_double,
                                 C.c_double, dp, dp]
        L.or_vjp_grad.argtypes = [C.c_int, dp, dp, dp, ip, C.c_int, C.c_double, dp, C.c_double,
                                  dp, dp]
        L.or_fsi_step_vjp.argtypes = [C.c_int, dp, dp, dp, ip, C.c_int, C.c_double, C.c_double,
                                      dp, dp, dp, dp, dp]
        L.or_kick_drift.argtypes = [C.c_int, dp, dp, dp, ip, C.c_int, C.c_double, C.c_double]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_get_threads.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _idx(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _n(idx, N):
    return N if idx is None else int(idx.shape[0])


def _check(code, what):
    if code != OK:
        raise OracleError(code, what)


def acc(pos, mass, A=None, B=None, eps2=0.0):
    """acc(A <- B), shape (3, |A|)."""
    pos, mass, A, B = _f64(pos), _f64(mass), _idx(A), _idx(B)
    N = mass.shape[0]
    nA, nB = _n(A, N), _n(B, N)
    out = np.zeros((3, nA))
    _check(lib().or_acc(N, _d(pos), _d(mass), _i(A), nA, _i(B), nB, float(eps2), _d(out)),
           "acc")
    return out


def grad(pos, mass, accg, A=None, B=None, eps2=0.0):
    """Gradient sum G(A <- B) with accelerations accg (3, N) indexed by global id."""
    pos, mass, accg, A, B = _f64(pos), _f64(mass), _f64(accg), _idx(A), _idx(B)
    N = mass.shape[0]
    nA, nB = _n(A, N), _n(B, N)
    out = np.zeros((3, nA))
    _check(lib().or_grad(N, _d(pos), _d(mass), _d(accg), _i(A), nA, _i(B), nB, float(eps2),
                         _d(out)), "grad")
    return out


def accel_grad(pos, mass, A=None, B=None, eps2=0.0):
    """(acc(A <- B), G(A <- B)) of one splitting term; A, B identical or disjoint."""
    pos, mass, A, B = _f64(pos), _f64(mass), _idx(A), _idx(B)
    N = mass.shape[0]
    nA, nB = _n(A, N), _n(B, N)
    a = np.zeros((3, nA))
    g = np.zeros((3, nA))
    _check(lib().or_accel_grad(N, _d(pos), _d(mass), _i(A), nA, _i(B), nB, float(eps2),
                               _d(a), _d(g)), "accel_grad")
    return a, g


def pn_acc(pos, vel, mass, is_bh, c, A=None, B=None):
    pos, vel, mass, A, B = _f64(pos), _f64(vel), _f64(mass), _idx(A), _idx(B)
    bh = np.ascontiguousarray(is_bh, dtype=np.uint8)
    N = mass.shape[0]
    nA, nB = _n(A, N), _n(B, N)
    out = np.zeros((3, nA))
    _check(lib().or_pn_acc(N, _d(pos), _d(vel), _d(mass), bh.ctypes.data_as(C.POINTER(C.c_ubyte)),
                           float(c), _i(A), nA, _i(B), nB, _d(out)), "pn_acc")
    return out


def energy(pos, vel, mass, P=None, eps2=0.0):
    """(kinetic, potential) energy of the listed set."""
    pos, vel, mass, P = _f64(pos), _f64(vel), _f64(mass), _idx(P)
    N = mass.shape[0]
    t, w = C.c_double(), C.c_double()
    _check(lib().or_energy(N, _d(pos), _d(vel), _d(mass), _i(P), _n(P, N), float(eps2),
                           C.byref(t), C.byref(w)), "energy")
    return t.value, w.value


def fsi_step(pos, vel, mass, h, P=None, eps2=0.0, c=0.0, is_bh=None, steps=1):
    """Return (pos, vel) after `steps` FSI cycles of step h on set P (copies)."""
    pos, vel, mass, P = _f64(pos).copy(), _f64(vel).copy(), _f64(mass), _idx(P)
    N = mass.shape[0]
    bh = None
    fp = _ForceParams(float(eps2), float(c), None)
    if c > 0:
        bh = np.ascontiguousarray(is_bh, dtype=np.uint8)
        fp.is_bh = bh.ctypes.data_as(C.POINTER(C.c_ubyte))
    for _ in range(steps):
        _check(lib().or_fsi_step(N, _d(pos), _d(vel), _d(mass), _i(P), _n(P, N), float(h),
                                 C.byref(fp)), "fsi_step")
    return pos, vel


def kick_drift(pos, vel, acc, c_kick, c_drift, P=None):
    """Return (pos, vel) after v_i += c_kick a_k, then x_i += c_drift v_i for i = P[k]
    (copies; acc: 3 x n compact rows or None for a drift only)."""
    pos, vel, P = _f64(pos).copy(), _f64(vel).copy(), _idx(P)
    N = pos.shape[1]
    n = _n(P, N)
    a = None if acc is None else _f64(acc)
    _check(lib().or_kick_drift(N, _d(pos), _d(vel), None if a is None else _d(a), _i(P), n,
                               float(c_kick), float(c_drift)), "kick_drift")
    return pos, vel


def timesteps(pos, vel, mass, P=None, eta_ff=0.2, eta_fb=0.2, eta_jerk=0.1, eps2=0.0,
              eta_grad=0.0, eta_va=0.0):
    """Time steps of the set P against itself (Sect. 3.4): free fall, fly-by and jerk, plus
    the gradient (eta_grad > 0) and velocity-per-acceleration (eta_va > 0) criteria."""
    pos, vel, mass, P = _f64(pos), _f64(vel), _f64(mass), _idx(P)
    N = mass.shape[0]
    n = _n(P, N)
    out = np.zeros(n)
    if eta_grad > 0 or eta_va > 0:
        sp = _StepParams(float(eta_ff), float(eta_fb), float(eta_jerk), float(eta_grad),
                         float(eta_va))
        _check(lib().or_timesteps_all(N, _d(pos), _d(vel), _d(mass), _i(P), n, C.byref(sp),
                                      float(eps2), _d(out)), "timesteps_all")
        return out
    _check(lib().or_timesteps(N, _d(pos), _d(vel), _d(mass), _i(P), n, float(eta_ff),
                              float(eta_fb), float(eta_jerk), float(eps2), _d(out)), "timesteps")
    return out


def hhs_interval(pos, vel, mass, tau, eta_ff=0.2, eta_fb=0.2, eta_jerk=0.1, eps2=0.0,
                 c=0.0, is_bh=None, max_level=40, allow_maxlevel=False, fixed_steps=None,
                 eta_grad=0.0, eta_va=0.0):
    """Return (pos, vel, level_counts, status) after one HHS interval of length tau.

    fixed_steps (N,) forces every particle's time step at every level (a frozen
    hierarchy, for convergence tests); None assigns steps from the criteria.
    """
    pos, vel, mass = _f64(pos).copy(), _f64(vel).copy(), _f64(mass)
    N = mass.shape[0]
    p = _HHSParams(float(eta_ff), float(eta_fb), float(eta_jerk), float(eps2), float(c),
                   None, int(max_level), None, float(eta_grad), float(eta_va))
    fs = None
    if fixed_steps is not None:
        fs = _f64(fixed_steps)
        p.fixed_steps = _d(fs)
    bh = None
    if c > 0:
        bh = np.ascontiguousarray(is_bh, dtype=np.uint8)
        p.is_bh = bh.ctypes.data_as(C.POINTER(C.c_ubyte))
    counts = np.zeros(max_level + 1, dtype=np.int64)
    code = lib().or_hhs_interval(N, _d(pos), _d(vel), _d(mass), float(tau), C.byref(p),
                                 counts.ctypes.data_as(C.POINTER(C.c_longlong)))
    if code != OK and not (allow_maxlevel and code == ERR_MAXLEVEL):
        raise OracleError(code, "hhs_interval")
    return pos, vel, counts, code


def hhs_interval_restart(pos, vel, mass, tau, eta_restart, max_restarts=8, eta_ff=0.2,
                         eta_fb=0.2, eta_jerk=0.1, eps2=0.0, eta_grad=0.0, eta_va=0.0,
                         max_level=40):
    """One HHS interval with adaptive energy-error restarts (Sect. 3.12).
    Returns (pos, vel, level_counts, restarts, rel_err, status)."""
    pos, vel, mass = _f64(pos).copy(), _f64(vel).copy(), _f64(mass)
    N = mass.shape[0]
    p = _HHSParams(float(eta_ff), float(eta_fb), float(eta_jerk), float(eps2), 0.0,
                   None, int(max_level), None, float(eta_grad), float(eta_va))
    counts = np.zeros(max_level + 1, dtype=np.int64)
    k = C.c_int()
    e = C.c_double()
    code = lib().or_hhs_interval_restart(N, _d(pos), _d(vel), _d(mass), float(tau), C.byref(p),
                                         float(eta_restart), int(max_restarts),
                                         counts.ctypes.data_as(C.POINTER(C.c_longlong)),
                                         C.byref(k), C.byref(e))
    if code not in (OK, ERR_MAXLEVEL):
        raise OracleError(code, "hhs_interval_restart")
    return pos, vel, counts, k.value, e.value, code


def subsystem_ids(N, pairs):
    """sub (N,) int32: the pair index of each member of `pairs` ((n_pairs, 2) global ids),
    -1 for single particles."""
    sub = np.full(N, -1, dtype=np.int32)
    for s, (i, j) in enumerate(np.asarray(pairs, dtype=np.int64).reshape(-1, 2)):
        sub[i] = sub[j] = s
    return sub


def acc_sub(pos, mass, pairs, A=None, B=None, eps2=0.0):
    """acc(A <- B) without the pairs inside one subsystem (Algorithm 1)."""
    pos, mass, A, B = _f64(pos), _f64(mass), _idx(A), _idx(B)
    N = mass.shape[0]
    sub = subsystem_ids(N, pairs)
    nA = _n(A, N)
    out = np.zeros((3, nA))
    _check(lib().or_acc_sub(N, _d(pos), _d(mass), _i(sub), _i(A), nA, _i(B), _n(B, N),
                            float(eps2), _d(out)), "acc_sub")
    return out


def grad_sub(pos, mass, pairs, accg, A=None, B=None, eps2=0.0):
    """grad(A <- B) without intra-subsystem pairs; accg (3, N) global-id field."""
    pos, mass, accg, A, B = _f64(pos), _f64(mass), _f64(accg), _idx(A), _idx(B)
    N = mass.shape[0]
    sub = subsystem_ids(N, pairs)
    nA = _n(A, N)
    out = np.zeros((3, nA))
    _check(lib().or_grad_sub(N, _d(pos), _d(mass), _i(sub), _d(accg), _i(A), nA, _i(B),
                             _n(B, N), float(eps2), _d(out)), "grad_sub")
    return out


def fsi_step_sub(pos, vel, mass, pairs, h, P=None, eps2=0.0, steps=1):
    """FSI cycles with binary subsystems (Sect. 2.3, Algorithm 1); returns (pos, vel)."""
    pos, vel, mass, P = _f64(pos).copy(), _f64(vel).copy(), _f64(mass), _idx(P)
    N = mass.shape[0]
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
    sub = subsystem_ids(N, pairs)
    for _ in range(steps):
        _check(lib().or_fsi_step_sub(N, _d(pos), _d(vel), _d(mass), _i(sub), _i(pr),
                                     int(pr.shape[0] // 2), _i(P), _n(P, N), float(h),
                                     float(eps2)), "fsi_step_sub")
    return pos, vel


def vjp_acc(pos, mass, u, P=None, eps2=0.0):
    """(xbar (3, N), mbar (N,)) of the acceleration's VJP with cotangent u (3, N) over P."""
    pos, mass, u, P = _f64(pos), _f64(mass), _f64(u), _idx(P)
    N = mass.shape[0]
    xb = np.zeros((3, N))
    mb = np.zeros(N)
    _check(lib().or_vjp_acc(N, _d(pos), _d(mass), _i(P), _n(P, N), float(eps2), _d(u), 1.0, 1.0,
                            _d(xb), _d(mb)), "vjp_acc")
    return xb, mb


def vjp_grad(pos, mass, acc, w, P=None, eps2=0.0):
    """(xbar, mbar) of the gradient sum's VJP through r and m (a held fixed)."""
    pos, mass, acc, w, P = _f64(pos), _f64(mass), _f64(acc), _f64(w), _idx(P)
    N = mass.shape[0]
    xb = np.zeros((3, N))
    mb = np.zeros(N)
    _check(lib().or_vjp_grad(N, _d(pos), _d(mass), _d(acc), _i(P), _n(P, N), float(eps2), _d(w),
                             1.0, _d(xb), _d(mb)), "vjp_grad")
    return xb, mb


def fsi_step_vjp(pos0, vel0, mass, h, gx_out, gv_out, P=None, eps2=0.0):
    """Cotangents (gx_in, gv_in, gm) of one FSI step's input given the output cotangents."""
    pos0, vel0, mass, P = _f64(pos0), _f64(vel0), _f64(mass), _idx(P)
    gx_out, gv_out = _f64(gx_out), _f64(gv_out)
    N = mass.shape[0]
    gx = np.zeros((3, N))
    gv = np.zeros((3, N))
    gm = np.zeros(N)
    _check(lib().or_fsi_step_vjp(N, _d(pos0), _d(vel0), _d(mass), _i(P), _n(P, N), float(h),
                                 float(eps2), _d(gx_out), _d(gv_out), _d(gx), _d(gv), _d(gm)),
           "fsi_step_vjp")
    return gx, gv, gm
