"""Thin ctypes binding of libzeitlin (argument marshalling only).

Every operation runs in the library's CUDA kernels; this module only passes
device pointers, sizes and the current CUDA stream.  Tensors are torch
complex128, contiguous, on a CUDA device (PyTorch supplies device memory and
streams).  There is no CPU fallback: if the shared library is missing or a
call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

ZT_OK = 0
ZT_NOT_CONVERGED = 1
ZT_EINVAL = -1
ZT_ENOMEM = -2
ZT_ECUDA = -3
ZT_ENONFINITE = -4
ZT_ETIMEOUT = -5
PRECISION_FP64 = 0
PRECISION_SPLIT = 1
FINAL_FRESH = 0
FINAL_REUSE = 1
FIRST_EXTRAPOLATED = 0
FIRST_WN = 1
KERNEL_PRODUCT = 0
KERNEL_SOLVE = 1
KERNEL_SPLIT = 2
KERNEL_UPDATE = 3

HEADER = os.path.join(_build.ROOT, "include", "zeitlin.h")


class Tuning(ctypes.Structure):
    _fields_ = [("slices", ctypes.c_int), ("digit_bits", ctypes.c_int), ("exact_groups", ctypes.c_int),
                ("final_mode", ctypes.c_int), ("sweeps_per_sync", ctypes.c_int), ("dense", ctypes.c_int),
                ("tile_order", ctypes.c_int), ("no_persistent", ctypes.c_int), ("wait_us", ctypes.c_int),
                ("debug_stall_loads", ctypes.c_int), ("slices2", ctypes.c_int), ("first_iterate", ctypes.c_int),
                ("second_form", ctypes.c_int)]


class StepStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("residual", ctypes.c_double)]


class RunStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_long), ("total_iters", ctypes.c_long), ("max_iters", ctypes.c_int),
                ("all_converged", ctypes.c_int), ("max_residual", ctypes.c_double)]


class ZeitlinError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libzeitlin status {code}: {msg}")
        self.code = code


_lib = None


def declared_functions() -> list[str]:
    """Names of the functions include/zeitlin.h declares."""
    txt = open(HEADER).read()
    return re.findall(r"^ZT_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt, flags=re.M)


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libzeitlin.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.is_stale():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libzeitlin.so not found at {_build.LIB}; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    vp, i, d, l = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
    L.zt_plan_create.argtypes = [i, i, ctypes.POINTER(Tuning), ctypes.POINTER(vp)]
    L.zt_plan_create.restype = i
    L.zt_plan_destroy.argtypes = [vp]
    L.zt_plan_destroy.restype = None
    L.zt_last_error.argtypes = []
    L.zt_last_error.restype = ctypes.c_char_p
    L.zeitlin_laplacian_apply.argtypes = [vp, vp, vp, vp]
    L.zeitlin_laplacian_apply.restype = i
    L.zeitlin_stream_solve.argtypes = [vp, vp, vp, vp]
    L.zeitlin_stream_solve.restype = i
    L.isomp_step.argtypes = [vp, vp, d, d, i, ctypes.POINTER(StepStats), vp]
    L.isomp_step.restype = i
    L.isomp_run.argtypes = [vp, vp, d, l, d, i, ctypes.POINTER(RunStats), vp]
    L.isomp_run.restype = i
    L.zt_zgemm_skew.argtypes = [vp, vp, vp, vp, vp]
    L.zt_zgemm_skew.restype = i
    L.zeitlin_casimirs.argtypes = [vp, vp, ctypes.POINTER(d), vp]
    L.zeitlin_casimirs.restype = i
    L.zt_basis_create.argtypes = [vp, i, ctypes.POINTER(vp)]
    L.zt_basis_create.restype = i
    L.zt_basis_destroy.argtypes = [vp]
    L.zt_basis_destroy.restype = None
    L.zt_basis_vector.argtypes = [vp, i, i, ctypes.POINTER(d)]
    L.zt_basis_vector.restype = i
    L.zeitlin_w_from_omega.argtypes = [vp, vp, vp, vp]
    L.zeitlin_w_from_omega.restype = i
    L.zeitlin_omega_from_w.argtypes = [vp, vp, vp, vp]
    L.zeitlin_omega_from_w.restype = i
    L.zeitlin_energy_spectrum.argtypes = [vp, vp, vp, vp]
    L.zeitlin_energy_spectrum.restype = i
    L.zt_plan_launch_count.argtypes = [vp]
    L.zt_plan_launch_count.restype = l
    L.zt_plan_reset_history.argtypes = [vp]
    L.zt_plan_reset_history.restype = None
    L.zt_plan_set_timing.argtypes = [vp, i]
    L.zt_plan_set_timing.restype = i
    dp, lp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long)
    L.zt_plan_kernel_time.argtypes = [vp, i, lp, dp, dp, dp]
    L.zt_plan_kernel_time.restype = i
    P = ctypes.POINTER
    L.zt_plan_estimate_bytes.argtypes = [i, i, P(Tuning)]
    L.zt_plan_estimate_bytes.restype = ctypes.c_longlong
    L.zt_batch_create.argtypes = [i, P(vp), P(vp), P(d), P(vp)]
    L.zt_batch_create.restype = i
    L.zt_batch_destroy.argtypes = [vp]
    L.zt_batch_destroy.restype = None
    L.zt_batch_set_graph.argtypes = [vp, i]
    L.zt_batch_set_graph.restype = i
    L.isomp_step_batched.argtypes = [vp, d, i, P(StepStats), vp]
    L.isomp_step_batched.restype = i
    L.isomp_run_batched.argtypes = [vp, l, d, i, P(RunStats), vp]
    L.isomp_run_batched.restype = i
    L.zt_batch_launch_count.argtypes = [vp]
    L.zt_batch_launch_count.restype = l
    _lib = L
    return L


def _check(rc, allow=(ZT_OK,)):
    if rc not in allow:
        raise ZeitlinError(rc, load().zt_last_error().decode())
    return rc


def _ptr(t, N):
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
        raise TypeError("expected a complex128 CUDA tensor")
    if tuple(t.shape) != (N, N) or not t.is_contiguous():
        raise ValueError(f"expected a contiguous ({N}, {N}) tensor, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A zt_plan: constant Laplacian factors plus step workspace for one N."""

    def __init__(self, N: int, precision: int = PRECISION_FP64, slices=0, digit_bits=0,
                 exact_groups=0, final_mode=FINAL_FRESH, sweeps_per_sync=0, dense=0, tile_order=0,
                 no_persistent=0, wait_us=0, debug_stall_loads=0, slices2=0, first_iterate=0, second_form=0):
        L = load()
        self.N = int(N)
        self.precision = precision
        tun = Tuning(slices, digit_bits, exact_groups, final_mode, sweeps_per_sync, 1 if dense else 0,
                     int(tile_order), int(no_persistent), int(wait_us), int(debug_stall_loads), int(slices2),
                     int(first_iterate), int(second_form))
        h = ctypes.c_void_p()
        _check(L.zt_plan_create(self.N, precision, ctypes.byref(tun), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().zt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        return load().zt_plan_launch_count(self._h)

    def reset_history(self):
        """The next step starts from W_n (for callers that rewrite W in place)."""
        load().zt_plan_reset_history(self._h)

    def set_timing(self, enable: bool = True):
        _check(load().zt_plan_set_timing(self._h, 1 if enable else 0))

    def kernel_time(self, kind: int) -> dict:
        n = ctypes.c_long()
        ms, work, alg = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().zt_plan_kernel_time(self._h, kind, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(work),
                                          ctypes.byref(alg)))
        return {"launches": n.value, "total_ms": ms.value, "work": work.value, "work_alg": alg.value}


def zeitlin_laplacian_apply(plan: Plan, P, W, stream=None):
    _check(load().zeitlin_laplacian_apply(plan.handle, _ptr(P, plan.N), _ptr(W, plan.N), _stream(stream)))
    return W


def zeitlin_stream_solve(plan: Plan, W, P, stream=None):
    _check(load().zeitlin_stream_solve(plan.handle, _ptr(W, plan.N), _ptr(P, plan.N), _stream(stream)))
    return P


def isomp_step(plan: Plan, W, h: float, tol: float = 1e-12, maxit: int = 50, stream=None,
               allow_not_converged: bool = False):
    st = StepStats()
    allow = (ZT_OK, ZT_NOT_CONVERGED) if allow_not_converged else (ZT_OK,)
    rc = _check(load().isomp_step(plan.handle, _ptr(W, plan.N), float(h), float(tol), int(maxit),
                                  ctypes.byref(st), _stream(stream)), allow)
    return {"status": rc, "iters": st.iters, "converged": bool(st.converged), "residual": st.residual}


def isomp_run(plan: Plan, W, h: float, nsteps: int, tol: float = 1e-12, maxit: int = 50, stream=None,
              allow_not_converged: bool = False):
    st = RunStats()
    allow = (ZT_OK, ZT_NOT_CONVERGED) if allow_not_converged else (ZT_OK,)
    rc = _check(load().isomp_run(plan.handle, _ptr(W, plan.N), float(h), int(nsteps), float(tol), int(maxit),
                                 ctypes.byref(st), _stream(stream)), allow)
    return {"status": rc, "steps": st.steps, "total_iters": st.total_iters, "max_iters": st.max_iters,
            "all_converged": bool(st.all_converged), "max_residual": st.max_residual}


def zeitlin_casimirs(plan: Plan, W, stream=None) -> dict:
    """Casimirs {k: tr(W^k)} for k = 2..5, computed on the device (waits for the stream)."""
    out = (ctypes.c_double * 8)()
    _check(load().zeitlin_casimirs(plan.handle, _ptr(W, plan.N), out, _stream(stream)))
    return {k: complex(out[2 * (k - 2)], out[2 * (k - 2) + 1]) for k in (2, 3, 4, 5)}


class Basis:
    """Quantised spherical-harmonic basis T^_lm, l <= lmax, on the plan's device."""

    def __init__(self, plan: Plan, lmax: int):
        self.plan = plan
        self.N = plan.N
        self.lmax = int(lmax)
        h = ctypes.c_void_p()
        _check(load().zt_basis_create(plan.handle, self.lmax, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().zt_basis_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vector(self, l: int, m: int):
        """The N - m diagonal entries of T^_lm (0 <= m <= l <= lmax), as a NumPy array."""
        import numpy as np

        out = np.empty(self.N - m, dtype=np.float64)
        _check(load().zt_basis_vector(self._h, int(l), int(m),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out


def _ptr_flat(t, n):
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
        raise TypeError("expected a complex128 CUDA tensor")
    if t.numel() != n or not t.is_contiguous():
        raise ValueError(f"expected a contiguous tensor of {n} entries, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def zeitlin_w_from_omega(basis: Basis, omega, W, stream=None):
    """W = sum i omega_lm T^_lm; omega: (lmax+1)^2 complex128 entries at l*l + l + m."""
    _check(load().zeitlin_w_from_omega(basis.handle, _ptr_flat(omega, (basis.lmax + 1) ** 2), _ptr(W, basis.N),
                                       _stream(stream)))
    return W


def zeitlin_omega_from_w(basis: Basis, W, omega, stream=None):
    """omega_lm = -i tr(T^_lm^H W) for l <= lmax."""
    _check(load().zeitlin_omega_from_w(basis.handle, _ptr(W, basis.N), _ptr_flat(omega, (basis.lmax + 1) ** 2),
                                       _stream(stream)))
    return omega


def zeitlin_energy_spectrum(plan: Plan, W, E=None, stream=None):
    """E_l = sum_m |omega_lm|^2 / (2 l(l+1)), l = 0..N-1 (E_0 = 0), as a float64 CUDA tensor."""
    import torch

    if E is None:
        E = torch.empty(plan.N, dtype=torch.float64, device=W.device)
    if not isinstance(E, torch.Tensor) or E.dtype != torch.float64 or not E.is_cuda or E.numel() != plan.N \
            or not E.is_contiguous():
        raise ValueError(f"E must be a contiguous float64 CUDA tensor of {plan.N} entries")
    _check(load().zeitlin_energy_spectrum(plan.handle, _ptr(W, plan.N), ctypes.c_void_p(E.data_ptr()),
                                          _stream(stream)))
    return E


def zt_zgemm_skew(plan: Plan, X, Y, C, stream=None):
    _check(load().zt_zgemm_skew(plan.handle, _ptr(X, plan.N), _ptr(Y, plan.N), _ptr(C, plan.N),
                                _stream(stream)))
    return C


class Batch:
    """A zt_batch: grouped IsoMP steps over several plans (any mix of N and precision).

    The state tensors are bound for the batch's lifetime; each step advances
    every instance exactly as isomp_step would.
    """

    def __init__(self, plans, Ws, hs):
        L = load()
        if not (len(plans) == len(Ws) == len(hs)) or not plans:
            raise ValueError("plans, Ws and hs must be non-empty and of equal length")
        n = len(plans)
        self.n = n
        self._plans = list(plans)
        self._Ws = list(Ws)
        parr = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
        warr = (ctypes.c_void_p * n)(*[_ptr(W, p.N).value for W, p in zip(Ws, plans)])
        harr = (ctypes.c_double * n)(*[float(h) for h in hs])
        h = ctypes.c_void_p()
        _check(L.zt_batch_create(n, parr, warr, harr, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().zt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_graph(self, enable: bool = True):
        _check(load().zt_batch_set_graph(self._h, 1 if enable else 0))

    def launch_count(self) -> int:
        return load().zt_batch_launch_count(self._h)

    def step(self, tol: float = 1e-12, maxit: int = 50, stream=None, allow_not_converged: bool = False):
        st = (StepStats * self.n)()
        allow = (ZT_OK, ZT_NOT_CONVERGED) if allow_not_converged else (ZT_OK,)
        rc = _check(load().isomp_step_batched(self._h, float(tol), int(maxit), st, _stream(stream)), allow)
        return rc, [{"iters": x.iters, "converged": bool(x.converged), "residual": x.residual} for x in st]

    def run(self, nsteps: int, tol: float = 1e-12, maxit: int = 50, stream=None, allow_not_converged: bool = False):
        st = RunStats()
        allow = (ZT_OK, ZT_NOT_CONVERGED) if allow_not_converged else (ZT_OK,)
        rc = _check(load().isomp_run_batched(self._h, int(nsteps), float(tol), int(maxit), ctypes.byref(st),
                                             _stream(stream)), allow)
        return {"status": rc, "steps": st.steps, "total_iters": st.total_iters, "max_iters": st.max_iters,
                "all_converged": bool(st.all_converged), "max_residual": st.max_residual}


def plan_estimate_bytes(N: int, precision: int = PRECISION_FP64, **tuning) -> int:
    """Device bytes a plan would allocate (library formula)."""
    t = Tuning(tuning.get("slices", 0), tuning.get("digit_bits", 0), tuning.get("exact_groups", 0),
               tuning.get("final_mode", 0), tuning.get("sweeps_per_sync", 0), 1 if tuning.get("dense", 0) else 0,
               tuning.get("tile_order", 0), tuning.get("no_persistent", 0), tuning.get("wait_us", 0),
               tuning.get("debug_stall_loads", 0), tuning.get("slices2", 0), tuning.get("first_iterate", 0),
               tuning.get("second_form", 0))
    v = load().zt_plan_estimate_bytes(int(N), int(precision), ctypes.byref(t))
    if v < 0:
        raise ValueError(f"invalid N={N}")
    return int(v)
