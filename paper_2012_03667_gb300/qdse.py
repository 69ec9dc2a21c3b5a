"""Python binding of libqdse (include/qdse.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all arithmetic of the solver
runs in the CUDA kernels of ``libqdse.so``.  PyTorch supplies device memory (tensors' data_ptr())
and the current CUDA stream.  There is no CPU fallback: if the library has not been built, or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqdse.so")

QDSE_OK, QDSE_ERR_ARG, QDSE_ERR_CUDA, QDSE_ERR_OOM = 0, 1, 2, 3
QDSE_ERR_NOT_CONVERGED, QDSE_ERR_NONFINITE, QDSE_ERR_TIMEOUT, QDSE_ERR_UNSUPPORTED = 4, 5, 6, 7
QDSE_COLLOCATED, QDSE_STAGGERED = 0, 1
QDSE_VERTEX_BC, QDSE_VERTEX_RL = 0, 1
QDSE_FP64, QDSE_MIXED, QDSE_FP64_PRE, QDSE_FP32 = 0, 1, 2, 3
STATUS_NAMES = {0: "ok", 1: "bad argument", 2: "cuda error", 3: "out of memory",
                4: "not converged", 5: "non-finite", 6: "timeout", 7: "unsupported"}

# Every symbol include/qdse.h declares (checked by the test-suite).
EXPORTS = ("qdse_default_options", "qdse_create", "qdse_create_ragged", "qdse_destroy",
           "qdse_last_error", "qdse_sizes", "qdse_layout", "qdse_grid_nodes", "qdse_set_options",
           "qdse_iterate", "qdse_solve", "qdse_solve_host", "qdse_residual", "qdse_jvp",
           "qdse_vjp", "qdse_adjoint", "qdse_condensate", "qdse_condensate_vjp",
           "qdse_last_stats", "qdse_last_work", "qdse_last_instance_stats",
           "qdse_set_profiling", "qdse_profile", "qdse_autotune", "qdse_sweep_fp64_noalloc")


class qdse_grid(ctypes.Structure):
    _fields_ = [("n_p", ctypes.c_int), ("n_theta", ctypes.c_int), ("s_min", ctypes.c_double),
                ("s_max", ctypes.c_double), ("grid_mode", ctypes.c_int)]


class qdse_params(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("omega", ctypes.c_double), ("m", ctypes.c_double),
                ("mu", ctypes.c_double)]


class qdse_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("vertex", ctypes.c_int), ("cf", ctypes.c_double),
                ("tol", ctypes.c_double), ("alpha", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("time_limit", ctypes.c_double), ("reuse_kernels", ctypes.c_int),
                ("stall_window", ctypes.c_int), ("stop_cycles", ctypes.c_int),
                ("shared_kernels", ctypes.c_int), ("stream", ctypes.c_void_p)]


class QdseError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libqdse.so (built by ``paper_2012_03667_gb300.build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libqdse.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    ctx_pp = P(vp)
    sig = {
        "qdse_default_options": (qdse_options, []),
        "qdse_create": (ip, [P(qdse_grid), ip, P(qdse_options), ctx_pp]),
        "qdse_create_ragged": (ip, [P(qdse_grid), ip, P(qdse_options), ctx_pp]),
        "qdse_destroy": (None, [vp]),
        "qdse_last_error": (ctypes.c_char_p, [vp]),
        "qdse_sizes": (ip, [vp, P(ip), P(ip)]),
        "qdse_layout": (ip, [vp, vp]),
        "qdse_grid_nodes": (ip, [vp, vp, vp, vp]),
        "qdse_set_options": (ip, [vp, P(qdse_options)]),
        "qdse_iterate": (ip, [vp, P(qdse_params), vp, vp, ip, vp]),
        "qdse_solve": (ip, [vp, P(qdse_params), vp, vp, vp, vp]),
        "qdse_solve_host": (ip, [vp, P(qdse_params), vp, vp, vp, vp]),
        "qdse_residual": (ip, [vp, P(qdse_params), vp, vp, vp, vp, vp]),
        "qdse_jvp": (ip, [vp, P(qdse_params), vp, vp, vp, vp, vp, vp]),
        "qdse_vjp": (ip, [vp, P(qdse_params), vp, vp, vp, vp, vp, vp]),
        "qdse_adjoint": (ip, [vp, P(qdse_params), vp, vp, vp, vp, vp, vp, vp]),
        "qdse_condensate": (ip, [vp, vp, vp, vp]),
        "qdse_condensate_vjp": (ip, [vp, vp, vp, vp, vp, vp]),
        "qdse_last_stats": (ip, [vp, P(ctypes.c_longlong), P(ctypes.c_longlong),
                                 P(ctypes.c_longlong), P(ctypes.c_longlong)]),
        "qdse_last_work": (ip, [vp, P(dp), P(dp)]),
        "qdse_last_instance_stats": (ip, [vp, vp, vp]),
        "qdse_set_profiling": (ip, [vp, ip]),
        "qdse_profile": (ip, [vp, P(dp), P(ctypes.c_longlong)]),
        "qdse_autotune": (ip, [vp, vp, vp, vp, ip, P(ip), P(dp)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(t) -> Optional[int]:
    """Device (torch CUDA tensor) or host (numpy / torch CPU tensor) pointer, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous(), "arrays passed to libqdse must be contiguous"
    return t.data_ptr()


def _check_dev(t, dtype_name: str):
    import torch
    assert t.is_cuda, "device array expected (torch CUDA tensor)"
    assert t.dtype == getattr(torch, dtype_name), f"{dtype_name} array expected, got {t.dtype}"
    assert t.is_contiguous()


def _current_stream() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


def qdse_default_options() -> qdse_options:
    return load_library().qdse_default_options()


def make_params(rows) -> ctypes.Array:
    """Host array of qdse_params from an iterable of (D, omega, m[, mu]) or an (n, 3|4) array."""
    rows = np.asarray(rows, dtype=np.float64)
    if rows.ndim == 1:
        rows = rows[None, :]
    arr = (qdse_params * len(rows))()
    for b, r in enumerate(rows):
        arr[b] = qdse_params(r[0], r[1], r[2], r[3] if len(r) > 3 else 0.0)
    return arr


@dataclass
class Grid:
    """Radial/angular grid of one instance (include/qdse.h: qdse_grid)."""
    n_p: int = 64
    n_theta: int = 32
    s_min: float = 1e-4
    s_max: float = 1e4
    grid_mode: int = QDSE_COLLOCATED

    def c(self) -> qdse_grid:
        return qdse_grid(self.n_p, self.n_theta, self.s_min, self.s_max, self.grid_mode)


class Context:
    """Owns a ``qdse_ctx``; every method marshals arguments into the C call of the same name."""

    def __init__(self, grid, n_inst: int = 1, precision: int = QDSE_MIXED,
                 vertex: int = QDSE_VERTEX_BC, cf: float = 4.0 / 3.0, tol: float = 1e-10,
                 alpha: float = 1.0, max_iter: int = 20000, time_limit: float = 0.0,
                 reuse_kernels: int = 0, stall_window: int = 0, stop_cycles: int = 1,
                 shared_kernels: int = 0):
        self.lib = load_library()
        self.ptr = ctypes.c_void_p()
        o = self.lib.qdse_default_options()
        o.precision, o.vertex, o.cf, o.tol, o.alpha = precision, vertex, cf, tol, alpha
        o.max_iter, o.time_limit, o.reuse_kernels = max_iter, time_limit, reuse_kernels
        o.stall_window, o.stop_cycles = stall_window, stop_cycles
        o.shared_kernels = shared_kernels
        try:
            o.stream = _current_stream()
        except Exception:
            o.stream = None
        self.options = o
        if isinstance(grid, (list, tuple)):
            n_inst = len(grid)
            arr = (qdse_grid * n_inst)(*[g.c() for g in grid])
            st = self.lib.qdse_create_ragged(arr, n_inst, ctypes.byref(o), ctypes.byref(self.ptr))
        else:
            g = grid.c()
            st = self.lib.qdse_create(ctypes.byref(g), n_inst, ctypes.byref(o),
                                      ctypes.byref(self.ptr))
        if st != QDSE_OK:
            raise QdseError(st, self.lib.qdse_last_error(None).decode())
        ni, nt = ctypes.c_int(), ctypes.c_int()
        self.lib.qdse_sizes(self.ptr, ctypes.byref(ni), ctypes.byref(nt))
        self.n_inst, self.n_total = ni.value, nt.value

    # -- lifetime ---------------------------------------------------------------------------
    def close(self):
        if self.ptr:
            self.lib.qdse_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st: int):
        if st != QDSE_OK:
            raise QdseError(st, self.lib.qdse_last_error(self.ptr).decode())

    def _sync_stream(self):
        s = _current_stream()
        if self.options.stream != s:
            self.options.stream = s
            self._raise(self.lib.qdse_set_options(self.ptr, ctypes.byref(self.options)))

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        self._raise(self.lib.qdse_set_options(self.ptr, ctypes.byref(self.options)))

    # -- layout ------------------------------------------------------------------------------
    def layout(self) -> np.ndarray:
        x = np.zeros(self.n_inst + 1, dtype=np.int32)
        self._raise(self.lib.qdse_layout(self.ptr, x.ctypes.data))
        return x

    def grid_nodes(self):
        sp, sq, W = (np.zeros(self.n_total) for _ in range(3))
        self._raise(self.lib.qdse_grid_nodes(self.ptr, sp.ctypes.data, sq.ctypes.data,
                                             W.ctypes.data))
        return sp, sq, W

    # -- solver entry points -------------------------------------------------------------------
    def qdse_iterate(self, params, A, B, n_sweeps: int, max_rel_change=None):
        self._sync_stream()
        self._raise(self.lib.qdse_iterate(self.ptr, make_params(params), _ptr(A), _ptr(B),
                                          n_sweeps, _ptr(max_rel_change)))

    def qdse_solve(self, params, A, B, iters=None, inst_status=None):
        self._sync_stream()
        self._raise(self.lib.qdse_solve(self.ptr, make_params(params), _ptr(A), _ptr(B),
                                        _ptr(iters), _ptr(inst_status)))

    def qdse_solve_host(self, params, A: np.ndarray, B: np.ndarray, iters=None, inst_status=None):
        self._sync_stream()
        st = self.lib.qdse_solve_host(self.ptr, make_params(params), _ptr(A), _ptr(B),
                                      _ptr(iters), _ptr(inst_status))
        self._raise(st)

    def qdse_residual(self, params, A, B, FA=None, FB=None, rel_res=None):
        self._sync_stream()
        self._raise(self.lib.qdse_residual(self.ptr, make_params(params), _ptr(A), _ptr(B),
                                           _ptr(FA), _ptr(FB), _ptr(rel_res)))

    def qdse_jvp(self, params, A, B, vA, vB, JvA, JvB):
        self._sync_stream()
        self._raise(self.lib.qdse_jvp(self.ptr, make_params(params), _ptr(A), _ptr(B), _ptr(vA),
                                      _ptr(vB), _ptr(JvA), _ptr(JvB)))

    def qdse_vjp(self, params, A, B, wA, wB, JtA, JtB):
        self._sync_stream()
        self._raise(self.lib.qdse_vjp(self.ptr, make_params(params), _ptr(A), _ptr(B), _ptr(wA),
                                      _ptr(wB), _ptr(JtA), _ptr(JtB)))

    def qdse_adjoint(self, params, A, B, gA, gB, g_params, lambda_out=None, inst_status=None):
        self._sync_stream()
        self._raise(self.lib.qdse_adjoint(self.ptr, make_params(params), _ptr(A), _ptr(B),
                                          _ptr(gA), _ptr(gB), _ptr(g_params), _ptr(lambda_out),
                                          _ptr(inst_status)))

    def qdse_condensate(self, A, B, out):
        self._sync_stream()
        self._raise(self.lib.qdse_condensate(self.ptr, _ptr(A), _ptr(B), _ptr(out)))

    def qdse_condensate_vjp(self, A, B, cbar, gA, gB):
        self._sync_stream()
        self._raise(self.lib.qdse_condensate_vjp(self.ptr, _ptr(A), _ptr(B), _ptr(cbar), _ptr(gA),
                                                 _ptr(gB)))

    def qdse_last_work(self) -> dict:
        b, e = ctypes.c_double(), ctypes.c_double()
        self._raise(self.lib.qdse_last_work(self.ptr, ctypes.byref(b), ctypes.byref(e)))
        return {"sweep_bytes": b.value, "kernel_evals": e.value}

    def qdse_last_instance_stats(self) -> dict:
        """Per-instance record of the last solve: FP32 and FP64 sweeps, the longest run of
        Picard sweeps without a new lowest change, kernel entries per plane, final phase, and the
        period of a cycle the cycle stop found with the sweep that found it."""
        out = np.zeros((self.n_inst, 5), dtype=np.int64)
        cyc = np.zeros((self.n_inst, 2), dtype=np.int64)
        self._raise(self.lib.qdse_last_instance_stats(self.ptr, out.ctypes.data, cyc.ctypes.data))
        return {"fp32_sweeps": out[:, 0], "fp64_sweeps": out[:, 1], "longest_stall": out[:, 2],
                "nnz": out[:, 3], "phase": out[:, 4], "cycle_period": cyc[:, 0],
                "cycle_found_at": cyc[:, 1]}

    def qdse_set_profiling(self, on: bool):
        self._raise(self.lib.qdse_set_profiling(self.ptr, int(bool(on))))

    SWEEP_KERNELS = ("ring 12x2", "ring 8x3", "ring 6x4", "slab", "register-only groups")

    def qdse_autotune(self, params, A, B, max_sweeps: int = 0):
        """qdse_autotune: solve the batch once from the start A, B (not modified) with each of the
        five FP32 sweep kernels (sweeps capped at max_sweeps when > 0) and keep the fastest.
        Returns (index, solve ms per candidate)."""
        self._sync_stream()
        choice = ctypes.c_int(-1)
        ms = (ctypes.c_double * 5)()
        self._raise(self.lib.qdse_autotune(self.ptr, make_params(params), _ptr(A), _ptr(B),
                                           int(max_sweeps), ctypes.byref(choice), ms))
        return choice.value, list(ms)

    def qdse_profile(self) -> dict:
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_longlong * 4)()
        self._raise(self.lib.qdse_profile(self.ptr, ms, n))
        names = ("precompute", "sweep", "update", "other")
        return {k: {"ms": ms[i], "launches": n[i]} for i, k in enumerate(names)}

    def qdse_last_stats(self) -> dict:
        v = [ctypes.c_longlong() for _ in range(4)]
        self._raise(self.lib.qdse_last_stats(self.ptr, *[ctypes.byref(x) for x in v]))
        return dict(zip(("kernel_launches", "fp32_sweeps", "fp64_sweeps", "polls"),
                        [x.value for x in v]))
