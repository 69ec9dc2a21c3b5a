"""Python binding of the finite chemical potential sweep (include/qdse_mu.h): argument marshalling
only.

The arithmetic runs in the CUDA kernels of ``libqdse.so`` (``csrc/k_mu.cu``); PyTorch supplies
device memory and the current stream.  There is no CPU fallback: without the built library or a
CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import qdse as Q

EXPORTS = ("qdse_mu_grid_create", "qdse_mu_grid_create_product", "qdse_mu_solve",
           "qdse_mu_grid_info", "qdse_mu_sweep", "qdse_mu_set_profiling", "qdse_mu_profile",
           "qdse_mu_set_ray_quotient", "qdse_mu_solve_continued", "qdse_mu_grid_destroy",
           "qdse_mu_last_error")

_lib = None


def load_library() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    lib = Q.load_library()
    P = ctypes.POINTER
    vp, ip, dp, llp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, P(ctypes.c_longlong)
    sig = {
        "qdse_mu_grid_create": (ip, [ip, vp, vp, ip, vp, ip, vp, vp, ip, vp, vp, dp, ip, vp,
                                     P(vp)]),
        "qdse_mu_grid_create_product": (ip, [ip, vp, ip, vp, ip, vp, ip, vp, vp, ip, vp, vp, dp,
                                             ip, vp, P(vp)]),
        "qdse_mu_solve": (ip, [vp, vp, ip, vp, dp, dp, dp, ip, dp, dp, dp, ip, vp, vp, vp, vp]),
        "qdse_mu_solve_continued": (ip, [vp, vp, ip, vp, dp, dp, dp, ip, dp, dp, dp, ip, ip, vp,
                                         vp, vp, vp, vp]),
        "qdse_mu_grid_info": (ip, [vp, llp, llp]),
        "qdse_mu_sweep": (ip, [vp, ip, vp, dp, dp, dp, ip, vp, vp, vp, vp]),
        "qdse_mu_set_profiling": (ip, [vp, ip]),
        "qdse_mu_set_ray_quotient": (ip, [vp, dp]),
        "qdse_mu_profile": (ip, [vp, P(dp), P(ctypes.c_longlong)]),
        "qdse_mu_grid_destroy": (None, [vp]),
        "qdse_mu_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _host(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


class MuGrid:
    """Owns a ``qdse_mu_grid``: external points (|p_vec|, p_4), the product grid of internal points
    (q_abs x q4 with weights w_q, row-major [r][f]), the angular rule and omega."""

    def __init__(self, p_abs, p4, q_abs, q4, w_q, z, w_z, omega: float,
                 precision: int = Q.QDSE_FP64, product: bool = False):
        """product=False: p_abs, p4 are the external points [n_ext] (qdse_mu_grid_create).
        product=True: they are the axes [n_pr], [n_p4] of the external product grid
        (qdse_mu_grid_create_product), which qdse_mu_solve needs."""
        self.lib = load_library()
        arrs = [_host(a) for a in (p_abs, p4, q_abs, q4, w_q, z, w_z)]
        self._keep = arrs
        p_abs, p4, q_abs, q4, w_q, z, w_z = arrs
        self.n_r, self.n_4 = len(q_abs), len(q4)
        self.n_int = self.n_r * self.n_4
        self.n_ext = len(p_abs) * len(p4) if product else len(p_abs)
        assert (product or len(p4) == self.n_ext) and w_q.size == self.n_int
        assert len(w_z) == len(z)
        self.precision = precision
        self.ptr = ctypes.c_void_p()
        tail = (self.n_r, q_abs.ctypes.data, self.n_4, q4.ctypes.data, w_q.ctypes.data, len(z),
                z.ctypes.data, w_z.ctypes.data, float(omega), precision, Q._current_stream(),
                ctypes.byref(self.ptr))
        if product:
            st = self.lib.qdse_mu_grid_create_product(len(p_abs), p_abs.ctypes.data, len(p4),
                                                      p4.ctypes.data, *tail)
        else:
            st = self.lib.qdse_mu_grid_create(self.n_ext, p_abs.ctypes.data, p4.ctypes.data, *tail)
        if st != Q.QDSE_OK:
            raise Q.QdseError(st, self.lib.qdse_mu_last_error().decode())

    def solve(self, mu: Sequence[float], D: float, m: float, F, alpha: float = 1.0,
              tol: float = 1e-10, max_iter: int = 500, vertex: int = Q.QDSE_VERTEX_BC,
              cf: float = 4.0 / 3.0, refine: "MuGrid" = None, switch_tol: float = 1e-5):
        """qdse_mu_solve: F (torch.complex128 CUDA [n_mu, 3, n_ext]) holds the start and receives
        the result.  Returns (iters, status) as numpy int32 arrays."""
        import torch
        mu = _host(mu)
        n_mu = len(mu)
        assert F.is_cuda and F.dtype == torch.complex128 and F.is_contiguous()
        assert tuple(F.shape) == (n_mu, 3, self.n_ext)
        iters = np.zeros(n_mu, dtype=np.int32)
        status = np.zeros(n_mu, dtype=np.int32)
        self._raise(self.lib.qdse_mu_solve(self.ptr, refine.ptr if refine is not None else None,
                                           n_mu, mu.ctypes.data, float(D), float(m), float(cf),
                                           vertex, float(alpha), float(tol), float(switch_tol),
                                           int(max_iter), F.data_ptr(), iters.ctypes.data,
                                           status.ctypes.data, Q._current_stream()))
        return iters, status

    def solve_continued(self, mu: Sequence[float], D: float, m: float, F, max_rounds: int = 4,
                        alpha: float = 1.0, tol: float = 1e-10, max_iter: int = 500,
                        vertex: int = Q.QDSE_VERTEX_BC, cf: float = 4.0 / 3.0,
                        refine: "MuGrid" = None, switch_tol: float = 1e-5):
        """qdse_mu_solve_continued: as solve(), then rounds in which each unconverged mu restarts
        from its nearest converged neighbour.  Returns (iters, status, rounds)."""
        import torch
        mu = _host(mu)
        n_mu = len(mu)
        assert F.is_cuda and F.dtype == torch.complex128 and F.is_contiguous()
        assert tuple(F.shape) == (n_mu, 3, self.n_ext)
        iters = np.zeros(n_mu, dtype=np.int32)
        status = np.zeros(n_mu, dtype=np.int32)
        rounds = np.zeros(n_mu, dtype=np.int32)
        self._raise(self.lib.qdse_mu_solve_continued(
            self.ptr, refine.ptr if refine is not None else None, n_mu, mu.ctypes.data, float(D),
            float(m), float(cf), vertex, float(alpha), float(tol), float(switch_tol),
            int(max_iter), int(max_rounds), F.data_ptr(), iters.ctypes.data, status.ctypes.data,
            rounds.ctypes.data, Q._current_stream()))
        return iters, status, rounds

    def info(self) -> dict:
        n, b = ctypes.c_longlong(), ctypes.c_longlong()
        self._raise(self.lib.qdse_mu_grid_info(self.ptr, ctypes.byref(n), ctypes.byref(b)))
        return {"n_pairs": n.value, "table_bytes": b.value}

    def sweep(self, mu: Sequence[float], D: float, m: float, F_ext, F_int, F_out,
              vertex: int = Q.QDSE_VERTEX_BC, cf: float = 4.0 / 3.0):
        """F_ext, F_out: torch.complex128 CUDA tensors [n_mu, 3, n_ext] (A, C, B); F_int:
        [n_mu, 3, n_r * n_4]."""
        import torch
        mu = _host(mu)
        n_mu = len(mu)
        for t, n in ((F_ext, self.n_ext), (F_int, self.n_int), (F_out, self.n_ext)):
            assert t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()
            assert tuple(t.shape) == (n_mu, 3, n), f"expected {(n_mu, 3, n)}, got {tuple(t.shape)}"
        self._raise(self.lib.qdse_mu_sweep(self.ptr, n_mu, mu.ctypes.data, float(D), float(m),
                                           float(cf), vertex, F_ext.data_ptr(), F_int.data_ptr(),
                                           F_out.data_ptr(), Q._current_stream()))

    def set_ray_quotient(self, eta: float):
        """Reading M8 of the BC vertex's difference quotients (include/qdse_mu.h): eta in GeV^2,
        0 turns it off.  Product grids only."""
        self._raise(self.lib.qdse_mu_set_ray_quotient(self.ptr, float(eta)))

    def set_profiling(self, on: bool):
        self._raise(self.lib.qdse_mu_set_profiling(self.ptr, int(bool(on))))

    def profile(self) -> dict:
        """Event-timed milliseconds and launches of the prep and sweep kernels since the last
        read (waits for the last recorded sweep)."""
        ms = (ctypes.c_double * 2)()
        n = (ctypes.c_longlong * 2)()
        self._raise(self.lib.qdse_mu_profile(self.ptr, ms, n))
        return {k: {"ms": ms[i], "launches": n[i]} for i, k in enumerate(("prep", "sweep"))}

    def _raise(self, st: int):
        if st != Q.QDSE_OK:
            raise Q.QdseError(st, self.lib.qdse_mu_last_error().decode())

    def close(self):
        if self.ptr:
            self.lib.qdse_mu_grid_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
