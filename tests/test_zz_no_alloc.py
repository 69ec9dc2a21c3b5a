"""The allocation-free sweep entry point (qdse_sweep_fp64_noalloc), through the C interface.

Some callers cannot allocate device memory (a fixed arena or pool that owns every byte, or a loop
that must not synchronise the device through cudaMalloc/cudaFree).  This entry point gives them one
FP64 sweep F(x) of a single instance using only their input/output arrays and a scratch array
compiled into the library.  Its output must equal the context-based qdse_residual (FP64) to the
FP64-map tolerance of the parity tests (1e-12 relative), on two calls in a row.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2012_03667_gb300 import build as Bld
from paper_2012_03667_gb300 import qdse as Q

pytestmark = pytest.mark.gpu


def _lib():
    Bld.build()
    lib = Q.load_library()
    f = lib.qdse_sweep_fp64_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(Q.qdse_grid), ctypes.POINTER(Q.qdse_params), ctypes.c_int,
                  ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]
    return lib


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_noalloc_sweep_equals_context_sweep_on_two_calls_in_a_row():
    lib = _lib()
    torch.cuda.set_device(0)
    cases = [(Q.Grid(64, 32, 1e-4, 1e4, Q.QDSE_COLLOCATED), (0.93, 0.5, 0.005, 0.0), 1),
             (Q.Grid(100, 48, 1e-3, 1e3, Q.QDSE_STAGGERED), (0.55, 0.678, 0.02, 0.0), 2)]
    inputs, outputs = [], []
    stream = torch.cuda.current_stream().cuda_stream
    err = ctypes.create_string_buffer(256)
    for g, prm, seed in cases:  # two calls in a row, nothing in between
        rng = np.random.default_rng(seed)
        A = _dev(1 + rng.uniform(0, 1.5, g.n_p))
        B = _dev(rng.uniform(0.01, 0.8, g.n_p))
        FA = torch.empty_like(A)
        FB = torch.empty_like(B)
        st = lib.qdse_sweep_fp64_noalloc(ctypes.byref(g.c()), ctypes.byref(Q.qdse_params(*prm)),
                                         Q.QDSE_VERTEX_BC, 4.0 / 3.0, A.data_ptr(), B.data_ptr(),
                                         FA.data_ptr(), FB.data_ptr(), stream, err, len(err))
        assert st == Q.QDSE_OK, err.value
        inputs.append((A, B))
        outputs.append((FA, FB))
    torch.cuda.synchronize()
    for (g, prm, _), (A, B), (FA, FB) in zip(cases, inputs, outputs):
        ctx = Q.Context(g, 1, precision=Q.QDSE_FP64)
        RA = torch.empty_like(A)
        RB = torch.empty_like(B)
        ctx.qdse_residual([prm], A, B, RA, RB)
        torch.cuda.synchronize()
        assert _rel(FA.cpu().numpy(), RA.cpu().numpy()) < 1e-12
        assert _rel(FB.cpu().numpy(), RB.cpu().numpy()) < 1e-12
        ctx.close()


def test_noalloc_sweep_rejects_sizes_beyond_its_scratch():
    lib = _lib()
    err = ctypes.create_string_buffer(256)
    x = torch.ones(600, dtype=torch.float64, device="cuda")
    g = Q.Grid(600, 32).c()
    st = lib.qdse_sweep_fp64_noalloc(ctypes.byref(g), ctypes.byref(Q.qdse_params(0.93, 0.5, 0.005, 0.0)),
                                     Q.QDSE_VERTEX_BC, 4.0 / 3.0, x.data_ptr(), x.data_ptr(),
                                     x.data_ptr(), x.data_ptr(), None, err, len(err))
    assert st == Q.QDSE_ERR_ARG
    assert b"n_p <= 512" in err.value
