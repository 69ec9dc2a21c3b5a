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

from oracle import oracle as O
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


def _call(lib, g, prm, vertex, A, B, FA, FB, err):
    return lib.qdse_sweep_fp64_noalloc(ctypes.byref(g.c()), ctypes.byref(Q.qdse_params(*prm)),
                                       vertex, 4.0 / 3.0, A.data_ptr(), B.data_ptr(),
                                       FA.data_ptr(), FB.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream, err, len(err))


@pytest.mark.parametrize("n_p,n_theta,mode,vertex", [
    (63, 40, Q.QDSE_STAGGERED, Q.QDSE_VERTEX_BC),   # odd n_p: the middle Gauss-Legendre node x = 0
    (63, 40, Q.QDSE_COLLOCATED, Q.QDSE_VERTEX_RL),  # the rainbow vertex
    (512, 256, Q.QDSE_COLLOCATED, Q.QDSE_VERTEX_BC),  # the largest sizes the scratch admits
    (512, 256, Q.QDSE_STAGGERED, Q.QDSE_VERTEX_BC),
])
def test_noalloc_sweep_equals_context_sweep_at_odd_rainbow_and_largest_sizes(n_p, n_theta, mode,
                                                                             vertex):
    """The on-device grid of the allocation-free sweep (its own Gauss-Legendre construction) and
    the context's host-built grid give the same map: odd n_p, both vertices, both grid modes and the
    largest admitted sizes, to 1e-12."""
    lib = _lib()
    torch.cuda.set_device(0)
    g = Q.Grid(n_p, n_theta, 1e-4, 1e4, mode)
    prm = (0.8, 0.55, 0.03, 0.0)
    rng = np.random.default_rng(n_p + n_theta + 7 * mode + 11 * vertex)
    A = _dev(1 + rng.uniform(0, 1.5, n_p))
    B = _dev(rng.uniform(0.01, 0.8, n_p))
    FA, FB = torch.empty_like(A), torch.empty_like(B)
    err = ctypes.create_string_buffer(256)
    assert _call(lib, g, prm, vertex, A, B, FA, FB, err) == Q.QDSE_OK, err.value
    ctx = Q.Context(g, 1, precision=Q.QDSE_FP64, vertex=vertex)
    RA, RB = torch.empty_like(A), torch.empty_like(B)
    ctx.qdse_residual([prm], A, B, RA, RB)
    torch.cuda.synchronize()
    assert _rel(FA.cpu().numpy(), RA.cpu().numpy()) < 1e-12
    assert _rel(FB.cpu().numpy(), RB.cpu().numpy()) < 1e-12
    ctx.close()


@pytest.mark.parametrize("mode", [Q.QDSE_COLLOCATED, Q.QDSE_STAGGERED])
def test_noalloc_sweep_matches_the_oracle(mode):
    """The allocation-free sweep against the FP64 oracle's sweep directly (not only through the
    context's map), both grid modes, an odd ragged size, to 1e-12."""
    lib = _lib()
    torch.cuda.set_device(0)
    n_p, n_theta = 45, 24
    g = Q.Grid(n_p, n_theta, 1e-4, 1e4, mode)
    prm = (0.93, 0.5, 0.005, 0.0)
    rng = np.random.default_rng(5 + mode)
    a = 1 + rng.uniform(0, 1.5, n_p)
    b = rng.uniform(0.01, 0.8, n_p)
    A, B = _dev(a), _dev(b)
    FA, FB = torch.empty_like(A), torch.empty_like(B)
    err = ctypes.create_string_buffer(256)
    assert _call(lib, g, prm, Q.QDSE_VERTEX_BC, A, B, FA, FB, err) == Q.QDSE_OK, err.value
    pr = O.Problem(n=n_p, n_theta=n_theta, s_min=1e-4, s_max=1e4,
                   grid_mode=O.STAGGERED if mode == Q.QDSE_STAGGERED else O.COLLOCATED,
                   D=prm[0], omega=prm[1], m=prm[2])
    Ao, Bo = O.sweep(pr, a, b)
    torch.cuda.synchronize()
    assert _rel(FA.cpu().numpy(), Ao) < 1e-12
    assert _rel(FB.cpu().numpy(), Bo) < 1e-12


def test_noalloc_sweep_rejects_too_many_angles_and_nonzero_mu():
    lib = _lib()
    err = ctypes.create_string_buffer(256)
    x = torch.ones(64, dtype=torch.float64, device="cuda")
    st = _call(lib, Q.Grid(64, 257), (0.93, 0.5, 0.005, 0.0), Q.QDSE_VERTEX_BC, x, x, x, x, err)
    assert st == Q.QDSE_ERR_ARG and b"n_theta <= 256" in err.value
    st = _call(lib, Q.Grid(64, 32), (0.93, 0.5, 0.005, 0.1), Q.QDSE_VERTEX_BC, x, x, x, x, err)
    assert st == Q.QDSE_ERR_ARG and b"mu must be 0" in err.value
