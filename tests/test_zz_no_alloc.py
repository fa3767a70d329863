"""The allocation-free transposed product gir_gemv_t_noalloc against gir_gemv(trans = 1).

Some callers cannot let the library allocate device memory when they call it (an allocator
that forbids cudaMalloc in a hot loop, a real-time loop, a fixed memory budget); this entry
point takes its scratch from a fixed array in the library instead. This file is collected
last so that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2201_09827_gb300 import gir
    gir.load()
    return gir


def _noalloc(G, A, v):
    w = torch.full_like(v, np.nan)
    st = G.load().gir_gemv_t_noalloc(ctypes.c_void_p(A.data_ptr()), A.shape[0], A.stride(0),
                                     ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, w


def test_noalloc_matches_allocating_entry_point_twice(G):
    rng = np.random.default_rng(42)
    # two calls in a row with different sizes: the shared fixed scratch must not leak state
    for n, lda in ((1000, 1000), (777, 800)):
        Af = rng.standard_normal((n, lda))
        A = torch.from_numpy(Af).cuda()[:, :n]
        v = torch.from_numpy(rng.standard_normal(n)).cuda()
        st, w = _noalloc(G, A, v)
        assert st == G.GIR_OK
        ref = G.gemv(A, v, trans=True)
        bound = 2 * n * 2.0 ** -53 * (A.abs().t() @ v.abs())
        assert bool(((w - ref).abs() <= bound + 1e-300).all())


def test_noalloc_allocates_nothing(G):
    """A call after the first (which looks up the fixed array's address) leaves the device's free
    memory unchanged: the library takes no device memory in it."""
    rng = np.random.default_rng(7)
    n = 2048
    A = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    v = torch.from_numpy(rng.standard_normal(n)).cuda()
    w = torch.empty_like(v)
    lib = G.load()
    args = (ctypes.c_void_p(A.data_ptr()), n, n, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(w.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert lib.gir_gemv_t_noalloc(*args) == G.GIR_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.gir_gemv_t_noalloc(*args) == G.GIR_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref = G.gemv(A, v, trans=True)
    assert bool(((w - ref).abs() <= 2 * n * 2.0 ** -53 * (A.abs().t() @ v.abs()) + 1e-300).all())


def test_noalloc_size_limit_boundary(G):
    """n = 11520 is the largest order whose partial sums (ceil(n / 256) * n doubles) fit the 2^19
    doubles of the fixed array: it runs and matches gir_gemv(trans = 1); n = 11521 is rejected."""
    n = 11520
    g = torch.Generator(device="cuda")
    g.manual_seed(11520)
    A = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g)
    v = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    st, w = _noalloc(G, A, v)
    assert st == G.GIR_OK
    ref = G.gemv(A, v, trans=True)
    bound = 2 * n * 2.0 ** -53 * (A.abs().t() @ v.abs())
    assert bool(((w - ref).abs() <= bound + 1e-300).all())
    del A
    torch.cuda.empty_cache()
    n = 11521
    A = torch.zeros(1, 1, dtype=torch.float64, device="cuda")
    st = G.load().gir_gemv_t_noalloc(ctypes.c_void_p(A.data_ptr()), n, n, ctypes.c_void_p(v.data_ptr()),
                                     ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(0))
    assert st == G.GIR_INVALID_ARG
