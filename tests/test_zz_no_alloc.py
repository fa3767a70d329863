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


def test_noalloc_rejects_too_large(G):
    n = 11586
    A = torch.zeros(1, 1, dtype=torch.float64, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = G.load().gir_gemv_t_noalloc(ctypes.c_void_p(A.data_ptr()), n, n, ctypes.c_void_p(v.data_ptr()),
                                     ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(0))
    assert st == G.GIR_INVALID_ARG
