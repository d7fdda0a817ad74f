"""The allocation-free entry point ozaki2_gemm_noalloc.

It serves callers that cannot allocate device memory while they run (a
memory-capped or custom-allocator setting, or a thread that must not call
cudaMalloc/cudaFree because they synchronise the device): every intermediate
lives in fixed static device arrays of the library.  These tests call it
through the C ABI twice in a row, on different products, and compare each
result with the allocating entry point ozaki2_gemm bit for bit (the tolerance
of every final-result test here).  The file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def ozk():
    from paper_2609_27831_gb300 import build
    build.build()
    import paper_2609_27831_gb300 as pkg
    return pkg


def _noalloc(ozk, A, B, p):
    M, K = A.shape
    N = B.shape[1]
    Cm = ozk.MPMatrix.empty(M, N, p)
    a, b, c = A.desc(), B.desc(), Cm.desc()
    st = ozk.lib().ozaki2_gemm_noalloc(M, N, K, p, C.byref(a), C.byref(b), C.byref(c),
                                       torch.cuda.current_stream().cuda_stream)
    return st, Cm


def test_noalloc_matches_allocating_entry_point_twice(ozk):
    rng = np.random.Generator(np.random.PCG64(4001))
    cases = [(96, 130, 70, 256), (200, 64, 150, 113)]
    outs = []
    for (M, N, K, p) in cases:
        A = ozk.MPMatrix.from_host(synth.mp_matrix(rng, M, K, p, -8, 8))
        B = ozk.MPMatrix.from_host(synth.mp_matrix(rng, K, N, p, -8, 8))
        st, Cn = _noalloc(ozk, A, B, p)
        assert st == 0, ozk._lib.strerror(st)
        outs.append((A, B, Cn, p))
    torch.cuda.synchronize()
    for A, B, Cn, p in outs:
        Ca = ozk.gemm(A, B, p)
        torch.cuda.synchronize()
        for key in ("limbs", "exp", "sign"):
            assert torch.equal(getattr(Cn, key), getattr(Ca, key)), key


def test_noalloc_rejects_products_above_its_scratch(ozk):
    rng = np.random.Generator(np.random.PCG64(4002))
    A = ozk.MPMatrix.from_host(synth.mp_matrix(rng, 1024, 1024, 256, -8, 8))
    B = ozk.MPMatrix.from_host(synth.mp_matrix(rng, 1024, 1024, 256, -8, 8))
    st, _ = _noalloc(ozk, A, B, 256)
    assert st == ozk._lib.OZ2_ERANGE
