"""The allocation-free entry point ozaki2_gemm_noalloc.

It serves callers that cannot allocate device memory while they run (a
memory-capped or custom-allocator setting, or a thread that must not call
cudaMalloc/cudaFree because they synchronise the device): every intermediate
lives in fixed static device arrays of the library.  These tests call it
through the C ABI twice in a row, on different products, and compare each
result with the allocating entry point ozaki2_gemm bit for bit (the tolerance
of every final-result test here) and one of them with the CPU oracle; they
read its status word, check that a call allocates no device memory, and that
a product above its fixed scratch is refused.  The file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import ozaki2_oracle as o

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


def _noalloc(ozk, A, B, p, Cm=None):
    M, K = A.shape
    N = B.shape[1]
    Cm = Cm if Cm is not None else ozk.MPMatrix.empty(M, N, p)
    a, b, c = A.desc(), B.desc(), Cm.desc()
    st = ozk.lib().ozaki2_gemm_noalloc(M, N, K, p, C.byref(a), C.byref(b), C.byref(c),
                                       torch.cuda.current_stream().cuda_stream)
    return st, Cm


def test_noalloc_matches_allocating_entry_point_twice(ozk):
    rng = np.random.Generator(np.random.PCG64(4001))
    cases = [(96, 130, 70, 256), (200, 64, 150, 113)]
    outs = []
    for (M, N, K, p) in cases:
        Ah = synth.mp_matrix(rng, M, K, p, -8, 8)
        Bh = synth.mp_matrix(rng, K, N, p, -8, 8)
        A, B = ozk.MPMatrix.from_host(Ah), ozk.MPMatrix.from_host(Bh)
        st, Cn = _noalloc(ozk, A, B, p)
        assert st == 0, ozk._lib.strerror(st)
        outs.append((Ah, Bh, A, B, Cn, p))
    assert ozk.lib().ozaki2_noalloc_check(torch.cuda.current_stream().cuda_stream) == 0
    for Ah, Bh, A, B, Cn, p in outs:
        Ca = ozk.gemm(A, B, p)
        torch.cuda.synchronize()
        for key in ("limbs", "exp", "sign"):
            assert torch.equal(getattr(Cn, key), getattr(Ca, key)), key
    # the second product against the oracle's stage-by-stage result
    Ah, Bh, _, _, Cn, p = outs[1]
    ref = o.ozaki2_full(Ah, Bh, p)["C"]
    got = Cn.to_host()
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(got[key], ref[key]), key


def test_noalloc_allocates_no_device_memory(ozk):
    """Once both shapes have run (so that every kernel they use is loaded),
    calls of the two shapes in turn leave the device's free memory unchanged
    (inputs and outputs are allocated before)."""
    rng = np.random.Generator(np.random.PCG64(4003))
    A1 = ozk.MPMatrix.from_host(synth.mp_matrix(rng, 64, 80, 200, -8, 8))
    B1 = ozk.MPMatrix.from_host(synth.mp_matrix(rng, 80, 50, 200, -8, 8))
    A2 = ozk.MPMatrix.from_host(synth.mp_matrix(rng, 150, 120, 320, -8, 8))
    B2 = ozk.MPMatrix.from_host(synth.mp_matrix(rng, 120, 90, 320, -8, 8))
    C1 = ozk.MPMatrix.empty(64, 50, 200)
    C2 = ozk.MPMatrix.empty(150, 90, 320)
    for A, B, Cm, p in ((A1, B1, C1, 200), (A2, B2, C2, 320)):
        assert _noalloc(ozk, A, B, p, Cm)[0] == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for A, B, Cm, p in ((A2, B2, C2, 320), (A1, B1, C1, 200), (A2, B2, C2, 320)):
        assert _noalloc(ozk, A, B, p, Cm)[0] == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert ozk.lib().ozaki2_noalloc_check(torch.cuda.current_stream().cuda_stream) == 0


def test_noalloc_rejects_products_above_its_scratch(ozk):
    rng = np.random.Generator(np.random.PCG64(4002))
    A = ozk.MPMatrix.from_host(synth.mp_matrix(rng, 1024, 1024, 256, -8, 8))
    B = ozk.MPMatrix.from_host(synth.mp_matrix(rng, 1024, 1024, 256, -8, 8))
    st, _ = _noalloc(ozk, A, B, 256)
    assert st == ozk._lib.OZ2_ERANGE
