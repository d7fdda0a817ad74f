"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and
its host-side planner (t, modulus prefix, CRT tables) agrees with the oracle.
No GPU is needed: only host-only entry points are called."""
import ctypes as C
import os
import re

import pytest

from oracle import ozaki2_oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ozk():
    from paper_2609_27831_gb300 import build
    build.build()
    import paper_2609_27831_gb300 as pkg
    return pkg


def _declared():
    with open(os.path.join(ROOT, "include", "ozaki2.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"OZ2_API\s+(?:const\s+char\s*\*|int)\s+(ozaki2_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol(ozk):
    names = _declared()
    assert len(names) >= 20
    h = C.CDLL(ozk._lib.LIB_PATH)
    for n in names:
        assert hasattr(h, n), n
    # and the binding knows all of them
    assert set(names) <= set(ozk._lib._SIGS)


def test_strerror_and_defaults(ozk):
    lib = ozk.lib()
    for st in range(8):
        assert lib.ozaki2_strerror(st)
    o_ = ozk.opts()
    assert o_.guard_bits == 16 and o_.engine == 0 and o_.schedule == 0
    assert lib.ozaki2_version().startswith(b"ozaki2")


@pytest.mark.parametrize("M,N,K,p", [(256, 256, 256, 53), (1024, 1024, 1024, 256), (100, 70, 4096, 1024),
                                     (64, 64, 4096, 2048), (3, 5, 1, 2), (4096, 4096, 4096, 53)])
def test_plan_parameters_match_oracle(ozk, M, N, K, p):
    plan = ozk.Plan((M, N, K, p))
    par = o.Params(K, p)
    assert plan.info["t"] == par.t
    assert plan.info["L"] == par.L
    assert plan.info["G"] == par.G
    assert plan.info["L1"] == sum(1 for m in par.moduli if m <= 255)
    assert plan.moduli() == par.moduli
    D = plan.info["crt_digits"]
    assert D == -(-par.tab.P.bit_length() // 32) + 2
    P, Md, inv = plan.crt_tables()
    as_int = lambda ds: sum(int(d) << (32 * i) for i, d in enumerate(ds))
    assert as_int(P) == par.tab.P
    assert [as_int(r) for r in Md] == par.tab.M
    assert inv == par.tab.Minv
    assert plan.workspace_bytes > 0
    off, kp = plan.layout()
    assert kp % 8 == 0 and kp >= K and all(x % 256 == 0 for x in off)


def test_moduli_table_through_the_library(ozk):
    """The library's planner reproduces the paper's moduli table (Sec. 4.3)."""
    import json
    with open(os.path.join(ROOT, "tests", "golden", "moduli_table.json")) as fh:
        g = json.load(fh)
    for row in g["rows"]:
        plan = ozk.Plan((8, 8, g["K"], row["p"]))
        assert (plan.info["t"], plan.info["L"], plan.info["G"]) == (row["t"], row["L"], row["gemms"])


def test_batched_plan(ozk):
    shapes = [(100, 200, 300, 113), (64, 64, 64, 512), (2048, 128, 1000, 256)]
    plan = ozk.Plan(shapes)
    assert plan.info["count"] == 3
    for i, (M, N, K, p) in enumerate(shapes):
        assert plan.moduli(i)[: o.Params(K, p).L] == o.Params(K, p).moduli


@pytest.mark.parametrize("args,status", [
    ((0, 4, 4, 53), 1), ((4, 4, 4, 1), 1), ((4, -1, 4, 53), 1),
    ((4, 4, 133001, 53), 2), ((4, 4, 4, 4096), 2),
])
def test_argument_errors(ozk, args, status):
    h = C.c_void_p()
    st = ozk.lib().ozaki2_plan_create(*args, None, C.byref(h))
    assert st == status and not h.value


def test_bad_options(ozk):
    h = C.c_void_p()
    for kw in ({"k_chunk": 100}, {"k_chunk": 2048}, {"engine": 7}, {"schedule": 9}, {"crt_engine": 4},
               {"crt_engine": -1}, {"res_engine": 4}):
        st = ozk.lib().ozaki2_plan_create(64, 64, 64, 53, C.byref(ozk.opts(**kw)), C.byref(h))
        assert st == 1, kw


def test_null_pointer_errors(ozk):
    lib = ozk.lib()
    assert lib.ozaki2_plan_create(4, 4, 4, 53, None, None) == 1
    assert lib.ozaki2_plan_destroy(None) == 1
    assert lib.ozaki2_execute(None, None, None, None, None, 0, None) == 1
    assert lib.ozaki2_check(None, None) == 1
    assert lib.ozaki2_cache_destroy(None) == 1
    assert lib.ozaki2_dgemm_bwd(None, None, 0, None, 0, None, 0, None) == 1


@pytest.mark.parametrize("p, cw_want", [(1024, 160), (2048, 160)])
def test_crt_sum_engine_workspace(ozk, p, cw_want):
    """crt_engine 2 adds the group sums ([groups of 32 columns formed][9][M N
    rounded to 8] uint32) and the quotient estimates ([M N rounded to 8]
    uint32) to the workspace where it applies, and nothing where it does not.  The table
    has np 7-bit pieces of P and five quotient columns, padded to groups of 32;
    the chunk width: two TMEM slots beside V (kpad / 2 of 512 columns) unless
    that makes them narrower than 128 columns, then one slot."""
    shape = (256, 256, 64, p)
    base = ozk.Plan(shape, crt_engine=3).info
    plan = ozk.Plan(shape, crt_engine=2)
    P = 1
    for m in plan.moduli():
        P *= m
    L = plan.info["L"]
    kpad = -(-2 * L // 64) * 64
    np_ = -(-P.bit_length() // 7) + 1
    npad = -(-(np_ + 5) // 32) * 32
    need = npad
    cw = min(256, ((512 - kpad // 2) // 2) // 32 * 32)
    if cw < 128 and cw < need:
        cw = min(256, (512 - kpad // 2) // 32 * 32)
    cw = min(cw, need)
    assert cw == cw_want
    # the long finish (more than 24 digits) reads the group sums from group
    # g0 - 1 on in its fast form (g0: the group just below its window of the
    # 2 nl + 4 highest digits); the sums below are not formed
    D, nl = plan.info["crt_digits"], -(-p // 64)
    W = 2 * nl + 4
    wbase = D - W if D > W else 0
    g0 = (wbase - 1) // 7 if wbase > 7 else 0
    gskip = g0 - 1 if D > 24 and g0 >= 2 else 0
    assert gskip > 0 and plan.info["crt_skip_groups"] == gskip
    ngrp, up = -(-(npad - 32 * gskip) // cw) * cw // 32, 256 * 256
    a256 = lambda x: -(-x // 256) * 256
    assert plan.info["workspace_bytes"] - base["workspace_bytes"] == a256(4 * ngrp * 9 * up) + a256(4 * up)
    small = (4, 4, 4, 53)                        # M N < 128: the CUDA-core CRT
    assert ozk.Plan(small, crt_engine=2).info["workspace_bytes"] == ozk.Plan(small, crt_engine=3).info["workspace_bytes"]


def test_crt_engine_choice(ozk):
    """The automatic CRT choice: tensor-core sums where the accumulator needs
    more than 20 digits; engine 3 keeps the CUDA cores; engine 2 asks for the
    sums wherever the shape qualifies (L >= 32, M N >= 128)."""
    lo, mid, hi = (64, 64, 64, 200), (64, 64, 64, 384), (64, 64, 64, 1024)
    assert ozk.Plan(lo).info["crt_digits"] <= 20 and ozk.Plan(lo).info["crt_mode"] == 0
    assert ozk.Plan((1024, 1024, 1024, 256)).info["crt_digits"] == 21
    assert ozk.Plan((1024, 1024, 1024, 256)).info["crt_mode"] == 2
    assert ozk.Plan(mid).info["crt_digits"] > 20 and ozk.Plan(mid).info["crt_mode"] == 2
    assert ozk.Plan(hi).info["crt_digits"] > 40 and ozk.Plan(hi).info["crt_mode"] == 2
    assert ozk.Plan(hi, crt_engine=3).info["crt_mode"] == 0
    assert ozk.Plan(lo, crt_engine=2).info["crt_mode"] == 2
    assert ozk.Plan((8, 8, 64, 1024)).info["crt_mode"] == 0          # M N < 128
    assert ozk.Plan((64, 64, 64, 53), crt_engine=2).info["crt_mode"] == 0   # L < 32


def test_residue_engine_choice(ozk):
    """The automatic residue choice: the warp-specialised tensor-core kernel for
    integers of more than 72 bytes (t + 1 bits), the CUDA cores below; engine 3
    forces the CUDA cores, engine 2 asks for the tensor cores up to 448 bytes."""
    assert ozk.Plan((64, 64, 64, 2048)).info["res_mode"] == 2
    assert ozk.Plan((64, 64, 64, 1024)).info["res_mode"] == 2
    t = ozk.Plan((64, 64, 64, 553)).info["t"]
    assert -(-(t + 1) // 8) == 72 and ozk.Plan((64, 64, 64, 553)).info["res_mode"] == 0
    t = ozk.Plan((64, 64, 64, 554)).info["t"]
    assert -(-(t + 1) // 8) == 73 and ozk.Plan((64, 64, 64, 554)).info["res_mode"] == 2
    assert ozk.Plan((64, 64, 64, 512)).info["res_mode"] == 0
    assert ozk.Plan((64, 64, 64, 2048), res_engine=3).info["res_mode"] == 0
    assert ozk.Plan((64, 64, 64, 256), res_engine=2).info["res_mode"] == 2


def test_planes_streamed_in_modulus_groups(ozk):
    """Large products stream their residue planes through the workspace in
    groups of consecutive moduli: one group's bf16 plane stacks at a time
    (at most 32 GiB automatically, or opts.plane_group planes), the reduced
    products and the CRT of every modulus kept whole."""
    big = (4096, 4096, 4096, 2048)
    whole = ozk.Plan(big, plane_group=-1).info
    auto = ozk.Plan(big).info
    G, L = whole["G"], whole["L"]
    assert whole["plane_groups"] == 1 and whole["group_planes"] == G == 879
    per_plane = 2 * (4096 + 4096) * 4096
    assert auto["plane_groups"] == 2 and auto["group_planes"] * per_plane <= 32 << 30
    # the workspace shrinks by the planes no longer resident
    assert whole["workspace_bytes"] - auto["workspace_bytes"] == (G - auto["group_planes"]) * per_plane
    # explicit group sizes: about equal groups, each at most the request
    for req in (3, 64, 300, 878):
        inf = ozk.Plan(big, plane_group=req).info
        assert inf["group_planes"] <= req
        assert inf["plane_groups"] in (-(-G // req), -(-G // req) + 1)
        assert inf["t"] == whole["t"] and inf["L"] == L and inf["crt_digits"] == whole["crt_digits"]
    assert ozk.Plan(big, plane_group=879).info["plane_groups"] == 1
    # small products stay in one group unless asked
    assert ozk.Plan((1024, 1024, 1024, 256)).info["plane_groups"] == 1
    assert ozk.Plan((200, 150, 300, 256), plane_group=20).info["plane_groups"] > 1
    # batched plans and the binary64 mode never stream
    assert ozk.Plan([(200, 150, 300, 256), (64, 64, 64, 53)], plane_group=20).info["plane_groups"] == 1


def test_automatic_groups_take_the_fewest_residue_chunks(ozk):
    """Among the group boundaries that give the fewest groups within the plane
    budget, the automatic split takes the one whose groups need the fewest
    tensor-core residue chunks (96 table columns each at p = 2048): 4096^3
    at p = 2048 splits its 54 one-limb and 275 two-limb moduli as 54 + 131
    and 144 (447 + 432 planes, 4 + 3 chunks) rather than in equal halves
    (441 + 438 planes, whose second group's 292 columns need a fourth chunk
    of 4 columns)."""
    inf = ozk.Plan((4096, 4096, 4096, 2048)).info
    assert inf["plane_groups"] == 2 and inf["group_planes"] == 447
    cols = [54 + 2 * 131, 2 * 144]
    assert [-(-(-(-c // 16) * 16) // 96) for c in cols] == [4, 3]
    assert 54 + 3 * 131 == 447 and 3 * 144 == 432 and 447 + 432 == 879
    # an explicit group size keeps the smallest cap that gives the count
    assert ozk.Plan((4096, 4096, 4096, 2048), plane_group=441).info["group_planes"] == 441


def test_plane_group_option_errors(ozk):
    for bad in (-2, 1, 2):
        with pytest.raises(ozk.OzakiError) as ei:
            ozk.Plan((200, 150, 300, 256), plane_group=bad)
        assert ei.value.status == ozk._lib.OZ2_EINVAL
    # streaming runs the grouped tensor-core GEMM: other engines or schedules refuse an explicit group size
    for kw in ({"engine": 1}, {"schedule": 1}):
        with pytest.raises(ozk.OzakiError):
            ozk.Plan((200, 150, 300, 256), plane_group=20, **kw)
        assert ozk.Plan((200, 150, 300, 256), **kw).info["plane_groups"] == 1


def test_injected_host_allocation_failure(ozk):
    """A host allocation failure while a plan is built is reported as
    OZ2_ENOMEM (nothing aborts, nothing half-made is kept); the next call
    succeeds."""
    lib = ozk.lib()
    h = C.c_void_p()
    assert lib.ozaki2_debug_inject_alloc_failure(1) == 0
    assert lib.ozaki2_plan_create(64, 64, 64, 53, None, C.byref(h)) == ozk._lib.OZ2_ENOMEM
    assert not h.value
    assert lib.ozaki2_plan_create(64, 64, 64, 53, None, C.byref(h)) == 0 and h.value
    lib.ozaki2_plan_destroy(h)
    # batched plans take the same path
    arr = (ozk._lib.Problem * 2)()
    for i, (M, N, K, p) in enumerate([(64, 64, 64, 53), (32, 16, 8, 113)]):
        arr[i].M, arr[i].N, arr[i].K, arr[i].p = M, N, K, p
    assert lib.ozaki2_debug_inject_alloc_failure(2) == 0
    assert lib.ozaki2_plan_create_batched(2, arr, None, C.byref(h)) == ozk._lib.OZ2_ENOMEM
    assert lib.ozaki2_plan_create_batched(2, arr, None, C.byref(h)) == ozk._lib.OZ2_ENOMEM
    assert lib.ozaki2_plan_create_batched(2, arr, None, C.byref(h)) == 0
    lib.ozaki2_plan_destroy(h)
    assert lib.ozaki2_debug_inject_alloc_failure(-1) == ozk._lib.OZ2_EINVAL
    assert lib.ozaki2_debug_inject_alloc_failure(0) == 0


def test_fault_injection_setters(ozk):
    lib = ozk.lib()
    assert lib.ozaki2_plan_set_wait_limit(None, 5) == ozk._lib.OZ2_EINVAL
    assert lib.ozaki2_plan_debug_corrupt_crt(None, 0) == ozk._lib.OZ2_EINVAL
    plan = ozk.Plan((64, 64, 64, 256))
    assert lib.ozaki2_plan_set_wait_limit(plan._h, 1) == 0
    assert lib.ozaki2_plan_set_wait_limit(plan._h, 0) == 0
    assert lib.ozaki2_plan_debug_corrupt_crt(plan._h, 1) == ozk._lib.OZ2_EINVAL
    assert lib.ozaki2_plan_debug_corrupt_crt(plan._h, 0) == 0


def test_operand_reuse_needs_a_previous_execute(ozk):
    """ozaki2_execute_reuse keeps one operand's planes from the previous
    execute with the same workspace: without one it refuses (host check)."""
    lib = ozk.lib()
    plan = ozk.Plan((64, 64, 64, 113))
    m = ozk._lib.Mat(1, 1, 1, 64, 64 * 64)
    c = ozk._lib.Mat(1, 1, 1, 64, 64 * 64)
    for keep in (0, 1):
        assert lib.ozaki2_execute_reuse(plan._h, keep, C.byref(m), C.byref(c), 256, 1 << 30, None) == \
            ozk._lib.OZ2_EINVAL
    assert lib.ozaki2_execute_reuse(plan._h, 2, C.byref(m), C.byref(c), 256, 1 << 30, None) == ozk._lib.OZ2_EINVAL
    assert lib.ozaki2_execute_reuse(None, 0, C.byref(m), C.byref(c), 256, 1 << 30, None) == ozk._lib.OZ2_EINVAL


def test_complex_plan_host_facts(ozk):
    """A complex plan: three real products sharing exponents, t and the
    modulus set chosen for inner length 2K; batched executes refuse it."""
    M, N, K, p = 100, 80, 60, 256
    plan = ozk.ComplexPlan((M, N, K, p))
    par = o.complex_params(K, p)
    assert plan.info["count"] == 3 and plan.info["t"] == par.t and plan.info["L"] == par.L
    assert plan.moduli() == par.moduli
    lib = ozk.lib()
    arr = (ozk._lib.Problem * 3)()
    assert lib.ozaki2_execute_batched(plan._h, 3, arr, 256, 1 << 30, None) == ozk._lib.OZ2_EINVAL


@pytest.mark.parametrize("p", [256, 300, 600, 800, 1024, 1500, 2048])
def test_crt_groups_skipped_below_the_fast_finish(ozk, p):
    """The CRT sums leave unformed exactly the groups of 32 column sums below
    group g0 - 1, g0 being the group whose lowest digit lies just below the
    long finish's window of 2 nl + 4 digits (the same rule the finish applies
    to choose its fast form), and only for the long finish (more than 24
    digits)."""
    plan = ozk.Plan((256, 256, 64, p), crt_engine=2)
    inf = plan.info
    D, nl = inf["crt_digits"], -(-p // 64)
    W = 2 * nl + 4
    wbase = D - W if D > W else 0
    g0 = (wbase - 1) // 7 if wbase > 7 else 0
    want = g0 - 1 if inf["crt_mode"] == 2 and D > 24 and g0 >= 2 else 0
    assert inf["crt_skip_groups"] == want
    if p >= 1024:
        assert want > 0
    if D <= 24:                                          # the short finish reads every group
        assert want == 0
    assert ozk.Plan((256, 256, 64, p), crt_engine=3).info["crt_skip_groups"] == 0
