"""GB300 (sm_103a) Ozaki-scheme-II multiple-precision GEMM.

Python front end of the C ABI in ``include/ozaki2.h``.  PyTorch provides
device memory and streams; every step of the product runs in this package's
CUDA kernels (``libozaki2_gb300.so``).  Matrices use the storage format of the
C ABI: limb planes ``[nl, rows, cols]`` (uint64 bit patterns held in int64
tensors), ``exp`` int32 ``[rows, cols]`` and ``sign`` int8 ``[rows, cols]``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from ._lib import OzakiError, check, lib, opts  # noqa: F401

__all__ = ["MPMatrix", "Plan", "ComplexPlan", "Graph", "gemm", "gemm_batched", "zgemm", "OzakiError", "lib",
           "opts"]


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class MPMatrix:
    """A p-bit matrix in device (or host) memory, struct-of-arrays layout."""

    def __init__(self, limbs: torch.Tensor, exp: torch.Tensor, sign: torch.Tensor, p: int):
        assert limbs.dtype == torch.int64 and exp.dtype == torch.int32 and sign.dtype == torch.int8
        assert limbs.dim() == 3 and limbs.is_contiguous() and exp.is_contiguous() and sign.is_contiguous()
        self.limbs, self.exp, self.sign, self.p = limbs, exp, sign, int(p)

    @property
    def shape(self):
        return tuple(self.exp.shape)

    @property
    def nl(self) -> int:
        return self.limbs.shape[0]

    @classmethod
    def empty(cls, rows: int, cols: int, p: int, device="cuda") -> "MPMatrix":
        nl = (p + 63) // 64
        return cls(torch.empty((nl, rows, cols), dtype=torch.int64, device=device),
                   torch.empty((rows, cols), dtype=torch.int32, device=device),
                   torch.empty((rows, cols), dtype=torch.int8, device=device), p)

    @classmethod
    def from_host(cls, m: dict, device="cuda") -> "MPMatrix":
        """From a host dict {'p', 'limbs' (uint64 [nl,R,C]), 'exp', 'sign'}."""
        limbs = torch.from_numpy(np.ascontiguousarray(m["limbs"]).view(np.int64))
        return cls(limbs.to(device), torch.from_numpy(np.ascontiguousarray(m["exp"])).to(device),
                   torch.from_numpy(np.ascontiguousarray(m["sign"])).to(device), m["p"])

    def to_host(self) -> dict:
        return {"p": self.p, "limbs": self.limbs.cpu().numpy().view(np.uint64),
                "exp": self.exp.cpu().numpy(), "sign": self.sign.cpu().numpy()}

    def desc(self) -> L.Mat:
        R, Cc = self.shape
        return L.Mat(self.limbs.data_ptr(), self.exp.data_ptr(), self.sign.data_ptr(), Cc, R * Cc)


class Graph:
    """A captured execute of a plan (replay with ``launch``)."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def launch(self, stream=None):
        check(lib().ozaki2_graph_launch(self._h, _stream_handle(stream)), "ozaki2_graph_launch")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ozaki2_graph_destroy(self._h)
            self._h = None


class Plan:
    """A plan for one product or for a batch of independent products."""

    def __init__(self, shapes, per_problem=None, **kw):
        """``shapes``: (M, N, K, p) or a list of such tuples (batched);
        ``per_problem`` (batched): one dict of per-problem options each
        (guard_bits, t_bits, k_chunk, crt_engine, res_engine)."""
        self._o = opts(**kw)
        h = C.c_void_p()
        if isinstance(shapes, tuple):
            M, N, K, p = shapes
            st = lib().ozaki2_plan_create(M, N, K, p, C.byref(self._o), C.byref(h))
            self.shapes = [shapes]
            self.batched = False
        else:
            arr = (L.Problem * len(shapes))()
            for i, (M, N, K, p) in enumerate(shapes):
                arr[i].M, arr[i].N, arr[i].K, arr[i].p = M, N, K, p
            if per_problem is not None:
                po = (L.Opts * len(shapes))()
                for i, d in enumerate(per_problem):
                    po[i] = opts(**d)
                st = lib().ozaki2_plan_create_batched_ex(len(shapes), arr, C.byref(self._o), po, C.byref(h))
            else:
                st = lib().ozaki2_plan_create_batched(len(shapes), arr, C.byref(self._o), C.byref(h))
            self.shapes = list(shapes)
            self.batched = True
        check(st, "ozaki2_plan_create")
        self._h = h
        inf = L.Info()
        check(lib().ozaki2_plan_info(h, C.byref(inf)), "ozaki2_plan_info")
        self.info = {f: getattr(inf, f) for f, _ in L.Info._fields_}
        self.workspace_bytes = inf.workspace_bytes

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ozaki2_plan_destroy(self._h)
            self._h = None

    def moduli(self, prob: int = 0) -> list[int]:
        out = (C.c_int32 * 40000)()
        check(lib().ozaki2_plan_moduli(self._h, prob, out, 40000), "ozaki2_plan_moduli")
        n = self.info["L"] if prob == 0 else None
        vals = list(out)
        if n is None:
            n = next(i for i, v in enumerate(vals) if v == 0)
        return vals[:n]

    def crt_tables(self, prob: int = 0, L_: int | None = None, D: int | None = None):
        L_ = L_ or self.info["L"]
        D = D or self.info["crt_digits"]
        P = (C.c_uint32 * D)()
        Md = (C.c_uint32 * (L_ * D))()
        inv = (C.c_uint32 * L_)()
        check(lib().ozaki2_plan_crt_tables(self._h, prob, P, Md, inv), "ozaki2_plan_crt_tables")
        return list(P), [list(Md[l * D:(l + 1) * D]) for l in range(L_)], list(inv)

    def layout(self, prob: int = 0):
        off = (C.c_size_t * 5)()
        kp = C.c_int64()
        check(lib().ozaki2_plan_layout(self._h, prob, off, C.byref(kp)), "ozaki2_plan_layout")
        return list(off), kp.value

    def workspace(self, device="cuda") -> torch.Tensor:
        return torch.empty(self.workspace_bytes, dtype=torch.uint8, device=device)

    def launches(self) -> int:
        """Kernel launches of the library per execute (after the first execute)."""
        n = C.c_int()
        check(lib().ozaki2_plan_launches(self._h, C.byref(n)), "ozaki2_plan_launches")
        return n.value

    def set_debug_prods(self, prob: int, buf: torch.Tensor | None):
        """Exact plane sums before reduction, int32 [G][M][N] (K within one chunk)."""
        check(lib().ozaki2_plan_set_debug_prods(self._h, prob, None if buf is None else buf.data_ptr()),
              "ozaki2_plan_set_debug_prods")

    def set_debug_chat(self, prob: int, buf: torch.Tensor | None):
        check(lib().ozaki2_plan_set_debug_chat(self._h, prob, None if buf is None else buf.data_ptr()),
              "ozaki2_plan_set_debug_chat")

    def execute(self, A: MPMatrix, B: MPMatrix, Cm: MPMatrix, ws: torch.Tensor, stream=None):
        a, b, c = A.desc(), B.desc(), Cm.desc()
        check(lib().ozaki2_execute(self._h, C.byref(a), C.byref(b), C.byref(c), ws.data_ptr(),
                                   ws.numel(), _stream_handle(stream)), "ozaki2_execute")

    def execute_reuse(self, keep: int, X: MPMatrix, Cm: MPMatrix, ws: torch.Tensor, stream=None):
        """C = A X (keep=0: A's planes from the previous execute with ``ws``) or
        C = X B (keep=1: B's planes kept)."""
        x, c = X.desc(), Cm.desc()
        check(lib().ozaki2_execute_reuse(self._h, keep, C.byref(x), C.byref(c), ws.data_ptr(), ws.numel(),
                                         _stream_handle(stream)), "ozaki2_execute_reuse")

    def _problems(self, triples):
        arr = (L.Problem * len(triples))()
        for i, ((M, N, K, p), (A, B, Cm)) in enumerate(zip(self.shapes, triples)):
            arr[i].M, arr[i].N, arr[i].K, arr[i].p = M, N, K, p
            arr[i].A, arr[i].B, arr[i].C = A.desc(), B.desc(), Cm.desc()
        return arr

    def execute_batched(self, triples, ws: torch.Tensor, stream=None):
        arr = self._problems(triples)
        check(lib().ozaki2_execute_batched(self._h, len(triples), arr, ws.data_ptr(), ws.numel(),
                                           _stream_handle(stream)), "ozaki2_execute_batched")

    def graph(self, triples, ws: torch.Tensor, stream) -> Graph:
        arr = self._problems(triples)
        g = C.c_void_p()
        check(lib().ozaki2_graph_create(self._h, len(triples), arr, ws.data_ptr(), ws.numel(),
                                        _stream_handle(stream), C.byref(g)), "ozaki2_graph_create")
        return Graph(g, (triples, ws))

    def check(self, stream=None):
        check(lib().ozaki2_check(self._h, _stream_handle(stream)), "ozaki2_check")

    def timings(self):
        ms = (C.c_float * 5)()
        check(lib().ozaki2_last_timings(self._h, ms), "ozaki2_last_timings")
        return dict(zip(["scan", "residues", "gemm", "crt", "total"], list(ms)))

    def crt_split(self):
        """The CRT stage of the last timed execute: tensor-core column sums
        (about 0 where none ran) and the rest, in ms."""
        ms = (C.c_float * 2)()
        check(lib().ozaki2_last_crt_split(self._h, ms), "ozaki2_last_crt_split")
        return {"crt_sums": ms[0], "crt_finish": ms[1]}


class ComplexPlan(Plan):
    """A plan for one complex product (Ar + i Ai)(Br + i Bi), 3M form."""

    def __init__(self, shape, **kw):
        self._o = opts(**kw)
        h = C.c_void_p()
        M, N, K, p = shape
        check(lib().ozaki2_plan_create_complex(M, N, K, p, C.byref(self._o), C.byref(h)),
              "ozaki2_plan_create_complex")
        self.shapes = [shape]
        self.batched = False
        self._h = h
        inf = L.Info()
        check(lib().ozaki2_plan_info(h, C.byref(inf)), "ozaki2_plan_info")
        self.info = {f: getattr(inf, f) for f, _ in L.Info._fields_}
        self.workspace_bytes = inf.workspace_bytes

    def execute_complex(self, Ar: MPMatrix, Ai: MPMatrix, Br: MPMatrix, Bi: MPMatrix, Cr: MPMatrix, Ci: MPMatrix,
                        ws: torch.Tensor, stream=None):
        d = [x.desc() for x in (Ar, Ai, Br, Bi, Cr, Ci)]
        check(lib().ozaki2_execute_complex(self._h, *[C.byref(x) for x in d], ws.data_ptr(), ws.numel(),
                                           _stream_handle(stream)), "ozaki2_execute_complex")


def zgemm(Ar: MPMatrix, Ai: MPMatrix, Br: MPMatrix, Bi: MPMatrix, p: int | None = None, stream=None, **kw):
    """(Cr, Ci) = (Ar + i Ai)(Br + i Bi) rounded to p bits per part (cached plan)."""
    p = p or Ar.p
    M, K = Ar.shape
    N = Br.shape[1]
    Cr = MPMatrix.empty(M, N, p, device=Ar.limbs.device)
    Ci = MPMatrix.empty(M, N, p, device=Ar.limbs.device)
    o = opts(**kw)
    d = [x.desc() for x in (Ar, Ai, Br, Bi, Cr, Ci)]
    check(lib().ozaki2_zgemm(M, N, K, p, *[C.byref(x) for x in d], C.byref(o), _stream_handle(stream)),
          "ozaki2_zgemm")
    return Cr, Ci


def gemm(A: MPMatrix, B: MPMatrix, p: int | None = None, stream=None, **kw) -> MPMatrix:
    """C = A B rounded to p bits (default: A's precision) through a cached plan."""
    p = p or A.p
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Cm = MPMatrix.empty(M, N, p, device=A.limbs.device)
    o = opts(**kw)
    a, b, c = A.desc(), B.desc(), Cm.desc()
    check(lib().ozaki2_gemm(M, N, K, p, C.byref(a), C.byref(b), C.byref(c), C.byref(o),
                            _stream_handle(stream)), "ozaki2_gemm")
    return Cm


def gemm_batched(pairs, ps=None, stream=None, **kw):
    """Batched products [(A, B)] -> [C] through a cached batched plan."""
    outs = []
    arr = (L.Problem * len(pairs))()
    for i, (A, B) in enumerate(pairs):
        p = ps[i] if ps else A.p
        M, K = A.shape
        N = B.shape[1]
        Cm = MPMatrix.empty(M, N, p, device=A.limbs.device)
        outs.append(Cm)
        arr[i].M, arr[i].N, arr[i].K, arr[i].p = M, N, K, p
        arr[i].A, arr[i].B, arr[i].C = A.desc(), B.desc(), Cm.desc()
    o = opts(**kw)
    check(lib().ozaki2_gemm_batched(len(pairs), arr, C.byref(o), _stream_handle(stream)),
          "ozaki2_gemm_batched")
    return outs
