"""Host arithmetic of the benchmark's per-kernel roofline objects (CPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _info(**kw):
    base = {"L": 70, "L1": 54, "G": 102, "t": 282, "crt_digits": 21}
    base.update(kw)
    return base


def test_cuda_core_crt_stage():
    M = N = K = 1024
    st = {"scan": 0.02, "residues": 0.2, "gemm": 0.18, "crt": 0.25}
    out = bench.stage_rooflines(_info(), M, N, K, 256, st, "none")
    assert set(out) == {"scan", "residues", "gemm", "crt"}
    assert out["crt"]["bound"] == "alu"
    # M N L (D - 2) multiply-adds in 0.25 ms
    assert out["crt"]["achieved"] == pytest.approx(M * N * 70 * 19 / 0.25e-3 / 1e12, rel=1e-3)
    assert out["gemm"]["achieved"] == pytest.approx(2.0 * M * N * K * 102 / 0.18e-3 / 1e12, rel=1e-3)


def test_tensor_core_crt_stages():
    M = N = K = 1024
    st = {"scan": 0.02, "residues": 0.2, "gemm": 0.18, "crt_sums": 0.15, "crt_finish": 0.09}
    out = bench.stage_rooflines(_info(crt_pieces=83), M, N, K, 256, st, "none")
    assert set(out) == {"scan", "residues", "gemm", "crt_sums", "crt_finish"}
    s, f = out["crt_sums"], out["crt_finish"]
    assert s["bound"] == "tensor" and f["bound"] == "hbm"
    assert s["achieved"] == pytest.approx(2.0 * M * N * 140 * 83 / 0.15e-3 / 1e12, abs=0.05)
    # group words D + 2 ceil(D/7), the 4-byte quotient estimate, 4 limbs + exponent + sign out
    per = 4 * (21 + 2 * 3) + 4 + 8 * 4 + 5
    assert f["achieved"] == pytest.approx(M * N * per / 0.09e-3 / 1e9, abs=0.05)
    assert 0 < f["frac"] < 1.5 and 0 < s["frac"] < 1.5


def test_every_stage_reports_its_hbm_rate():
    M = N = K = 1024
    info = _info(crt_pieces=83)
    st = {"scan": 0.02, "residues": 0.2, "gemm": 0.18, "crt_sums": 0.15, "crt_finish": 0.09}
    out = bench.stage_rooflines(info, M, N, K, 256, st, "none")
    for name, ms in st.items():
        h = out[name]["hbm"]
        assert h["unit"] == "GB/s" and h["achieved"] == pytest.approx(h["bytes"] / (ms * 1e-3) / 1e9, abs=0.05)
    # residues: inputs (4 limbs + exponent + sign per entry) and 102 planes of 1024 x 1024 bf16 per side
    assert out["residues"]["hbm"]["bytes"] == 2 * M * K * (8 * 4 + 5) + 102 * 2 * M * K * 2
    # GEMM: both plane stacks and 70 values v_l per output
    assert out["gemm"]["hbm"]["bytes"] == 102 * 2 * M * K * 2 + 70 * M * N * 2
    # CRT sums: v_l in, three 9-word groups and the estimate out
    assert out["crt_sums"]["hbm"]["bytes"] == 70 * M * N * 2 + M * N * (3 * 9 * 4 + 4)
    cpu = bench.stage_rooflines(_info(), M, N, K, 256, {"scan": 0.02, "residues": 0.2, "gemm": 0.18, "crt": 0.25},
                                "none")
    assert cpu["crt"]["hbm"]["bytes"] == 70 * M * N * 2 + M * N * (8 * 4 + 5)


def test_tensor_core_residues_against_the_tensor_peak():
    """res_mode 2 runs the residue byte products on the tensor cores: 2 flops
    per byte multiply-add against the bf16 peak, not the dp4a rate."""
    M = N = K = 1024
    info = _info(res_mode=2, crt_pieces=83)
    st = {"scan": 0.02, "residues": 0.5, "gemm": 0.18, "crt_sums": 0.15, "crt_finish": 0.09}
    out = bench.stage_rooflines(info, M, N, K, 256, st, "none")
    r = out["residues"]
    macs = (M + N) * K * -(-283 // 8) * (54 + 2 * 16)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(2.0 * macs / 0.5e-3 / 1e12, abs=0.05)


def test_skipped_crt_groups_are_not_counted():
    """Where the long finish's fast form leaves the lowest groups of 32 column
    sums unformed (crt_skip_groups), the CRT sums count only the formed
    columns' products and the group words written, and the finish the group
    words it reads."""
    M = N = 256
    K = 4096
    info = _info(L=329, L1=54, G=879, t=2076, crt_digits=133, crt_pieces=635, crt_skip_groups=8)
    st = {"scan": 0.02, "residues": 2.0, "gemm": 4.0, "crt_sums": 1.0, "crt_finish": 0.3}
    out = bench.stage_rooflines(info, M, N, K, 2048, st, "none")
    assert out["crt_sums"]["achieved"] == pytest.approx(2.0 * M * N * 658 * (635 - 256) / 1e-3 / 1e12, abs=0.05)
    ngrp = -(-(635 + 5) // 32) - 8                       # 20 groups, 12 formed
    assert out["crt_sums"]["hbm"]["bytes"] == 329 * M * N * 2 + M * N * (ngrp * 9 * 4 + 4)
    per = 4 * 9 * ngrp + 4 + 8 * 32 + 5
    assert out["crt_finish"]["achieved"] == pytest.approx(M * N * per / 0.3e-3 / 1e9, abs=0.05)
