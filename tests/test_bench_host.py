"""Host logic of bench.py (no GPU): the byte models behind the roofline and
the yardstick, the measured-traffic lookup and the dominant-family roofline."""
import os
import sys
from types import SimpleNamespace

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_byte_model_zq_update_and_diagonal_level():
    n, nnz, s = 1000, 6400, 4
    V = 8 * n
    bm = bench.byte_model(n, nnz, 4, s, "df64", fused=False, dia=True)
    # z / Q update with a constant diagonal: U_1..U_{s+1}, P_old, Q_old, x in; P, Q, x, z out
    assert bm["update"] == (5 * s + 4) * V
    # a diagonal-form level: the masks, u_j gathered, u_{j+1} written
    assert bm["level_avg"] == 4 * n + 2 * V
    csr = bench.byte_model(n, nnz, 4, s, "df64", fused=False, dia=False)
    M = 4 * (n + 1) + nnz * 8
    assert csr["level_avg"] == M + 3 * V and csr["update"] == (5 * s + 5) * V


def test_yardstick_is_fixed_algorithm3_bytes():
    n, nnz, s = 4096, 27000, 4
    y = bench.yardstick(n, nnz, s)
    V, M = 8 * n, 4 * (n + 1) + 12 * nnz
    # Algorithm 3 on CSR FP64: every level reads A and u_j, writes A u_j (and u_{j+1} but the last)
    assert y["level"] == [M + 2 * V + 2 * V] * (s - 1) + [M + 2 * V]
    assert y["update"] == (6 * s + 6) * V
    # independent of how the library stores the matrix
    assert bench.yardstick(n, nnz, s) == bench.byte_model(n, nnz, 8, s, "f64", fused=True, dia=False)


def test_traffic_only_for_the_captured_configuration():
    a = SimpleNamespace(s=4, arith="df64", fused_mpk=False)
    t = bench.traffic(a, "update", 4_096_000, True)
    assert t == round(732.694e6)
    assert bench.traffic(SimpleNamespace(s=4, arith="f64", fused_mpk=False), "update", 4_096_000, True) == \
        round(734.1e6)
    assert bench.traffic(SimpleNamespace(s=8, arith="df64", fused_mpk=False), "update", 4_096_000, True) is None
    assert bench.traffic(a, "update", 4_096_000, False) is None
    assert bench.traffic(a, "dir", 4_096_000, True) is None


def test_family_roofline_picks_the_dominant_family(monkeypatch):
    monkeypatch.setattr(bench, "hbm_peak", lambda: (8000.0, "test peak"))
    res = SimpleNamespace(profile={"t_mpk_ms": 10.0, "n_mpk": 100, "t_dir_ms": 30.0, "n_dir": 10,
                                   "t_update_ms": 20.0, "n_update": 10})
    r = bench.family_roofline(res, {"mpk": 1e6, "dir": 3e9, "update": 2e9},
                              {"mpk": "levels", "dir": "gram", "update": "update"})
    assert r["kernel"] == "gram"
    # 3 GB per record, 10 records in 30 ms: 1000 GB/s
    assert r["achieved"] == pytest.approx(1000.0) and r["frac"] == pytest.approx(0.125)
    assert r["bound"] == "hbm" and r["traffic"] is None and r["peak"] == 8000.0


def test_value_is_kernel_bytes_over_time_and_stays_below_the_copy_bandwidth():
    """value = the bytes the solve's kernels move per second; at the 256^3
    s = 4 solve measured on the GB300 (130 outer steps in 122.2 ms, the
    double-float run) it sits below the measured copy bandwidth, while the
    Algorithm 3 yardstick over the same time would read 1.9x above it."""
    n, nnz, s, outer, ms, hbm = 256 ** 3, 117_047_296, 4, 130, 122.155, 6786.6
    bm = bench.byte_model(n, nnz, 4, s, "df64", fused=False, dia=True)
    value = bench.sstep_bytes(bm, outer) / (ms * 1e-3) / 1e9
    assert value <= 1.2 * hbm and value == pytest.approx(4872, rel=1e-3)
    yard = bench.sstep_bytes(bench.yardstick(n, nnz, s), outer) / (ms * 1e-3) / 1e9
    assert yard > hbm


def test_fp64_operation_model():
    ops = bench.fp64_ops_model(4, K=7)
    # level: the neighbour sum on the integer units and its conversion to FP64;
    # u_{j+1} and two moments (one on the last level)
    assert ops["level"] == [4, 4, 4, 3]
    # update: s^2 for P and Q each, s for x and z each, one for sum z^2
    assert ops["update"] == 2 * 16 + 2 * 4 + 1 and ops["update_first"] == 9
    assert (ops["pcg_spmv"], ops["pcg_update"], ops["pcg_dir"]) == (3, 3, 2)
    assert bench.fp64_ops_model(2, K=27)["level"] == [4, 3]
    # the fixed-point update: P and Q on the integer units, one conversion each;
    # x and z FMAs and sum z^2 left
    assert bench.fp64_ops_model(4, fixed_update=True)["update"] == 2 * 4 + 2 * 4 + 1


def test_fixed_update_is_used_where_the_library_uses_it():
    import argparse

    def args(**kw):
        d = dict(arith="f64", s=4, fma_update=False, fused_mpk=False)
        d.update(kw)
        return argparse.Namespace(**d)

    assert bench.fixed_update_used(args())
    assert bench.fixed_update_used(args(s=1))
    assert bench.fixed_update_used(args(s=6))
    assert not bench.fixed_update_used(args(s=8))  # the 64-bit sums hold s + 1 <= 7 terms
    assert not bench.fixed_update_used(args(arith="df64"))
    assert not bench.fixed_update_used(args(fma_update=True))
    assert not bench.fixed_update_used(args(fused_mpk=True))


def test_fp64_alu_peak_is_two_per_clock_per_sm():
    # 2 x 152 SMs x 2070 MHz = 629.3 G operations/s, the nominal 1.25 TFLOP/s (FMA = 2 FLOPs)
    assert bench.alu_peak(152) == pytest.approx(629.28e9)
    assert 2 * bench.alu_peak(152) == pytest.approx(1.25e12, rel=0.01)
