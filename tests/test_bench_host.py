"""Host arithmetic of bench.py, on CPU: the flop count of the trailing
updates, the roofline fields and the clock-record parser.  No GPU is used."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _brute_update_flops(T, b):
    """Right-looking tiled Cholesky (Sec. 4.2, Fig. 1): after factoring diagonal
    tile k, every tile (i, j) with k < j <= i < T takes one update; a diagonal
    tile is a SYRK (b^3 flops on its lower half), an off-diagonal one a GEMM
    (2 b^3)."""
    tot = 0
    for k in range(T):
        for i in range(k + 1, T):
            for j in range(k + 1, i + 1):
                tot += b ** 3 if i == j else 2 * b ** 3
    return tot


@pytest.mark.parametrize("T,b", [(1, 64), (2, 8), (5, 16), (16, 32), (33, 7)])
def test_update_flops_counts_every_tile_update(T, b):
    assert bench.update_flops(T, b) == _brute_update_flops(T, b)


def test_update_flops_tends_to_the_cholesky_count():
    # The trailing updates carry all but O(N^2 b) of the Cholesky's N^3 / 3 flops.
    T, b = 128, 256
    n = T * b
    r = bench.update_flops(T, b) / (n ** 3 / 3.0)
    assert 1.0 - 2.0 / T < r < 1.0


def _args(**kw):
    a = dict(n=32768, m=8192, precision="mixed")
    a.update(kw)
    return types.SimpleNamespace(**a)


def _prof(oz_ms, oz_launches, upd_ms, upd_launches):
    return {"ozaki": (oz_ms, oz_launches), "update": (upd_ms, upd_launches)}


def test_roofline_mixed_counts_the_methods_work(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1750.0})
    T, b = 128, 256
    prof = _prof(294.2, 2, 45.0, T - 1)
    r = bench.roofline(_args(), prof, T, b)
    flops = 2.0 * 8192 * 32768 ** 2                       # K x~0 for all test points
    achieved = flops / 0.1471 / 1e12                       # one launch of 147.1 ms
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["peak"] == 1750.0 and "sustained" in r["peak_note"]
    assert r["algorithmic_flops_per_launch"] == pytest.approx(flops)
    assert r["achieved"] == pytest.approx(achieved)
    assert r["frac"] == pytest.approx(achieved / 1750.0)
    assert r["tensor_op_frac"] == pytest.approx(bench.OZAKI_PAIRS * achieved / 1750.0)
    assert r["traffic"] == pytest.approx(1.647e9 * 64)
    upd = bench.update_flops(T, b) / (T - 1)
    assert r["second"]["achieved"] == pytest.approx(upd / (45.0 / (T - 1) * 1e-3) / 1e12)
    assert r["second"]["tensor_op_frac"] == pytest.approx(6.0 * r["second"]["frac"])


def test_roofline_traffic_only_for_the_captured_scaling(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: None)
    r = bench.roofline(_args(n=8192, m=2048), _prof(2.6, 1, 1.0, 31), 32, 256)
    assert r["traffic"] is None
    assert r["peak"] == 1700.0 and "fallback" in r["peak_note"]


def test_roofline_fp64_paths(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: {"bf16_tflops_sustained": 1750.0})
    monkeypatch.setattr(bench, "_FP64_PEAK", (1.056, "of measured (test)"))
    T, b = 64, 128
    upd = bench.update_flops(T, b) / (T - 1)
    r = bench.roofline(_args(precision="fp64"), _prof(0.0, 0, 630.0, T - 1), T, b)
    assert r["peak"] == 1.056
    assert r["frac"] == pytest.approx(upd / (10e-3) / 1e12 / 1.056)
    r = bench.roofline(_args(precision="fp64_ozaki"), _prof(0.0, 0, 630.0, T - 1), T, b)
    assert r["peak"] == 1750.0
    assert r["tensor_op_frac"] == pytest.approx(28.0 * r["frac"])
    assert r["fp64_equivalent_frac_of_fp64_peak"] == pytest.approx(r["achieved"] / 1.056)


def test_clock_summary_parses_reasons(tmp_path):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "short line",
    ]
    with open(cs.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    cs.proc = object()                       # as if nvidia-smi had been started
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_flags_thermal_slowdown(tmp_path):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    with open(cs.path, "w") as f:
        f.write("0, 1500, 2070, 1000, 0x40, Not Active, Active, Not Active, Not Active\n")
    cs.proc = object()
    assert cs.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_without_sampler():
    assert bench.ClockSampler(0).summary() is None


def test_workload_config_names_the_workload():
    c = bench.workload_config(types.SimpleNamespace(n=32768, m=8192, d=8, tiles=128, precision="mixed"))
    assert c["n_train"] == 32768 and c["n_test"] == 8192 and c["tiles_per_dim"] == 128
    assert "N=32768" in c["workload"] and "M=8192" in c["workload"]
    assert "model" not in c
