"""bench.py's bookkeeping on CPU: the roofline's algorithmic units, the
committed-traffic lookup and the clock-sample summary (no GPU needed)."""
import json
import os
from types import SimpleNamespace

import bench


def _w(N=1000, D=64, K=256, G=26):
    return SimpleNamespace(N=N, D=D, K=K, G=G)


def _it(i, path, surv=0, scan=0, nd=0):
    return {"iter": i, "path": path, "n_survivors": surv, "n_scanned": scan, "n_dist": nd}


def test_dense_bytes_per_launch():
    w = _w()
    out = dict(bench.algorithmic("dense_assign", w, [_it(0, 2)], 1))
    # X (4 bytes per coordinate), label/u/lbg/stamp, and the lb row with G rounded to 4
    assert out["hbm"] == w.N * (4 * 64 + 16 + 4 * 28)
    assert out["tensor"] == 6.0 * w.N * w.K * w.D and "alu" not in out  # BF16x3 on the tensor cores
    out = dict(bench.algorithmic("dense_assign", w, [_it(0, 1)], 1))
    assert out["alu"] == 3.0 * w.N * w.K * w.D and "tensor" not in out  # FP32 engine: every distance


def test_survivor_units_count_filtered_iterations_only():
    w = _w()
    stats = [_it(0, 2, nd=w.N * w.K), _it(1, 2, surv=w.N, nd=w.N * w.K), _it(2, 0, surv=400, scan=300, nd=1200),
             _it(3, 0, surv=200, scan=100, nd=600)]
    out = dict(bench.algorithmic("survivor", w, stats, 4))
    surv, scan, nd = 300.0, 200.0, 900.0  # means over iterations 2 and 3
    assert out["hbm"] == surv * (4 + 12 + 4 * 64 + 8) + scan * (8 * 28 + 16)
    assert out["alu"] == 3.0 * 64 * nd


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", {"dense_assign": ["k.cu"]})
    rec = {"dense_assign": {"source_sha": bench.source_sha(["k.cu"]), "dram_bytes_per_launch": 123}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic("dense_assign") == 123
    assert bench.ncu_traffic("dense_assign", "highdim4m") is None  # another workload
    assert bench.ncu_traffic("survivor") is None                   # no record
    src.write_text("kernel v2\n")                                  # the kernel changed since
    assert bench.ncu_traffic("dense_assign") is None


def test_clock_summary_and_energy(tmp_path):
    c = bench.ClockSampler(None)
    c.path = str(tmp_path / "clocks.csv")
    c.proc = object()  # a sampler that ran
    rows = [
        "0, 2070, 2070, 400.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 420.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 410.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert abs(s["power_w_mean"] - 410.0) < 1e-9
    e = bench.energy_of(4.1e9, s)
    assert abs(e["value"] - 1e7) < 1e-3 and e["mean_power_w"] == s["power_w_mean"]
    assert bench.energy_of(1.0, {"power_w_mean": None}) is None


def test_clock_summary_without_sampler(tmp_path):
    c = bench.ClockSampler(None)
    c.path = os.path.join(str(tmp_path), "missing.csv")
    assert c.summary()["sm_mhz"] is None
