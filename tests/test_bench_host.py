"""CPU checks of the benchmark's host arithmetic: roofline figures, the ncu launch-list summary and
the source-hash gate on recorded DRAM traffic (no GPU)."""

import json
import os

import pytest

import bench


def test_roofline_entry_flops_and_bytes():
    n = 257
    r = bench.roofline_entry(("pass64:matvec", (3, 3.0)), n, 1.2, 6674.5)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(44.5 * n ** 3 / 1e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.2)
    # a level-1 kernel counts (n + 1) / 2 nodes per axis
    r = bench.roofline_entry(("pass27:jacobi:L1", (2, 0.128)), n, 1.2, 6674.5, s=4)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(68.0 * 129 ** 3 / 64e-6 / 1e9)  # 14 coefficients + x, b, e
    # the method's bytes (x, k, b in, e out, the FP32 q of the fused dot); BF16 halves the stored
    # values; the precomputed (1/2) L k and 1/diag are reported apart
    assert bench.bytes_per_node("pass:jacobi:L0", 2) == 12 and bench.bytes_per_node("pass:jacobi:L0", 4) == 20
    assert bench.aux_bytes_per_node("pass:jacobi:L0", 4) == 8
    r = bench.roofline_entry(("pass:jacobi:L0", (1, 0.1)), n, 1.2, 6674.5, s=4)
    assert r["frac"] == pytest.approx(20 * n ** 3 / 1e-4 / 1e9 / 6674.5)
    assert r["frac_with_aux"] == pytest.approx(28 * n ** 3 / 1e-4 / 1e9 / 6674.5)
    assert bench.bytes_per_node("restrict:L0", 4) == 4.5
    assert bench.roofline_entry(("unknown", (1, 1.0)), n, 1.2, 6674.5)["bound"] is None


def _csv(tmp_path, rows):
    head = '"ID","Kernel Name","Grid Size","Metric Name","Metric Unit","Metric Value"\n'
    body = "".join(",".join(f'"{v}"' for v in r) + "\n" for r in rows)
    p = tmp_path / "launches.csv"
    p.write_text("==PROF== Connected\n" + head + body)
    return str(p)


def test_ncu_summary_groups_launches(tmp_path, capsys):
    k1 = "void nn4::<unnamed>::k_pass<float, 3, 2>(nn4::<unnamed>::Maps, nn4::PassArgs)"
    k2 = "void nn4::<unnamed>::k_restrict<float>(const T1 *, T1 *, nn4::LevelGeom, nn4::LevelGeom)"
    rows = [
        ("0", k1, "(9, 17, 8)", "gpu__time_duration.sum", "us", "70"),
        ("0", k1, "(9, 17, 8)", "dram__bytes_read.sum", "Mbyte", "300"),
        ("0", k1, "(9, 17, 8)", "dram__bytes_write.sum", "Mbyte", "60"),
        ("1", k2, "(5, 33, 65)", "gpu__time_duration.sum", "ns", "20,000"),
        ("2", k1, "(9, 17, 8)", "gpu__time_duration.sum", "ms", "0.080"),
    ]
    bench.ncu_summary(_csv(tmp_path, rows), False)
    out = capsys.readouterr().out
    lines = [ln for ln in out.splitlines() if ln.startswith("| `")]
    assert lines[0].startswith("| `k_pass<float, 3, 2>` | (9, 17, 8) | 2 | 150.0 | 0.8824 | 75.00 | 180.00 |")
    assert lines[1].startswith("| `k_restrict<float>` | (5, 33, 65) | 1 | 20.0 | 0.1176 | 20.00 | 0.00 |")
    assert "total 170.0 us over 3 launches" in out


def test_recorded_traffic_needs_matching_source_hash(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2401_06755_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "outer.cu").write_text("kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"inner": "f32", "kernels": {"inner:update": {"dram_bytes_per_launch": 4.0e8,
                                                          "source_sha256": bench._source_sha(("outer.cu",))}}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert bench._traffic("inner:update", "f32") == 4.0e8
    assert bench._traffic("inner:update", "bf16") is None  # captured with another storage type
    (csrc / "outer.cu").write_text("kernel v2")
    assert bench._traffic("inner:update", "f32") is None   # the kernel changed since the capture
