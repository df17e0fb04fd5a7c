"""Host arithmetic of the bench's roofline (CPU only): the algorithmic byte counts against hand-computed
figures for the single-source 256^2 x 64 case (data 0.26 MB, FP64 class table 4.3 MB, xi 16.8 MB), and the
rule that DRAM traffic recorded by ncu is reported only while the kernel's sources are the ones it was
taken on."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_fused_bytes_match_the_printed_single_source_figures():
    # 256^2 x 64, one source, M = 1: data 0.26 MB + FP64 class table 4.3 MB + xi 16.8 MB = about 21 MB,
    # 5.1 B per voxel; the two-pass form adds 8 B per voxel: about 55 MB
    n, mp = 256, 64
    vox = n * n * mp
    b = bench.fused_algorithmic_bytes(n, mp, 1)
    assert abs(b["minimum"] / 1e6 - 21.4) < 0.3
    assert abs(b["minimum"] / vox - 5.1) < 0.05
    assert abs(b["two_pass"] / 1e6 - 55.0) < 1.0
    assert b["two_pass"] - b["minimum"] == 8 * vox
    # each further source adds its data spectra and 8 B per voxel of intermediate
    b8 = bench.fused_algorithmic_bytes(n, mp, 8)
    ps = (n // 2 + 1) * n
    assert b8["two_pass"] - b["two_pass"] == 7 * (8 * ps + 8 * vox)


def test_design_bytes_of_the_fused_inverse_include_the_weight_table():
    n, mp, q = 256, 64, 8
    d = bench.stage_bytes("inv_fused", n, mp, q, mp)
    w_table = 4 * q * n * n * mp
    assert d > w_table and abs(d / 1e6 - 161.7) < 0.1
    assert bench.stage_bytes("no such stage", n, mp, q, mp) == 0.0


def test_recorded_traffic_follows_the_kernel_sources(monkeypatch):
    rows = {}
    for line in open(os.path.join(ROOT, "profiles", "traffic.md")):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 3 and cells[0] in ("inv_fused/v3", "alpha"):
            rows[cells[0]] = (cells[1], float(cells[2]))
    assert set(rows) == {"inv_fused/v3", "alpha"}
    for stage, (h, nbytes) in rows.items():
        monkeypatch.setattr(bench, "kernel_source_hash", lambda s, h=h: h)
        assert bench.recorded_traffic(stage) == nbytes
        monkeypatch.setattr(bench, "kernel_source_hash", lambda s: "0000000000000000")
        assert bench.recorded_traffic(stage) is None
    monkeypatch.undo()
    # another tile variant of the fused kernel has no row
    assert bench.recorded_traffic("inv_fused/v0") is None


def test_source_hash_changes_with_any_listed_file(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1703_01216_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.STAGE_SOURCES["alpha"]:
        (csrc / f).write_text(f"// {f}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash("alpha")
    (csrc / bench.STAGE_SOURCES["alpha"][-1]).write_text("// changed\n")
    assert bench.kernel_source_hash("alpha") != h0


def test_hbm_peak_reads_the_measured_copy_bandwidth_or_falls_back(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak() == (6800.0, "fallback 6800 GB/s")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6792.4, "bf16_tflops": 1932.2}')
    peak, src = bench.hbm_peak()
    assert peak == 6792.4 and "measured" in src
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"bf16_tflops": 1932.2}')
    assert bench.hbm_peak()[0] == 6800.0
