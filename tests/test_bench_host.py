"""Host-side pieces of bench.py that decide what its JSON line claims: the
algorithmic bytes and flops behind `roofline`, and which ncu traffic record
(if any) applies to a run."""
import json
import os
import shutil
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_per_cell_update():
    # read b, n, sigma and write b, n once per pass (FP32: 4 B each)
    assert bench.bytes_per_cell("f32", "euler", "static", 1) == 20
    assert bench.bytes_per_cell("f32", "euler", "static", 2) == 10     # two steps per pass
    assert bench.bytes_per_cell("f64", "euler", "static", 1) == 40
    assert bench.bytes_per_cell("f32", "euler", "per-step", 1) == 16   # sigma regenerated
    assert bench.bytes_per_cell("f32", "heun", "per-step", 2) == 16    # one Heun step per pass


def test_flop_count_of_the_scheme():
    # 14 per face, two faces per cell, 15 for the update; Heun: two stages and the mean
    assert bench.FLOPS_PER_CELL_UPDATE == {"euler": 43, "heun": 90}


def _scratch_root(tmp_path):
    """A copy of the repository's records and kernel sources in a scratch
    root, with each record's source hashes set to the copied sources, so that
    the matching logic is tested whether or not the records are current and
    source edits can be simulated without touching the tree."""
    import hashlib
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "profiles"), root / "profiles")
    csrc = root / "paper_1301_5058_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_1301_5058_gb300", "csrc"), csrc)
    for rec_path in (root / "profiles").glob("*_traffic.json"):
        rec = json.load(open(rec_path))
        rec["sources_sha256_16"] = {f: hashlib.sha256((csrc / f).read_bytes()).hexdigest()[:16]
                                    for f in rec["sources_sha256_16"]}
        json.dump(rec, open(rec_path, "w"))
    return root


def test_traffic_record_applies_only_to_its_run(tmp_path, monkeypatch):
    root = _scratch_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = json.load(open(root / "profiles" / "fused_kernel_traffic.json"))
    entries = {(e["scheme"], e["noise"]): e["dram_bytes_per_launch_16384sq"] for e in rec["f32"]}
    want = entries[("euler", "static")]
    assert bench.kernel_traffic("f32", "fused_kernel", 16384, 16384, "euler", "static") == want
    assert bench.kernel_traffic("f32", "fused_kernel", 16384, 16384, "heun", "per-step") == \
        entries[("heun", "per-step")]
    # another grid, scheme, noise mode or precision: no record
    assert bench.kernel_traffic("f32", "fused_kernel", 4096, 4096, "euler", "static") is None
    assert bench.kernel_traffic("f32", "fused_kernel", 16384, 16384, "heun", "static") is None
    assert bench.kernel_traffic("f32", "fused_kernel", 16384, 16384, "euler", "per-step") is None
    assert bench.kernel_traffic("f64", "fused_kernel", 16384, 16384, "euler", "static") is None
    # a kernel source that changed since the capture voids the record
    src = root / "paper_1301_5058_gb300" / "csrc" / "cx_fused.cuh"
    src.write_text(src.read_text() + "\n// edited\n")
    assert bench.kernel_traffic("f32", "fused_kernel", 16384, 16384, "euler", "static") is None


def test_sweep_traffic_record_applies_only_to_its_tuning(tmp_path, monkeypatch):
    root = _scratch_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = json.load(open(root / "profiles" / "batch_fused_kernel_traffic.json"))["f32"]
    tuning = dict(rec["tuning"], graph_steps=64)
    assert bench.sweep_traffic(512, tuning) == rec["dram_bytes_per_launch"]
    assert bench.sweep_traffic(256, tuning) is None                       # another sweep
    other = 32 if tuning["tile_rows"] != 32 else 64
    assert bench.sweep_traffic(512, dict(tuning, tile_rows=other)) is None  # other tiles
    assert bench.sweep_traffic(512, dict(tuning, time_block=1)) is None    # one stage per pass


def test_issue_roofline_from_the_recorded_instruction_counts(tmp_path, monkeypatch):
    root = _scratch_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = json.load(open(root / "profiles" / "fused_kernel_traffic.json"))
    want = {(e["scheme"], e["noise"]): e["warp_instructions_per_launch_16384sq"] for e in rec["f32"]}
    assert bench.kernel_issue_count("f32", "fused_kernel", 16384, 16384, "euler", "static") == \
        want[("euler", "static")]
    assert bench.kernel_issue_count("f32", "fused_kernel", 4096, 4096, "euler", "static") is None
    # one warp instruction per scheduler and clock: 4 x 152 SMs x 2000 MHz = 1.216e12 / s
    r = bench.issue_roofline(2000, 1000, 3e11, 2000.0)
    assert r["warp_instructions_per_cell_update"] == 2.0
    assert abs(r["peak"] - 1.216e12) < 1.0 and abs(r["frac"] - 6e11 / 1.216e12) < 1e-12
    assert bench.issue_roofline(None, 1000, 3e11, 2000.0) is None
    batch = json.load(open(root / "profiles" / "batch_fused_kernel_traffic.json"))["f32"]
    assert bench.sweep_issue_count(512, dict(batch["tuning"])) == batch["warp_instructions_per_launch"]
    src = root / "paper_1301_5058_gb300" / "csrc" / "cx_stencil.cuh"
    src.write_text(src.read_text() + "\n// edited\n")
    assert bench.kernel_issue_count("f32", "fused_kernel", 16384, 16384, "euler", "static") is None
    assert bench.sweep_issue_count(512, dict(batch["tuning"])) is None
