"""Host logic of bench.py on CPU: the reference arm's JSON line (the CPU
oracle on a bounded sample), the workload table, and how the DRAM traffic of
a committed ncu summary is looked up, scaled by rows and dropped once the
kernel sources change."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--rows", "65536",
                        "--steps", "2", "--warmup", "3", "--ref-budget-s", "2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "rows/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "decode + evaluate" in cb["sample"] and cb["cpu_model"]
    assert d["e2e"] == {"value": d["value"], "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("star_join")


@pytest.mark.parametrize("name", ["star", "star_unsorted", "star_year", "star_year_unsorted", "star_bigint", "scan",
                                  "strings", "strings_all", "groups_hot", "strings_text", "strings_fsst", "chain", "chain_sparse"])
def test_every_workload_name_builds(name):
    w = bench._workload(name, 1 << 12)
    assert w["tables"][w["fact"]]["rows"] == 1 << 12
    assert w["query"]["aggs"]


def _profile(tmp_path, workload, source_hash, rows, dram):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / f"fused_kernel_{workload}.txt").write_text(
        f"title line\n\nsource_hash: {source_hash}\ncaptured_rows: {rows}\n"
        f"dram_bytes_per_launch: {dram}\n  indented: lines are notes\n")


def test_stored_traffic_scales_by_rows_and_drops_stale_captures(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()  # of the real kernel sources
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _profile(tmp_path, "star", h, 1 << 25, 1000)
    traffic, src = bench.stored_traffic("star", 1 << 26)
    assert traffic == 2000 and "scaled" in src
    _profile(tmp_path, "star", "0" * 16, 1 << 25, 1000)
    assert bench.stored_traffic("star", 1 << 26) == (None, "stale (kernel changed since capture)")
    assert bench.stored_traffic("chain", 1 << 26) == (None, "no capture")


def test_cpu_baselines_and_percentiles():
    import synth
    w = synth.scan_filter_aggregate(rows=1 << 16, page_rows=4096)
    cb = bench.cpu_baselines(w)
    assert cb["cores"] == cb["nproc"] >= 1 and cb["value"] > 0 and cb["one_thread"]["cores"] == 1
    q = bench.pcts([3.0, 1.0, 2.0, 4.0, 5.0])
    assert q["p50"] == 3.0 and q["p90"] == 5.0 and q["mean"] == 3.0 and q["n"] == 5


def test_kernel_source_hash_ignores_comments_only():
    """The hash that ties stored ncu counters to the kernel code changes with
    the code and not with comments or blank lines."""
    a = "int f(int x) {  // doubles x\n  return 2 * x; /* no overflow check */\n}\n"
    b = "// a header comment\nint f(int x) {\n\n  return 2 * x;\n}\n"
    c = "int f(int x) {\n  return 3 * x;\n}\n"
    s = 'const char* p = "// not a comment"; char q = \'"\';\n'
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
    assert bench._code_only(s) == s.rstrip("\n")


def test_stored_traffic_by_algorithmic_bytes_and_link_bytes(tmp_path, monkeypatch):
    """A batch's capture scales by algorithmic bytes; the host-resident
    variant's link bytes come from its own capture when present, and the
    lookup reports a missing or stale one."""
    h = "ab" * 8
    monkeypatch.setattr(bench, "kernel_source_hash", lambda *a: h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "fused_kernel_batched.txt").write_text(
        f"source_hash: {h}\ncaptured_rows: 100\ndram_bytes_per_launch: 900\n"
        "algorithmic_bytes_per_launch: 1000\n")
    traffic, src = bench.stored_traffic("batched", 0, alg_bytes=4000)
    assert traffic == 3600 and "algorithmic bytes" in src
    assert bench.stored_link_bytes("star", 1 << 26) == (None, "no capture")
    (tmp_path / "profiles" / "fused_kernel_star_host.txt").write_text(
        f"source_hash: {h}\ncaptured_rows: {1 << 25}\nlink_bytes_per_launch: 1000\n")
    link, src = bench.stored_link_bytes("star", 1 << 26)
    assert link == 2000 and "scaled" in src
    (tmp_path / "profiles" / "fused_kernel_star_host.txt").write_text(
        f"source_hash: {'0' * 16}\ncaptured_rows: 1\nlink_bytes_per_launch: 1\n")
    assert bench.stored_link_bytes("star", 1 << 26) == (None, "stale (kernel changed since capture)")
