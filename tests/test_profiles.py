"""The committed profile summaries stay consistent with the source they describe.

The benchmark reports the dominant kernel's DRAM traffic from
``profiles/traffic.txt`` only while the kernel's source is unchanged since the
capture (a record of another source reads as null); every summary is short
text and gives an ncu command that leaves the GPU clocks alone.
"""

import hashlib
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")
KERNEL_FILES = {
    "fold_tc_kernel": "paper_2607_00488_gb300/csrc/fold_tc.cu",
    "fold_simt_kernel": "paper_2607_00488_gb300/csrc/fold_simt.cu",
}


def test_traffic_records_are_well_formed():
    lines = [ln.split() for ln in open(os.path.join(PROFILES, "traffic.txt")) if ln.strip()]
    assert lines
    for parts in lines:
        tag, dram_bytes, sha = parts[:3]
        assert tag.split(":")[0] in KERNEL_FILES, tag
        assert float(dram_bytes) > 0
        assert re.fullmatch(r"[0-9a-f]{16}", sha), sha


def test_bench_reports_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    # a record taken on another version of the kernel's source reads as null
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(b"__global__ void k() {}\n").hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.txt").write_text("k:fp16x3 1234 %s\nk:bf16x3 99 0000000000000000\n" % sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k.cu", "k:fp16x3") == 1234.0
    assert bench.recorded_traffic("k.cu", "k:bf16x3") is None
    (tmp_path / "k.cu").write_text("__global__ void k() { }\n")
    assert bench.recorded_traffic("k.cu", "k:fp16x3") is None


def test_summaries_are_short_text_with_an_unlocked_clock_command():
    names = sorted(os.listdir(PROFILES))
    assert names
    for name in names:
        path = os.path.join(PROFILES, name)
        assert name.endswith((".md", ".txt")), name
        assert os.path.getsize(path) < 16 * 1024, name
        if not name.endswith(".md"):
            continue
        text = re.sub(r"\\\n\s*", " ", open(path).read())  # join continued command lines
        cmds = [ln for ln in text.splitlines() if re.search(r"\bncu\b.*--(set|metrics|section)", ln)]
        assert cmds, "%s gives no ncu command" % name
        for ln in cmds:
            assert "--clock-control none" in ln, (name, ln)
