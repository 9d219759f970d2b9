"""Host logic of bench.py that needs no GPU: the roofline's DRAM traffic is
taken from the committed ncu summary only while the kernel's sources are the
ones that summary was captured from."""
import os
import shutil

import bench

SOURCES = ("k_gemm_f16.cu", "tc_common.cuh")
SUMMARY = "gemm_f16_zgemm16384.txt"


def _tree(tmp_path):
    """A copy of the summary and the kernel sources in the layout bench.py reads."""
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2512_08321_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", SUMMARY), root / "profiles" / SUMMARY)
    for f in SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2512_08321_gb300", "csrc", f), csrc / f)
    return root


def test_traffic_read_while_sources_match(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    v = bench.profile_traffic(SOURCES, SUMMARY)
    assert v is not None and v > 0


def test_traffic_dropped_when_either_source_changes(tmp_path, monkeypatch):
    for changed in SOURCES:
        root = _tree(tmp_path / changed)
        monkeypatch.setattr(bench, "ROOT", str(root))
        with open(root / "paper_2512_08321_gb300" / "csrc" / changed, "a") as fh:
            fh.write("\n// edited\n")
        assert bench.profile_traffic(SOURCES, SUMMARY) is None


def test_traffic_missing_summary_is_none(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profile_traffic(SOURCES, "no_such_summary.txt") is None
