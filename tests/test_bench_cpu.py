"""Host logic of bench.py that needs no GPU: the roofline's DRAM traffic is
taken from the committed ncu summary only while the kernel's sources are the
ones that summary was captured from."""
import os
import shutil

import bench

SOURCES = ("k_gemm_f16.cu", "tc_common.cuh")
SUMMARY = "gemm_f16_zgemm16384.txt"


def _tree(tmp_path):
    """The kernel sources in the layout bench.py reads, and a summary in the
    committed summaries' format recording their current sha256."""
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2512_08321_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2512_08321_gb300", "csrc", f), csrc / f)
    import hashlib
    h = hashlib.sha256()
    for f in SOURCES:
        h.update((csrc / f).read_bytes())
    (root / "profiles" / SUMMARY).write_text(
        "# a summary\nkernel: gemm_f16_kernel\ndram_bytes_per_launch_full_size: 1.5e11\n"
        f"source_sha256: {h.hexdigest()}\n")
    return root


def test_traffic_read_while_sources_match(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profile_traffic(SOURCES, SUMMARY) == 1.5e11


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


# ---------------------------------------------------------------- comparators
def _calls_in_main():
    """(callee name, argument names) of every call in bench.main."""
    import ast
    import inspect
    tree = ast.parse(inspect.getsource(bench.main))
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Call) and isinstance(node.func, ast.Name):
            out.append((node.func.id, [a.id for a in node.args if isinstance(a, ast.Name)]))
    return out


def test_plain_comparator_reference_is_a_private_snapshot():
    """The buffer the unfused pipeline is checked against is passed to no other
    comparator, and cuBLAS's 3M GEMM writes into a buffer of its own."""
    import inspect
    calls = _calls_in_main()
    plain = [args for name, args in calls if name == "plain_emulation"]
    assert plain, "main() no longer runs the plain comparator"
    ref = plain[0][-1]
    assert ref not in ("C", "A", "B")
    others = [name for name, args in calls if ref in args and name != "plain_emulation"]
    assert not others, f"the comparator's reference buffer {ref} is also passed to {others}"
    assert "C" not in inspect.signature(bench.gemm3m).parameters


def test_plain_comparator_compares_against_the_reference(monkeypatch):
    import torch
    wl = dict(m=4, n=3, k=5, N=2, single=False)
    ref = torch.arange(12, dtype=torch.float64).reshape(3, 4).to(torch.complex128)
    monkeypatch.setattr(bench, "plain_emulation_run", lambda *a: (ref.clone(), 1.0))
    assert bench.plain_emulation(None, torch, None, None, wl, ref)["bitexact_vs_fused"] is True
    other = ref.clone()
    other[1, 2] += 1.0
    monkeypatch.setattr(bench, "plain_emulation_run", lambda *a: (other, 1.0))
    assert bench.plain_emulation(None, torch, None, None, wl, ref)["bitexact_vs_fused"] is False
