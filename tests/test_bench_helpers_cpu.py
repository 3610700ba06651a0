"""Host-side helpers of the benchmark (no GPU): the hash-form bytes per window
that every variant's path fraction divides by, and the rule that a kernel's
DRAM traffic is read from its profile summary only while the kernel's device
sources are unchanged."""
import os
import shutil

import pytest

import bench


def test_hash_form_bytes_per_window():
    # the 2-Gbase metagenome at k = 31: 1.595 G windows, 539 M distinct, 114 M survivors
    b = bench.hash_form_bytes_per_window(31, 150, 1_595_046_060, 539_029_809, 114_076_936)
    assert b == pytest.approx(77.38, abs=0.01)
    # its parts: packed input 0.5 B/base over 120 windows of 150 bases, one 64-byte
    # table sector read and written back per window, the sweep and the survivors
    inp = 0.5 * 150 / 120
    sweep = 539_029_809 * (8 + 4 + 16) / 1_595_046_060
    out = 114_076_936 * (8 + 4 + 32 + 2) / 1_595_046_060
    assert b == pytest.approx(inp + 64 + sweep + out)
    # two-word keys read and write two sectors' worth
    assert bench.hash_form_bytes_per_window(55, 150, 1000, 0, 0) == pytest.approx(0.5 * 150 / 96 + 96)


def test_kernel_traffic_follows_the_sources(tmp_path, monkeypatch):
    root = tmp_path
    csrc = root / "paper_1809_07014_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (root / "profiles").mkdir()
    for f in bench.KERNEL_SOURCES["leaf_kernel"]:
        shutil.copy(os.path.join(bench.ROOT, "paper_1809_07014_gb300", "csrc", f), csrc / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench.kernel_source_sha("leaf_kernel")
    prof = root / "profiles" / "leaf_kernel.md"
    prof.write_text(f"source_sha256: {sha}\ndram_bytes_per_launch_full_size: 12345\n")
    assert bench.kernel_traffic("leaf_kernel") == 12345.0
    # a change to any of the kernel's device sources makes the figure stale
    with open(csrc / bench.KERNEL_SOURCES["leaf_kernel"][0], "a") as f:
        f.write("// changed\n")
    assert bench.kernel_traffic("leaf_kernel") is None
    assert bench.kernel_traffic("no_such_kernel") is None
