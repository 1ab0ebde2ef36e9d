"""The benchmark's capture-derived figures (traffic per receiver-block, executed
instructions per sample*channel) are tied to the kernel sources they were captured
on: every entry that carries a source hash names a summary under profiles/ that
quotes the same hash, and the hash function covers the files that define the
kernel (so a change to any of them makes the figures read as null)."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _summaries():
    out = {}
    for f in os.listdir(PROFILES):
        if f.endswith(".md") or f.endswith(".txt"):
            out[f] = open(os.path.join(PROFILES, f)).read()
    return out


def test_every_hashed_figure_has_a_summary_quoting_its_hash():
    docs = _summaries()
    entries = list(bench.PROFILED.values()) + list(bench.PROFILED_CONFIG.values())
    hashed = [e for e in entries if re.fullmatch(r"[0-9a-f]{64}", e["src_sha256"])]
    assert hashed
    for e in hashed:
        h = e["src_sha256"]
        quote = f"{h[:8]}...{h[-8:]}"
        assert any(quote in t or h in t for t in docs.values()), quote


def test_source_hash_covers_the_segment_kernel_files():
    files = bench.KERNEL_SOURCES["segment"]
    assert "rx_cseg.cu" in files and "rx_device.cuh" in files and "rx_item.cuh" in files
    for f in files:
        assert os.path.exists(os.path.join(ROOT, "paper_1907_00463_gb300", "csrc", f)), f
    h = bench.kernel_sources_sha256("segment")
    assert re.fullmatch(r"[0-9a-f]{64}", h)
    assert bench.kernel_sources_sha256("no such schedule") != h
