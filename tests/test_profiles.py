"""The committed ncu summaries (CPU only).

bench.py reports a kernel's DRAM traffic from its committed summary only
while the summary's kernel-source hash equals the current sources' hash, so
a kernel change without a new capture silently turns `traffic` into null.
These tests keep the evidence and the code in step: every summary names the
command that produced it, carries the current hash, and (where bench.py
reads it) a positive per-launch traffic figure."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _summaries():
    return sorted(f for f in os.listdir(PROFILES) if f.endswith(".md"))


def test_every_summary_gives_its_command():
    for f in _summaries():
        s = open(os.path.join(PROFILES, f)).read()
        assert "ncu " in s and "--clock-control none" in s, f
        assert "python bench.py" in s, f   # committed files only


def test_summaries_match_the_kernel_sources():
    sha = bench.kernel_src_sha()
    for f in _summaries():
        s = open(os.path.join(PROFILES, f)).read()
        m = re.search(r"Kernel source sha256 prefix at capture: `([0-9a-f]+)`", s)
        if m:
            assert m.group(1) == sha, f"{f} was captured from other kernel sources"


def test_traffic_read_by_the_bench():
    for tag in ("scatter_c2_64KiB", "split_hash_c2_64KiB", "crz_encode_c2_f32"):
        t = bench.profile_traffic(tag)
        assert t is not None and t > 0, tag
