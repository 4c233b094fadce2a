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
    """Each summary names the translation unit it was captured from, and its
    hash equals that unit's (and its device headers') current hash."""
    for f in _summaries():
        s = open(os.path.join(PROFILES, f)).read()
        shas = bench.summary_sha_ok(s)
        if shas is None:
            continue
        unit = bench.SHA_LINE.search(s).group(2)
        assert unit in bench.KERNEL_UNITS, f"{f} names no kernel translation unit"
        assert shas[0] == shas[1], f"{f} was captured from other {unit} sources"


def test_unit_hash_follows_its_headers():
    """A unit's hash covers the headers it includes: every kernel unit's hash
    differs from the hash of the unit's own file alone."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2008_10596_gb300", "csrc")
    for u in bench.KERNEL_UNITS:
        h = hashlib.sha256()
        h.update(u.encode())
        h.update(open(os.path.join(csrc, u), "rb").read())
        assert bench.kernel_src_sha(u) != h.hexdigest()[:16], u


def test_traffic_read_by_the_bench():
    for tag in ("scatter_c2_64KiB", "split_hash_c2_64KiB", "crz_encode_c2_f32"):
        t = bench.profile_traffic(tag)
        assert t is not None and t > 0, tag
