"""The committed ncu summaries that bench.py reads (DRAM traffic per launch of
the scoring kernel) were taken on the kernel source as it stands: the hash of
the kernel's source recorded with each capture equals the current one, so the
bench line's roofline `traffic` is not silently dropped after a kernel change."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("form", ["bf16x2", "exact"])
def test_scoring_profile_matches_kernel_source(form):
    sys.path.insert(0, ROOT)
    import bench
    d = json.load(open(os.path.join(ROOT, "profiles", f"score_tc_{form}_n4096.json")))
    assert d["kernel_sha"] == bench._kernel_hash(form)
    assert bench._traffic(form) == d["dram_bytes_per_launch"] > 0
