"""The committed ncu summaries that bench.py reads (DRAM traffic per launch of
the scoring kernel) were taken on the kernel source as it stands: the hash of
the kernel's source recorded with each capture equals the current one, so the
bench line's roofline `traffic` is not silently dropped after a kernel change."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("form", ["bf16x2", "exact", "exact_pair", "bf16x2_pair"])
def test_scoring_profile_matches_kernel_source(form):
    sys.path.insert(0, ROOT)
    import bench
    d = json.load(open(os.path.join(ROOT, "profiles", f"score_tc_{form}_n4096.json")))
    assert d["kernel_sha"] == bench._kernel_hash(form)
    assert bench._traffic(form) == d["dram_bytes_per_launch"] > 0


def test_exact_epilogue_label():
    """The bench names the exact kernel's epilogue mode by the library's rule:
    one int32 sum per warp unless 32 max|q|^2 2^(r-1) Nv_pad >= 2^31."""
    sys.path.insert(0, ROOT)
    import bench
    assert not bench._exact_split((10, 5, 0), [1.0, 2.0, 3.0, -2.0], 4096)      # the 16^3 cubic cell
    assert bench._exact_split((10, 5, 4), [49.0 / 16, 1.0, -1.0, -49.0 / 16], 512)   # charges x16, max 49
