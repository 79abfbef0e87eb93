"""The benchmark's roofline accounting for each scoring kernel and tile shape:
the executed tensor work per launch (the upper block triangle of the symmetric
operand, 528 blocks of 128 x 128 at Nv_pad = 4,096; on CTA pairs one more zero
block per pair-panel below the diagonal, 544; the configuration-lane kernel
over the batch rounded up to 128 instead of 256), the kernel named in the line,
and achieved = work / kernel time against the measured peak (TF32 at half the
BF16 rate).  CPU only: the function takes the kernel time as an argument."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def upper_blocks(nbm):
    return nbm * (nbm + 1) // 2


def pair_blocks(nbm):
    return sum(min(2, nbm - 2 * P) * (nbm - 2 * P) for P in range((nbm + 1) // 2))


def test_block_counts_of_the_benchmark_cell():
    assert upper_blocks(32) == 528
    assert pair_blocks(32) == 544            # 16 pair-panels, one zero block each
    assert pair_blocks(7) == upper_blocks(7) + 3   # odd panel count: the last pair-panel has one panel


@pytest.mark.parametrize("form,terms,tile_m,tile_n,split,kernel,blocks,ncfg", [
    ("exact", 5, 256, 256, False, "k_score_exact_pair<false>", 544, 4096),
    ("exact", 5, 128, 256, False, "k_score_exact<256, false>", 528, 4096),
    ("exact", 5, 128, 256, True, "k_score_exact<256, true>", 528, 4096),
    ("exact", 5, 256, 128, False, "k_score_exact_ct<false>", 528, 4096),
    ("bf16x2", 2, 256, 256, False, "k_score_tc_pair<2,false>", 544, 4096),
    ("bf16x2", 2, 128, 256, False, "k_score_tc<2,false,256>", 528, 4096),
    ("tf32x2", 2, 256, 256, False, "k_score_tc_pair<2,true>", 544, 4096),
    ("tf32x2", 2, 128, 256, False, "k_score_tc<2,true,256>", 528, 4096),
])
def test_executed_work_and_kernel_label(form, terms, tile_m, tile_n, split, kernel, blocks, ncfg):
    N = B = 4096
    kern_ms = 0.2
    r = bench._roofline(form, terms, kern_ms, 10, N, B, tile_m, split, tile_n)
    flops = terms * 2.0 * 128 * 128 * blocks * ncfg
    assert r["kernel"] == kernel
    assert r["flops_per_launch"] == flops
    assert r["useful_flops_per_launch"] == 2.0 * N * N * B
    peak, _, _ = bench._peaks()
    expect_peak = peak / 2.0 if "tf32" in form else peak
    assert r["peak"] == pytest.approx(expect_peak)
    assert r["achieved"] == pytest.approx(flops / (kern_ms / 1e3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / expect_peak)


def test_configuration_lane_kernel_counts_blocks_of_128():
    """The configuration-lane kernel covers the batch in blocks of 128, the
    other shapes the batch padded to 256: B = 1,000 gives 1,024 both ways,
    B = 600 gives 640 against 768."""
    for B, ncfg_ct, bpad in [(1000, 1024, 1024), (600, 640, 768)]:
        r = bench._roofline("exact", 5, 1.0, 1, 4096, B, 256, False, 128)
        assert r["flops_per_launch"] == 5 * 2.0 * 128 * 128 * 528 * ncfg_ct
        r = bench._roofline("exact", 5, 1.0, 1, 4096, B, 128, False, 256)
        assert r["flops_per_launch"] == 5 * 2.0 * 128 * 128 * 528 * bpad
