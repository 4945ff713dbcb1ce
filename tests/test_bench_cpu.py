"""Host logic of bench.py (CPU only): the per-search kernel count behind the
`gpu_launches` claim."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_kernels_per_search_follows_the_flags():
    import bench
    from paper_1808_09617_gb300 import nndtw
    base = bench.kernels_per_search(0, nndtw)
    assert base == 12
    # the cascade's second stage: query envelopes and the filter
    assert bench.kernels_per_search(nndtw.REVERSE, nndtw) == base + 2
    # the LB_Improved bridge also builds and packs the second envelopes
    assert bench.kernels_per_search(nndtw.IMPROVED, nndtw) == base + 4
    assert bench.kernels_per_search(nndtw.IMPROVED | nndtw.REVERSE, nndtw) == base + 4
    # switched off by the flags that disable the stage
    assert bench.kernels_per_search(nndtw.REVERSE | nndtw.NO_REVERSE, nndtw) == base
    assert bench.kernels_per_search(nndtw.IMPROVED | nndtw.NO_PRUNE, nndtw) == base
    # layout choices never change the count
    assert bench.kernels_per_search(nndtw.DTW_GROUP(8) | nndtw.IMPROVED, nndtw) == base + 4
