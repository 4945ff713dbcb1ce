"""Host logic of the autotuner (CPU only)."""
from paper_1808_09617_gb300 import autotune


def test_admissible_groups():
    # W=26: 27 diagonal pairs; G=32 would need one pair per lane with no short lanes
    assert autotune.admissible_groups(26) == [1, 2, 4, 8, 16]
    assert autotune.admissible_groups(31) == [1, 2, 4, 8, 16, 32]
    assert autotune.admissible_groups(0) == [1]
    assert autotune.admissible_groups(1023) == [32]
    assert autotune.admissible_groups(1024) == []
    assert autotune.admissible_groups(100)[0] == 4
    assert autotune.admissible_groups(255, 256)[-3:] == [64, 65, 66]  # full window: row layouts
    assert autotune.admissible_groups(599, 600)[-2:] == [64, 65]     # 8 lanes hold L <= 512
    assert 65 not in autotune.admissible_groups(1999, 2000)          # 16 lanes hold L <= 1024
    assert 64 not in autotune.admissible_groups(100, 256)
    assert 64 in autotune.admissible_groups(3000, 3001)      # a CTA per pair up to 4096


def test_key_buckets():
    k1 = autotune.key("GB300", 500, 500, 256, 26, 5)
    k2 = autotune.key("GB300", 400, 300, 256, 26, 5)
    assert k1 == k2
    assert autotune.key("GB300", 500, 500, 256, 300, 5) == autotune.key("GB300", 500, 500, 256, 255, 5)
