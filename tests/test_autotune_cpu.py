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
    assert 64 in autotune.admissible_groups(3000, 3001)      # a CTA per pair up to 8192
    assert 64 in autotune.admissible_groups(8191, 8192)


def test_key_buckets():
    k1 = autotune.key("GB300", 500, 500, 256, 26, 5)
    k2 = autotune.key("GB300", 400, 300, 256, 26, 5)
    assert k1 == k2
    assert autotune.key("GB300", 500, 500, 256, 300, 5) == autotune.key("GB300", 500, 500, 256, 255, 5)


def test_tune_search_flags_picks_fastest_cascade_and_tile(monkeypatch):
    """The cascade's second stage is the fastest of none / reverse bound /
    LB_Improved bridge, then the bound pass's tile shape the fastest of the
    three (or the library's own choice when none is faster), chosen once per
    data key and then remembered (timings faked: no GPU here)."""
    import torch

    from paper_1808_09617_gb300 import nndtw
    calls = []
    fake_ms = {0: 5.0, nndtw.REVERSE: 4.0, nndtw.IMPROVED: 3.0}
    tile_gain = {0: 0.0, 1: -1.0, 2: 0.0, 3: 0.5}

    def median_ms(train, labels, test, W, V, flags, workspace, out, reps):
        calls.append(flags)
        tile = (flags & nndtw.LB_TILE_MASK) >> 19
        return fake_ms[flags & (nndtw.REVERSE | nndtw.IMPROVED)] - tile_gain[tile]

    monkeypatch.setattr(autotune, "tune_search", lambda *a, **k: 8)
    monkeypatch.setattr(autotune, "_median_ms", median_ms)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "fake-gpu")
    monkeypatch.setattr(nndtw, "nn_dtw_workspace_size", lambda *a: 64)
    monkeypatch.setattr(autotune, "_mem", {})
    train = torch.zeros((100, 32))
    test = torch.zeros((40, 32))
    labels = torch.zeros(100, dtype=torch.int32)
    f = autotune.tune_search_flags(train, labels, test, 3, 2, reps=1)
    assert f == nndtw.DTW_GROUP(8) | nndtw.IMPROVED | nndtw.LB_TILE(3)
    cascade = nndtw.REVERSE | nndtw.IMPROVED
    untiled = [c for c in calls if not c & nndtw.LB_TILE_MASK]
    assert sorted(c & cascade for c in untiled) == sorted(autotune.CASCADE_CHOICES)
    tiled = [c for c in calls if c & nndtw.LB_TILE_MASK]
    assert sorted((c & nndtw.LB_TILE_MASK) >> 19 for c in tiled) == sorted(autotune.LB_TILE_CHOICES)
    assert all(c & cascade == nndtw.IMPROVED for c in tiled)    # with the chosen cascade
    assert all(c & nndtw.DTW_GROUP_MASK == nndtw.DTW_GROUP(8) for c in calls)
    n = len(calls)
    assert autotune.tune_search_flags(train, labels, test, 3, 2, reps=1) == f
    assert len(calls) == n                       # remembered
    fake_ms[nndtw.IMPROVED] = 9.0
    tile_gain[3] = -2.0                          # no tile shape beats the library's choice
    f2 = autotune.tune_search_flags(train, labels, test[:3], 3, 2, reps=1)   # another Q bucket
    assert f2 == nndtw.DTW_GROUP(8) | nndtw.REVERSE
