"""Autotuner for the search's launch shapes.

The shape with the largest effect is G, the number of lanes that share one
(query, train) pair in the FP32 DTW kernel: G = 1 gives every lane its own
pair (no shuffles, but many concurrent pairs, so uneven early-abandoning
leaves lanes idle when work is scarce); larger G sweeps each pair faster with
more exchange per cell; full windows also have the row layouts.  The tuner
times ``nn_dtw_search`` with every admissible G on the caller's data
(results never depend on G) and keeps the fastest, cached in memory and
optionally in a JSON file keyed by device, L, W, V and power-of-two buckets
of N and Q.  ``tune_search_flags`` then also picks the cascade's second
stage for that data: none, the reverse bound (``nndtw.REVERSE``) or the bound
with the LB_Improved bridge (``nndtw.IMPROVED``).
"""
from __future__ import annotations

import json
import os
import threading

from . import nndtw

_lock = threading.Lock()
_mem: dict = {}

# the cascade's second stage: none, the reverse bound, the LB_Improved bridge
CASCADE_CHOICES = (0, nndtw.REVERSE, nndtw.IMPROVED)
# the bound pass's tile shapes tried against the library's own choice
LB_TILE_CHOICES = (1, 2, 3)


def _bucket(n: int) -> int:
    b = 1
    while b < n:
        b <<= 1
    return b


def key(device_name: str, N: int, Q: int, L: int, W: int, V: int) -> str:
    return f"{device_name}|L{L}|W{min(W, L - 1)}|V{V}|N{_bucket(N)}|Q{_bucket(Q)}"


def admissible_groups(W: int, L: int | None = None):
    """Lanes-per-pair choices of the diagonal layout for window W, plus the
    row layouts when the window is full (W >= L-1): 32 lanes per pair for
    L <= 2048 (a CTA of 128 lanes per pair up to 4096, of 256 up to 8192),
    16 for L <= 1024, 8 for L <= 512."""
    out = []
    for g in (1, 2, 4, 8, 16, 32):
        h = (W + g) // g
        if h <= 32 and not (h == 1 and g != W + 1):
            out.append(g)
    if L is not None and W >= L - 1:
        if L <= nndtw.NNDTW_MAX_L:
            out.append(nndtw.ROWS_GROUP)
        if L <= 1024:
            out.append(nndtw.ROWS16_GROUP)
        if L <= 512:
            out.append(nndtw.ROWS8_GROUP)
    return out


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _median_ms(train, labels, test, W, V, flags, workspace, out, reps):
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nndtw.nn_dtw_search(train, labels, test, W, V, flags=flags, workspace=workspace, out=out)
    times = []
    for _ in range(reps):
        s.record()
        nndtw.nn_dtw_search(train, labels, test, W, V, flags=flags, workspace=workspace, out=out)
        e.record()
        e.synchronize()
        times.append(s.elapsed_time(e))
    return sorted(times)[len(times) // 2]


def tune_search(train, labels, test, W: int, V: int, workspace=None, out=None, reps: int = 3,
                cache_path: str | None = None) -> int:
    """Return the fastest lanes-per-pair G for this search (0 if nothing to tune)."""
    import torch
    N, L = train.shape
    Q = test.shape[0]
    Weff = min(W, L - 1)
    dev = torch.cuda.get_device_name(train.device)
    k = key(dev, N, Q, L, Weff, V)
    with _lock:
        if k in _mem:
            return _mem[k]
        if cache_path and k in _load(cache_path):
            _mem[k] = int(_load(cache_path)[k])
            return _mem[k]
    groups = admissible_groups(Weff, L)
    if not groups:
        return 0
    if workspace is None:
        workspace = torch.empty(nndtw.nn_dtw_workspace_size(N, Q, L, W, V), dtype=torch.uint8,
                                device=train.device)
    if out is None:
        out = (torch.empty(Q, dtype=torch.int32, device=train.device),
               torch.empty(Q, dtype=torch.int32, device=train.device),
               torch.empty(Q, dtype=torch.float64, device=train.device))
    best, best_ms = groups[0], float("inf")
    for g in groups:
        ms = _median_ms(train, labels, test, W, V, nndtw.DTW_GROUP(g), workspace, out, reps)
        if ms < best_ms:
            best, best_ms = g, ms
    with _lock:
        _mem[k] = best
        if cache_path:
            d = _load(cache_path)
            d[k] = best
            tmp = cache_path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(d, f, indent=1, sort_keys=True)
            os.replace(tmp, cache_path)
    return best


def tune_search_flags(train, labels, test, W: int, V: int, reps: int = 3,
                      cache_path: str | None = None) -> int:
    """Search flags for this data: the fastest lanes-per-pair choice, the
    cascade's second stage that makes the search fastest (none, the reverse
    bound ``nndtw.REVERSE`` or the bound with the LB_Improved bridge
    ``nndtw.IMPROVED``), then the fastest tile shape of the bound pass
    (``nndtw.LB_TILE``: 32 x 32, 64 x 64 or 128 x 64 queries x training
    series per CTA).  Results never depend on any of them."""
    import torch
    g = tune_search(train, labels, test, W, V, reps=reps, cache_path=cache_path)
    base = nndtw.DTW_GROUP(g) if g else 0
    N, L = train.shape
    Q = test.shape[0]
    k = "cascade|" + key(torch.cuda.get_device_name(train.device), N, Q, L, min(W, L - 1), V)
    with _lock:
        if k in _mem:
            return base | _mem[k]
    workspace = torch.empty(nndtw.nn_dtw_workspace_size(N, Q, L, W, V), dtype=torch.uint8,
                            device=train.device)
    out = (torch.empty(Q, dtype=torch.int32, device=train.device),
           torch.empty(Q, dtype=torch.int32, device=train.device),
           torch.empty(Q, dtype=torch.float64, device=train.device))
    best, best_ms = 0, None
    for extra in CASCADE_CHOICES:
        ms = _median_ms(train, labels, test, W, V, base | extra, workspace, out, reps)
        if best_ms is None or ms < best_ms:
            best, best_ms = extra, ms
    # the bound pass's tile shape, with the chosen layout and cascade
    tile, tile_ms = 0, best_ms
    for t in LB_TILE_CHOICES:
        ms = _median_ms(train, labels, test, W, V, base | best | nndtw.LB_TILE(t), workspace,
                        out, reps)
        if ms < tile_ms:
            tile, tile_ms = t, ms
    best |= nndtw.LB_TILE(tile) if tile else 0
    with _lock:
        _mem[k] = best
    return base | best


def tune_search_varlen(train, labels, test, W: int, V: int, workspace=None, out=None,
                       reps: int = 3) -> int:
    """Search flags for the unequal-length search (``nndtw.Ragged`` sets):
    the fastest lanes-per-pair choice of its diagonal DTW kernel (0 when the
    window has none to choose).  Results never depend on it."""
    import torch
    ml = max(train.max_len, test.max_len)
    groups = admissible_groups(min(W, ml - 1))
    if len(groups) < 2:
        return 0
    N, Q = train.n, test.n
    dev = train.values.device
    if workspace is None:
        workspace = torch.empty(nndtw.nn_dtw_varlen_workspace_size(N, Q, ml, W, V),
                                dtype=torch.uint8, device=dev)
    if out is None:
        out = (torch.empty(Q, dtype=torch.int32, device=dev),
               torch.empty(Q, dtype=torch.int32, device=dev),
               torch.empty(Q, dtype=torch.float64, device=dev))
    run = lambda f: nndtw.nn_dtw_search_varlen(train, labels, test, W, V, flags=f,
                                               workspace=workspace, out=out)
    best, best_ms = 0, float("inf")
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for g in groups:
        f = nndtw.DTW_GROUP(g)
        run(f)
        times = []
        for _ in range(reps):
            s.record()
            run(f)
            e.record()
            e.synchronize()
            times.append(s.elapsed_time(e))
        ms = sorted(times)[len(times) // 2]
        if ms < best_ms:
            best, best_ms = f, ms
    return best
