"""Continuous-batching server: results equal alone and in a mix of concurrent
requests across datasets, equal to the direct search and to the oracle."""
import numpy as np
import pytest

from paper_1808_09617_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sets():
    specs = [dict(L=128, N=700, W=13, V=5, n_classes=8), dict(L=512, N=400, W=51, V=5, n_classes=8),
             dict(L=300, N=900, W=30, V=3, n_classes=8)]
    out = {}
    for d, sp in enumerate(specs):
        ds = synth.make_serving_set(d, sp)
        out[d] = (ds.train, ds.train_labels, sp["W"], sp["V"], sp)
    return out


def _server(sets, **kw):
    from paper_1808_09617_gb300 import serving
    return serving.Server({k: v[:4] for k, v in sets.items()}, **kw)


def test_alone_equals_in_the_mix(lib, orc, sets):
    probe_set = 1
    q, _ = synth.serving_queries(probe_set, sets[probe_set][4], 1, offset=12345)
    srv = _server(sets, n_slots=4, max_batch=64)
    try:
        alone = srv.submit(q[0], probe_set).result(timeout=60)
        futs, mine = [], None
        rng = np.random.default_rng(3)
        for k in range(400):
            sid = int(rng.integers(0, 3))
            qq, _ = synth.serving_queries(sid, sets[sid][4], 1, offset=k)
            futs.append((sid, qq[0], srv.submit(qq[0], sid)))
            if k == 200:
                mine = srv.submit(q[0], probe_set)
        in_mix = mine.result(timeout=120)
        res = [(sid, qq, f.result(timeout=120)) for sid, qq, f in futs]
        st = srv.latency_stats()
    finally:
        srv.close()
    assert alone[0] == in_mix[0] and alone[1] == in_mix[1]
    np.testing.assert_allclose(in_mix[2], alone[2], rtol=1e-4)
    assert st["completed"] == 402 and st["batches"] >= 2
    # every result of the mix equals the oracle's 1-NN
    for sid in range(3):
        train, labels, W, V, _ = sets[sid]
        qs = np.stack([qq for s_, qq, _ in res if s_ == sid])
        got = [r for s_, _, r in res if s_ == sid]
        bi, bl, bd = orc.nn_brute(train, labels, qs, W)
        assert [g[0] for g in got] == list(bi)
        assert [g[1] for g in got] == list(bl)
        np.testing.assert_allclose([g[2] for g in got], bd, rtol=1e-4)
    train, labels, W, V, _ = sets[probe_set]
    bi, _, _ = orc.nn_brute(train, labels, q, W)
    assert alone[0] == bi[0]


def test_small_memory_budget_splits_batches(lib, sets):
    srv = _server(sets, n_slots=2, max_batch=256, memory_budget=6 << 20, tune=False)
    try:
        futs = []
        for k in range(150):
            qq, _ = synth.serving_queries(0, sets[0][4], 1, offset=k)
            futs.append(srv.submit(qq[0], 0))
        res = [f.result(timeout=120) for f in futs]
        st = srv.latency_stats()
    finally:
        srv.close()
    assert len(res) == 150 and st["batches"] > 2


def test_set_larger_than_the_budget_is_refused(lib, sets):
    """A set whose one-query batch cannot fit the memory budget would never be
    served: the server refuses it at construction instead of hanging."""
    from paper_1808_09617_gb300 import serving
    with pytest.raises(ValueError):
        serving.Server({0: sets[0][:4]}, memory_budget=1 << 16, tune=False)


def test_serving_workload_full_size_matches_oracle(lib):
    """The serving workload at its configured size: 16 resident training sets
    (L in {128, 512, 1500}, 1,000-20,000 series each, W = 0.1 L, V = 5), 24
    queries per set submitted in a shuffled mix; every result equals the
    oracle's stored 1-NN (tests/golden/make_full_golden.py)."""
    from golden import make_full_golden as fg
    from paper_1808_09617_gb300 import serving
    specs = synth.serving_specs(16)
    resident = {}
    for d, sp in enumerate(specs):
        ds = synth.make_serving_set(d, sp)
        resident[d] = (ds.train, ds.train_labels, sp["W"], sp["V"])
    k = fg.SERVING_QUERIES_PER_SET
    golden = {(r[0], r[1]): r[2:] for r in fg.read(fg.SERVING_PATH)}
    assert len(golden) == 16 * k
    order = [(d, j) for d in range(16) for j in range(k)]
    np.random.default_rng(1500).shuffle(order)
    srv = serving.Server(resident, n_slots=4, max_batch=128, tune=False)
    try:
        futs = []
        for d, j in order:
            q, _ = synth.serving_queries(d, specs[d], 1, offset=j)
            futs.append(((d, j), srv.submit(q[0], d)))
        got = [(key, f.result(timeout=300)) for key, f in futs]
    finally:
        srv.close()
    for key, (idx, lab, dist) in got:
        gi, gl, gd = golden[key]
        assert (idx, lab) == (gi, gl), key
        assert abs(dist - gd) <= 1e-4 * gd, key
