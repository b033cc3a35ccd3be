"""Host logic of the serving loop (no GPU): the seeded request stream, the
bytes a request would add to the cache, and admission with least-recently-used
eviction under a cache budget and a free-HBM reserve.  The server is built
without its slots (contexts and streams need a device); cache entries are
placed by hand in the layout the server keeps:
key -> [tensors, bytes, running users, ready event]."""
import collections

import numpy as np
import pytest


@pytest.fixture(scope="module")
def S():
    import __graft_entry__ as g
    g.build()
    from paper_2109_10375_gb300 import serve
    return serve


def _server(S, cache_bytes, free, hbm_reserve=0.0, keep_outputs=False):
    srv = S.Server.__new__(S.Server)  # no slots: no device needed
    srv.cache = collections.OrderedDict()
    srv.cache_bytes = cache_bytes
    srv.cached = 0
    srv.hbm_reserve = hbm_reserve
    srv.keep_outputs = keep_outputs
    srv.free_bytes = lambda: free[0]
    srv.waited = set()
    srv.evictions = 0
    return srv


def _add(srv, key, nbytes, users=0):
    srv.cache[key] = [None, nbytes, users, None]
    srv.cached += nbytes


def _req(S, r=0, n=128, l=5.0, dc=1.686):
    return S.Request(rid=0, arrival=0.0, realisation=r, n=n, l_mfp=l, delta_c=dc, history=(8.0, 4.0, 3.0))


def test_request_stream_is_seeded_and_follows_its_mix(S):
    a = S.poisson_requests(2000, 200.0, seed=3)
    b = S.poisson_requests(2000, 200.0, seed=3)
    assert [(q.arrival, q.n, q.realisation, q.l_mfp, q.delta_c, q.history) for q in a] == \
           [(q.arrival, q.n, q.realisation, q.l_mfp, q.delta_c, q.history) for q in b]
    t = np.array([q.arrival for q in a])
    assert np.all(np.diff(t) > 0)
    # Poisson arrivals at 200/s: mean gap 5 ms
    assert abs(np.mean(np.diff(t)) - 1 / 200.0) < 0.0005
    sizes = np.array([q.n for q in a])
    for n, p in zip((128, 256, 512), (0.6, 0.3, 0.1)):
        assert abs(np.mean(sizes == n) - p) < 0.04
    # a request repeats its (realisation, grid)'s last l_mfp and threshold,
    # or changes exactly one of them
    last = {}
    for q in a:
        key = (q.realisation, q.n)
        if key in last:
            l, dc = last[key]
            assert (q.l_mfp == l) + (q.delta_c == dc) >= 1
        last[key] = (q.l_mfp, q.delta_c)


def test_need_counts_only_the_missing_entries(S):
    srv = _server(S, 1e12, [1e12])
    q = _req(S, n=128)
    order_b, spec_b = S.Server._order_bytes(128), S.Server._spec_bytes(128)
    assert order_b == 8 * 128 ** 3
    assert spec_b > 4 * 128 ** 3  # the half spectrum and the masses
    assert srv._need(q) == order_b + spec_b
    _add(srv, S.Server._spec_key(q), spec_b)
    assert srv._need(q) == order_b  # a new l_mfp over a kept spectrum
    _add(srv, S.Server._order_key(q), order_b)
    assert srv._need(q) == 0  # history only
    srv.keep_outputs = True
    assert srv._need(_req(S, n=128, l=7.0)) == order_b + 4 * 128 ** 3


def test_admission_evicts_least_recently_used_idle_entries(S):
    q = _req(S, r=9, n=128)
    need = S.Server._order_bytes(128) + S.Server._spec_bytes(128)
    srv = _server(S, cache_bytes=need + 3 * 10 ** 6, free=[1e12])
    for i in range(5):
        _add(srv, ("order", i, 64, 5.0, 1.686), 10 ** 6)
    srv.cache[("order", 1, 64, 5.0, 1.686)][2] = 1  # in use by a running request
    assert srv._admissible(q)
    # two idle entries had to go, oldest first; the running one stays
    assert srv.evictions == 2
    assert list(srv.cache) == [("order", i, 64, 5.0, 1.686) for i in (1, 3, 4)]
    assert srv.cached == 3 * 10 ** 6


def test_admission_waits_when_only_running_entries_are_left(S):
    q = _req(S, r=9, n=128)
    srv = _server(S, cache_bytes=10 ** 6, free=[1e12])
    _add(srv, ("order", 1, 64, 5.0, 1.686), 10 ** 6, users=1)
    assert not srv._admissible(q)
    assert srv.evictions == 0 and srv.cached == 10 ** 6


def test_admission_keeps_the_free_hbm_reserve(S):
    q = _req(S, r=9, n=128)
    need = S.Server._order_bytes(128) + S.Server._spec_bytes(128)
    free = [need + 5 * 10 ** 6]
    srv = _server(S, cache_bytes=1e15, free=free, hbm_reserve=8 * 10 ** 6)
    for i in range(4):
        _add(srv, ("order", i, 64, 5.0, 1.686), 10 ** 6)
    # the fake's free bytes grow as entries are evicted, as the device's would
    orig = srv._evict_one

    def evict(protect=()):
        ok = orig(protect)
        if ok:
            free[0] += 10 ** 6
        return ok

    srv._evict_one = evict
    assert srv._admissible(q)
    assert srv.evictions == 3 and free[0] - need >= 8 * 10 ** 6


def test_admission_never_evicts_the_requests_own_entries(S):
    q = _req(S, r=2, n=128, l=9.0)
    spec_b = S.Server._spec_bytes(128)
    srv = _server(S, cache_bytes=spec_b + S.Server._order_bytes(128) - 1, free=[1e12])
    _add(srv, S.Server._spec_key(q), spec_b)  # idle, but the request will read it
    assert not srv._admissible(q)
    assert S.Server._spec_key(q) in srv.cache and srv.evictions == 0
