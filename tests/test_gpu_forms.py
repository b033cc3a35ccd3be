"""Batched (graph-captured) and cached-rerun forms of the path (needs a GB300).

Each form must reproduce the plain amber_solve result: the kernels are
deterministic, so results are compared bit for bit, and one case per form is
also checked against the FP64 oracle.
"""
import numpy as np
import pytest
import torch

from oracle import amber_oracle as O
from paper_2109_10375_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2109_10375_gb300 import binding
    return binding


def test_solve_ex_keeps_order_and_rank_masses(B):
    n, box, l = 64, 100.0, 3.0
    S, m = synth.realisation(n, box, 3)
    h = B.history(8.0, 4.0, 3.0)
    with B.Context(n ** 3) as ctx:
        Sd, md = S.cuda(), m.cuda()
        J = torch.empty_like(Sd)
        z1 = ctx.solve(Sd, md, box, l, h, J_out=J)
        order = torch.empty(n ** 3, dtype=torch.int32, device="cuda")
        mrank = torch.empty(n ** 3, device="cuda")
        z2 = torch.empty_like(Sd)
        ctx.solve_ex(Sd, md, box, l, h, z2, order, mrank)
        assert ctx.sync_status() == 0
        assert torch.equal(z1, z2)
        o = order.cpu().numpy().astype(np.int64)
        np.testing.assert_array_equal(o, np.argsort(-J.cpu().numpy().reshape(-1), kind="stable"))
        np.testing.assert_array_equal(mrank.cpu().numpy(), m.numpy().reshape(-1)[o])


def test_history_only_rerun_from_cached_order(B):
    n, box, l = 64, 100.0, 3.0
    S, m = synth.realisation(n, box, 4)
    with B.Context(n ** 3) as ctx:
        Sd, md = S.cuda(), m.cuda()
        order = torch.empty(n ** 3, dtype=torch.int32, device="cuda")
        mrank = torch.empty(n ** 3, device="cuda")
        z = torch.empty_like(Sd)
        ctx.solve_ex(Sd, md, box, l, B.history(8.0, 4.0, 3.0), z, order, mrank)
        for hist in [(7.0, 3.0, 2.0), (9.0, 5.0, 4.0), (6.5, 6.0, 1.5)]:
            h = B.history(*hist)
            z_hit = ctx.assign_zre_ranked(order, mrank, h, torch.empty(n ** 3, device="cuda"))
            z_full = ctx.solve(Sd, md, box, l, h)
            assert ctx.sync_status() == 0
            assert torch.equal(z_hit, z_full.reshape(-1))
            zo = O.assign_zre(order.cpu().numpy().astype(np.int64), m.double().numpy().reshape(-1),
                              O.history_table(*hist))
            assert np.max(np.abs(z_hit.cpu().numpy() - zo)) < 5e-5


def test_batch_graph_matches_individual_solves(B, monkeypatch):
    # the references are solved before the batch exists: keep the batch on
    # the same (default) choices, so the results must agree bit for bit
    monkeypatch.setenv("AMBER_AUTOTUNE", "0")
    rng = np.random.default_rng(5)
    specs = [(32, 50.0)] * 5 + [(64, 100.0)] * 3 + [(128, 100.0)] * 2
    items, ref = [], []
    ctxs = [B.Context(128 ** 3) for _ in range(3)]
    try:
        for i, (n, box) in enumerate(specs):
            S, m = synth.realisation(n, box, 100 + i, device="cuda")
            l = float(rng.uniform(1, 20))
            hist = (float(rng.uniform(6.5, 9)), float(rng.uniform(2, 6)), float(rng.uniform(1.5, 5)))
            h = B.history(*hist)
            z = torch.full_like(S, -1.0)
            items.append((S, m, box, l, h, z))
            ref.append(ctxs[0].solve(S, m, box, l, h))
        assert ctxs[0].sync_status() == 0
        batch = B.Batch(ctxs, items)
        for rep in range(2):  # replays give the same answer
            for it in items:
                it[5].fill_(-1.0)
            batch.launch()
            torch.cuda.synchronize()
            for c in ctxs:
                assert c.sync_status() == 0
            for it, r in zip(items, ref):
                assert torch.equal(it[5], r)
        # one item against the oracle
        S, m, box, l, h, z = items[-1]
        hist = (h.z_mid, h.dz, h.Az)
        _, _, zo = O.solve(S.double().cpu().numpy(), m.double().cpu().numpy(), box, l, *hist)
        assert np.mean(np.abs(z.cpu().numpy().reshape(-1) - zo) > 1e-3) <= 1e-4
        batch.close()
    finally:
        for c in ctxs:
            c.close()


def test_serving_results_same_alone_and_in_the_mix(B):
    from paper_2109_10375_gb300 import serve
    reqs = serve.poisson_requests(40, rate=2000.0, seed=11, sizes=(32, 64), size_p=(0.5, 0.5), n_realisations=4)

    def clone(qs):
        return [serve.Request(q.rid, q.arrival, q.realisation, q.n, q.l_mfp, q.delta_c, q.history) for q in qs]

    alone = clone(reqs)
    srv = serve.Server(n_slots=1, max_n=64, cache_bytes=1e9, hbm_reserve=0, keep_outputs=True)
    srv.prepare(alone)
    for q in alone:  # one at a time, nothing else on the GPU
        srv.run([q], realtime=False)
    srv.close()
    mix = clone(reqs)
    srv = serve.Server(n_slots=4, max_n=64, cache_bytes=1e9, hbm_reserve=0, keep_outputs=True)
    srv.prepare(mix)
    srv.run(mix, realtime=True)
    stats = serve.summarize(mix)
    srv.close()
    assert stats["hit_rate"] > 0.3
    overlapped = sum(1 for a in mix for b in mix if a is not b and a.start < b.done and b.start < a.done)
    assert overlapped > 0  # requests really ran concurrently
    for a, b in zip(alone, mix):
        assert torch.equal(a.z, b.z), a.rid
    # one 64^3 request against the oracle, at the stated tolerance: > 1e-3 in at
    # most 1e-4 of the cells
    q = next(x for x in reversed(mix) if x.n == 64)
    box = serve.BOX_PER_CELL.get(q.n, 100.0 / 128) * q.n
    from paper_2109_10375_gb300 import synth as sy
    d = sy.gaussian_density(q.n, box, 1000 + q.realisation).float().double().numpy()
    So, mo = O.source_field(d, q.delta_c, 0.7)
    _, _, zo = O.solve(So, mo, box, q.l_mfp, *q.history)
    assert np.mean(np.abs(q.z.cpu().numpy().reshape(-1) - zo) > 1e-3) <= 1e-4


@pytest.mark.parametrize("n,variant", [(32, 0), (64, 0), (128, 0), (128, 1)])
def test_solve_from_a_kept_spectrum_equals_the_full_solve(B, n, variant):
    # amber_source_spectrum + amber_solve_spectrum (two l_mfp values from one
    # kept spectrum) against amber_solve_ex on the source field: bit-equal
    box = 100.0 * n / 128
    S, m = synth.realisation(n, box, 5, device="cuda")
    h = B.history(7.5, 4.0, 3.0)
    with B.Context(n ** 3) as ctx:
        ctx.set_tuning(n, fft_variant=variant)
        spec = ctx.source_spectrum(S)
        assert spec.numel() == B.spectrum_bytes(n) == n * n * (n // 2 + 2) * 8
        kept = spec.clone()
        for l in (3.0, 11.0):
            outs = []
            for from_spec in (False, True):
                z = torch.empty_like(S)
                J = torch.empty_like(S)
                order = torch.empty(n ** 3, dtype=torch.int32, device="cuda")
                mr = torch.empty(n ** 3, device="cuda")
                if from_spec:
                    ctx.solve_spectrum(spec, m, box, l, h, z, order, mr, J_out=J)
                else:
                    ctx.solve_ex(S, m, box, l, h, z, order, mr, J_out=J)
                outs.append((z, J, order, mr))
            assert ctx.sync_status() == 0
            for a, b in zip(*outs):
                assert torch.equal(a, b)
        assert torch.equal(spec, kept)  # read only


def test_serving_admission_waits_and_evicts_with_the_same_results(B):
    # a device-memory budget that holds the cache entries of only a couple of
    # requests at a time: requests wait for running ones to end, entries are
    # evicted, and every result is the one the request gets alone
    from paper_2109_10375_gb300 import serve
    reqs = serve.poisson_requests(30, rate=3000.0, seed=13, sizes=(32, 64), size_p=(0.4, 0.6), n_realisations=3)

    def clone(qs):
        return [serve.Request(q.rid, q.arrival, q.realisation, q.n, q.l_mfp, q.delta_c, q.history) for q in qs]

    alone = clone(reqs)
    srv = serve.Server(n_slots=1, max_n=64, cache_bytes=1e9, hbm_reserve=0, keep_outputs=True)
    srv.prepare(alone)
    for q in alone:
        srv.run([q], realtime=False)
    srv.close()
    tight = clone(reqs)
    srv = serve.Server(n_slots=4, max_n=64, cache_bytes=1e9, hbm_reserve=0, keep_outputs=True)
    miss64 = srv._order_bytes(64) + srv._spec_bytes(64) + 4 * 64 ** 3
    budget = int(2.2 * miss64)
    srv.free_bytes = lambda: budget - srv.cached
    srv.prepare(tight)
    # every request queued at once, and each held on the GPU a few
    # milliseconds (a fixed-length busy wait ahead of its work on the slot's
    # stream), so running requests keep their entries while later ones ask
    # for room
    launch = srv._launch

    def slow_launch(slot, q, now):
        with torch.cuda.stream(slot.stream):
            torch.cuda._sleep(10_000_000)
        launch(slot, q, now)

    srv._launch = slow_launch
    srv.run(tight, realtime=False)
    waits, evictions = srv.waiting_hbm, srv.evictions
    srv.close()
    assert waits > 0 and evictions > 0, (waits, evictions)
    for a, b in zip(alone, tight):
        assert torch.equal(a.z, b.z), a.rid


def test_batch_is_one_launch_per_stage_with_mixed_tunings_and_weightings(B, monkeypatch):
    # three grid sizes, two digit widths, FFT variant 1 on one size, mass and
    # growth-rescaled weightings: bit-equal to individual solves with the same
    # choices, and a graph whose kernel nodes do not grow with the item count
    monkeypatch.setenv("AMBER_AUTOTUNE", "0")
    rng = np.random.default_rng(9)
    specs = [(16, 25.0)] * 3 + [(64, 100.0)] * 6 + [(128, 100.0)] * 4
    ctx = B.Context(128 ** 3)
    try:
        ctx.set_tuning(16, sort_digit_bits=9)
        ctx.set_tuning(64, sort_digit_bits=8)
        ctx.set_tuning(128, fft_variant=1, sort_digit_bits=9)
        items, ref = [], []
        for i, (n, box) in enumerate(specs):
            S, m = synth.realisation(n, box, 300 + i, device="cuda")
            l = float(rng.uniform(1, 20))
            w = B.AMBER_WEIGHT_MASS_GROWTH if i % 3 == 1 else B.AMBER_WEIGHT_MASS
            h = B.history(float(rng.uniform(6.5, 9)), float(rng.uniform(2, 6)), float(rng.uniform(1.5, 5)), weighting=w)
            items.append((S, m, box, l, h, torch.full_like(S, -1.0)))
            ref.append(ctx.solve(S, m, box, l, h))
        assert ctx.sync_status() == 0
        batch = B.Batch([ctx], items)
        # 5 transform passes x 3 sizes, (histogram + offsets + 4 digit passes)
        # x 2 widths, thresholds + 2 scan forms + scatter
        assert batch.kernel_nodes() == 5 * 3 + 6 * 2 + 4
        batch.launch()
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
        for it, r in zip(items, ref):
            assert torch.equal(it[5], r)
        batch.close()
    finally:
        ctx.close()


@pytest.mark.parametrize("n,pinned", [(32, False), (64, True), (128, True)])
def test_solve_from_host_buffers_equals_the_device_solve(B, n, pinned):
    # amber_solve_host: host inputs copied in, solved, z_re copied out on the
    # stream; the result is the device solve's, bit for bit, call after call
    box, l = 100.0 * n / 128, 4.0
    S, m = synth.realisation(n, box, 7)
    h = B.history(7.8, 3.5, 2.5)
    with B.Context(n ** 3) as ctx:
        ref = ctx.solve(S.cuda(), m.cuda(), box, l, h).cpu()
        Sh, mh = (S.pin_memory(), m.pin_memory()) if pinned else (S.contiguous(), m.contiguous())
        for rep in range(2):
            zh = torch.full(S.shape, -1.0, pin_memory=pinned)
            ctx.solve_host(Sh, mh, box, l, h, zh)
            torch.cuda.synchronize()
            assert ctx.sync_status() == 0
            assert torch.equal(zh, ref)


def test_host_buffer_solves_on_contexts_in_turn(B):
    # contexts used in turn on their own streams: each call's solve waits for
    # the previous call's (copies in do not), and every result is the device
    # solve's
    n, box, l = 64, 50.0, 4.0
    S, m = synth.realisation(n, box, 8)
    h = B.history(8.0, 4.0, 3.0)
    ctxs = [B.Context(n ** 3) for _ in range(3)]
    try:
        ref = ctxs[0].solve(S.cuda(), m.cuda(), box, l, h).cpu()
        Sh, mh = S.pin_memory(), m.pin_memory()
        streams = [torch.cuda.Stream() for _ in ctxs]
        outs = [torch.full(S.shape, -1.0, pin_memory=True) for _ in range(7)]
        for i, zh in enumerate(outs):
            k = i % len(ctxs)
            ctxs[k].solve_host(Sh, mh, box, l, h, zh, stream=streams[k])
        torch.cuda.synchronize()
        for c in ctxs:
            assert c.sync_status() == 0
        for zh in outs:
            assert torch.equal(zh, ref)
    finally:
        for c in ctxs:
            c.close()
