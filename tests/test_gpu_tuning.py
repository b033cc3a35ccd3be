"""Autotuning of the FP32 solve path (needs a GB300).

Every choice the tuner can make is checked on its own: the alternative FFT
tiles against the FP64 oracle (the intensity tolerance of the plain path) and
a plane wave at the sizes the oracle cannot transform quickly; the 8-bit and
warp-match rankings bit-exact against a stable sort, with z_re equal to the
default choice's.  Then the tuner itself, and the batch that tunes its sizes.
"""
import math

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


def _j_errors(Jg, Jo):
    Jg = np.asarray(Jg, np.float64).reshape(-1)
    Jo = np.asarray(Jo, np.float64).reshape(-1)
    d = np.abs(Jg - Jo)
    rms = math.sqrt(float(np.mean(Jo * Jo)))
    return float(np.linalg.norm(d) / np.linalg.norm(Jo)), float(np.max(d / np.maximum(np.abs(Jo), 5e-2 * rms)))


@pytest.mark.parametrize("n", [128, 256])
def test_fft_variant_1_vs_oracle(B, n):
    box, l = 100.0 * n / 128, 3.0
    S, _ = synth.realisation(n, box, 2)
    with B.Context(n ** 3) as ctx:
        ctx.set_tuning(n, fft_variant=1)
        J = ctx.radiation_field(S.cuda(), box, l)
        assert ctx.sync_status() == 0
        assert ctx.get_tuning(n)["fft_variant"] == 1
    rel_l2, max_rel = _j_errors(J.cpu().numpy(), O.radiation_field(S.double().numpy(), box, l))
    assert rel_l2 <= 1e-5 and max_rel <= 1e-4, (rel_l2, max_rel)


@pytest.mark.parametrize("n", [512, 1024])
def test_fft_variant_1_plane_wave(B, n):
    # S = cos(2 pi (3 x - 5 y + 7 z) / n) is an eigenfunction: J = K(|k|) S
    box, l = 1000.0 * n / 1024, 5.0
    i = torch.arange(n, device="cuda", dtype=torch.float64)
    ph = (7.0 * i.view(n, 1, 1) - 5.0 * i.view(1, n, 1) + 3.0 * i.view(1, 1, n)) * (2.0 * math.pi / n)
    S = torch.cos(ph).float()
    del ph
    K = float(O.kernel_transform(2.0 * math.pi / box * math.sqrt(83.0), l))
    with B.Context(n ** 3) as ctx:
        ctx.set_tuning(n, fft_variant=1)
        J = ctx.radiation_field(S, box, l)
        assert ctx.sync_status() == 0
    assert float((J - K * S).abs().max()) <= 1e-5 * K


@pytest.mark.parametrize("n,variant", [(64, 0), (128, 0), (128, 1), (256, 1), (512, 0), (512, 1), (1024, 0)])
def test_tma_z_pass_gives_the_same_solve(B, n, variant):
    # the z pass with TMA-staged tiles (one to four boxes of up to 256 rows
    # per tile; the last column tile holds one column, the rest zero fill)
    # does the plain z pass's arithmetic: intensities, z_re, order and masses
    # bit-equal, from the source and from a kept spectrum
    box, l = 100.0 * n / 128, 3.0
    S, m = synth.realisation(n, box, 43, device="cuda")
    h = B.history(8.0, 4.0, 3.0)
    outs = []
    with B.Context(n ** 3) as ctx:
        ctx.set_tuning(n, fft_variant=variant)
        spec = ctx.source_spectrum(S)  # the x and y passes of this variant's tiles
        for tma in (0, 1):
            ctx.set_tuning(n, zpass_tma=tma)
            assert ctx.get_tuning(n)["zpass_tma"] == tma
            z = torch.empty_like(S)
            J = torch.empty_like(S)
            order = torch.empty(n ** 3, dtype=torch.int32, device="cuda")
            mr = torch.empty(n ** 3, device="cuda")
            ctx.solve_ex(S, m, box, l, h, z, order, mr, J_out=J)
            z2 = torch.empty_like(S)
            ctx.solve_spectrum(spec, m, box, l, h, z2)
            Jr = ctx.radiation_field(S, box, l)
            assert ctx.sync_status() == 0
            assert torch.equal(z2, z) and torch.equal(Jr, J)
            outs.append((z, J, order, mr))
            del z2, Jr
    for a, b in zip(*outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("bits,match", [(8, 0), (8, 1), (9, 1)])
@pytest.mark.parametrize("n", [4, 8, 64, 128])
def test_ranking_choices_bit_exact(B, n, bits, match):
    # 4^3 and 8^3 leave the single sort tile ragged
    box, l = 100.0 * n / 128, 3.0
    S, m = synth.realisation(n, box, 5, device="cuda")
    h = B.history(8.0, 4.0, 3.0)
    with B.Context(n ** 3) as ctx:
        J = torch.empty_like(S)
        z0 = ctx.solve(S, m, box, l, h, J_out=J)
        ctx.set_tuning(n, 0, bits, match)
        order = torch.empty(n ** 3, dtype=torch.int32, device="cuda")
        mr = torch.empty(n ** 3, device="cuda")
        z1 = torch.empty_like(S)
        ctx.solve_ex(S, m, box, l, h, z1, order, mr)
        assert ctx.sync_status() == 0
        o = order.cpu().numpy().astype(np.int64)
        np.testing.assert_array_equal(o, np.argsort(-J.cpu().numpy().reshape(-1), kind="stable"))
        np.testing.assert_array_equal(mr.cpu().numpy(), m.cpu().numpy().reshape(-1)[o])
        assert torch.equal(z1, z0)


def test_set_tuning_rejects_bad_choices(B):
    with B.Context(64 ** 3) as ctx:
        for args in [(64, 1, 9, 0), (64, 0, 7, 0), (64, 0, 9, 2), (256, 0, 9, 0), (48, 0, 9, 0)]:
            with pytest.raises(B.AmberError):
                ctx.set_tuning(*args)
        for kw in [{"fuse_histogram": 2}, {"zpass_tma": 2}, {"zpass_tma": -1}]:
            with pytest.raises(B.AmberError):
                ctx.set_tuning(64, **kw)


def test_autotune_keeps_the_fastest_choice(B):
    n, box, l = 128, 100.0, 3.0
    S, m = synth.realisation(n, box, 6, device="cuda")
    h = B.history(8.0, 4.0, 3.0)
    with B.Context(n ** 3) as ctx:
        t = ctx.autotune(S, m, box, l)
        assert t["tuned"] == 1 and t["n"] == n
        assert min(t["fft_ms"]) > 0 and min(t["sort_ms"]) > 0
        assert t["fft_variant"] == int(np.argmin(t["fft_ms"]))
        assert t["fft_tma_ms"] > 0
        assert t["zpass_tma"] == int(t["fft_tma_ms"] < 0.98 * t["fft_ms"][t["fft_variant"]])
        k = int(np.argmin(t["sort_ms"]))
        assert (t["sort_digit_bits"], t["sort_match"]) == [(9, 0), (9, 1), (8, 0), (8, 1)][k]
        assert ctx.get_tuning(n) == t
        J = torch.empty_like(S)
        z = ctx.solve(S, m, box, l, h, J_out=J)
        assert ctx.sync_status() == 0
    # the tuned solve against the oracle's matching of the same intensities
    Jn = J.cpu().numpy().reshape(-1)
    order = np.argsort(-Jn, kind="stable")
    zo = O.assign_zre(order, m.double().cpu().numpy().reshape(-1), O.history_table(8.0, 4.0, 3.0))
    assert np.max(np.abs(z.cpu().numpy().reshape(-1) - zo)) < 5e-5


def test_batch_tunes_each_size_once(B, monkeypatch):
    monkeypatch.delenv("AMBER_AUTOTUNE", raising=False)
    specs = [(64, 100.0)] * 2 + [(128, 100.0)]
    ctxs = [B.Context(128 ** 3) for _ in range(2)]
    try:
        items = []
        for i, (n, box) in enumerate(specs):
            S, m = synth.realisation(n, box, 200 + i, device="cuda")
            items.append((S, m, box, 3.0, B.history(8.0, 4.0, 3.0), torch.empty_like(S)))
        batch = B.Batch(ctxs, items)
        for n in (64, 128):
            t = [c.get_tuning(n) for c in ctxs]
            assert t[0]["tuned"] == 1 and t[0] == t[1], t
        batch.launch()
        torch.cuda.synchronize()
        for it in items:  # the batch uses the tuned choices, as a plain solve now does
            z = ctxs[0].solve(*it[:5])
            assert torch.equal(z, it[5])
        assert all(c.sync_status() == 0 for c in ctxs)
        batch.close()
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("n,variant", [(8, 0), (64, 0), (256, 0), (256, 1), (512, 0)])
def test_fused_digit_counts_give_the_same_solve(B, n, variant):
    # 8-bit digits with the digit counts taken in the inverse x pass (raw
    # keys, no histogram pass) against the separate histogram of key - min:
    # the stable order is unique and the prefix sums exact, so z_re, the
    # order and the rank-order masses are bit-equal; the order is the stable
    # descending order of the intensities
    box, l = 100.0 * n / 128, 3.0
    S, m = synth.realisation(n, box, 41, device="cuda")
    h = B.history(8.0, 4.0, 3.0)
    outs = []
    with B.Context(n ** 3) as ctx:
        for fuse in (0, 1):
            ctx.set_tuning(n, fft_variant=variant, sort_digit_bits=8, fuse_histogram=fuse)
            z = torch.empty_like(S)
            J = torch.empty_like(S)
            order = torch.empty(n ** 3, dtype=torch.int32, device="cuda")
            mr = torch.empty(n ** 3, device="cuda")
            ctx.solve_ex(S, m, box, l, h, z, order, mr, J_out=J)
            assert ctx.sync_status() == 0
            assert ctx.get_tuning(n)["fuse_histogram"] == fuse
            if fuse:
                assert ctx.sort_passes() == 4  # raw 32-bit keys
            outs.append((z, J, order, mr))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    Jn = outs[1][1].cpu().numpy().reshape(-1).astype(np.float64)
    np.testing.assert_array_equal(outs[1][2].cpu().numpy(), np.argsort(-Jn, kind="stable"))
