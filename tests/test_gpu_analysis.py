"""Analysis of z_re fields on the GPU (Sec. 2.3) against the FP64 oracle, through the C ABI.

Tolerances: the transforms are FP32 and the shell sums FP64, so shell spectra
agree to ~1e-5 relative (the FFT's own rounding); the mode counts are exact
integers; delta_z is an FP32 field with an FP64 mean.
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


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(128 ** 3)
    yield c
    c.close()


def _cpu(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check_spectra(got, ref, rtol=2e-5):
    k, Paa, Pbb, Pab, modes = ref
    np.testing.assert_array_equal(got["modes"], modes)
    live = modes > 0
    np.testing.assert_allclose(got["k"][live], k[live], rtol=1e-6)
    for key, P in (("Paa", Paa), ("Pbb", Pbb), ("Pab", Pab)):
        scale = np.max(np.abs(P))
        np.testing.assert_allclose(got[key], P, rtol=rtol, atol=1e-6 * scale, err_msg=key)


@pytest.mark.parametrize("n", [4, 8, 16, 64, 128])
def test_power_spectrum_vs_oracle(ctx, B, n):
    g = np.random.default_rng(n)
    a = g.normal(size=(n, n, n)).astype(np.float32)
    b = (0.5 * a + g.normal(size=(n, n, n))).astype(np.float32)
    box = 37.0
    got = _cpu(ctx.power_spectrum(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), box))
    assert ctx.sync_status() == 0
    _check_spectra(got, O.power_spectrum(a.astype(np.float64), b.astype(np.float64), box))


def test_power_spectrum_auto_only(ctx, B):
    n = 32
    a = np.random.default_rng(1).normal(size=(n, n, n)).astype(np.float32)
    ta = torch.from_numpy(a).cuda()
    one = _cpu(ctx.power_spectrum(ta, None, 10.0))
    two = _cpu(ctx.power_spectrum(ta, ta, 10.0))
    np.testing.assert_array_equal(one["Paa"], two["Paa"])
    assert np.all(one["Pbb"] == 0) and np.all(one["Pab"] == 0)
    np.testing.assert_allclose(two["Pab"], two["Paa"], rtol=1e-6)


@pytest.mark.parametrize("m0", [(1, 0, 0), (3, -2, 5), (8, 8, 8)])
def test_power_spectrum_plane_wave(ctx, B, m0):
    n, box, A = 16, 25.0, 0.8
    x = np.arange(n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    # C order [z][y][x]: the fastest axis is x
    a = (A * np.cos(2 * np.pi * (m0[0] * Z + m0[1] * Y + m0[2] * X) / n)).astype(np.float32)
    got = _cpu(ctx.power_spectrum(torch.from_numpy(a).cuda(), None, box))
    b = int(round(math.sqrt(sum(c * c for c in m0))))
    nyq = all(abs(c) == n // 2 for c in m0)
    power = (A * n ** 3) ** 2 if nyq else 2 * (A * n ** 3 / 2) ** 2
    assert abs(got["Paa"][b] / (box ** 3 / n ** 6 * power / got["modes"][b]) - 1) < 1e-5
    assert np.all(np.abs(np.delete(got["Paa"], b)) < 1e-9 * got["Paa"][b])


def test_power_spectrum_of_z_fields_and_derived(ctx, B):
    # z_re of one 64^3 realisation with and without growth rescaling:
    # normalised fields (Eq. deltaz), their spectra, bias and cross-correlation
    n, box = 64, 100.0
    S, m = synth.realisation(n, box, 0, device="cuda")
    za = ctx.solve(S, m, box, 3.0, B.history(8.0, 4.0, 3.0))
    zb = ctx.solve(S, m, box, 3.0, B.history(8.0, 4.0, 3.0, weighting=B.AMBER_WEIGHT_MASS_GROWTH))
    da, zbar_a = ctx.delta_z(za)
    db, _ = ctx.delta_z(zb)
    got = ctx.power_spectrum(da, db, box)
    assert ctx.sync_status() == 0
    oa, zbar_o = O.delta_z(za.cpu().numpy())
    ob, _ = O.delta_z(zb.cpu().numpy())
    assert abs(float(zbar_a) / zbar_o - 1) < 1e-12
    np.testing.assert_allclose(da.cpu().numpy(), oa, rtol=0, atol=2e-6)
    ref = O.power_spectrum(oa, ob, box)
    _check_spectra(_cpu(got), ref, rtol=1e-4)
    der = {k: v.cpu().numpy() for k, v in ctx.derived_spectra(got).items()}
    assert ctx.sync_status() == 0
    live = ref[4] > 0
    live[0] = False  # k = 0: the mean of a normalised field, rounding noise on both sides
    # Eqs. Dk, bias and rcc formed in the library against the oracle's (pinned) forms
    np.testing.assert_allclose(der["Delta2_aa"][live], O.dimensionless_power(ref[0], ref[1])[live], rtol=1e-4)
    np.testing.assert_allclose(der["Delta2_bb"][live], O.dimensionless_power(ref[0], ref[2])[live], rtol=1e-4)
    np.testing.assert_allclose(der["bias"][live], O.bias(ref[1], ref[2])[live], rtol=1e-4)
    np.testing.assert_allclose(der["r"][live], O.cross_correlation(ref[3], ref[1], ref[2])[live], rtol=1e-4)
    # a shell without modes: Delta^2 = 0, NaN ratios
    empty = ~(ref[4] > 0)
    if empty.any():
        assert np.all(der["Delta2_aa"][empty] == 0.0) and np.all(np.isnan(der["bias"][empty]))


def test_power_derived_on_given_shells(ctx, B):
    # the derived statistics of fixed shell averages (no transform): exact
    # FP64 arithmetic against the oracle's forms, and argument checks
    nb = 37
    g = np.random.default_rng(9)
    k = np.linspace(0.0, 3.0, nb)
    Paa, Pbb = g.uniform(0.5, 2.0, nb), g.uniform(0.5, 2.0, nb)
    Pab = g.uniform(-0.4, 0.4, nb)
    t = lambda a: torch.from_numpy(a).cuda()
    s = {"k": t(k), "Paa": t(Paa), "Pbb": t(Pbb), "Pab": t(Pab)}
    der = {key: v.cpu().numpy() for key, v in ctx.derived_spectra(s).items()}
    np.testing.assert_allclose(der["Delta2_aa"], O.dimensionless_power(k, Paa), rtol=1e-14)
    np.testing.assert_allclose(der["Delta2_bb"], O.dimensionless_power(k, Pbb), rtol=1e-14)
    np.testing.assert_allclose(der["bias"], O.bias(Paa, Pbb), rtol=1e-14)
    np.testing.assert_allclose(der["r"], O.cross_correlation(Pab, Paa, Pbb), rtol=1e-14)
    vp = __import__("ctypes").c_void_p
    out = torch.empty(nb, dtype=torch.float64, device="cuda")
    # a bias without P_bb, and a misaligned array, are refused before any launch
    assert B.lib.amber_power_derived(ctx._h, vp(s["k"].data_ptr()), vp(s["Paa"].data_ptr()), None, None, nb,
                                     vp(out.data_ptr()), None, vp(out.data_ptr()), None, None) == B.AMBER_ERR_INVALID_ARG
    assert B.lib.amber_power_derived(ctx._h, vp(s["k"].data_ptr() + 4), vp(s["Paa"].data_ptr()), None, None, nb,
                                     vp(out.data_ptr()), None, None, None, None) == B.AMBER_ERR_INVALID_ARG


def test_power_spectrum_parseval_512(B):
    # at a size the oracle cannot transform quickly: the shell sums must still
    # add up to box^3/n^3 sum_x a^2 (a property that holds at any size)
    n, box = 512, 400.0
    with B.Context(n ** 3) as c:
        a = torch.randn((n, n, n), device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
        got = c.power_spectrum(a, None, box)
        assert c.sync_status() == 0
        total = float((got["modes"] * got["Paa"]).sum())
        ref = box ** 3 / n ** 3 * float((a.double() ** 2).sum())
        assert abs(total / ref - 1) < 1e-5
        assert float(got["modes"].sum()) == n ** 3


def test_delta_z_vs_oracle(ctx, B):
    g = np.random.default_rng(2)
    z = g.uniform(5.0, 16.0, 1_000_003).astype(np.float32)
    d, zbar = ctx.delta_z(torch.from_numpy(z).cuda())
    od, ozbar = O.delta_z(z.astype(np.float64))
    assert abs(float(zbar) / ozbar - 1) < 1e-12
    np.testing.assert_allclose(d.cpu().numpy(), od, rtol=0, atol=2e-6)


def test_epsilon_pdf_vs_oracle(ctx, B):
    g = np.random.default_rng(6)
    n = 2_000_000
    zr = g.uniform(5.0, 15.0, n).astype(np.float32)
    z = (zr * (1 + g.normal(scale=0.01, size=n)) + 0.02).astype(np.float32)
    lo, hi, nb = -0.03, 0.03, 120
    counts, mom = ctx.epsilon_z_pdf(torch.from_numpy(z).cuda(), torch.from_numpy(zr).cuda(), lo, hi, nb)
    counts = counts.cpu().numpy()
    e = O.epsilon_z(z.astype(np.float64), zr.astype(np.float64))
    ref = np.concatenate([[np.sum(e < lo)], np.histogram(e[(e >= lo) & (e < hi)], bins=nb, range=(lo, hi))[0],
                          [np.sum(e >= hi)]])
    assert counts.sum() == n
    # FP32 vs FP64 epsilon: only values within rounding of a bin edge may move
    assert np.abs(counts - ref).sum() <= 2e-4 * n
    mom = mom.cpu().numpy()
    assert abs(mom[0] / e.sum() - 1) < 1e-5 and abs(mom[1] / (e * e).sum() - 1) < 1e-5


def test_analysis_rejects_bad_arguments(ctx, B):
    a = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(B.AmberError):
        ctx.power_spectrum(a, None, -1.0)
    with pytest.raises(B.AmberError):
        ctx.power_spectrum(torch.zeros((6, 6, 6), device="cuda"), None, 1.0)
    z = torch.ones(10, device="cuda")
    with pytest.raises(B.AmberError):
        ctx.epsilon_z_pdf(z, z, 1.0, 1.0, 10)
