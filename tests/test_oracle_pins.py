"""Pins for the FP64 oracle against what the paper and the mathematics fix.

No GPU.  Each test ties one oracle function to something other than itself:
the paper's Table 1 worked values, closed forms (kernel transform, plane-wave
eigenfunctions, uniform fields), brute-force sums on tiny grids, and the
invariants of abundance matching (Sec. 3.4.2).
"""
import math
import os

import numpy as np
import pytest

from oracle import amber_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "weibull_table1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            rows.append((name, *map(float, vals)))
    return rows


# ----------------------------------------------------------------------------
# Reionization history: Sec. 3.1, Appendix A, Table 1
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("row", _table1(), ids=lambda r: r[0])
def test_weibull_coeffs_match_table1(row):
    _, z_mid, dz, Az, a_w, b_w, c_w = row
    a, b, c = o.weibull_coeffs(z_mid, dz, Az)
    assert abs(a - a_w) <= 0.01 and abs(b - b_w) <= 0.01 and abs(c - c_w) <= 0.01, (a, b, c)


@pytest.mark.parametrize("params", [(8, 4, 3), (7.5, 4, 3), (6.5, 6, 1.5), (9, 2, 5), (8, 4, 1), (8, 4, 14)])
def test_weibull_passes_through_ionization_points(params):
    z_mid, dz, Az = params
    a, b, c = o.weibull_coeffs(z_mid, dz, Az)
    z_ear, _, z_lat = o.ionization_redshifts(z_mid, dz, Az)
    x = o.weibull_x([z_ear, z_mid, z_lat], a, b, c)
    np.testing.assert_allclose(x, [0.05, 0.5, 0.95], rtol=0, atol=1e-12)
    # duration and asymmetry definitions (Eqs. duration, asymmetry)
    assert abs((z_ear - z_lat) - dz) < 1e-12
    assert abs((z_ear - z_mid) / (z_mid - z_lat) - Az) < 1e-12


def test_weibull_quartile_convention():
    # the other convention named in Sec. 3.1.1: (x_ear, x_lat) = (0.25, 0.75)
    a, b, c = o.weibull_coeffs(8.0, 2.0, 2.0, x_points=(0.25, 0.5, 0.75))
    z_ear, z_mid, z_lat = o.ionization_redshifts(8.0, 2.0, 2.0)
    np.testing.assert_allclose(o.weibull_x([z_ear, z_mid, z_lat], a, b, c), [0.25, 0.5, 0.75], atol=1e-12)


def test_weibull_symmetric_case_and_monotone():
    a, b, c = o.weibull_coeffs(8.0, 4.0, 1.0)
    z = np.linspace(0, 30, 3001)
    x = o.weibull_x(z, a, b, c)
    assert np.all(np.diff(x) <= 0)            # monotone non-increasing in z
    assert np.all(x[z <= a] == 1.0)           # fully ionized below a_w
    assert np.all((x > 0) & (x <= 1))


def test_weibull_rejects_bad_points():
    with pytest.raises(ValueError):
        o.weibull_coeffs(8, 4, 3, x_points=(0.5, 0.05, 0.95))
    with pytest.raises(ValueError):
        o.weibull_coeffs(8, -1, 3)


def test_analytic_inverse_roundtrip():
    a, b, c = o.weibull_coeffs(7.91, 5.45, 2.69)
    xs = np.linspace(0.001, 0.999, 500)
    np.testing.assert_allclose(o.weibull_x(o.weibull_inverse(xs, a, b, c), a, b, c), xs, rtol=1e-12)


def test_table_lowers_z_lo_to_reach_plateau():
    t = o.history_table(6.5, 6.0, 1.5)        # a_w ~ 3.22 < 5
    assert abs(t.z[0] - t.a_w) < 1e-12 and t.x[0] == 1.0 and t.z[-1] == 20.0
    t2 = o.history_table(8.0, 4.0, 3.0)       # a_w ~ 6.89 > 5
    assert t2.z[0] == 5.0 and len(t2.z) == 2000


def test_table_interpolation_vs_analytic_inverse():
    t = o.history_table(8.0, 4.0, 3.0)
    F = np.linspace(t.x[-1] * 1.01, 0.999, 20001)
    z_tab = o.assign_from_fraction(F, t)
    z_ana = o.weibull_inverse(F, t.a_w, t.b_w, t.c_w)
    # linear interpolation in z between table nodes: error <= local node spacing
    assert np.max(np.abs(z_tab - z_ana)) < (t.z[1] - t.z[0])
    # and much better where x(z) is nearly linear on the node scale
    mid = (F > 0.05) & (F < 0.95)
    assert np.max(np.abs(z_tab[mid] - z_ana[mid])) < 1e-4


# ----------------------------------------------------------------------------
# Source field: Sec. 3.3, Eq. fcoll (ESF-E density)
# ----------------------------------------------------------------------------

def test_source_field_closed_forms():
    dc, sf = 1.686, 0.7
    d = np.array([dc, -50.0, 0.0, 3.0, -0.995, 10.0])
    S, m = o.source_field(d, dc, sf)
    np.testing.assert_allclose(m, [1 + dc, 0.01, 1.0, 4.0, 0.01, 11.0], rtol=1e-14)
    raw = np.array([mi * math.erfc((dc - di) / (math.sqrt(2) * sf)) for di, mi in zip(d, m)])
    np.testing.assert_allclose(S, raw / raw.mean(), rtol=1e-14)
    assert abs(S.mean() - 1.0) < 1e-14
    # at the barrier erfc(0) = 1: the raw density is the mass itself
    assert abs(raw[0] - (1 + dc)) < 1e-14
    # deep voids collapse nothing; a high peak collapses (almost) everything
    assert raw[1] < 1e-300 and abs(raw[5] / m[5] - 2.0) < 1e-12


# ----------------------------------------------------------------------------
# Radiation kernel: Sec. 3.4.1, Eq. intensity
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("l", [0.5, 3.0, 20.0])
def test_kernel_transform_matches_radial_quadrature(l):
    from scipy.integrate import quad
    for k in [0.01, 0.3, 1.0, 4.0]:
        # 3D transform of G(r) = exp(-r/l)/(4 pi r^2): 4 pi int r^2 G(r) sin(kr)/(kr) dr
        f = lambda r: 4 * math.pi * r * r * (math.exp(-r / l) / (4 * math.pi * r * r)) * math.sin(k * r) / (k * r)
        a = 1.0 / k
        head, _ = quad(f, 0, a, epsabs=1e-14, epsrel=1e-13, limit=400)
        # oscillatory tail by the Fourier-integral rule (sin weight on [a, inf))
        tail, _ = quad(lambda r: math.exp(-r / l) / (k * r), a, np.inf, weight="sin", wvar=k, epsabs=1e-14, limlst=200)
        val = head + tail
        assert abs(o.kernel_transform(np.array([k]), l)[0] - val) <= 1e-10 * abs(val)


def test_kernel_transform_limits():
    l = 3.0
    assert o.kernel_transform(np.array([0.0]), l)[0] == l
    k = np.array([1e-9])
    assert abs(o.kernel_transform(k, l)[0] - l) < 1e-12
    # l -> infinity: pure inverse-square kernel, transform pi/(2k)
    kk = np.array([0.5, 2.0])
    np.testing.assert_allclose(o.kernel_transform(kk, 1e12), math.pi / (2 * kk), rtol=1e-10)


def _brute_force_field(S, box, l):
    """J by explicit complex sums over every k and x (no FFT)."""
    n = S.shape[0]
    C = n ** 3
    m = np.arange(n)
    sm = np.where(m < n // 2, m, m - n)
    kf = 2 * math.pi / box
    xs = np.array([(z, y, x) for z in range(n) for y in range(n) for x in range(n)])
    Sflat = S.reshape(-1)
    J = np.zeros(C)
    for a in range(n):
        for b in range(n):
            for c in range(n):
                kv = kf * np.array([sm[a], sm[b], sm[c]])       # (kz, ky, kx)
                phase = xs @ (np.array([a, b, c]) * 2 * math.pi / n)
                Sk = np.sum(Sflat * np.exp(-1j * phase))
                K = o.kernel_transform(np.array([np.linalg.norm(kv)]), l)[0]
                J += (Sk * K * np.exp(1j * phase)).real
    return (J / C).reshape(S.shape)


@pytest.mark.parametrize("n", [4, 6])
def test_radiation_field_vs_brute_force_dft(n):
    rng = np.random.default_rng(7)
    S = rng.random((n, n, n))
    box, l = 10.0, 2.5
    np.testing.assert_allclose(o.radiation_field(S, box, l), _brute_force_field(S, box, l), rtol=1e-11, atol=1e-12)


def test_uniform_source_gives_uniform_intensity():
    S = np.full((16, 16, 16), 2.5)
    J = o.radiation_field(S, 50.0, 3.0)
    np.testing.assert_allclose(J, 2.5 * 3.0, rtol=1e-12)


@pytest.mark.parametrize("mvec", [(0, 0, 1), (0, 3, 0), (2, 0, 0), (1, -2, 3), (0, 0, 8), (8, 8, 8), (-5, 7, 2)])
def test_plane_wave_is_eigenfunction(mvec):
    n, box, l, eps = 16, 40.0, 3.0, 0.3
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    mz, my, mx = mvec
    phase = 2 * math.pi * (mz * z + my * y + mx * x) / n
    S = 1.0 + eps * np.cos(phase)
    kmag = 2 * math.pi / box * math.sqrt(mz * mz + my * my + mx * mx)
    K = math.atan(kmag * l) / kmag
    np.testing.assert_allclose(o.radiation_field(S, box, l), l + eps * K * np.cos(phase), rtol=0, atol=1e-12)


def test_point_source_recovers_attenuated_inverse_square():
    n, box, l = 64, 64.0, 6.0
    dx = box / n
    S = np.zeros((n, n, n))
    S[0, 0, 0] = 1.0 / dx ** 3
    J = o.radiation_field(S, box, l)

    def G_images(d):
        tot = 0.0
        for i in range(-3, 4):
            for j in range(-3, 4):
                for k in range(-3, 4):
                    r = np.linalg.norm(np.array(d) * dx + np.array([i, j, k]) * box)
                    tot += math.exp(-r / l) / (4 * math.pi * r * r)
        return tot

    # along lattice diagonals the band-limited field matches exp(-r/l)/(4 pi r^2)
    for c in [3, 4, 6, 8, 12, 16]:
        assert abs(J[c, c, c] / G_images((c, c, c)) - 1) < 1e-3
        assert abs(J[0, c, c] / G_images((0, c, c)) - 1) < 2e-2


# ----------------------------------------------------------------------------
# Ranking and abundance matching: Sec. 3.4.2
# ----------------------------------------------------------------------------

def test_rank_matches_brute_force_and_is_stable():
    rng = np.random.default_rng(3)
    J = rng.integers(0, 7, size=300).astype(np.float64)   # many ties
    order = o.rank(J)
    brute = sorted(range(len(J)), key=lambda i: (-J[i], i))
    assert list(order) == brute
    assert sorted(order.tolist()) == list(range(len(J)))


def test_rank_rejects_nan():
    with pytest.raises(ValueError):
        o.rank(np.array([1.0, np.nan]))


def test_equal_mass_fraction_is_n_over_C_and_matches_analytic_inverse():
    C = 5000
    order = np.arange(C)[::-1].copy()
    F = o.cumulative_mass_fraction(order, np.ones(C))
    np.testing.assert_array_equal(F, np.arange(1, C + 1) / C)
    t = o.history_table(8.0, 4.0, 3.0)
    z = o.assign_zre(order, np.ones(C), t)
    Fn = np.arange(1, C + 1) / C
    inside = (Fn < 0.999) & (Fn > t.x[-1])
    ana = o.weibull_inverse(Fn, t.a_w, t.b_w, t.c_w)
    assert np.max(np.abs(z[order][inside] - ana[inside])) < (t.z[1] - t.z[0])


def _brute_assign(order, mass, t):
    C = len(order)
    T = 0.0
    for i in range(C):
        T += float(mass[order[i]])
    zre = np.zeros(C)
    M = 0.0
    for n in range(C):
        M += float(mass[order[n]])
        F = M / T
        js = [j for j in range(len(t.x)) if t.x[j] >= F]
        if not js:
            zn = t.z[0]
        elif js[-1] == len(t.x) - 1:
            zn = t.z[-1]
        else:
            j = js[-1]
            tt = (t.x[j] - F) / (t.x[j] - t.x[j + 1])
            zn = t.z[j] + tt * (t.z[j + 1] - t.z[j])
        zre[order[n]] = zn
    return zre


def test_assign_vs_brute_force_loop():
    rng = np.random.default_rng(11)
    C = 400
    mass = rng.uniform(0.01, 5.0, C)
    order = rng.permutation(C)
    t = o.history_table(8.0, 4.0, 3.0, n_table=200)
    np.testing.assert_allclose(o.assign_zre(order, mass, t), _brute_assign(order, mass, t), rtol=0, atol=1e-12)


def _fraction_invariant(z_re, mass, t):
    T = mass.sum()
    mmax = mass.max() / T
    for zj, xj in zip(t.z, t.x):
        frac = mass[z_re >= zj].sum() / T
        assert xj - mmax - 1e-12 <= frac <= xj + 1e-12, (zj, xj, frac)


def test_ionized_mass_fraction_follows_history_within_one_cell():
    rng = np.random.default_rng(5)
    C = 20000
    mass = rng.uniform(0.01, 3.0, C)
    J = rng.normal(size=C)
    t = o.history_table(7.5, 4.0, 3.0, n_table=300)
    z = o.assign_zre(o.rank(J), mass, t)
    _fraction_invariant(z, mass, t)


def test_tiny_grid_whole_path_brute_force():
    """N = 4 (64 cells): J by explicit sums, ranking by selection, loop assign."""
    n, box, l = 4, 8.0, 1.7
    rng = np.random.default_rng(2)
    S = rng.random((n, n, n))
    mass = rng.uniform(0.5, 1.5, n ** 3)
    Jb = _brute_force_field(S, box, l).reshape(-1)
    remaining = list(range(n ** 3))
    order_b = []
    while remaining:
        best = remaining[0]
        for i in remaining[1:]:
            if Jb[i] > Jb[best]:
                best = i
        order_b.append(best)
        remaining.remove(best)
    t = o.history_table(8.0, 4.0, 3.0, n_table=50)
    zb = _brute_assign(np.array(order_b), mass, t)
    J, order, z = o.solve(S, mass, box, l, 8.0, 4.0, 3.0, n_table=50)
    np.testing.assert_allclose(J.reshape(-1), Jb, rtol=1e-12)
    assert list(order) == order_b
    np.testing.assert_allclose(z, zb, atol=1e-12)


def test_solve_monotone_in_intensity():
    import sys
    from paper_2109_10375_gb300 import synth
    S, m = synth.realisation(16, 25.0, 0)
    J, order, z = o.solve(S.numpy(), m.numpy(), 25.0, 3.0, 8.0, 4.0, 3.0)
    Jf = J.reshape(-1)
    # J_a > J_b  =>  z(a) >= z(b): z along descending-J order is non-increasing
    assert np.all(np.diff(z[order]) <= 0)
    assert np.all(np.diff(Jf[order]) <= 0)


# ---------------------------------------------------------------------------
# Weighted abundance matching (Sec. 3.4.2 with linear growth; volume weighting)
# ---------------------------------------------------------------------------

def test_growth_factor_einstein_de_sitter():
    # Omega_m = 1: the growing mode is exactly D = a
    z = np.array([0.0, 0.5, 3.0, 8.0, 20.0])
    np.testing.assert_allclose(o.growth_factor(z, 1.0), 1.0 / (1.0 + z), rtol=1e-12)


def test_growth_factor_matches_growth_ode():
    # D'' + (3/a + dlnE/da) D' - 3 Om / (2 a^5 E^2) D = 0 from the matter era
    # (D = a, D' = 1 at a = 1e-3, where the Lambda term is ~1e-9 of the matter
    # term), integrated independently of the quadrature form
    from scipy.integrate import solve_ivp
    om = 0.3
    E2 = lambda a: om * a ** -3 + 1.0 - om
    dlnE = lambda a: -1.5 * om * a ** -4 / E2(a)

    def rhs(a, y):
        D, dD = y
        return [dD, -(3.0 / a + dlnE(a)) * dD + 1.5 * om / (a ** 5 * E2(a)) * D]

    z = np.array([0.0, 1.0, 5.0, 8.0, 15.0])
    a_eval = np.sort(1.0 / (1.0 + z))
    sol = solve_ivp(rhs, (1e-3, 1.0), [1e-3, 1.0], t_eval=a_eval, rtol=1e-12, atol=1e-15, method="DOP853")
    D_ode = dict(zip(np.round(sol.t, 12), sol.y[0]))
    for zz in z:
        a = round(1.0 / (1.0 + zz), 12)
        assert abs(o.growth_factor(zz, om) / D_ode[a] - 1.0) < 1e-7, (zz, o.growth_factor(zz, om), D_ode[a])


def test_growth_factor_hypergeometric_closed_form():
    # flat LCDM: D(a) = a 2F1(1/3, 1; 11/6; -a^3 Omega_L / Omega_m)
    from scipy.special import hyp2f1
    for om in (0.3, 0.5):
        for zz in (0.0, 2.0, 6.0, 12.0):
            a = 1.0 / (1.0 + zz)
            ref = a * hyp2f1(1.0 / 3.0, 1.0, 11.0 / 6.0, -a ** 3 * (1.0 - om) / om)
            assert abs(o.growth_factor(zz, om) / ref - 1.0) < 1e-11


def _weighted_case(n=3000, seed=5, lo=0.01, hi=8.0):
    g = np.random.default_rng(seed)
    return g.permutation(n), g.uniform(lo, hi, n)


def test_weighted_mass_weighting_is_the_plain_rule():
    order, mass = _weighted_case()
    t = o.history_table(8.0, 4.0, 3.0)
    np.testing.assert_allclose(o.assign_zre_weighted(order, mass, t, o.WEIGHT_MASS), o.assign_zre(order, mass, t),
                               rtol=0, atol=1e-12)


def test_weighted_volume_is_rank_over_count():
    # every cell weighs 1: F_n = n / N exactly, whatever the masses
    order, mass = _weighted_case()
    t = o.history_table(7.5, 4.0, 3.0)
    z = o.assign_zre_weighted(order, mass, t, o.WEIGHT_VOLUME)
    n = len(order)
    zo = o.assign_from_fraction(np.arange(1, n + 1) / n, t)
    np.testing.assert_allclose(z[order], zo, rtol=0, atol=1e-12)


def test_weighted_growth_of_uniform_density_is_volume():
    # delta = 0 everywhere: every grown weight is 1 at every z
    order, _ = _weighted_case()
    t = o.history_table(8.0, 4.0, 3.0)
    ones = np.ones(len(order))
    np.testing.assert_allclose(o.assign_zre_weighted(order, ones, t, o.WEIGHT_MASS_GROWTH, 8.0),
                               o.assign_zre_weighted(order, ones, t, o.WEIGHT_VOLUME), rtol=0, atol=1e-12)


def test_weighted_growth_matches_continuous_root():
    # modest overdensities (weights stay positive): solve the paper's equation
    #   sum_{m<=n} (1 + g(z) d_m) / sum_m (1 + g(z) d_m) = x(z)
    # per cell on continuous z (analytic Weibull x, quadrature g), taking the
    # highest root; the table result must agree to the interpolation error
    n = 400
    order, mass = _weighted_case(n, seed=9, lo=0.8, hi=1.2)
    z_mid, dz, Az = 8.0, 4.0, 3.0
    t = o.history_table(z_mid, dz, Az)
    z_tab = o.assign_zre_weighted(order, mass, t, o.WEIGHT_MASS_GROWTH, z_mid)[order]
    d = mass[order] - 1.0
    A = np.cumsum(d)
    ranks = np.arange(1, n + 1)
    Dmid = o.growth_factor(z_mid)

    def margin(zz, k):
        g = o.growth_factor(zz) / Dmid
        F = (ranks[k] + g * A[k]) / (n + g * A[-1])
        return o.weibull_x(zz, t.a_w, t.b_w, t.c_w) - F

    grid = np.linspace(t.z[0], t.z[-1], 301)
    checked = 0
    for k in range(0, n, 7):
        x_here = o.weibull_x(z_tab[k], t.a_w, t.b_w, t.c_w)
        if not (0.02 < x_here < 0.98):
            continue
        vals = np.array([margin(zz, k) for zz in grid])
        idx = np.nonzero(vals >= 0)[0]
        top = idx.max()  # highest grid z still ionized
        lo, hi = grid[top], grid[top + 1]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if margin(mid, k) >= 0:
                lo = mid
            else:
                hi = mid
        assert abs(z_tab[k] - lo) < 5e-4, (k, z_tab[k], lo)
        checked += 1
    assert checked > 20


def test_weighted_takes_the_first_ionization_brute_force():
    # six cells whose grown weights turn negative at low z: the margin is
    # evaluated with explicit loops, and z_n must come from the largest table
    # point that ionizes the cell, interpolated where its margin changes sign
    mass = np.array([0.01, 0.01, 0.01, 0.01, 1.297, 0.01])
    order = np.arange(6)
    t = o.history_table(8.0, 4.0, 3.0, n_table=60)
    g = o.growth_factor(t.z) / o.growth_factor(8.0)
    z = o.assign_zre_weighted(order, mass, t, o.WEIGHT_MASS_GROWTH, 8.0)
    for nn in range(6):
        h = []
        for j in range(len(t.z)):
            w = [1.0 + g[j] * (mass[m] - 1.0) for m in range(6)]
            h.append(t.x[j] * sum(w) - sum(w[: nn + 1]))
        ion = [j for j in range(len(t.z)) if h[j] >= 0.0]
        if not ion:
            ref = t.z[0]
        elif ion[-1] == len(t.z) - 1:
            ref = t.z[-1]
        else:
            k = ion[-1]
            tt = min(max(h[k] / (h[k] - h[k + 1]), 0.0), np.nextafter(1.0, 0.0))
            ref = t.z[k] + tt * (t.z[k + 1] - t.z[k])
        assert abs(z[nn] - ref) < 1e-12, (nn, z[nn], ref)
    # the case does have a cell with more than one crossing
    assert o.non_prefix_cells(order, mass, t, o.WEIGHT_MASS_GROWTH, 8.0) >= 1


# ---------------------------------------------------------------------------
# Analysis of z_re (Sec. 2.3): delta_z, epsilon_z, shell power spectra
# ---------------------------------------------------------------------------

def test_power_spectrum_parseval():
    # sum over shells of modes x P equals box^3/n^6 sum_k |A_k|^2 = box^3/n^3 sum_x a^2
    g = np.random.default_rng(21)
    n, box = 12, 37.0
    a = g.normal(size=(n, n, n))
    k, Paa, Pbb, Pab, modes = o.power_spectrum(a, 2.0 * a, box)
    assert modes.sum() == n ** 3
    np.testing.assert_allclose(np.sum(modes * Paa), box ** 3 / n ** 3 * np.sum(a * a), rtol=1e-12)
    np.testing.assert_allclose(Pbb, 4.0 * Paa, rtol=1e-12)
    np.testing.assert_allclose(Pab, 2.0 * Paa, rtol=1e-12)


@pytest.mark.parametrize("m0", [(1, 0, 0), (0, 3, 2), (2, -1, 4), (4, 4, 4)])
def test_power_spectrum_plane_wave(m0):
    # a = A cos(2 pi m0.x / n): modes +-m0 carry (A n^3 / 2)^2 each, all in shell round(|m0|)
    n, box, A = 8, 20.0, 1.7
    x = np.arange(n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    a = A * np.cos(2 * np.pi * (m0[0] * X + m0[1] * Y + m0[2] * Z) / n)
    k, P, _, _, modes = o.power_spectrum(a, a, box)
    mag = math.sqrt(sum(c * c for c in m0))
    b = int(round(mag))
    nyq = all(abs(c) == n // 2 for c in m0)  # the mode is its own conjugate
    power = (A * n ** 3) ** 2 if nyq else 2 * (A * n ** 3 / 2) ** 2
    assert abs(P[b] - box ** 3 / n ** 6 * power / modes[b]) <= 1e-9 * P[b]
    others = np.delete(P, b)
    assert np.all(np.abs(others) <= 1e-20 * P[b])
    np.testing.assert_allclose(o.dimensionless_power(k[b], P[b]), k[b] ** 3 * P[b] / (2 * np.pi ** 2), rtol=1e-14)


def _integral_dlnk(fn, lo, hi, npts=40001):
    """Trapezoid rule of fn(k) over ln k on [lo, hi]."""
    u = np.linspace(math.log(lo), math.log(hi), npts)
    f = fn(np.exp(u))
    return float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(u)))


@pytest.mark.parametrize("n_index", [0.0, -2.5, 1.0])
def test_dimensionless_power_integrates_to_the_variance_closed_form(n_index):
    # sigma^2 = int P(k) d^3k / (2 pi)^3 = int Delta^2(k) dln k.  For
    # P = A k^n exp(-(k R)^2) the left side is, by the Gamma integral,
    # A Gamma((3 + n)/2) / (4 pi^2 R^(3 + n)): a dropped 2 pi^2, a k^2 for k^3
    # or any other slip in Eq. Dk breaks the equality
    A, R = 2.7, 1.3
    closed = A * math.gamma((3.0 + n_index) / 2.0) / (4.0 * math.pi ** 2 * R ** (3.0 + n_index))
    num = _integral_dlnk(lambda k: o.dimensionless_power(k, A * k ** n_index * np.exp(-(k * R) ** 2)),
                         1e-18 / R, 12.0 / R)
    assert abs(num / closed - 1.0) < 1e-6


def test_dimensionless_power_of_a_band_limited_field_sums_to_its_variance():
    # a Gaussian random field whose power sits in shells 10..25 of a 64^3 grid
    # (where the mode count of shell b is close to 4 pi b^2): the shell sum of
    # Delta^2 over ln k (width kf / k per shell) recovers the field's variance
    n, box = 64, 80.0
    g = np.random.default_rng(5)
    w = np.fft.rfftn(g.normal(size=(n, n, n)))
    m = np.fft.fftfreq(n, 1.0 / n)
    mr = np.fft.rfftfreq(n, 1.0 / n)
    mag = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + mr[None, None, :] ** 2)
    field = np.fft.irfftn(w * np.exp(-((mag - 17.0) / 4.0) ** 2), s=(n, n, n), axes=(0, 1, 2))
    k, P, _, _, modes = o.power_spectrum(field, field, box)
    kf = 2.0 * math.pi / box
    live = (modes > 0) & (k > 0)
    D2 = o.dimensionless_power(k[live], P[live])
    shell_sum = float(np.sum(D2 * kf / k[live]))
    assert abs(shell_sum / field.var() - 1.0) < 0.02


def test_power_shell_counts_brute_force():
    # lattice points with round(|m|) = b, counted by explicit loops
    n = 6
    cnt = [0] * o.power_bins(n)
    r = range(-n // 2, n // 2)
    for i in r:
        for j in r:
            for l in r:
                cnt[int(round(math.sqrt(i * i + j * j + l * l)))] += 1
    _, _, _, _, modes = o.power_spectrum(np.ones((n, n, n)), np.ones((n, n, n)), 1.0)
    np.testing.assert_array_equal(modes, np.array(cnt, dtype=np.float64))


def test_bias_and_cross_correlation_identities():
    g = np.random.default_rng(3)
    a = g.normal(size=(8, 8, 8))
    k, Paa, Pbb, Pab, modes = o.power_spectrum(a, -a, 10.0)
    live = modes > 0
    np.testing.assert_allclose(o.cross_correlation(Pab[live], Paa[live], Pbb[live]), -1.0, rtol=1e-12)
    k, Paa, Pbb, Pab, modes = o.power_spectrum(3.0 * a, a, 10.0)
    np.testing.assert_allclose(o.bias(Paa[live], Pbb[live]), 3.0, rtol=1e-12)
    np.testing.assert_allclose(o.cross_correlation(Pab[live], Paa[live], Pbb[live]), 1.0, rtol=1e-12)


def test_white_noise_power_is_flat():
    # <|A_k|^2> = n^3 sigma^2 for white noise: P = sigma^2 box^3 / n^3 at every k
    g = np.random.default_rng(8)
    n, box, sig = 32, 50.0, 0.7
    a = g.normal(scale=sig, size=(n, n, n))
    k, P, _, _, modes = o.power_spectrum(a, a, box)
    flat = sig ** 2 * box ** 3 / n ** 3
    live = modes > 500
    assert np.all(np.abs(P[live] / flat - 1.0) < 0.2)
    assert abs(np.sum(modes[1:] * P[1:]) / np.sum(modes[1:]) / flat - 1.0) < 0.02


def test_delta_z_and_epsilon_z_closed_forms():
    g = np.random.default_rng(5)
    z = g.uniform(5.0, 15.0, 1000)
    d, zbar = o.delta_z(z)
    assert abs(zbar - z.mean()) < 1e-12 and abs(d.mean()) < 1e-15
    np.testing.assert_allclose((1.0 + zbar) * (1.0 + d), 1.0 + z, rtol=1e-14)
    np.testing.assert_array_equal(o.epsilon_z(z, z), np.zeros_like(z))
    np.testing.assert_allclose(o.epsilon_z(z + 0.5, z), 0.5 / (1.0 + z), rtol=1e-12)


# ---------------------------------------------------------------------------
# Source-field pipeline (Sec. 3.2, 3.2.1, 3.3)
# ---------------------------------------------------------------------------

def _xyz(n, box):
    x = np.arange(n) * box / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def test_lpt_plane_wave_is_zeldovich():
    # delta = A cos(k x): phi1 = -A cos(kx)/k^2, no second-order source, so
    # psi_x = -D1 A sin(k x)/k exactly and psi_y = psi_z = 0
    n, box, A, D1 = 16, 32.0, 0.3, 0.8
    X, Y, Z = _xyz(n, box)
    k = 2 * np.pi * 3 / box
    px, py, pz = o.lpt_displacement(A * np.cos(k * X), box, D1, -3.0 / 7.0 * D1 ** 2)
    np.testing.assert_allclose(px, -D1 * A * np.sin(k * X) / k, atol=1e-12)
    assert np.max(np.abs(py)) < 1e-13 and np.max(np.abs(pz)) < 1e-13


def test_lpt_two_orthogonal_waves_second_order():
    # delta = A cos(k1 x) + B cos(k2 y): source = A B cos(k1 x) cos(k2 y) and
    # phi2 = -A B cos(k1 x) cos(k2 y)/(k1^2 + k2^2)
    n, box, A, Bm, D1 = 16, 20.0, 0.4, 0.25, 1.3
    D2 = -3.0 / 7.0 * D1 ** 2
    X, Y, Z = _xyz(n, box)
    k1, k2 = 2 * np.pi * 2 / box, 2 * np.pi * 5 / box
    px, py, pz = o.lpt_displacement(A * np.cos(k1 * X) + Bm * np.cos(k2 * Y), box, D1, D2)
    c = A * Bm / (k1 ** 2 + k2 ** 2)
    np.testing.assert_allclose(px, -D1 * A * np.sin(k1 * X) / k1 + D2 * c * k1 * np.sin(k1 * X) * np.cos(k2 * Y),
                               atol=1e-12)
    np.testing.assert_allclose(py, -D1 * Bm * np.sin(k2 * Y) / k2 + D2 * c * k2 * np.cos(k1 * X) * np.sin(k2 * Y),
                               atol=1e-12)
    assert np.max(np.abs(pz)) < 1e-13


def test_assignment_weights_are_the_b_splines():
    # B-spline windows of order 1, 2, 3 at a quarter-cell offset
    assert o.assignment_weights_1d(0.25, 1) == {0: 1.0}
    assert o.assignment_weights_1d(0.25, 2) == {0: 0.75, 1: 0.25}
    assert o.assignment_weights_1d(-0.25, 2) == {0: 0.75, -1: 0.25}
    w = o.assignment_weights_1d(0.25, 3)
    assert abs(w[-1] - 0.03125) < 1e-15 and abs(w[0] - 0.6875) < 1e-15 and abs(w[1] - 0.28125) < 1e-15


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_mesh_assign_uniform_lattice_and_translation(p, shift):
    n, box = 6, 12.0
    zero = np.zeros((n, n, n))
    rho = o.mesh_assign((zero, zero, zero), None, box, p, shift)
    np.testing.assert_allclose(rho, 1.0, atol=1e-14)
    # a whole-cell translation of every particle shifts the mesh exactly
    g = np.random.default_rng(p)
    psi = tuple(g.uniform(-0.4, 0.4, (n, n, n)) * box / n for _ in range(3))
    m = g.uniform(0.5, 2.0, (n, n, n))
    r0 = o.mesh_assign(psi, m, box, p, shift)
    r1 = o.mesh_assign((psi[0] + box / n, psi[1], psi[2]), m, box, p, shift)
    np.testing.assert_allclose(r1, np.roll(r0, 1, axis=2), atol=1e-12)
    assert abs(r0.mean() - 1.0) < 1e-14


@pytest.mark.parametrize("p", [0, 2, 3])
def test_interlace_realigns_and_deconvolves_a_plane_wave(p):
    # rho1 = f(x_n), rho2 = f(x_n - dX): the second mesh's particles moved
    # by +dX, so its point x_n sees what sat at x_n - dX; the combination is
    # f(x_n) with the mode divided by W(k)
    n, box, eps = 16, 30.0, 0.2
    X, Y, Z = _xyz(n, box)
    m = np.array([2, -3, 5])
    kv = 2 * np.pi * m / box
    dx = box / n
    f = lambda sx: 1 + eps * np.cos(kv[0] * (X - sx) + kv[1] * (Y - sx) + kv[2] * (Z - sx))
    got = o.interlace_deconvolve(f(0.0), f(dx / 2), box, p)
    W = np.prod([np.sin(k * dx / 2) / (k * dx / 2) for k in kv]) ** p
    np.testing.assert_allclose(got, 1 + eps / W * np.cos(kv[0] * X + kv[1] * Y + kv[2] * Z), atol=1e-12)


def test_filters_on_plane_waves():
    n, box = 16, 40.0
    X, Y, Z = _xyz(n, box)
    k1, k2 = 2 * np.pi * 1 / box, 2 * np.pi * 4 / box
    d = np.cos(k1 * X) + np.cos(k2 * Z)
    R = 1.0 / (0.5 * (k1 + k2))  # between the two modes
    np.testing.assert_allclose(o.filter_field(d, box, R, "sharpk"), np.cos(k1 * X), atol=1e-12)
    th = lambda x: 3 * (np.sin(x) - x * np.cos(x)) / x ** 3
    np.testing.assert_allclose(o.filter_field(d, box, R, "tophat"),
                               th(k1 * R) * np.cos(k1 * X) + th(k2 * R) * np.cos(k2 * Z), atol=1e-12)


def test_fcoll_closed_forms():
    from scipy.special import erfc
    dc, ds2 = 1.686 / 0.1, 4.0
    np.testing.assert_allclose(o.fcoll_esf([dc, dc - math.sqrt(2 * ds2), -1e9], dc, ds2), [1.0, erfc(1.0), 0.0],
                               atol=1e-15)


def test_sigma2_tophat_small_radius_limit():
    # Delta^2 = 1 on [k1, k2], R -> 0: W -> 1, sigma^2 -> ln(k2/k1)
    k = np.geomspace(0.1, 10.0, 20001)
    s2 = o.sigma2_tophat(k, np.ones_like(k), 1e-4)
    assert abs(s2 / math.log(100.0) - 1.0) < 1e-6


# ---------------------------------------------------------------------------
# Tomographic abundance matching
# ---------------------------------------------------------------------------

def test_tomographic_with_one_field_is_the_plain_rule():
    g = np.random.default_rng(31)
    C = 5000
    mass = g.uniform(0.01, 3.0, C)
    J = g.normal(size=C)
    t = o.history_table(8.0, 4.0, 3.0, n_table=400)
    plain = o.assign_zre(o.rank(J), mass, t)
    for bounds in ([20.0, 5.0], [20.0, 9.0, 7.5, 5.0], [20.0, 12.0, 8.0, 7.9, 6.0, 5.0]):
        z = o.assign_zre_tomographic([J] * (len(bounds) - 1), bounds, mass, t)
        # the ionized prefix is summed in cell order rather than rank order
        np.testing.assert_allclose(z, plain, rtol=0, atol=1e-12)


def test_tomographic_follows_the_history_within_one_cell():
    # fields that decorrelate from interval to interval: at every table
    # redshift the ionized mass fraction still matches x(z) to one cell
    g = np.random.default_rng(32)
    C = 20000
    mass = g.uniform(0.01, 3.0, C)
    base = g.normal(size=C)
    fields = [base + s * g.normal(size=C) for s in (0.0, 0.7, 1.5)]
    t = o.history_table(7.5, 4.0, 3.0, n_table=300)
    z = o.assign_zre_tomographic(fields, [20.0, 8.5, 7.0, 5.0], mass, t)
    assert not np.any(np.isnan(z))
    _fraction_invariant(z, mass, t)
    # every cell's redshift lies in the interval that assigned it, and the
    # first interval follows the first field's ranking alone
    early = z >= 8.5
    first = o.assign_zre(o.rank(fields[0]), mass, t)
    np.testing.assert_array_equal(z[early], first[early])


def test_tomographic_two_interval_brute_force():
    # eight cells, two intervals, the second field reversing the ranking: the
    # cells left neutral after the first interval are matched in reversed
    # order after the ionized ones (explicit loops)
    mass = np.array([1.0, 2.0, 0.5, 1.5, 1.0, 3.0, 0.25, 0.75])
    J1 = np.arange(8, 0, -1, dtype=np.float64)  # cell 0 brightest
    J2 = -J1
    t = o.history_table(8.0, 4.0, 3.0, n_table=200)
    z = o.assign_zre_tomographic([J1, J2], [20.0, 8.0, 5.0], mass, t)
    T = mass.sum()
    z1 = [None] * 8
    acc = 0.0
    for c in range(8):  # first interval: ranking 0, 1, ..., 7
        acc += mass[c]
        z1[c] = float(o.assign_from_fraction(np.array([acc / T]), t)[0])
    ref = [zz if zz >= 8.0 else None for zz in z1]
    acc = sum(mass[c] for c in range(8) if ref[c] is not None)
    for c in range(7, -1, -1):  # second interval: the neutral cells by J2, cell 7 first
        if ref[c] is None:
            acc += mass[c]
            ref[c] = float(o.assign_from_fraction(np.array([acc / T]), t)[0])
    np.testing.assert_allclose(z, ref, rtol=0, atol=1e-12)


def test_rank_blocks_is_the_stable_descending_order():
    # the block-parallel merge sort gives rank()'s order exactly, ties included
    # (few distinct values, ties spread across blocks), for block counts that
    # do and do not divide the cell count
    g = np.random.default_rng(12)
    for C, workers in ((1, 3), (1000, 1), (10007, 3), (65536, 4)):
        J = np.round(g.normal(size=C), 1)
        J[::7] = 0.25
        ref = o.rank(J)
        got = o.rank_blocks(J, workers)
        np.testing.assert_array_equal(got, ref)


def test_solve_large_is_solve():
    # the multi-core form of the whole oracle path gives solve()'s results:
    # the same order and z, J up to the FFT's rounding
    from paper_2109_10375_gb300 import synth
    for n, box in ((16, 25.0), (32, 50.0)):
        S, m = synth.realisation(n, box, 3)
        S, m = S.double().numpy(), m.double().numpy()
        J0, o0, z0 = o.solve(S, m, box, 3.0, 8.0, 4.0, 3.0)
        J1, o1, z1 = o.solve_large(S, m, box, 3.0, 8.0, 4.0, 3.0, workers=3, block=1000)
        assert np.max(np.abs(J1 - J0)) <= 1e-13 * np.max(np.abs(J0))
        np.testing.assert_array_equal(o1, o0)
        np.testing.assert_array_equal(z1, z0)
