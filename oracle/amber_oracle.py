"""FP64 CPU oracle for the AMBER reionization-redshift assignment z_re(x).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain, obviously-correct
statement of what the GPU path computes.  Only the test-suite, the smoke check
of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it;
the library itself never does, and this module imports nothing from the
library.  Everything is float64 numpy; library primitives (an FFT, a stable
sort, a cumulative sum, a binary search) serve as single steps, with no
blocking, fusion or reordering beyond what the paper's definition states.

Paper: Trac, Chen, Hoffmann & Cen, "AMBER: Abundance Matching Box for the
Epoch of Reionization", arXiv 2109.10375.

Steps and the passages they follow
----------------------------------
* Reionization history (Sec. 3.1.1, Eqs. duration/asymmetry/zear/zlat):
  z_ear = z_mid + dz*Az/(1+Az), z_lat = z_ear - dz.  The printed first form of
  the z_lat equation repeats z_ear's fraction with a minus sign; it contradicts
  the asymmetry definition, so the second printed form z_ear - dz is used.
* Weibull history (Sec. 3.1.2, Eq. weibull) and its inverse.
* Weibull coefficients (Appendix A): root of f(c) for c, then the algebraic
  a_w, b_w.  The appendix suggests a secant iteration; this oracle brackets the
  root on a log grid and bisects, because a secant started at (1, 2) leaves the
  valid region for large asymmetry.
* Radiation field (Sec. 3.4.1, Eq. intensity): J = S * G with
  G(r) = exp(-r/l)/(4 pi r^2), done by FFT (the paper computes it "using
  FFTs").  The transform of G is arctan(k l)/k with value l at k = 0, from the
  radial Fourier integral int_0^inf exp(-r/l) sin(kr)/(kr) dr.
* Ranking and abundance matching (Sec. 3.4.2): rank cells by J descending
  (ties: ascending cell index), F_n = sum_{m<=n} mass_m / sum_all mass, and z_n
  from the tabulated history x(z_j) by linear interpolation in z between the
  two table points that bracket F_n.
* Source-field pipeline (Sec. 3.2, Eq. xlpt; Sec. 3.2.1, Eqs. interlace and
  Wofk; Sec. 3.3, Eqs. fcoll and variance): second-order Lagrangian
  displacements from spectral potentials, NGP/CIC/TSC assignment by plain
  loops over particles, the interlaced and deconvolved mesh, and the ESF
  collapsed fraction of a filtered linear field.
* Tomographic matching (Sec. 3.4.2 mentions it without detail): one
  correlated field per redshift interval, cells ionized in earlier intervals
  ranked first, each still-neutral cell keeping the redshift the interval's
  matching gives it when that redshift lies inside the interval.
* Analysis (Sec. 2.3, Eqs. epsz, deltaz, Pk, Dk, bias, rcc): the normalised
  and fractional-difference redshift fields, and spherical-shell auto and
  cross power spectra with the bias and cross-correlation built from them
  (full complex FFT, every mode counted once).
* Weighted matching (Sec. 3.4.2, the cumulative-fraction equation with the
  linearly grown overdensity delta_m(z) = D(z)/D(z_mid) delta_m(z_mid); the
  volume-weighted fraction of Sec. 2.3 and 3.1.1): the weight of a cell at
  redshift z is linear in its mass, the ionized set at each table redshift
  is the ranks whose weighted cumulative fraction is at most x(z_j), and z_n
  is interpolated where that margin changes sign.  D(z) of flat LCDM with
  Omega_m = 0.3 (Sec. 2) by quadrature of its integral form.

parity status: every function here is pinned by tests under tests/ (worked
Table 1 values, closed forms, brute force on tiny grids, invariants).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ---------------------------------------------------------------------------
# Reionization history (Sec. 3.1.1 and 3.1.2, Appendix A)
# ---------------------------------------------------------------------------

DEFAULT_X_POINTS = (0.05, 0.50, 0.95)  # (x_ear, x_mid, x_lat), Sec. 3.1.1 default


def ionization_redshifts(z_mid: float, dz: float, Az: float) -> tuple[float, float, float]:
    """(z_ear, z_mid, z_lat) from midpoint, duration and asymmetry (Sec. 3.1.1).

    z_ear follows Eq. zear; z_lat = z_ear - dz is the duration definition
    (Eq. duration) and the second form of Eq. zlat.
    """
    z_ear = z_mid + dz * Az / (1.0 + Az)
    z_lat = z_ear - dz
    return z_ear, z_mid, z_lat


def weibull_x(z, a_w: float, b_w: float, c_w: float):
    """Modified Weibull history x(z) = exp(-max((z-a)/b, 0)^c)  (Eq. weibull)."""
    z = np.asarray(z, dtype=np.float64)
    u = np.maximum((z - a_w) / b_w, 0.0)
    return np.exp(-(u ** c_w))


def weibull_inverse(x, a_w: float, b_w: float, c_w: float):
    """Analytic inverse z(x) = a + b |ln x|^(1/c)  (Sec. 3.1.2)."""
    x = np.asarray(x, dtype=np.float64)
    return a_w + b_w * np.abs(np.log(x)) ** (1.0 / c_w)


def _a_from_mid_lat(c, z_mid, z_lat, L_mid, L_lat):
    """Offset a(c) from the mid and late points (Appendix A)."""
    pm = L_mid ** (1.0 / c)
    pl = L_lat ** (1.0 / c)
    return (z_lat * pm - z_mid * pl) / (pm - pl)


def weibull_coeffs(z_mid: float, dz: float, Az: float,
                   x_points=DEFAULT_X_POINTS) -> tuple[float, float, float]:
    """(a_w, b_w, c_w) through the three ionization points (Appendix A).

    Solve f(c) = (ln x_ear / ln x_mid)^(1/c) - (z_ear - a(c))/(z_mid - a(c)) = 0
    for c by a sign change on a log grid over [0.05, 100] followed by bisection
    to machine precision, then a_w from the early and late points and
    b_w = (z_mid - a_w) / |ln x_mid|^(1/c).  Raises ValueError when no root is
    bracketed or a coefficient is not positive (the paper requires all three
    to be positive).
    """
    x_ear, x_mid, x_lat = x_points
    if not (0.0 < x_ear < x_mid < x_lat < 1.0):
        raise ValueError("need 0 < x_ear < x_mid < x_lat < 1")
    if not (dz > 0.0 and Az > 0.0):
        raise ValueError("need dz > 0 and Az > 0")
    z_ear, z_mid, z_lat = ionization_redshifts(z_mid, dz, Az)
    L_ear, L_mid, L_lat = abs(math.log(x_ear)), abs(math.log(x_mid)), abs(math.log(x_lat))

    def f(c):
        a = _a_from_mid_lat(c, z_mid, z_lat, L_mid, L_lat)
        return (L_ear / L_mid) ** (1.0 / c) - (z_ear - a) / (z_mid - a)

    grid = np.exp(np.linspace(math.log(0.05), math.log(100.0), 401))
    vals = [f(c) for c in grid]
    for i in range(len(grid) - 1):
        f0, f1 = vals[i], vals[i + 1]
        if not (math.isfinite(f0) and math.isfinite(f1)) or f0 * f1 > 0.0:
            continue
        lo, hi, flo = grid[i], grid[i + 1], f0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            fm = f(mid)
            if fm == 0.0:
                lo = hi = mid
                break
            if (fm > 0.0) == (flo > 0.0):
                lo, flo = mid, fm
            else:
                hi = mid
            if hi - lo <= 1e-15 * hi:
                break
        c = 0.5 * (lo + hi)
        pe, pl = L_ear ** (1.0 / c), L_lat ** (1.0 / c)
        a = (z_ear * pl - z_lat * pe) / (pl - pe)
        b = (z_mid - a) / L_mid ** (1.0 / c)
        if a > 0.0 and b > 0.0 and c > 0.0:
            return float(a), float(b), float(c)
    raise ValueError("no Weibull root bracketed with positive coefficients")


@dataclass
class HistoryTable:
    """Tabulated history: z_j uniform on [z_lo, z_hi], x_j = x(z_j)."""
    z: np.ndarray
    x: np.ndarray
    a_w: float
    b_w: float
    c_w: float


def history_table(z_mid: float, dz: float, Az: float, z_lo: float = 5.0, z_hi: float = 20.0,
                  n_table: int = 2000, x_points=DEFAULT_X_POINTS) -> HistoryTable:
    """x(z) tabulated on n_table uniform redshifts.

    The low end is lowered to a_w when a_w < z_lo so that the table reaches the
    fully ionized plateau x = 1 (otherwise the fraction at the lowest table
    redshift could not equal x there).
    """
    a, b, c = weibull_coeffs(z_mid, dz, Az, x_points)
    lo = min(z_lo, a)
    j = np.arange(n_table, dtype=np.float64)
    z = lo + (z_hi - lo) * j / (n_table - 1)
    return HistoryTable(z=z, x=weibull_x(z, a, b, c), a_w=a, b_w=b, c_w=c)


# ---------------------------------------------------------------------------
# Source field (Sec. 3.3): excursion-set collapsed fraction, ESF-E density
# ---------------------------------------------------------------------------

def source_field(delta, delta_c: float = 1.686, sigma_f: float = 0.7):
    """(S, mass) from a density field, float64.

    f_coll = erfc((delta_c - delta) / sqrt(2 sigma_f^2))  (Eq. fcoll, with
    sigma_f^2 standing for sigma^2(M_min) - sigma^2(M_s)); the halo density
    is f_coll (1 + delta) (ESF-E form), with 1 + delta floored at 0.01;
    S is that density divided by its mean; mass = 1 + max(delta, -0.99).
    """
    from scipy.special import erfc
    d = np.asarray(delta, dtype=np.float64)
    mass = 1.0 + np.maximum(d, -0.99)
    S = mass * erfc((delta_c - d) / (math.sqrt(2.0) * sigma_f))
    return S / S.mean(), mass


# ---------------------------------------------------------------------------
# Radiation field (Sec. 3.4.1, Eq. intensity)
# ---------------------------------------------------------------------------

def kernel_transform(k, l_mfp: float):
    """Fourier transform of G(r) = exp(-r/l)/(4 pi r^2): arctan(k l)/k, l at k=0."""
    k = np.asarray(k, dtype=np.float64)
    out = np.empty_like(k)
    nz = k > 0.0
    out[nz] = np.arctan(k[nz] * l_mfp) / k[nz]
    out[~nz] = l_mfp
    return out


def wavenumbers(n: int, box: float):
    """Angular wavenumbers 2 pi m / L for FFT index m, signed (numpy order)."""
    return 2.0 * np.pi / box * np.fft.fftfreq(n, d=1.0 / n)


def kmag_half(n: int, box: float):
    """|k| on the half-spectrum grid [z][y][x<=n/2] of a real n^3 field."""
    k = wavenumbers(n, box)
    kx = np.abs(k[: n // 2 + 1])
    kx[-1] = 2.0 * np.pi / box * (n // 2)  # Nyquist: same |k| either sign
    return np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + kx[None, None, :] ** 2)


def radiation_field(S, box: float, l_mfp: float, workers: int | None = None):
    """J = IDFT(DFT(S) * K(|k|)) in float64, cell order [z][y][x].

    The discrete convolution on the periodic grid: forward sum
    S_hat(k) = sum_x S(x) e^{-i k.x}, inverse with the 1/C normalisation.
    workers: if given, the two FFTs run on that many threads (scipy.fft, the
    same real-input transforms); the product is formed in place.
    """
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    assert S.shape == (n, n, n)
    if workers:
        import scipy.fft as sfft
        S_hat = sfft.rfftn(S, workers=workers)
    else:
        S_hat = np.fft.rfftn(S)
    S_hat *= kernel_transform(kmag_half(n, box), l_mfp)
    if workers:
        return sfft.irfftn(S_hat, s=S.shape, axes=(0, 1, 2), workers=workers)
    return np.fft.irfftn(S_hat, s=S.shape, axes=(0, 1, 2))


# ---------------------------------------------------------------------------
# Ranking and abundance matching (Sec. 3.4.2)
# ---------------------------------------------------------------------------

def rank(J):
    """order[r] = cell index of rank r: descending J, ties by ascending index."""
    J = np.asarray(J).reshape(-1)
    if not np.all(np.isfinite(J)):
        raise ValueError("non-finite intensity")
    return np.argsort(-J, kind="stable")


def _sort_block(args):
    """Worker of rank_blocks: stable descending order of one block of cells,
    read from and written to shared memory (global cell indices)."""
    from multiprocessing import shared_memory
    jname, oname, C, lo, hi = args
    js = shared_memory.SharedMemory(name=jname)
    os_ = shared_memory.SharedMemory(name=oname)
    try:
        J = np.ndarray((C,), dtype=np.float64, buffer=js.buf)
        out = np.ndarray((C,), dtype=np.int32, buffer=os_.buf)
        out[lo:hi] = np.argsort(-J[lo:hi], kind="stable") + lo
    finally:
        js.close()
        os_.close()
    return hi - lo


def rank_blocks(J, workers: int):
    """rank(J) for fields too large for one process to sort in reasonable time.

    The same stable descending order, as a merge sort over contiguous blocks:
    `workers` spawned processes each sort one block of consecutive cells
    stably (ties keep ascending cell index), then one stable sort of the
    concatenated, already sorted blocks merges them -- equal intensities from
    different blocks keep block order, which is ascending cell index.  Both
    sorts are numpy's stable argsort.  Returns int32 cell indices."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    J = np.asarray(J, dtype=np.float64).reshape(-1)
    if not np.all(np.isfinite(J)):
        raise ValueError("non-finite intensity")
    C = J.shape[0]
    bounds = np.linspace(0, C, max(1, int(workers)) + 1).astype(np.int64)
    js = shared_memory.SharedMemory(create=True, size=max(8 * C, 8))
    os_ = shared_memory.SharedMemory(create=True, size=max(4 * C, 4))
    try:
        np.ndarray((C,), dtype=np.float64, buffer=js.buf)[:] = J
        jobs = [(js.name, os_.name, C, int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            pool.map(_sort_block, jobs, chunksize=1)
        g = np.array(np.ndarray((C,), dtype=np.int32, buffer=os_.buf))
    finally:
        js.close()
        js.unlink()
        os_.close()
        os_.unlink()
    vals = J[g]
    np.negative(vals, out=vals)
    perm = np.argsort(vals, kind="stable")  # merges the sorted blocks
    del vals
    return g[perm]


def cumulative_mass_fraction(order, mass):
    """F_n = sum_{m<=n} mass[order[m]] / sum_all mass (inclusive, float64)."""
    m = np.asarray(mass, dtype=np.float64).reshape(-1)[np.asarray(order)]
    M = np.cumsum(m)
    return M / M[-1]


def assign_from_fraction(F, table: HistoryTable):
    """z_n from F_n by the tabulated inverse of x(z).

    j* = largest j with x_j >= F.  No such j: z_lo.  j* = last: z_hi.
    Otherwise t = (x_j* - F)/(x_j* - x_j*+1) in [0,1) and
    z = z_j* + t (z_j*+1 - z_j*).
    """
    F = np.asarray(F, dtype=np.float64)
    x, z = table.x, table.z
    M = len(x)
    # x is non-increasing in j, so {j : x_j >= F} is a prefix of length cnt.
    cnt = M - np.searchsorted(x[::-1], F, side="left")
    j = cnt - 1
    out = np.empty_like(F)
    none = j < 0
    last = j == M - 1
    mid = ~(none | last)
    jm = j[mid]
    t = (x[jm] - F[mid]) / (x[jm] - x[jm + 1])
    t = np.minimum(np.maximum(t, 0.0), np.nextafter(1.0, 0.0))
    out[mid] = z[jm] + t * (z[jm + 1] - z[jm])
    out[none] = z[0]
    out[last] = z[-1]
    return out


def assign_zre(order, mass, table: HistoryTable):
    """z_re in cell order: z_re[order[n]] = z_n (Sec. 3.4.2)."""
    order = np.asarray(order)
    z_n = assign_from_fraction(cumulative_mass_fraction(order, mass), table)
    z_re = np.empty(order.shape[0], dtype=np.float64)
    z_re[order] = z_n
    return z_re


# ---------------------------------------------------------------------------
# Weighted abundance matching: the growth-rescaled equation and the
# volume-weighted fraction (Sec. 3.4.2; Sec. 2.3 and 3.1.1 on the weightings)
# ---------------------------------------------------------------------------

WEIGHT_MASS, WEIGHT_MASS_GROWTH, WEIGHT_VOLUME = 0, 1, 2


def growth_factor(z, omega_m: float = 0.3):
    """Linear density growth factor D(z) of a flat universe of matter and a
    cosmological constant (the simulations' Omega_m = 0.3, Omega_L = 0.7,
    Sec. 2), normalised so that D = a = 1/(1+z) at early times:

        D(a) = (5 Omega_m / 2) E(a) int_0^a da' / (a' E(a'))^3,
        E(a) = sqrt(Omega_m a^-3 + 1 - Omega_m),

    the growing solution of the linear growth equation for pressureless
    matter.  The integral is evaluated with scipy's adaptive quadrature."""
    from scipy import integrate
    zs = np.atleast_1d(np.asarray(z, dtype=np.float64))
    E = lambda a: math.sqrt(omega_m * a ** -3 + 1.0 - omega_m)
    out = np.empty_like(zs)
    for i, zz in enumerate(zs):
        a = 1.0 / (1.0 + zz)
        I = integrate.quad(lambda x: 1.0 / (x * E(x)) ** 3 if x > 0 else 0.0, 0.0, a,
                           epsabs=0.0, epsrel=1e-13, limit=200)[0]
        out[i] = 2.5 * omega_m * E(a) * I
    return out if np.ndim(z) else float(out[0])


def weight_coeffs(table: HistoryTable, weighting: int, z_mid: float = 8.0, omega_m: float = 0.3):
    """(alpha_j, beta_j) with the weight of cell m at table redshift z_j equal
    to alpha_j + beta_j mass_m:

    * mass (the plain path): weight = mass_m                      -> (0, 1)
    * mass with growth (Sec. 3.4.2): 1 + delta_m(z_j), delta_m(z) =
      D(z)/D(z_mid) delta_m(z_mid) and delta_m(z_mid) = mass_m - 1 (the
      mass field is 1 + delta at the midpoint)                     -> (1 - g_j, g_j)
    * volume: every cell weighs 1                                  -> (1, 0)
    """
    M = len(table.z)
    if weighting == WEIGHT_MASS:
        return np.zeros(M), np.ones(M)
    if weighting == WEIGHT_VOLUME:
        return np.ones(M), np.zeros(M)
    if weighting == WEIGHT_MASS_GROWTH:
        g = growth_factor(table.z, omega_m) / growth_factor(z_mid, omega_m)
        return 1.0 - g, g
    raise ValueError("unknown weighting")


def weighted_margins(order, mass, table: HistoryTable, alpha, beta):
    """h[j, n] = x_j W_N(z_j) - W_n(z_j) for all table points and ranks, where
    W_n(z) = sum_{m<=n} weight_m(z) (inclusive): the rank-n cell counts as
    ionized at z_j when h >= 0, i.e. when its cumulative weighted fraction
    W_n/W_N is at most x_j (small cases only: M x N values)."""
    m = np.asarray(mass, dtype=np.float64).reshape(-1)[np.asarray(order)]
    N = m.shape[0]
    n = np.arange(1, N + 1, dtype=np.float64)
    Mn = np.cumsum(m)
    WN = alpha * N + beta * Mn[-1]
    return table.x[:, None] * WN[:, None] - (alpha[:, None] * n[None, :] + beta[:, None] * Mn[None, :])


def assign_zre_weighted(order, mass, table: HistoryTable, weighting: int = WEIGHT_MASS,
                        z_mid: float = 8.0, omega_m: float = 0.3, coeffs=None):
    """z_re in cell order for a weighted cumulative fraction (Sec. 3.4.2).

    The rank-n cell is ionized at table redshift z_j when its cumulative
    weighted fraction is at most x_j (h_j(n) >= 0, see weighted_margins).
    z_n is the largest table z_j at which it is ionized, refined linearly in
    z between z_j* and z_j*+1 where h crosses zero:
    t = h_j*/(h_j* - h_j*+1) in [0, 1), z_n = z_j* + t (z_j*+1 - z_j*);
    z_lo if it is ionized at no table point, z_hi if at the last one.
    With the mass weighting h_j = x_j T - M_n and this is assign_zre.
    The paper does not say which root to take when the fraction crosses x(z)
    more than once (linearly grown weights can turn negative in deep voids):
    the largest z, i.e. the cell's first ionization, is taken.
    coeffs: explicit (alpha_j, beta_j) instead of the weighting's."""
    order = np.asarray(order)
    alpha, beta = coeffs if coeffs is not None else weight_coeffs(table, weighting, z_mid, omega_m)
    m = np.asarray(mass, dtype=np.float64).reshape(-1)[order]
    N = m.shape[0]
    Mtab = len(table.z)
    n = np.arange(1, N + 1, dtype=np.float64)
    Mn = np.cumsum(m)
    WN = alpha * N + beta * Mn[-1]
    jstar = np.full(N, -1, dtype=np.int64)
    for j in range(Mtab):  # the last assignment wins: the largest such j
        jstar[table.x[j] * WN[j] - (alpha[j] * n + beta[j] * Mn) >= 0.0] = j
    h = lambda j: table.x[j] * WN[j] - (alpha[j] * n_sel + beta[j] * M_sel)
    z_n = np.empty(N, dtype=np.float64)
    none, last = jstar < 0, jstar == Mtab - 1
    mid = ~(none | last)
    jm = jstar[mid]
    n_sel, M_sel = n[mid], Mn[mid]
    h0, h1 = h(jm), h(jm + 1)
    t = np.minimum(np.maximum(h0 / (h0 - h1), 0.0), np.nextafter(1.0, 0.0))
    z_n[mid] = table.z[jm] + t * (table.z[jm + 1] - table.z[jm])
    z_n[none] = table.z[0]
    z_n[last] = table.z[-1]
    z_re = np.empty(N, dtype=np.float64)
    z_re[order] = z_n
    return z_re


def non_prefix_cells(order, mass, table: HistoryTable, weighting: int, z_mid: float = 8.0,
                     omega_m: float = 0.3) -> int:
    """How many ranks have an ionized set {j : h_j(n) >= 0} that is not a
    prefix of the table (more than one crossing in z).  The paper speaks of
    the reionization redshift of a cell, i.e. assumes a single crossing;
    tests check their inputs have none."""
    alpha, beta = weight_coeffs(table, weighting, z_mid, omega_m)
    ion = weighted_margins(order, mass, table, alpha, beta) >= 0.0
    cnt = ion.sum(axis=0)
    prefix = np.arange(len(table.z))[:, None] < cnt[None, :]
    return int(np.sum(np.any(ion != prefix, axis=0)))


# ---------------------------------------------------------------------------
# Analysis of z_re (Sec. 2.3: Eqs. epsz, deltaz, Pk, Dk, bias, rcc)
# ---------------------------------------------------------------------------

def delta_z(z_re):
    """Normalised redshift field (Eq. deltaz): ((1 + z) - (1 + zbar)) / (1 + zbar)
    with zbar the volume-weighted (per-cell) mean.  Returns (delta_z, zbar)."""
    z = np.asarray(z_re, dtype=np.float64)
    zbar = float(z.mean())
    return ((1.0 + z) - (1.0 + zbar)) / (1.0 + zbar), zbar


def epsilon_z(z_re, z_ref):
    """Fractional difference field (Eq. epsz): ((1 + z) - (1 + z_ref)) / (1 + z_ref)."""
    z = np.asarray(z_re, dtype=np.float64)
    z1 = np.asarray(z_ref, dtype=np.float64)
    return ((1.0 + z) - (1.0 + z1)) / (1.0 + z1)


def power_bins(n: int) -> int:
    """Number of spherical shells: shell b holds the integer wave vectors m
    (components in [-n/2, n/2)) with round(|m|) = b, so b runs to
    round(sqrt(3) n / 2)."""
    return int(np.rint(math.sqrt(3.0) * n / 2.0)) + 1


def power_spectrum(a, b, box: float):
    """Auto and cross power spectra of real fields a, b on an n^3 periodic
    grid of side box (Eqs. Pk, Dk): P_ij(k) = <delta_i(k) delta_j(k)*> over the
    modes of a spherical shell, in the continuum normalisation
    delta(k) = (box/n)^3 sum_x delta(x) exp(-i k.x), P = |delta(k)|^2 / box^3.
    Shell b holds every wave vector m of the full n^3 transform with
    round(|m|) = b (k = 2 pi m / box).  Returns (k_mean, P_aa, P_bb, P_ab,
    modes) per shell, k_mean the mean |k| of the shell's modes."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.shape[0]
    A = np.fft.fftn(a)
    Bf = np.fft.fftn(b)
    m = np.fft.fftfreq(n, 1.0 / n)  # integer frequencies in [-n/2, n/2)
    mx, my, mz = np.meshgrid(m, m, m, indexing="ij")
    mag = np.sqrt(mx ** 2 + my ** 2 + mz ** 2)
    shell = np.rint(mag).astype(np.int64).reshape(-1)
    nb = power_bins(n)
    modes = np.bincount(shell, minlength=nb).astype(np.float64)
    norm = box ** 3 / float(n) ** 6
    Paa = np.bincount(shell, weights=(np.abs(A) ** 2).reshape(-1), minlength=nb)
    Pbb = np.bincount(shell, weights=(np.abs(Bf) ** 2).reshape(-1), minlength=nb)
    Pab = np.bincount(shell, weights=(A * np.conj(Bf)).real.reshape(-1), minlength=nb)
    ksum = np.bincount(shell, weights=mag.reshape(-1), minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        inv = np.where(modes > 0, 1.0 / modes, 0.0)
    kf = 2.0 * math.pi / box
    return kf * ksum * inv, norm * Paa * inv, norm * Pbb * inv, norm * Pab * inv, modes


def dimensionless_power(k, P):
    """Delta^2(k) = k^3 P(k) / (2 pi^2) (Eq. Dk)."""
    return np.asarray(k) ** 3 * np.asarray(P) / (2.0 * math.pi ** 2)


def bias(P_ii, P_jj):
    """b_ij = sqrt(P_ii / P_jj) (Eq. bias)."""
    return np.sqrt(np.asarray(P_ii) / np.asarray(P_jj))


def cross_correlation(P_ij, P_ii, P_jj):
    """r_ij = P_ij / sqrt(P_ii P_jj) (Eq. rcc)."""
    return np.asarray(P_ij) / np.sqrt(np.asarray(P_ii) * np.asarray(P_jj))


# ---------------------------------------------------------------------------
# Source-field pipeline (Sec. 3.2: 2LPT, mesh assignment with interlacing and
# deconvolution; Sec. 3.3: ESF-L collapsed fraction)
# ---------------------------------------------------------------------------

def _int_freqs(n):
    """Signed integer frequencies m in [-n/2, n/2) along one axis."""
    return np.fft.fftfreq(n, 1.0 / n)


def _kgrid(n, box):
    """k components [z][y][x] for numpy's full fftn layout, and the Nyquist masks."""
    m = _int_freqs(n)
    kf = 2.0 * math.pi / box
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    nyq = -(n // 2)
    return (kf * mx, kf * my, kf * mz), (mx == nyq, my == nyq, mz == nyq)


def lpt_displacement(delta_lin, box: float, D1: float, D2: float):
    """Second-order Lagrangian displacement psi(q) = x - q (Eq. xlpt):
    x = q - D1 grad phi1 + D2 grad phi2 with
      lap phi1 = delta_lin,
      lap phi2 = sum_{i<j} [phi1,ii phi1,jj - (phi1,ij)^2],
    derivatives taken spectrally on the periodic n^3 lattice of side box
    (phi at k = 0 is 0).  A derivative along an axis whose wave number is the
    Nyquist one is set to 0 for odd orders along that axis (it has no real
    counterpart).  Returns (psi_x, psi_y, psi_z), arrays [z][y][x], in box
    length units."""
    d = np.asarray(delta_lin, dtype=np.float64)
    n = d.shape[0]
    (kx, ky, kz), (nx, ny, nz) = _kgrid(n, box)
    k2 = kx * kx + ky * ky + kz * kz
    D = np.fft.fftn(d)
    inv_k2 = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    phi1 = -D * inv_k2
    ks = (kx, ky, kz)
    nq = (nx, ny, nz)

    def deriv2(P, a, b):
        out = -ks[a] * ks[b] * P
        if a != b:
            out = np.where(nq[a] | nq[b], 0.0, out)
        return np.fft.ifftn(out).real

    def grad(P, a):
        return np.fft.ifftn(np.where(nq[a], 0.0, 1j * ks[a] * P)).real

    p = {(a, b): deriv2(phi1, a, b) for a in range(3) for b in range(a, 3)}
    src = (p[0, 0] * p[1, 1] + p[0, 0] * p[2, 2] + p[1, 1] * p[2, 2]
           - p[0, 1] ** 2 - p[0, 2] ** 2 - p[1, 2] ** 2)
    phi2 = -np.fft.fftn(src) * inv_k2
    return tuple(-D1 * grad(phi1, a) + D2 * grad(phi2, a) for a in range(3))


def assignment_weights_1d(d, p: int):
    """Weights of the mesh points at offsets -1, 0, +1 (and the point itself
    for NGP) from a particle at signed distance d in cells from its nearest
    mesh point (|d| <= 1/2): NGP (p = 1), CIC (p = 2) and TSC (p = 3), the
    assignment windows whose transforms are Eq. Wofk."""
    if p == 1:
        return {0: 1.0}
    if p == 2:
        return {0: 1.0 - abs(d), (1 if d >= 0 else -1): abs(d)}
    return {-1: 0.5 * (0.5 - d) ** 2, 0: 0.75 - d * d, 1: 0.5 * (0.5 + d) ** 2}


def mesh_assign(psi, mass, box: float, p: int, shift: float = 0.0):
    """rho(x_n) / mean: particles at lattice points q_i = i dx displaced by psi
    (box units, periodic), optionally all shifted by `shift` cells in each
    direction, assigned to the mesh points x_n = n dx with the order-p window
    (Sec. 3.2.1).  mass: per-particle masses [z][y][x] or None (all equal).
    Plain loops over particles (small n only)."""
    px, py, pz = (np.asarray(c, dtype=np.float64) for c in psi)
    n = px.shape[0]
    dx = box / n
    m = np.ones((n, n, n)) if mass is None else np.asarray(mass, dtype=np.float64)
    rho = np.zeros((n, n, n))
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                pos = [ix + px[iz, iy, ix] / dx + shift, iy + py[iz, iy, ix] / dx + shift,
                       iz + pz[iz, iy, ix] / dx + shift]
                base = [int(math.floor(c + 0.5)) for c in pos]  # nearest mesh point
                w = [assignment_weights_1d(pos[a] - base[a], p) for a in range(3)]
                for oz, wz in w[2].items():
                    for oy, wy in w[1].items():
                        for ox, wx in w[0].items():
                            rho[(base[2] + oz) % n, (base[1] + oy) % n, (base[0] + ox) % n] += \
                                m[iz, iy, ix] * wx * wy * wz
    return rho * (n ** 3 / m.sum())


def interlace_deconvolve(rho1, rho2, box: float, p: int):
    """Eqs. interlace and Wofk: rho(k) = [rho1(k) + e^{i k.dX} rho2(k)] / 2 /
    W(k), dX = (dx/2)(1, 1, 1) the shift of the second mesh's particles, and
    W(k) = [prod_a sin(k_a dx/2)/(k_a dx/2)]^p.  Modes with a Nyquist
    component are set to 0: after the half-cell twiddle they have no real
    counterpart.  Returns the real field."""
    r1 = np.fft.fftn(np.asarray(rho1, dtype=np.float64))
    r2 = np.fft.fftn(np.asarray(rho2, dtype=np.float64))
    n = r1.shape[0]
    dx = box / n
    (kx, ky, kz), (nx, ny, nz) = _kgrid(n, box)
    sinc = lambda t: np.where(t == 0, 1.0, np.sin(t) / np.where(t == 0, 1.0, t))
    W = (sinc(kx * dx / 2) * sinc(ky * dx / 2) * sinc(kz * dx / 2)) ** p
    tw = np.exp(1j * (kx + ky + kz) * dx / 2)
    out = 0.5 * (r1 + tw * r2) / W
    out = np.where(nx | ny | nz, 0.0, out)
    return np.fft.ifftn(out).real


def filter_field(delta, box: float, R: float, kind: str):
    """delta_f(k) = delta(k) W_f(k) (Sec. 3.3): sharp k-space filter (W = 1
    for k R <= 1, else 0) or spherical top hat W = 3 (sin x - x cos x)/x^3,
    x = k R."""
    D = np.fft.fftn(np.asarray(delta, dtype=np.float64))
    n = D.shape[0]
    (kx, ky, kz), _ = _kgrid(n, box)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    if kind == "sharpk":
        W = (kk * R <= 1.0).astype(np.float64)
    else:
        x = kk * R
        xs = np.where(x > 0, x, 1.0)
        W = np.where(x > 0, 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3, 1.0)
    return np.fft.ifftn(D * W).real


def fcoll_esf(delta_f, delta_c: float, dsigma2: float):
    """Collapsed fraction (Eq. fcoll): erfc[(delta_c - delta_f) / sqrt(2 dsigma2)],
    dsigma2 = sigma^2(M_min) - sigma^2(M_s)."""
    from scipy.special import erfc
    return erfc((delta_c - np.asarray(delta_f, dtype=np.float64)) / math.sqrt(2.0 * dsigma2))


def sigma2_tophat(k, Delta2, R: float):
    """Eq. variance: sigma^2(R) = int Delta^2_lin(k) |W_th(kR)|^2 dln k by the
    trapezoid rule over a tabulated Delta^2 on increasing k."""
    k = np.asarray(k, dtype=np.float64)
    x = k * R
    W = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    f = np.asarray(Delta2, dtype=np.float64) * W * W
    lk = np.log(k)
    return float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(lk)))


# ---------------------------------------------------------------------------
# Tomographic abundance matching (Sec. 3.4.2 names matching over several
# redshift intervals as an option and gives no further detail)
# ---------------------------------------------------------------------------

def assign_zre_tomographic(J_list, z_bounds, mass, table: HistoryTable):
    """z_re in cell order from one correlated field per redshift interval.

    Intervals k = 0..K-1 run from high to low redshift, interval k covering
    [z_bounds[k+1], z_bounds[k]).  In interval k the cells ionized in earlier
    intervals rank first (they hold the earliest share of the ionized mass),
    the rest follow by descending J_k (ties by cell index); abundance matching
    over that order gives each still-neutral cell a redshift, which it keeps
    if it falls inside the interval (always, in the last interval) and
    otherwise carries over to the next interval.  With the same field in
    every interval this is assign_zre of that field's ranking (up to the
    rounding of summing the ionized prefix in another order)."""
    K = len(J_list)
    if len(z_bounds) != K + 1:
        raise ValueError("need K+1 interval bounds")
    m = np.asarray(mass, dtype=np.float64).reshape(-1)
    z_re = np.full(m.shape[0], np.nan)
    for k, J in enumerate(J_list):
        Jk = np.asarray(J, dtype=np.float64).reshape(-1)
        done = ~np.isnan(z_re)
        key = np.where(done, np.inf, Jk)
        order = np.argsort(-key, kind="stable")
        z_tmp = assign_zre(order, m, table)
        take = ~done & ((z_tmp >= z_bounds[k + 1]) | (k == K - 1))
        z_re[take] = z_tmp[take]
    return z_re


def solve_large(S, mass, box: float, l_mfp: float, z_mid: float, dz: float, Az: float, workers: int,
                z_lo: float = 5.0, z_hi: float = 20.0, n_table: int = 2000, block: int = 1 << 26):
    """solve() for grids too large for one core (1024^3 in minutes): the same
    steps in the same order, with the two FFTs on `workers` threads, the
    ranking by rank_blocks (the same stable order), and the table inverse --
    which acts on each F_n alone -- applied to `block` ranks at a time.
    Returns J (float64 [n][n][n]), order (int32) and z_re (float64, cell order)."""
    J = radiation_field(S, box, l_mfp, workers=workers)
    order = rank_blocks(J, workers)
    table = history_table(z_mid, dz, Az, z_lo, z_hi, n_table)
    F = cumulative_mass_fraction(order, mass)
    z_n = assign_from_fraction_blocks(F, table, workers, block)
    del F
    z_re = np.empty(z_n.shape[0], dtype=np.float64)
    z_re[order] = z_n
    return J, order, z_re


def _assign_block(args):
    """Worker of assign_from_fraction_blocks: the table inverse of ranks
    [lo, hi), read from and written to shared memory."""
    from multiprocessing import shared_memory
    fname, zname, C, lo, hi, table = args
    fs = shared_memory.SharedMemory(name=fname)
    zs = shared_memory.SharedMemory(name=zname)
    try:
        F = np.ndarray((C,), dtype=np.float64, buffer=fs.buf)
        z = np.ndarray((C,), dtype=np.float64, buffer=zs.buf)
        z[lo:hi] = assign_from_fraction(F[lo:hi], table)
    finally:
        fs.close()
        zs.close()
    return hi - lo


def assign_from_fraction_blocks(F, table: HistoryTable, workers: int, block: int = 1 << 26):
    """assign_from_fraction(F, table), which acts on each F_n alone, applied
    to `block` ranks at a time by `workers` spawned processes."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    F = np.asarray(F, dtype=np.float64).reshape(-1)
    C = F.shape[0]
    if workers <= 1 or C <= block:
        return assign_from_fraction(F, table)
    fs = shared_memory.SharedMemory(create=True, size=8 * C)
    zs = shared_memory.SharedMemory(create=True, size=8 * C)
    try:
        np.ndarray((C,), dtype=np.float64, buffer=fs.buf)[:] = F
        jobs = [(fs.name, zs.name, C, a, min(a + block, C), table) for a in range(0, C, block)]
        with mp.get_context("spawn").Pool(min(int(workers), len(jobs))) as pool:
            pool.map(_assign_block, jobs, chunksize=1)
        return np.array(np.ndarray((C,), dtype=np.float64, buffer=zs.buf))
    finally:
        fs.close()
        fs.unlink()
        zs.close()
        zs.unlink()


def solve(S, mass, box: float, l_mfp: float, z_mid: float, dz: float, Az: float,
          z_lo: float = 5.0, z_hi: float = 20.0, n_table: int = 2000):
    """The whole path: J, order, z_re (cell order, flattened) in float64."""
    J = radiation_field(S, box, l_mfp)
    order = rank(J)
    table = history_table(z_mid, dz, Az, z_lo, z_hi, n_table)
    z_re = assign_zre(order, mass, table)
    return J, order, z_re
