"""Plant plausible mistakes in the oracle (CPU only) and check that the pins catch each.

Every mutation below is a slip one could make when writing the oracle from
the paper: a dropped or wrong term, a sign, an index or a transposed axis.
Each must make at least one pin in test_oracle_pins fail.
"""
import math

import numpy as np
import pytest

from oracle import amber_oracle as o
import tests.test_oracle_pins as pins

PINS = [
    lambda: pins.test_radiation_field_vs_brute_force_dft(4),
    lambda: pins.test_uniform_source_gives_uniform_intensity(),
    lambda: [pins.test_plane_wave_is_eigenfunction(m) for m in [(0, 0, 1), (0, 3, 0), (2, 0, 0), (1, -2, 3)]],
    lambda: pins.test_point_source_recovers_attenuated_inverse_square(),
    lambda: pins.test_rank_matches_brute_force_and_is_stable(),
    lambda: pins.test_equal_mass_fraction_is_n_over_C_and_matches_analytic_inverse(),
    lambda: pins.test_assign_vs_brute_force_loop(),
    lambda: pins.test_ionized_mass_fraction_follows_history_within_one_cell(),
    lambda: [pins.test_weibull_coeffs_match_table1(r) for r in pins._table1()],
    lambda: pins.test_table_interpolation_vs_analytic_inverse(),
    lambda: pins.test_growth_factor_einstein_de_sitter(),
    lambda: pins.test_growth_factor_matches_growth_ode(),
    lambda: pins.test_growth_factor_hypergeometric_closed_form(),
    lambda: pins.test_weighted_mass_weighting_is_the_plain_rule(),
    lambda: pins.test_weighted_volume_is_rank_over_count(),
    lambda: pins.test_weighted_growth_of_uniform_density_is_volume(),
    lambda: pins.test_weighted_growth_matches_continuous_root(),
    lambda: pins.test_weighted_takes_the_first_ionization_brute_force(),
    lambda: pins.test_power_spectrum_parseval(),
    lambda: [pins.test_power_spectrum_plane_wave(m) for m in [(1, 0, 0), (0, 3, 2), (2, -1, 4), (4, 4, 4)]],
    lambda: pins.test_power_shell_counts_brute_force(),
    lambda: pins.test_bias_and_cross_correlation_identities(),
    lambda: [pins.test_dimensionless_power_integrates_to_the_variance_closed_form(v) for v in (0.0, -2.5, 1.0)],
    lambda: pins.test_dimensionless_power_of_a_band_limited_field_sums_to_its_variance(),
    lambda: pins.test_white_noise_power_is_flat(),
    lambda: pins.test_delta_z_and_epsilon_z_closed_forms(),
    lambda: pins.test_lpt_plane_wave_is_zeldovich(),
    lambda: pins.test_lpt_two_orthogonal_waves_second_order(),
    lambda: pins.test_assignment_weights_are_the_b_splines(),
    lambda: [pins.test_mesh_assign_uniform_lattice_and_translation(p, sh) for p in (1, 2, 3) for sh in (0.0, 0.5)],
    lambda: [pins.test_interlace_realigns_and_deconvolves_a_plane_wave(p) for p in (0, 2, 3)],
    lambda: pins.test_filters_on_plane_waves(),
    lambda: pins.test_fcoll_closed_forms(),
    lambda: pins.test_tomographic_with_one_field_is_the_plain_rule(),
    lambda: pins.test_tomographic_follows_the_history_within_one_cell(),
    lambda: pins.test_tomographic_two_interval_brute_force(),
]

_tomo = o.assign_zre_tomographic


def _tomo_ionized_last(J_list, z_bounds, mass, table):
    # earlier-ionized cells ranked last instead of first
    m = np.asarray(mass, dtype=np.float64).reshape(-1)
    z_re = np.full(m.shape[0], np.nan)
    K = len(J_list)
    for k, J in enumerate(J_list):
        done = ~np.isnan(z_re)
        order = np.argsort(-np.where(done, -np.inf, np.asarray(J, dtype=np.float64).reshape(-1)), kind="stable")
        z_tmp = o.assign_zre(order, m, table)
        take = ~done & ((z_tmp >= z_bounds[k + 1]) | (k == K - 1))
        z_re[take] = z_tmp[take]
    return z_re

_weights = o.assignment_weights_1d


def _tsc_mirrored(d, p):
    w = _weights(d, p)
    return {-k: v for k, v in w.items()} if p == 3 else w


def _interlace_wrong_twiddle(rho1, rho2, box, p):
    # the half-cell twiddle applied with the opposite sign
    r1, r2 = np.fft.fftn(rho1), np.fft.fftn(rho2)
    n = r1.shape[0]
    dx = box / n
    (kx, ky, kz), (nx, ny, nz) = o._kgrid(n, box)
    sinc = lambda t: np.where(t == 0, 1.0, np.sin(t) / np.where(t == 0, 1.0, t))
    W = (sinc(kx * dx / 2) * sinc(ky * dx / 2) * sinc(kz * dx / 2)) ** p
    out = 0.5 * (r1 + np.exp(-1j * (kx + ky + kz) * dx / 2) * r2) / W
    return np.fft.ifftn(np.where(nx | ny | nz, 0.0, out)).real


_lpt = o.lpt_displacement


def _lpt_first_order_only(delta_lin, box, D1, D2):
    return _lpt(delta_lin, box, D1, 0.0)

_power = o.power_spectrum


def _power_no_volume(a, b, box):
    k, Paa, Pbb, Pab, modes = _power(a, b, box)
    return k, Paa / box ** 3, Pbb / box ** 3, Pab / box ** 3, modes


def _power_cross_swapped(a, b, box):
    k, Paa, Pbb, Pab, modes = _power(a, b, box)
    return k, Paa, Pbb, np.sqrt(Paa * Pbb), modes

_weight_coeffs = o.weight_coeffs


def _coeffs_swapped(table, weighting, z_mid=8.0, omega_m=0.3):
    a, b = _weight_coeffs(table, weighting, z_mid, omega_m)
    return (b, a) if weighting == o.WEIGHT_MASS_GROWTH else (a, b)


def _coeffs_unpivoted(table, weighting, z_mid=8.0, omega_m=0.3):
    if weighting != o.WEIGHT_MASS_GROWTH:
        return _weight_coeffs(table, weighting, z_mid, omega_m)
    g = o.growth_factor(table.z, omega_m)  # D(z) without dividing by D(z_mid)
    return 1.0 - g, g


def _kmag_transposed(n, box):
    k = o.wavenumbers(n, box)
    kx = np.abs(k[: n // 2 + 1])
    kx[-1] = 2.0 * np.pi / box * (n // 2)
    return np.sqrt(kx[None, None, :] ** 2 * 0 + k[None, :, None] ** 2 + k[:n // 2 + 1][None, None, :] ** 2
                   + np.zeros((n, 1, 1)))


MUTATIONS = {
    "kernel_k_squared": ("kernel_transform",
                         lambda k, l: np.where(np.asarray(k) > 0, np.arctan(np.asarray(k) * l) / np.maximum(np.asarray(k), 1e-300) ** 2, l)),
    "kernel_no_atan": ("kernel_transform",
                       lambda k, l: np.where(np.asarray(k) > 0, l / (1.0 + np.asarray(k) * l), l)),
    "kmag_drops_z_axis": ("kmag_half", _kmag_transposed),
    "rank_ascending": ("rank", lambda J: np.argsort(np.asarray(J).reshape(-1), kind="stable")),
    "fraction_exclusive": ("cumulative_mass_fraction",
                           lambda order, mass: (lambda m: (np.cumsum(m) - m) / m.sum())(
                               np.asarray(mass, dtype=np.float64).reshape(-1)[np.asarray(order)])),
    "zlat_printed_typo": ("ionization_redshifts",
                          lambda z_mid, dz, Az: (z_mid + dz * Az / (1 + Az), z_mid, z_mid - dz * Az / (1 + Az))),
    "growth_einstein_de_sitter_always": ("growth_factor",
                                         lambda z, omega_m=0.3: 1.0 / (1.0 + np.asarray(z, dtype=np.float64))),
    "growth_weights_swapped": ("weight_coeffs", _coeffs_swapped),
    "growth_not_pivoted_at_midpoint": ("weight_coeffs", _coeffs_unpivoted),
    "power_missing_volume": ("power_spectrum", _power_no_volume),
    "power_cross_is_geometric_mean": ("power_spectrum", _power_cross_swapped),
    "delta2_k_squared": ("dimensionless_power", lambda k, P: np.asarray(k) ** 2 * np.asarray(P) / (2.0 * math.pi ** 2)),
    "delta2_wrong_constant": ("dimensionless_power", lambda k, P: np.asarray(k) ** 3 * np.asarray(P) / (2.0 * math.pi)),
    "delta_z_not_normalised": ("delta_z", lambda z: (lambda zz: (zz - zz.mean(), float(zz.mean())))(
        np.asarray(z, dtype=np.float64))),
    "tsc_weights_mirrored": ("assignment_weights_1d", _tsc_mirrored),
    "interlace_twiddle_sign": ("interlace_deconvolve", _interlace_wrong_twiddle),
    "lpt_drops_second_order": ("lpt_displacement", _lpt_first_order_only),
    "tomographic_ionized_ranked_last": ("assign_zre_tomographic", _tomo_ionized_last),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(o, attr, fn)
    caught = 0
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError):
            caught += 1
    assert caught > 0, f"no pin caught mutation {name}"


def test_pins_pass_unmutated():
    for pin in PINS:
        pin()
