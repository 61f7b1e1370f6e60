"""Planted mistakes in the FP64 oracle, each caught by a pin (CPU only).

The pins in tests/test_oracle_pins.py tie the oracle to what the paper and the
mathematics fix.  This file checks that they are strong enough: each case below swaps
one oracle function for a plausible wrong version (a dropped factor, a flipped sign or
conjugate, an off-by-one index, a transposed or truncated factor, a wrong rounding or
window convention), rebuilds the pins' inputs under the mistake, and requires every pin
it names to fail.  The mistakes live only in this process's copy of the oracle, for the
duration of one test.
"""
import math

import numpy as np
import pytest

import oracle as O
import tests.test_oracle_pins as PINS


def _patch(monkeypatch, name, fn):
    """Replace an oracle function both where the pins call it (``oracle.<name>``) and
    where the oracle's own functions look it up (``oracle.srp.<name>``)."""
    monkeypatch.setattr(O.srp, name, fn)
    if hasattr(O, name):
        monkeypatch.setattr(O, name, fn)


class _Fixtures:
    """The pins' module fixtures, rebuilt lazily under the planted mistake."""

    def __init__(self):
        self._d = {}

    def getfixturevalue(self, name):
        if name not in self._d:
            self._d[name] = {"sq": lambda: PINS._small("square4", F=4, sub=7),
                             "uca": lambda: PINS._small("uca8", F=3, sub=211)}[name]()
        return self._d[name]


PIN_CALLS = {
    "pairs": lambda fx: PINS.test_pair_order_and_count(),
    "tdoa_range": lambda fx: PINS.test_tdoa_range_and_colinear_limit(),
    "hann": lambda fx: PINS.test_hann_window_closed_form(),
    "shift": lambda fx: PINS.test_stft_shift_theorem(),
    "P1_sq": lambda fx: PINS.test_P1_conv_equals_delay_and_sum_power("sq", fx),
    "P1_uca": lambda fx: PINS.test_P1_conv_equals_delay_and_sum_power("uca", fx),
    "P2": lambda fx: PINS.test_P2_source_on_grid_point_is_the_exact_peak(),
    "P2_win": lambda fx: PINS.test_P2_windowed_free_field_source_on_a_grid_point_is_the_argmax("hann"),
    "P3_ifft": lambda fx: PINS.test_P3_samples_direct_equal_ifft_selection(fx.getfixturevalue("sq")),
    "P3_int": lambda fx: PINS.test_P3_integer_lag_equals_conv_pair_term(fx.getfixturevalue("sq")),
    "nmod": lambda fx: PINS.test_lag_order_is_nmod(),
    "P5_si": lambda fx: PINS.test_P5_full_rank_and_full_support_reproduce_si(fx.getfixturevalue("uca")),
    "td": lambda fx: PINS.test_td_is_one_hot_interpolation(fx.getfixturevalue("sq")),
    "lr": lambda fx: PINS.test_lr_full_rank_equals_conv(fx.getfixturevalue("sq")),
    "P6": lambda fx: PINS.test_P6_rank_R_matches_gram_eigenprojector(fx.getfixturevalue("uca")),
    "P7": lambda fx: PINS.test_P7_sparse_selection_matches_full_sort(fx.getfixturevalue("sq")),
    "P9": lambda fx: PINS.test_P9_paper_worked_numbers(),
    "argmax": lambda fx: PINS.test_argmax_takes_the_lowest_index_on_ties(),
    "measures": lambda fx: PINS.test_error_measures_closed_forms(),
    "P10": lambda fx: PINS.test_P10_si_error_shrinks_with_aux_samples(fx.getfixturevalue("sq")),
    "ff": lambda fx: PINS.test_tdoa_ff_is_nf_limit(),
    "lr_rank": lambda fx: PINS.test_lr_rank_R_is_the_best_approximation(fx.getfixturevalue("sq")),
    "dirichlet": lambda fx: PINS.test_dirichlet_kernel_closed_form_and_exact_interpolation(),
    "peaks_line": lambda fx: PINS.test_peaks_worked_example_on_a_line(),
    "peaks_sort": lambda fx: PINS.test_peaks_without_separation_are_the_sorted_map(),
    "peaks_far": lambda fx: PINS.test_peaks_beyond_the_grid_diameter_leave_the_argmax_only(),
    "peaks_box": lambda fx: PINS.test_peaks_are_separated_and_greedy_on_a_box_grid(),
    "peaks_two": lambda fx: PINS.test_peaks_of_two_sources_on_grid_points_are_the_sources(),
}


# ---------------------------------------------------------------- the planted mistakes
def _peaks_generic(z, grid_xyz, K, d_min, tie_last=False, strict=False, last_only=False,
                   keep_self=False):
    """srp_peaks with one planted mistake switched on."""
    z = np.atleast_2d(np.asarray(z))
    F, J = z.shape
    q = np.asarray(grid_xyz, float).astype(np.float32)
    t = np.float32(float(d_min) * float(d_min))
    idx = np.full((F, K), -1, dtype=np.int64)
    val = np.full((F, K), np.nan)
    for f in range(F):
        allowed = np.ones(J, bool)
        picked = np.zeros(J, bool)
        for k in range(K):
            if not allowed.any():
                break
            v = np.where(allowed, z[f], -np.inf)
            i = int(J - 1 - np.argmax(v[::-1])) if tie_last else int(np.argmax(v))
            idx[f, k], val[f, k] = i, z[f, i]
            picked[i] = True
            d = q - q[i]
            d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
            ok = d2 > t if strict else d2 >= t
            allowed = (ok & ~picked) if last_only else (allowed & ok)
            if not keep_self:
                allowed[i] = False
            elif d_min == 0:
                allowed[i] = True
    return idx, val


def _peaks_tie_last(z, g, K, d):
    return _peaks_generic(z, g, K, d, tie_last=True)


def _peaks_strict(z, g, K, d):
    return _peaks_generic(z, g, K, d, strict=True)


def _peaks_last_only(z, g, K, d):
    return _peaks_generic(z, g, K, d, last_only=True)


def _peaks_keep_self(z, g, K, d):
    return _peaks_generic(z, g, K, d, keep_self=True)


def _peaks_radius_not_squared(z, g, K, d):
    return _peaks_generic(z, g, K, math.sqrt(d) if d > 0 else d)


def _pairs_reversed(M):
    return [(mp, m) for mp in range(M - 1) for m in range(mp + 1, M)]


def _tdoa_sign(mic_xyz, grid_xyz, c=340.0):
    return -O.srp.__dict__["_orig_tdoa_nf"](mic_xyz, grid_xyz, c)


def _tdoa_c343(mic_xyz, grid_xyz, c=343.0):
    return O.srp.__dict__["_orig_tdoa_nf"](mic_xyz, grid_xyz, c)


def _window_symmetric(N, kind="hann"):
    n = np.arange(N)
    hann = 0.5 - 0.5 * np.cos(2.0 * np.pi * n / (N - 1))
    return {"hann": hann, "sqrt-hann": np.sqrt(hann), "rect": np.ones(N)}[kind]


def _stft_plus_sign(frames, window="hann"):
    frames = np.asarray(frames, dtype=np.float64)
    return np.conj(np.fft.rfft(frames * O.srp.analysis_window(frames.shape[-1], window), axis=-1))


def _phat_conj_swapped(Y, tiny=1e-30):
    return np.conj(O.srp.__dict__["_orig_gcc_phat"](Y, tiny))


def _phat_unweighted(Y, tiny=1e-30):
    F, M, K1 = Y.shape
    pairs = O.srp.mic_pairs(M)
    y = Y[:, :, 1:K1 - 1]
    return np.stack([y[:, m] * np.conj(y[:, mp]) for m, mp in pairs], axis=1)


def _phat_with_dc(Y, tiny=1e-30):
    F, M, K1 = Y.shape
    pairs = O.srp.mic_pairs(M)
    y = Y[:, :, 0:K1 - 2]  # bins 0..K-2 instead of 1..K-1
    prod = np.stack([y[:, m] * np.conj(y[:, mp]) for m, mp in pairs], axis=1)
    mag = np.abs(prod)
    return np.where(mag > 0, prod / np.where(mag > 0, mag, 1.0), 0.0)


def _omega_off_by_one(K, fs):
    return np.arange(0, K - 1) * (np.pi * fs) / K


def _conv_half(psi, dt, fs, chunk=None):
    return 0.5 * O.srp.__dict__["_orig_srp_conv"](psi, dt, fs, chunk)


def _np_ceil(mic_xyz, fs, c=340.0, n_aux=2):
    out = []
    for (m, mp) in O.srp.mic_pairs(len(mic_xyz)):
        d = float(np.linalg.norm(np.asarray(mic_xyz[m], float) - np.asarray(mic_xyz[mp], float)))
        out.append(int(math.ceil(d / c * fs)) + n_aux)
    return np.array(out, dtype=np.int64)


def _np_no_aux(mic_xyz, fs, c=340.0, n_aux=2):
    return O.srp.__dict__["_orig_n_p_samples"](mic_xyz, fs, c, 0)


def _lags_ascending(Np):
    return [np.arange(-n, n + 1) for n in Np]


def _S_minus(n_lags, K):
    return np.conj(O.srp.__dict__["_orig_sampling_matrix_S"](n_lags, K))


def _ifft_normalised(psi, lags, K):
    re, im = O.srp.__dict__["_orig_gcc_samples_ifft"](psi, lags, K)
    return re / (2 * K), im / (2 * K)


def _sinc_unnormalised(x):
    x = np.asarray(x, float)
    return np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))


def _interp_plus(dt, fs, lags, kernel="sinc", K=None):
    return O.srp.__dict__["_orig_interp_matrix"](-dt, fs, lags, kernel, K)


def _slri_no_sigma(Lam, R):
    tall, fat, s = O.srp.__dict__["_orig_slri_factors"](Lam, R)
    return tall / s[:R], fat, s


def _slri_smallest(Lam, R):
    import scipy.linalg
    U, s, Vt = scipy.linalg.svd(Lam, full_matrices=False)
    return U[:, -R:] * s[-R:], Vt[-R:], s


def _sspi_smallest(Lam, lags, Q_Lambda):
    mask, tied, need = O.srp.__dict__["_orig_sspi_select"](-np.abs(Lam) + np.abs(Lam).max(), lags, Q_Lambda)
    return mask, tied, need


def _td_floor(dt, fs, lags):
    blocks = []
    for p, n in enumerate(lags):
        r = np.floor(dt[:, p] * fs)
        blocks.append((r[:, None] == np.asarray(n, float)[None, :]).astype(np.float64))
    return np.concatenate(blocks, axis=1)


def _lr_fat_conj(H2d, R_H):
    tall, fat = O.srp.__dict__["_orig_lr_factors"](H2d, R_H)
    return tall, np.conj(fat)


def _complexity_table_convention(J, P, K, **kw):
    out = O.srp.__dict__["_orig_complexity"](J, P, K, **kw)
    out["C"] = J * P * (K - 1)
    return out


def _argmax_last(z):
    z = np.asarray(z)
    return z.shape[-1] - 1 - np.argmax(z[..., ::-1], axis=-1)


def _rel_err_squared(approx, ref, axis=-1):
    return O.srp.__dict__["_orig_rel_err"](approx, ref, axis) ** 2


def _two_sided_no_conj(psi_p, K):
    out = np.zeros(psi_p.shape[:-1] + (2 * K,), dtype=np.complex128)
    out[..., 1:K] = psi_p
    out[..., K + 1:] = psi_p[..., ::-1]
    return out


def _tdoa_ff_sign(mic_xyz, dirs, c=340.0):
    return -O.srp.__dict__["_orig_tdoa_ff"](mic_xyz, dirs, c)


def _mean_samples_no_one(Np):
    return 2.0 * float(np.sum(Np)) / len(Np)


def _samples_direct_half(psi, lags, K):
    return 0.5 * O.srp.__dict__["_orig_gcc_samples_direct"](psi, lags, K)


def _srp_td_floor(dt, fs, xi_fn):
    out = None
    for p in range(dt.shape[1]):
        v = xi_fn(p, np.floor(dt[:, p] * fs).astype(np.int64))
        out = v if out is None else out + v
    return out


def _lr_smallest(H2d, R_H):
    import scipy.linalg
    U, s, Vh = scipy.linalg.svd(H2d, full_matrices=False)
    return U[:, -R_H:] * s[-R_H:], Vh[-R_H:]


def _dirichlet_with_nyquist(x, K):
    k = np.arange(-K + 1, K + 1)  # one term too many: the Nyquist bin
    x = np.asarray(x, float)
    return np.real(np.exp(1j * np.pi * x[..., None] * k / K).sum(axis=-1)) / (2 * K)


# (oracle function, mistake, pins that must fail)
MUTANTS = {
    "pairs_m_below_mprime": ("mic_pairs", _pairs_reversed, ["pairs"]),
    "tdoa_sign_flipped": ("tdoa_nf", _tdoa_sign, ["P1_sq", "P2", "P2_win", "tdoa_range"]),
    "tdoa_speed_343": ("tdoa_nf", _tdoa_c343, ["P2", "P2_win"]),
    "window_symmetric_hann": ("analysis_window", _window_symmetric, ["hann"]),
    "stft_plus_exponent": ("stft", _stft_plus_sign, ["shift", "P2", "P2_win"]),
    "phat_conjugate_swapped": ("gcc_phat", _phat_conj_swapped, ["P1_sq", "P2", "P2_win"]),
    "phat_weight_dropped": ("gcc_phat", _phat_unweighted, ["P1_sq", "P2"]),
    "phat_bins_off_by_one": ("gcc_phat", _phat_with_dc, ["P1_sq", "P2"]),
    "omega_off_by_one": ("_omega", _omega_off_by_one, ["P2"]),
    "conv_factor_two_dropped": ("srp_conv", _conv_half, ["P1_sq", "P1_uca", "P2"]),
    "np_ceil_not_floor": ("n_p_samples", _np_ceil, ["P9"]),
    "np_aux_dropped": ("n_p_samples", _np_no_aux, ["P9"]),
    "lags_ascending_not_nmod": ("pair_lags", _lags_ascending, ["nmod"]),
    "sampling_negative_exponent": ("sampling_matrix_S", _S_minus, ["P3_ifft", "P3_int"]),
    "ifft_normalised": ("gcc_samples_ifft", _ifft_normalised, ["P3_ifft"]),
    "two_sided_conjugate_dropped": ("two_sided", _two_sided_no_conj, ["P3_ifft"]),
    "sinc_unnormalised": ("sinc", _sinc_unnormalised, ["P3_int"]),
    "interp_lag_sign": ("interp_matrix", _interp_plus, ["P3_int", "P10"]),
    "slri_sigma_dropped": ("slri_factors", _slri_no_sigma, ["P5_si", "P6"]),
    "slri_smallest_triplets": ("slri_factors", _slri_smallest, ["P6"]),
    "sspi_keeps_smallest": ("sspi_select", _sspi_smallest, ["P7"]),
    "td_floor_not_round": ("td_matrix", _td_floor, ["td"]),
    "lr_fat_conjugated": ("lr_factors", _lr_fat_conj, ["lr"]),
    "complexity_table_convention": ("complexity", _complexity_table_convention, ["P9"]),
    "argmax_last_of_ties": ("argmax_map", _argmax_last, ["argmax"]),
    "rel_err_not_square_rooted": ("rel_err", _rel_err_squared, ["measures"]),
    "tdoa_ff_sign_flipped": ("tdoa_ff", _tdoa_ff_sign, ["ff"]),
    "mean_samples_without_centre": ("mean_samples", _mean_samples_no_one, ["P9"]),
    "samples_direct_factor_two": ("gcc_samples_direct", _samples_direct_half, ["P3_ifft"]),
    "td_lookup_floor_not_round": ("srp_td", _srp_td_floor, ["td"]),
    "lr_smallest_triplets": ("lr_factors", _lr_smallest, ["lr_rank"]),
    "dirichlet_with_nyquist_term": ("dirichlet", _dirichlet_with_nyquist, ["dirichlet"]),
    "peaks_last_of_ties": ("srp_peaks", _peaks_tie_last, ["peaks_line", "peaks_sort"]),
    "peaks_boundary_excluded": ("srp_peaks", _peaks_strict, ["peaks_line"]),
    "peaks_exclude_around_last_pick_only": ("srp_peaks", _peaks_last_only, ["peaks_line"]),
    "peaks_pick_not_excluded": ("srp_peaks", _peaks_keep_self, ["peaks_sort"]),
    "peaks_radius_compared_unsquared": ("srp_peaks", _peaks_radius_not_squared, ["peaks_box"]),
}


def test_pins_pass_on_the_oracle_as_it_stands():
    fx = _Fixtures()
    for name, call in PIN_CALLS.items():
        call(fx)


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_is_caught(monkeypatch, mutant):
    target, fn, pins = MUTANTS[mutant]
    monkeypatch.setattr(O.srp, "_orig_" + target, getattr(O.srp, target), raising=False)
    _patch(monkeypatch, target, fn)
    fx = _Fixtures()
    survived = []
    for pin in pins:
        try:
            PIN_CALLS[pin](fx)
        except AssertionError:
            continue
        survived.append(pin)
    assert not survived, f"{mutant}: pins {survived} did not catch the planted mistake"
