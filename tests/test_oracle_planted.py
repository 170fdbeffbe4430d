"""Plausible mistakes planted in the oracle (on the CPU) must make a pin fail.

Each case patches one oracle function with a typical slip (a sign, a missing
conjugate, an argmax for an argmin, a non-Gray map) and re-runs a pin from the
other test files; the pin has to raise.
"""

import numpy as np
import pytest

import oracle.bps as obps
import oracle.cdc as ocdc
import oracle.kk as okk
import oracle.mimo as omimo
import oracle.pam as opam
import oracle.qam as oqam
from tests import (test_oracle_bps, test_oracle_cdc, test_oracle_kk, test_oracle_mimo, test_oracle_pam, test_oracle_qam,
                   test_oracle_wl)


def test_flipped_dispersion_sign_is_caught(monkeypatch):
    real = ocdc.cdc_response
    monkeypatch.setattr(ocdc, "cdc_response", lambda n, fs, D, L, lam, *a, **k: real(n, fs, -D, L, lam, *a, **k))
    with pytest.raises(AssertionError):
        test_oracle_cdc.test_cd_all_pass_round_trip(50)


def test_missing_conjugate_in_gradient_is_caught(monkeypatch):
    monkeypatch.setattr(omimo, "gradient", lambda e, X: np.einsum("...qn,...pnk->...qpk", e, X))
    with pytest.raises(AssertionError):
        test_oracle_mimo.test_butterfly_and_gradient_by_explicit_loops()


def test_reversed_tap_index_is_caught(monkeypatch):
    real = omimo.gather
    monkeypatch.setattr(omimo, "gather", lambda x, n, T, off: real(x, n, T, off)[..., ::-1])
    with pytest.raises(AssertionError):
        test_oracle_mimo.test_butterfly_and_gradient_by_explicit_loops()


def test_argmax_instead_of_argmin_is_caught(monkeypatch):
    real = obps.window_sums
    monkeypatch.setattr(obps, "window_sums", lambda d, W, **k: -real(d, W))
    with pytest.raises(AssertionError):
        test_oracle_bps.test_bps_matches_brute_force_on_tiny_inputs(2, 4, 4)


def test_off_by_one_window_is_caught(monkeypatch):
    real = obps.window_sums
    monkeypatch.setattr(obps, "window_sums", lambda d, W, **k: real(d, W + 1))
    with pytest.raises(AssertionError):
        test_oracle_bps.test_bps_matches_brute_force_on_tiny_inputs(4, 4, 4)


def test_natural_binary_map_is_caught(monkeypatch):
    monkeypatch.setattr(oqam, "_level_to_gray", lambda l: l)
    with pytest.raises(AssertionError):
        test_oracle_qam.test_gray_map_is_a_bijection_with_single_bit_neighbours(4)


def test_fo_correction_with_wrong_sign_is_caught(monkeypatch):
    real = omimo.fo_correct_taps
    monkeypatch.setattr(omimo, "fo_correct_taps", lambda h, code, grid, fs: real(h, -code, grid, fs))
    with pytest.raises(AssertionError):
        test_oracle_mimo.test_large_offset_is_removed_on_noiseless_input()


def test_derotation_with_wrong_sign_is_caught(monkeypatch):
    real = omimo.derotate
    monkeypatch.setattr(omimo, "derotate", lambda x, code, grid, fs, g0: real(x, -code, grid, fs, g0))
    with pytest.raises(AssertionError):
        test_oracle_mimo.test_large_offset_is_removed_on_noiseless_input()


def test_widely_linear_without_the_conjugate_is_caught(monkeypatch):
    monkeypatch.setattr(omimo, "augment", lambda x: np.concatenate([x, x], axis=0))
    with pytest.raises(AssertionError):
        test_oracle_wl.test_one_segment_by_explicit_loops(2)
    with pytest.raises(AssertionError):
        test_oracle_wl.test_converges_to_the_closed_form_inverse_of_a_tx_iq_imbalance()


def test_widely_linear_step_on_the_wrong_taps_is_caught(monkeypatch):
    monkeypatch.setattr(omimo, "wl_step", lambda mu, mu_c: np.array([mu_c, mu_c, mu, mu])[:, None])
    with pytest.raises(AssertionError):
        test_oracle_wl.test_one_segment_by_explicit_loops(4)


def test_kk_hilbert_sign_flipped_is_caught(monkeypatch):
    real = okk.hilbert_sign
    monkeypatch.setattr(okk, "hilbert_sign", lambda N: -real(N))
    with pytest.raises(AssertionError):
        test_oracle_kk.test_kk_is_exact_for_an_analytic_log_field(0.0)


def test_kk_log_of_intensity_instead_of_amplitude_is_caught(monkeypatch):
    real = okk.front_end
    monkeypatch.setattr(okk, "front_end", lambda *a: (real(*a)[0], 2.0 * real(*a)[1]))
    with pytest.raises(AssertionError):
        test_oracle_kk.test_kk_is_exact_for_an_analytic_log_field(0.0)


def test_kk_missing_downshift_is_caught(monkeypatch):
    real = okk.reconstruct
    monkeypatch.setattr(okk, "reconstruct", lambda a, phi, tone: real(a, phi, 0.0))
    with pytest.raises(AssertionError):
        test_oracle_kk.test_kk_is_exact_for_an_analytic_log_field(0.13675)


def test_kk_wrong_decimation_bins_are_caught(monkeypatch):
    monkeypatch.setattr(okk, "decimation_bins", lambda N: np.arange(N // 2))
    with pytest.raises(AssertionError):
        test_oracle_kk.test_matched_decimation_of_grid_tones()


def test_pam_clock_product_conjugate_on_the_wrong_factor_is_caught(monkeypatch):
    monkeypatch.setattr(opam, "clock_products",
                        lambda X: np.sum(np.conj(X[:, :X.shape[1] // 2]) * X[:, X.shape[1] // 2:], axis=1))
    with pytest.raises(AssertionError):
        test_oracle_pam.test_clock_phase_returns_the_sampling_offset(0.2)


def test_pam_winding_sign_reversed_is_caught(monkeypatch):
    real = opam.winding
    monkeypatch.setattr(opam, "winding", lambda phi: -real(phi))
    with pytest.raises(AssertionError):
        test_oracle_pam.test_variable_rate_extraction_is_continuous(25.0, 0.1)


def test_pam_correction_ramp_sign_is_caught(monkeypatch):
    real = opam.correct
    monkeypatch.setattr(opam, "correct", lambda X, phi: real(X, -phi))
    with pytest.raises(AssertionError):
        test_oracle_pam.test_variable_rate_extraction_is_continuous(25.0, 0.1)


def _rebuild_variant(sign, reverse, conj):
    def f(h):
        h2 = h.copy()
        r = (lambda v: v[::-1]) if reverse else (lambda v: v)
        c = np.conj if conj else (lambda v: v)
        h2[1, 1, :] = c(r(h[0, 0]))
        h2[1, 0, :] = sign * c(r(h[0, 1]))
        return h2
    return f


@pytest.mark.parametrize("variant", [(1.0, True, True), (-1.0, False, True), (-1.0, True, False)],
                         ids=["no-minus", "no-reversal", "no-conjugate"])
def test_wrong_singularity_rebuild_is_caught(monkeypatch, variant):
    monkeypatch.setattr(omimo, "rebuild_second_row", _rebuild_variant(*variant))
    with pytest.raises(AssertionError):
        test_oracle_mimo.test_rebuilt_second_row_makes_a_scaled_unitary_at_every_frequency(15)


def test_lag_zero_only_singularity_check_is_caught(monkeypatch):
    real = omimo.output_correlation
    monkeypatch.setattr(omimo, "output_correlation", lambda y, max_lag: real(y, 0))
    with pytest.raises(AssertionError):
        test_oracle_mimo.test_output_correlation_of_a_delayed_copy_is_the_overlap_fraction(5)
