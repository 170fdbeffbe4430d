"""Pins for the closed forms: Q <-> BER at the paper's FEC thresholds, exact Gray-QAM BER."""

import json
import os

import numpy as np
import pytest
from scipy.special import erfc

from oracle import qam, theory

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_q_thresholds_printed_in_the_paper():
    # Sec. I / III-E: 8.4 dB (6.7 % OH HD-FEC); Sec. V-B: 5.7 dB (20 % OH HD-FEC)
    q1 = GOLDEN["hdfec_q_db_6p7pct"]["value"]
    q2 = GOLDEN["hdfec_q_db_20pct"]["value"]
    assert theory.ber_from_q(q1) == pytest.approx(4.27e-3, rel=2e-3)
    assert theory.ber_from_q(q2) == pytest.approx(2.70e-2, rel=3e-3)
    assert theory.q_from_ber(theory.ber_from_q(q1)) == pytest.approx(q1, abs=1e-12)


def test_qpsk_ber_reduces_to_textbook_q_function():
    for snr_db in (4.0, 8.0, 12.0, 14.0):
        g = 10 ** (snr_db / 10)
        assert theory.gray_qam_ber(2, snr_db) == pytest.approx(0.5 * erfc(np.sqrt(g) / np.sqrt(2)), rel=1e-12)


@pytest.mark.parametrize("m,snr,ref", [(2, 14, 2.70e-7), (4, 20, 2.90e-6), (6, 24, 1.58e-4),
                                       (2, 12, 3.43e-5), (4, 12, 2.81e-2), (6, 12, 0.115)])
def test_exact_gray_qam_ber_values(m, snr, ref):
    # reference values of the Cho-Yoon (2002) exact expression, 3 digits
    assert theory.gray_qam_ber(m, snr) == pytest.approx(ref, rel=6e-3)


def test_high_snr_16qam_approaches_nearest_neighbour_form():
    # BER -> (3/4) Q(sqrt(Es/(5 N0))) for Gray 16QAM as SNR grows
    snr = 10 ** (22 / 10)
    approx = 0.75 * 0.5 * erfc(np.sqrt(snr / 5) / np.sqrt(2))
    assert theory.gray_qam_ber(4, 22) == pytest.approx(approx, rel=2e-3)


@pytest.mark.parametrize("m,snr_db", [(4, 10.0), (6, 16.0)])
def test_ber_formula_against_brute_force_monte_carlo(m, snr_db):
    rng = np.random.default_rng(11)
    n = 400_000
    pts = qam.alphabet(m)
    idx = rng.integers(0, pts.size, n)
    sigma = np.sqrt(1 / (2 * 10 ** (snr_db / 10)))
    r = pts[idx] + sigma * (rng.normal(size=n) + 1j * rng.normal(size=n))
    L = qam.n_levels(m)
    dec = np.argmin(np.abs(r[:, None] - pts[None, :]), axis=1)   # exhaustive nearest point
    b_tx = qam.levels_to_bits(idx // L, idx % L, m)
    b_rx = qam.levels_to_bits(dec // L, dec % L, m)
    ber = np.mean(b_tx != b_rx)
    p = theory.gray_qam_ber(m, snr_db)
    assert abs(ber - p) < 4 * np.sqrt(p * (1 - p) / (n * m))
