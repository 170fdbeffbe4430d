"""Pins for the oracle's IM/DD PAM-M chain with FD clock recovery (Sec. III, Steps 1-9).

* Gray demapping inverts the generator's independent Gray mapping;
* the clock-phase estimate returns the generator's sampling-phase offset (sign and scale);
* with a receiver clock offset the unwrapped clock phase drifts by 2 pi ppm 1e-6 per symbol and
  the winding number counts the slipped symbols;
* across the slips the variable-rate extraction returns the transmitted symbols one for one
  (noiseless, away from the frame edges where the 105-block average is one-sided);
* over AWGN the bit error rate matches the closed form of Gray PAM-M at the matched-filter
  output: BER = 2 (1 - 1/M) Q(sqrt(2) / sigma) / log2 M, sigma^2 = E[a^2] / SNR, the matched
  filter's gain at the symbol instant being sqrt(2) (its response sqrt(2) RRC times the
  transmitter's RRC integrates to sqrt(2)) and its noise gain 1.
"""

import math

import numpy as np
import pytest

from oracle import pam
from synth.pam import PAMLink, generate_pam, gray_levels


@pytest.mark.parametrize("M", [2, 4, 8])
def test_demap_inverts_the_generator_map(M):
    m = int(math.log2(M))
    bits = np.random.default_rng(M).integers(0, 2, size=600 * m, dtype=np.uint8)
    a = gray_levels(bits, M)
    lev, out = pam.decide(a.astype(np.float64), M)
    assert np.array_equal(out, bits)
    assert np.array_equal(2 * lev - (M - 1), a)


@pytest.mark.parametrize("tau", [-0.3, 0.0, 0.2, 0.45])
def test_clock_phase_returns_the_sampling_offset(tau):
    """Sample n is taken at symbol time n/2 + tau, so a symbol appears tau early: the estimate
    -phi / (2 pi) (symbols of delay) is -tau."""
    fr = generate_pam(PAMLink(levels=4, n_samp=1 << 17, timing=tau), 1)
    r = pam.pam_receive(fr.codes, fr.scale, fr.dc, 4, 0.5)
    est = -r["phi"][60:-60] / (2 * np.pi)
    assert abs(np.median(est) + tau) < 1e-3, np.median(est)
    assert np.all(r["w"] == 0)


@pytest.mark.parametrize("ppm", [30.0, -20.0])
def test_clock_offset_drift_and_slips(ppm):
    fr = generate_pam(PAMLink(levels=4, n_samp=1 << 18, clock_ppm=ppm), 2)
    r = pam.pam_receive(fr.codes, fr.scale, fr.dc, 4, 0.5)
    Phi = r["phi"] + 2 * np.pi * r["w"]
    j = np.arange(Phi.size)
    sl = slice(60, Phi.size - 60)
    slope = np.polyfit(j[sl], Phi[sl], 1)[0]
    # a fast receiver clock sees each symbol later: the delay grows by ppm 1e-6 per symbol, 256 per block
    expect = -2 * np.pi * ppm * 1e-6 * 256
    assert abs(slope - expect) < 0.01 * abs(expect), (slope, expect)
    symbols = (1 << 18) // 2
    assert abs(r["w"][-1] + ppm * 1e-6 * symbols) <= 1.0
    assert r["y"].size == symbols + r["w"][-1] - r["w"][0]


@pytest.mark.parametrize("ppm,tau", [(25.0, 0.1), (-30.0, -0.2), (30.0, 0.45)])
def test_variable_rate_extraction_is_continuous(ppm, tau):
    fr = generate_pam(PAMLink(levels=4, n_samp=1 << 20, clock_ppm=ppm, timing=tau), 3)
    r = pam.pam_receive(fr.codes, fr.scale, fr.dc, 4, 0.5)
    assert np.any(np.diff(r["w"]) != 0)
    lev = r["levels"]
    tx = (fr.symbols[fr.first:fr.first + lev.size] + 3) // 2
    E = 60 * 256                      # the 105-block average is one-sided near the frame edges
    assert np.array_equal(lev[E:-E], tx[E:-E])


@pytest.mark.parametrize("M,snr_db", [(2, 6.0), (4, 12.0), (8, 18.0)])
def test_ber_matches_the_closed_form(M, snr_db):
    fr = generate_pam(PAMLink(levels=M, n_samp=1 << 20, snr_db=snr_db, timing=0.15), 5)
    r = pam.pam_receive(fr.codes, fr.scale, fr.dc, M, 0.5)
    m = int(math.log2(M))
    n = r["levels"].size
    E = 2000
    tx_bits = fr.bits[fr.first * m:(fr.first + n) * m]
    errs = int(np.sum(r["bits"][E * m:(n - E) * m] != tx_bits[E * m:(n - E) * m]))
    ber = errs / ((n - 2 * E) * m)
    sigma = math.sqrt((M * M - 1) / 3 / 10 ** (snr_db / 10))
    theory = 2 * (1 - 1 / M) * 0.5 * math.erfc(math.sqrt(2) / sigma / math.sqrt(2)) / m
    assert errs > 1000
    assert 0.85 < ber / theory < 1.2, (ber, theory)
