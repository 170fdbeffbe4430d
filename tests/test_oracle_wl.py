"""Pins for the oracle's widely-linear segmented DD-LMS (Sec. IV-D: the paper's TD
equaliser is widely linear so that it also undoes transmitter IQ imbalance).

* with the conjugate taps held at zero (zero start, zero step) it is the linear
  A4 DD-LMS, which the other oracle pins fix;
* one segment of blocks written out sample by sample (outputs with the
  conjugate terms, block phase, decisions, both tap updates);
* on a noiseless QPSK signal with a known transmitter IQ imbalance
  x' = mu x + nu conj(x) the taps converge to the closed-form inverse
  (conj(mu) x' - nu conj(x')) / (|mu|^2 - |nu|^2), up to the common phase
  the in-loop phase leaves free, while the linear equaliser cannot remove
  the image term.
"""

import numpy as np
import pytest

from oracle import mimo, qam
from synth import iq_coefficients


def _wl_by_loops(x, h0, n_sym, L_b, m, mu, mu_c):
    """One segment (no warm-up) of the widely-linear DD-LMS, sample by sample."""
    T = h0.shape[-1]
    c = (T - 1) // 2
    S = x.shape[1]
    h = h0.copy()

    def xs(p, i):
        return x[p, i] if 0 <= i < S else 0.0

    y = np.zeros((2, n_sym), dtype=np.complex128)
    for b0 in range(0, n_sym, L_b):
        L = min(L_b, n_sym - b0)
        hb = h.copy()
        for q in range(2):
            yq = []
            for n in range(b0, b0 + L):
                v = 0.0
                for p in range(2):
                    for k in range(T):
                        v += hb[q, p, k] * xs(p, 2 * n + c - k) + hb[q, 2 + p, k] * np.conj(xs(p, 2 * n + c - k))
                yq.append(v)
            s4 = sum(v ** 4 for v in yq)
            psi = np.arctan2((-s4).imag, (-s4).real) / 4
            for i, n in enumerate(range(b0, b0 + L)):
                d = qam.decide(np.array([yq[i] * np.exp(-1j * psi)]), m)[0]
                err = d * np.exp(1j * psi) - yq[i]
                for p in range(2):
                    for k in range(T):
                        xv = xs(p, 2 * n + c - k)
                        h[q, p, k] += mu * err * np.conj(xv)
                        h[q, 2 + p, k] += mu_c * err * xv
                y[q, n] = yq[i]
    return y, h


def test_frozen_conjugate_taps_give_the_linear_dd_lms():
    rng = np.random.default_rng(3)
    T, L_b, n_sym = 7, 16, 300
    x = 0.6 * (rng.normal(size=(2, 2 * n_sym + 20)) + 1j * rng.normal(size=(2, 2 * n_sym + 20)))
    h = mimo.identity_taps(T) + 0.05 * (rng.normal(size=(2, 2, T)) + 1j * rng.normal(size=(2, 2, T)))
    hw = np.zeros((2, 4, T), dtype=np.complex128)
    hw[:, :2] = h
    y_l, t_l = mimo.dd_lms(x, h, n_sym, L_b, 4, 2, 4, 0.01)
    y_w, t_w = mimo.dd_lms_wl(x, hw, n_sym, L_b, 4, 2, 4, 0.01, 0.0)
    assert np.array_equal(y_l, y_w)
    assert np.array_equal(t_l, t_w[:, :2])
    assert not np.any(t_w[:, 2:])


@pytest.mark.parametrize("m", [2, 4])
def test_one_segment_by_explicit_loops(m):
    rng = np.random.default_rng(10 + m)
    T, L_b, n_sym = 5, 8, 21
    x = 0.7 * (rng.normal(size=(2, 2 * n_sym + 9)) + 1j * rng.normal(size=(2, 2 * n_sym + 9)))
    h0 = mimo.wl_identity_taps(T) + 0.05 * (rng.normal(size=(2, 4, T)) + 1j * rng.normal(size=(2, 4, T)))
    mu, mu_c = 0.02, 0.013
    y, h = mimo.dd_lms_wl(x, h0, n_sym, L_b, 100, 0, m, mu, mu_c)
    y_ref, h_ref = _wl_by_loops(x, h0, n_sym, L_b, m, mu, mu_c)
    assert np.max(np.abs(y - y_ref)) < 1e-12
    assert np.max(np.abs(h - h_ref)) < 1e-12


def _iq_input(n_sym, iq, seed):
    """Noiseless QPSK at 2 samples/symbol (symbols on the even samples, zeros between) with a
    transmitter IQ imbalance per polarisation."""
    rng = np.random.default_rng(seed)
    s = qam.alphabet(2)[rng.integers(0, 4, size=(2, n_sym))]
    x = np.zeros((2, 2 * n_sym), dtype=np.complex128)
    for p in range(2):
        mu, nu = iq[p]
        x[p, ::2] = mu * s[p] + nu * np.conj(s[p])
    return s, x


IQ = [iq_coefficients(0.12, 0.10), iq_coefficients(-0.08, 0.15)]


def test_converges_to_the_closed_form_inverse_of_a_tx_iq_imbalance():
    T, L_b, n_sym = 7, 64, 64 * 240
    c = (T - 1) // 2
    s, x = _iq_input(n_sym, IQ, seed=5)
    y, h = mimo.dd_lms_wl(x, mimo.wl_identity_taps(T), n_sym, L_b, 10 ** 6, 0, 2, 0.004, 0.004)
    for p in range(2):
        mu, nu = IQ[p]
        D = abs(mu) ** 2 - abs(nu) ** 2
        hc, gc = h[p, p, c], h[p, 2 + p, c]
        # the in-loop phase leaves the overall phase of the solution free
        ph = np.exp(1j * np.angle(hc * mu))
        assert abs(hc - ph * np.conj(mu) / D) < 1e-6, (p, hc, ph * np.conj(mu) / D)
        assert abs(gc - ph * (-nu) / D) < 1e-6, (p, gc, -ph * nu / D)
        others = np.abs(h[p]).copy()
        others[p, c] = 0.0
        others[2 + p, c] = 0.0
        assert others.max() < 1e-6
    # last blocks: the derotated outputs sit on the QPSK points
    tail = y[:, -L_b * 8:]
    psi = np.angle(-np.sum(tail ** 4, axis=-1, keepdims=True)) / 4
    u = tail * np.exp(-1j * psi)
    evm = np.mean(np.abs(u - qam.decide(u, 2)) ** 2)
    assert 10 * np.log10(evm) < -100


def test_linear_dd_lms_cannot_remove_the_image():
    T, L_b, n_sym = 7, 64, 64 * 240
    s, x = _iq_input(n_sym, IQ, seed=5)
    y, _ = mimo.dd_lms(x, mimo.identity_taps(T), n_sym, L_b, 10 ** 6, 0, 2, 0.004)
    tail = y[:, -L_b * 8:]
    psi = np.angle(-np.sum(tail ** 4, axis=-1, keepdims=True)) / 4
    u = tail * np.exp(-1j * psi)
    evm = np.mean(np.abs(u - qam.decide(u, 2)) ** 2)
    # the image of a linear fit stays near |nu|^2 / |mu|^2 (-18 dB and -16 dB here)
    assert 10 * np.log10(evm) > -25


def test_segment_schedule_matches_the_serial_run_when_converged():
    """Every segment of the widely-linear schedule starts from the same taps and warms up on the
    blocks before it; started from the converged taps on a stationary channel its outputs equal the
    serial run's (both stay at the fixed point)."""
    T, L_b = 7, 64
    s, x = _iq_input(64 * 300, IQ, seed=6)
    _, h = mimo.dd_lms_wl(x, mimo.wl_identity_taps(T), 64 * 240, L_b, 10 ** 6, 0, 2, 0.004, 0.004)
    y_ser, _ = mimo.dd_lms_wl(x, h, 64 * 300, L_b, 10 ** 6, 0, 2, 0.004, 0.004)
    y_seg, _ = mimo.dd_lms_wl(x, h, 64 * 300, L_b, 16, 4, 2, 0.004, 0.004)
    assert np.max(np.abs(y_seg - y_ser)) < 1e-6


def test_generator_iq_imbalance_is_the_branch_model():
    """x -> mu x + nu conj(x) with (mu, nu) = iq_coefficients(eps, phi) is the I/Q branch model
    I' = (1 + eps)(I cos phi - Q sin phi), Q' = (1 - eps)(Q cos phi - I sin phi)."""
    rng = np.random.default_rng(4)
    for eps, phi in ((0.1, 0.08), (-0.2, 0.3), (0.0, -0.5)):
        mu, nu = iq_coefficients(eps, phi)
        for _ in range(5):
            I, Q = rng.normal(size=2)
            x = complex(I, Q)
            y = mu * x + nu * np.conj(x)
            assert abs(y.real - (1 + eps) * (I * np.cos(phi) - Q * np.sin(phi))) < 1e-12
            assert abs(y.imag - (1 - eps) * (Q * np.cos(phi) - I * np.sin(phi))) < 1e-12
