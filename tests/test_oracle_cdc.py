"""Pins for the generator's channel and the oracle's A0/A1 (CPU only)."""

import json
import os

import numpy as np
import pytest

from oracle import cdc, qam, theory
from synth import LinkParams, generate
from synth.channel import fibre_dispersion, modulate, rrc_spectrum

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _link(**kw):
    base = dict(bits_per_sym=2, symbol_rate=25e9, n_sym=4096, length=0.0, linewidth=0.0,
                freq_offset=0.0, snr_db=None, jones=False)
    base.update(kw)
    return LinkParams(**base)


def test_rrc_nyquist_round_trip_returns_the_symbols():
    """Tx RRC -> Rx RRC is a raised cosine: at the symbol instants it returns the symbols."""
    p = _link(n_sym=8192)
    fr = generate(p, 3)
    S = p.n_samp
    f = np.fft.fftfreq(S, 1 / p.fs)
    H = cdc.cdc_response(S, p.fs, 0.0, 0.0, p.wavelength, p.symbol_rate, p.rolloff)
    r = np.fft.ifft(np.fft.fft(fr.samples, axis=1) * H[None], axis=1)
    assert np.max(np.abs(r[:, ::2] - fr.symbols)) < 1e-12
    # the oracle's matched filter and the generator's pulse are written apart but equal
    assert np.allclose(cdc.rrc_amplitude(f, p.symbol_rate, p.rolloff),
                       rrc_spectrum(f, p.symbol_rate, p.rolloff), atol=1e-15)


@pytest.mark.parametrize("L_km", [50, 120, 2000])
def test_cd_all_pass_round_trip(L_km):
    p = _link(length=L_km * 1e3)
    f = np.fft.fftfreq(8192, 1 / p.fs)
    Hc = cdc.cdc_response(8192, p.fs, p.dispersion, p.length, p.wavelength)
    assert np.max(np.abs(Hc * fibre_dispersion(f, p) - 1)) < 1e-12
    assert np.allclose(np.abs(Hc), 1.0, atol=1e-15)


def test_generator_snr_calibration():
    p = _link(n_sym=1 << 16, snr_db=10.0, jones=True, linewidth=1e5, freq_offset=1e8)
    fr = generate(p, 7)
    clean = generate(p.with_(snr_db=None), 7).samples
    noise = fr.samples - clean
    for q in range(2):
        P = np.mean(np.abs(clean[q]) ** 2)
        assert np.mean(np.abs(noise[q]) ** 2) == pytest.approx(2 * P / 10.0, rel=0.02)
    # the Jones matrix is unitary
    assert np.allclose(fr.jones @ fr.jones.conj().T, np.eye(2), atol=1e-14)


@pytest.mark.parametrize("m,snr_db", [(2, 7.0), (4, 13.0), (6, 19.0)])
def test_awgn_ber_of_generator_plus_ideal_matched_filter(m, snr_db):
    """Generator + ideal RRC matched filter + oracle decisions = exact Gray-QAM BER (3 sigma)."""
    p = _link(bits_per_sym=m, n_sym=1 << 19, snr_db=snr_db)
    fr = generate(p, 21)
    H = cdc.cdc_response(p.n_samp, p.fs, 0.0, 0.0, p.wavelength, p.symbol_rate, p.rolloff)
    r = np.fft.ifft(np.fft.fft(fr.samples, axis=1) * H[None], axis=1)[:, ::2]
    li, lq = qam.decide_levels(r, m)
    bits = qam.levels_to_bits(li, lq, m).reshape(2, -1)
    nbits = bits.size
    ber = np.mean(bits != fr.bits)
    pth = theory.gray_qam_ber(m, snr_db)
    assert nbits >= 1 << 21
    assert abs(ber - pth) < 3 * np.sqrt(pth * (1 - pth) / nbits) * 1.5   # x1.5: bits of a symbol correlate


def test_power_scale_closed_form():
    x = np.stack([2.0 * np.exp(1j * np.linspace(0, 9, 1000)), np.zeros(1000)])
    x[1, :10] = 0.5
    s = cdc.power_scale(x, 10)
    assert s[0] == pytest.approx(0.5, rel=1e-15) and s[1] == pytest.approx(2.0, rel=1e-15)
    assert cdc.power_scale(np.zeros((2, 8)), 8).tolist() == [1.0, 1.0]


def test_overlap_save_blocks_by_direct_circular_convolution():
    """Each kept sample equals the block's circular convolution with ifft(H), summed term by term."""
    rng = np.random.default_rng(2)
    N, S = 32, 100
    x = rng.normal(size=(1, S)) + 1j * rng.normal(size=(1, S))
    H = np.exp(1j * rng.uniform(0, 2 * np.pi, N)) * rng.uniform(0.5, 1.5, N)
    h = np.array([np.sum(H * np.exp(2j * np.pi * np.arange(N) * t / N)) / N for t in range(N)])
    out = cdc.overlap_save(x, H)
    for i in range(S):
        j = i // (N // 2)
        start = j * (N // 2) - N // 4
        seg = np.array([x[0, start + mm] if 0 <= start + mm < S else 0 for mm in range(N)])
        nloc = i - start
        ref = sum(seg[mm] * h[(nloc - mm) % N] for mm in range(N))
        assert abs(out[0, i] - ref) < 1e-12


def test_paper_block_geometry_and_filter_length_rule():
    """Sec. III-A: 1024-pt FFT, 512 valid per block, 8192 blocks per 2^22 buffer; 503 taps add no cyclic ISI."""
    nfft = GOLDEN["fft_size"]["value"]
    assert GOLDEN["buffer_samples"]["value"] // (nfft // 2) == GOLDEN["blocks_per_buffer"]["value"]
    assert nfft // 2 == GOLDEN["valid_per_block"]["value"]
    assert 2 * GOLDEN["fd_threads"]["value"] == GOLDEN["buffer_samples"]["value"]
    assert GOLDEN["buffer_samples"]["value"] / 4e9 * 1e3 == pytest.approx(
        GOLDEN["buffer_duration_ms_at_4gsps"]["value"], abs=5e-4)
    rng = np.random.default_rng(4)
    S = 4096
    x = rng.normal(size=(1, S)) + 1j * rng.normal(size=(1, S))
    for taps, exact in ((GOLDEN["fd_fir_taps_max"]["value"], True), (601, False)):
        g = rng.normal(size=taps) + 1j * rng.normal(size=taps)        # two-sided FIR, centre tap (taps-1)/2
        c = (taps - 1) // 2
        gc = np.zeros(nfft, complex)
        gc[np.arange(-c, taps - c) % nfft] = g
        out = cdc.overlap_save(x, np.fft.fft(gc))
        lin = np.convolve(x[0], g)[c:c + S]
        err = np.max(np.abs(out[0] - lin))
        assert (err < 1e-9) == exact


def test_overlap_save_recovers_dispersed_symbols():
    p = _link(n_sym=1 << 14, length=200e3, symbol_rate=32e9)
    fr = generate(p, 9)
    H = cdc.cdc_response(4096, p.fs, p.dispersion, p.length, p.wavelength, p.symbol_rate, p.rolloff)
    out = cdc.overlap_save(fr.samples, H)
    mem = p.dispersion * p.length * p.wavelength**2 / 299792458.0 * p.symbol_rate * 1.1 * p.fs
    assert 4096 // 4 >= 2 * mem
    inner = slice(1024, p.n_sym - 1024)
    assert np.max(np.abs(out[:, ::2][:, inner] - fr.symbols[:, inner])) < 2e-3


def test_stream_overlap_save_equals_one_pass_over_the_concatenation():
    rng = np.random.default_rng(8)
    nfft, S, F = 256, 512, 5
    x = rng.normal(size=(2, S * F)) + 1j * rng.normal(size=(2, S * F))
    H = np.exp(1j * rng.uniform(0, 6, nfft))
    tail = np.zeros((2, nfft // 2), complex)
    outs = []
    for f in range(F):
        o, tail = cdc.overlap_save_stream(x[:, f * S:(f + 1) * S], H, tail)
        outs.append(o)
    stream = np.concatenate(outs, axis=1)
    whole = cdc.overlap_save(np.concatenate([np.zeros((2, nfft // 4)), x], axis=1), H)
    assert np.max(np.abs(stream - whole[:, :S * F])) < 1e-12
