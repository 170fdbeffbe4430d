"""Seeded single-polarisation self-coherent (Kramers-Kronig) QAM link, FP64 NumPy.

What it draws and applies, in this order (one periodic frame of ``n_sym``
symbols, 4 samples per symbol):

1. uniform bits mapped onto the Gray square M-QAM alphabet of unit average
   energy (``synth.channel.modulate``);
2. root-raised-cosine pulse shaping in the frequency domain over the whole
   frame, gain 2 (= sqrt(4)) so that an RRC matched filter of gain 2 returns
   the symbols at the symbol instants, optionally followed by a transmitter
   IQ imbalance s -> mu s + nu conj(s) (``iq_imbalance``, the model of
   ``synth.channel.iq_coefficients``); the mean sample power P_s is measured
   (about 1/4: one symbol of unit energy per 4 samples);
3. a carrier tone of amplitude A = sqrt(CSPR P_s) (CSPR = carrier-to-signal
   power ratio) ``tone_offset`` Hz below the signal centre. In the tone's frame the
   field is h(t) = A + s(t) exp(+j 2 pi f_t t): the signal lies above the
   tone, so h is minimum phase when A exceeds |s|;
4. optical noise: complex AWGN on the field with variance 4 P_s / SNR per
   sample (SNR = Es/N0 of the signal, as in ``synth.channel``);
5. square-law detection I = |h + n|^2;
6. an AC-coupled 12-bit ADC: the mean is removed, the rest quantised with the
   step delta = clip * std(I) / 2048 around code 2048 and clipped to
   [0, 4095]. ``scale`` = delta and ``dc`` = mean(I) - 2048 delta return
   v = scale * code + dc ~ I (the static DC offset the receiver adds back).

The paper's KK experiments used an IQ modulator with a transmitter-side tone
(Sec. IV-E: 1 GBd, 1 % roll-off, tone at 0.547 GHz); this module stands in
for the lab link with the textbook model above.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .channel import iq_coefficients, modulate, rrc_spectrum

SPS = 4


@dataclass
class KKLink:
    bits_per_sym: int = 4
    symbol_rate: float = 1e9
    n_sym: int = 1 << 14
    rolloff: float = 0.01
    tone_offset: float = 0.547e9     # tone below the signal centre [Hz]
    cspr_db: float = 11.0
    snr_db: float | None = None      # None = noiseless
    adc_clip: float = 6.0            # ADC full scale in standard deviations of I
    iq_imbalance: tuple | None = None  # transmitter IQ imbalance (amplitude eps, phase skew rad) of s(t)

    @property
    def fs(self) -> float:
        return SPS * self.symbol_rate


@dataclass
class KKFrame:
    link: KKLink
    seed: int
    codes: np.ndarray        # uint16 [S] 12-bit ADC codes
    scale: float             # volts (intensity units) per code
    dc: float                # static offset: v = scale * code + dc
    intensity: np.ndarray    # float64 [S] detected intensity before the ADC
    field: np.ndarray        # complex128 [S] h = A + s exp(j 2 pi f_t t) (noise included)
    signal: np.ndarray       # complex128 [S] s(t) at 4 sps, noiseless
    symbols: np.ndarray      # complex128 [n_sym]
    bits: np.ndarray         # uint8 [n_sym * m]
    carrier: float           # A


def generate_kk(p: KKLink, seed: int) -> KKFrame:
    ss = np.random.SeedSequence(seed).spawn(2)
    rng_bits, rng_noise = (np.random.Generator(np.random.PCG64(s)) for s in ss)
    m, N = p.bits_per_sym, p.n_sym
    S = SPS * N
    bits = rng_bits.integers(0, 2, size=(1, N * m), dtype=np.uint8)
    sym = modulate(bits, m)[0]
    x = np.zeros(S, dtype=np.complex128)
    x[::SPS] = sym
    f = np.fft.fftfreq(S, d=1.0 / p.fs)
    s = np.fft.ifft(np.fft.fft(x) * np.sqrt(SPS) * rrc_spectrum(f, p.symbol_rate, p.rolloff))
    if p.iq_imbalance is not None:
        mu, nu = iq_coefficients(*p.iq_imbalance)
        s = mu * s + nu * np.conj(s)
    P_s = float(np.mean(np.abs(s) ** 2))
    A = float(np.sqrt(10.0 ** (p.cspr_db / 10.0) * P_s))
    n = np.arange(S, dtype=np.float64)
    h = A + s * np.exp(2j * np.pi * p.tone_offset * n / p.fs)
    if p.snr_db is not None:
        var = SPS * P_s / 10.0 ** (p.snr_db / 10.0)
        h = h + np.sqrt(var / 2.0) * (rng_noise.standard_normal(S) + 1j * rng_noise.standard_normal(S))
    I = np.abs(h) ** 2
    mean, std = float(np.mean(I)), float(np.std(I))
    delta = p.adc_clip * std / 2048.0
    codes = np.clip(np.rint((I - mean) / delta) + 2048.0, 0, 4095).astype(np.uint16)
    return KKFrame(link=p, seed=seed, codes=codes, scale=delta, dc=mean - 2048.0 * delta, intensity=I, field=h,
                   signal=s, symbols=sym, bits=bits[0], carrier=A)
