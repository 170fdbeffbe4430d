"""Seeded IM/DD PAM-M link with a free-running receiver clock, FP64 NumPy.

What it draws and applies, in this order:

1. uniform bits mapped onto Gray-coded PAM-M levels a in {-(M-1), ..., M-1}
   (step 2; the first bit is the most significant of the Gray word);
2. root-raised-cosine pulses (roll-off ``rolloff``, impulse response truncated
   to +-``span`` symbols) at the transmitter's symbol clock: the electrical
   drive d(t) = sum_k a_k p(t - k T) on top of a bias, so the detected
   intensity is bias + d(t) (intensity modulation, direct detection);
3. the receiver's ADC samples at 2 samples/symbol of its own clock, which
   runs ``clock_ppm`` parts per million fast: t_n = n T / (2 (1 + ppm 1e-6))
   + ``timing`` T (a constant sampling-phase offset);
4. AWGN on the samples with variance E[d^2] / SNR (SNR = electrical signal
   power over noise power per sample);
5. an AC-coupled 12-bit ADC: the mean is removed, the rest quantised with the
   step delta = clip std / 2048 around code 2048, clipped to [0, 4095];
   ``scale`` = delta and ``dc`` = mean - 2048 delta give v = scale code + dc.

The paper's IM/DD experiments (Sec. III-D/E: 2 GBd PAM-N with 50 % roll-off,
free-running transmitter and receiver clocks) used lab hardware; this module
stands in for them with the textbook model above.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SPS = 2


@dataclass
class PAMLink:
    levels: int = 4                 # M: 2, 4 or 8
    n_samp: int = 1 << 16           # receiver samples (2 per nominal symbol)
    rolloff: float = 0.5
    span: int = 24                  # RRC truncation, symbols each side
    clock_ppm: float = 0.0          # receiver clock offset
    timing: float = 0.0             # sampling-phase offset, symbols
    snr_db: float | None = None     # None = noiseless
    bias: float = 10.0
    adc_clip: float = 6.0


@dataclass
class PAMFrame:
    link: PAMLink
    seed: int
    codes: np.ndarray       # uint16 [n_samp]
    scale: float
    dc: float
    samples: np.ndarray     # float64 [n_samp] detected signal before the ADC
    symbols: np.ndarray     # int64 [K] transmitted levels, symbol k at k T
    bits: np.ndarray        # uint8 [K * log2 M]
    first: int              # index into symbols of the symbol at time 0


def gray_levels(bits: np.ndarray, M: int) -> np.ndarray:
    """[..., K * m] bits -> [..., K] levels: the Gray word g (MSB first) -> level index l with
    g = l ^ (l >> 1) -> amplitude 2 l - (M - 1)."""
    m = int(np.log2(M))
    b = bits.reshape(bits.shape[:-1] + (-1, m)).astype(np.int64)
    g = (b * (1 << np.arange(m - 1, -1, -1))).sum(-1)
    l = g.copy()
    shift = g >> 1
    while np.any(shift):
        l ^= shift
        shift >>= 1
    return 2 * l - (M - 1)


def rrc_pulse(t: np.ndarray, rolloff: float) -> np.ndarray:
    """Root-raised-cosine impulse response, t in symbols, p(0) = 1 - b + 4 b / pi."""
    b = rolloff
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    at0 = np.abs(t) < 1e-12
    sing = np.abs(np.abs(4.0 * b * t) - 1.0) < 1e-9
    reg = ~(at0 | sing)
    tt = t[reg]
    out[reg] = (np.sin(np.pi * tt * (1 - b)) + 4 * b * tt * np.cos(np.pi * tt * (1 + b))) / (
        np.pi * tt * (1 - (4 * b * tt) ** 2))
    out[at0] = 1 - b + 4 * b / np.pi
    out[sing] = b / np.sqrt(2) * ((1 + 2 / np.pi) * np.sin(np.pi / (4 * b)) + (1 - 2 / np.pi) * np.cos(np.pi / (4 * b)))
    return out


def generate_pam(p: PAMLink, seed: int) -> PAMFrame:
    ss = np.random.SeedSequence(seed).spawn(2)
    rng_bits, rng_noise = (np.random.Generator(np.random.PCG64(s)) for s in ss)
    M = p.levels
    m = int(np.log2(M))
    r = 1.0 + p.clock_ppm * 1e-6
    t_end = (p.n_samp / (SPS * r)) + abs(p.timing) + 1
    first = p.span + 2
    K = int(np.ceil(t_end)) + 2 * first
    bits = rng_bits.integers(0, 2, size=K * m, dtype=np.uint8)
    a = gray_levels(bits, M).astype(np.float64)
    t = np.arange(p.n_samp, dtype=np.float64) / (SPS * r) + p.timing      # symbols, symbol k at time k - first
    d = np.zeros(p.n_samp)
    chunk = 1 << 15
    ks = np.arange(-p.span, p.span + 1)
    for c0 in range(0, p.n_samp, chunk):
        tc = t[c0:c0 + chunk]
        k0 = np.floor(tc).astype(np.int64)
        for dk in ks:
            k = k0 + dk
            d[c0:c0 + chunk] += a[k + first] * rrc_pulse(tc - k, p.rolloff)
    if p.snr_db is not None:
        var = np.mean(d ** 2) / 10.0 ** (p.snr_db / 10.0)
        d = d + np.sqrt(var) * rng_noise.standard_normal(p.n_samp)
    x = p.bias + d
    mean, std = float(np.mean(x)), float(np.std(x))
    delta = p.adc_clip * std / 2048.0
    codes = np.clip(np.rint((x - mean) / delta) + 2048.0, 0, 4095).astype(np.uint16)
    return PAMFrame(link=p, seed=seed, codes=codes, scale=delta, dc=mean - 2048.0 * delta, samples=x,
                    symbols=a.astype(np.int64), bits=bits, first=first)
