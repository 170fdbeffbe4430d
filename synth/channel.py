"""Seeded dual-polarisation transmitter + linear channel, FP64 NumPy.

What it draws and applies, in this order (one periodic frame of ``n_sym``
symbols per polarisation, ``sps`` samples per symbol):

1. uniform bits per polarisation, mapped onto a Gray-coded square M-QAM
   alphabet of unit average energy (the alphabet the receiver decides on);
2. root-raised-cosine pulse shaping, applied in the frequency domain over the
   whole frame (exact RRC spectrum, gain sqrt(sps) so that an RRC matched
   filter returns the symbols at the symbol instants);
   optionally followed by a transmitter IQ imbalance x -> mu x + nu conj(x)
   (``iq_imbalance``; see ``iq_coefficients``);
3. chromatic dispersion of a fibre of length L, written with the group-velocity
   dispersion beta2 = -D * lambda^2 / (2 pi c):  H(w) = exp(j beta2/2 w^2 L);
4. a Haar-random 2x2 unitary Jones matrix (QR of a complex Gaussian matrix with
   the phases of R's diagonal folded into Q);
5. a common laser phase: a Wiener process with per-sample increments
   N(0, 2 pi dnu / fs) (dnu = combined linewidth) plus a frequency offset;
6. complex AWGN per polarisation with variance sps * P / SNR, where P is the
   measured mean sample power of that polarisation, i.e. SNR = Es/N0.

The paper's own experiments used lab hardware (an AWG-driven IQ modulator, an
EDFA noise-loading setup and a field fibre ring; Sec. III-D, Sec. IV-E and
Sec. V-A); this module stands in for them with a textbook channel model.

Seeds: ``SeedSequence(seed).spawn(5)`` gives independent streams for
{bits, jones, phase, awgn, nonlinear}.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

C_LIGHT = 299_792_458.0  # m/s


@dataclass(frozen=True)
class LinkParams:
    """Transmitter and channel parameters of one synthetic link."""

    bits_per_sym: int = 2            # bits per symbol per polarisation: 2, 4, 6
    symbol_rate: float = 25e9        # Rs [Bd]
    n_sym: int = 2**14               # symbols per polarisation in the frame/stream
    sps: int = 2                     # samples per symbol at the ADC
    rolloff: float = 0.1             # RRC roll-off
    wavelength: float = 1550e-9      # [m]
    dispersion: float = 17e-6        # D [s/m^2] (17 ps/nm/km)
    length: float = 50e3             # fibre length [m]
    linewidth: float = 100e3         # combined Tx+LO linewidth [Hz]
    freq_offset: float = 200e6       # carrier frequency offset [Hz]
    snr_db: float | None = 14.0      # Es/N0 per polarisation; None = noiseless
    jones: bool = True               # apply a Haar-random Jones matrix
    tx_rrc: bool = True              # RRC pulse shaping (False = rectangular spectrum)
    iq_imbalance: tuple | None = None  # transmitter IQ imbalance (amplitude eps, phase skew rad), both pols

    @property
    def fs(self) -> float:
        return self.sps * self.symbol_rate

    @property
    def n_samp(self) -> int:
        return self.sps * self.n_sym

    def with_(self, **kw) -> "LinkParams":
        return replace(self, **kw)


@dataclass
class Frame:
    """One generated frame (or stream) and everything drawn to make it."""

    params: LinkParams
    seed: int
    samples: np.ndarray              # complex128 [2, S]   received field at sps
    bits: np.ndarray                 # uint8 [2, n_sym*m]  transmitted bits (0/1)
    ref_words: np.ndarray            # uint32 [2, ceil(n_sym*m/32)] packed bits
    symbols: np.ndarray              # complex128 [2, n_sym] transmitted symbols
    jones: np.ndarray                # complex128 [2, 2]
    phase: np.ndarray                # float64 [S] common laser phase (rad)
    noise_var: np.ndarray            # float64 [2] AWGN variance per sample
    extra: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# bits -> symbols (transmitter side)
# ----------------------------------------------------------------------------

def _gray_to_level(g: np.ndarray, nbits: int) -> np.ndarray:
    """Binary-reflected Gray code word -> its position on the PAM axis."""
    level = g.copy()
    shift = 1
    while shift < nbits:
        level ^= level >> shift
        shift <<= 1
    return level


def modulate(bits: np.ndarray, bits_per_sym: int) -> np.ndarray:
    """Gray square-QAM mapping, unit average energy.

    Per symbol, the first m/2 bits (MSB first) are the Gray word of the
    in-phase level and the last m/2 bits that of the quadrature level; level l
    of L = 2^(m/2) sits at amplitude (2l - (L-1)) / sqrt(2(M-1)/3).
    """
    m = bits_per_sym
    if m not in (2, 4, 6, 8):
        raise ValueError(f"bits_per_sym must be even in [2, 8], got {m}")
    h = m // 2
    L = 1 << h
    M = L * L
    b = bits.reshape(bits.shape[:-1] + (-1, m)).astype(np.int64)
    weights = 1 << np.arange(h - 1, -1, -1)
    gi = (b[..., :h] * weights).sum(-1)
    gq = (b[..., h:] * weights).sum(-1)
    li = _gray_to_level(gi, h)
    lq = _gray_to_level(gq, h)
    amp = 1.0 / np.sqrt(2.0 * (M - 1) / 3.0)
    return ((2 * li - (L - 1)) + 1j * (2 * lq - (L - 1))) * amp


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """uint8 0/1 bits [..., n] -> uint32 words [..., ceil(n/32)]; bit i -> word i//32, bit i%32."""
    n = bits.shape[-1]
    nw = (n + 31) // 32
    pad = np.zeros(bits.shape[:-1] + (nw * 32,), dtype=np.uint64)
    pad[..., :n] = bits
    pad = pad.reshape(bits.shape[:-1] + (nw, 32))
    words = (pad << np.arange(32, dtype=np.uint64)).sum(-1)
    return words.astype(np.uint32)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    """Inverse of :func:`pack_bits`."""
    w = words.astype(np.uint64)[..., :, None] >> np.arange(32, dtype=np.uint64)
    bits = (w & 1).astype(np.uint8).reshape(words.shape[:-1] + (-1,))
    return bits[..., :n]


# ----------------------------------------------------------------------------
# channel pieces
# ----------------------------------------------------------------------------

def rrc_spectrum(f: np.ndarray, symbol_rate: float, rolloff: float) -> np.ndarray:
    """Root-raised-cosine amplitude spectrum, H(0) = 1."""
    af = np.abs(f)
    f1 = (1.0 - rolloff) * symbol_rate / 2.0
    f2 = (1.0 + rolloff) * symbol_rate / 2.0
    H = np.zeros_like(af)
    H[af <= f1] = 1.0
    band = (af > f1) & (af <= f2)
    if rolloff > 0:
        H[band] = np.sqrt(0.5 * (1.0 + np.cos(np.pi / (rolloff * symbol_rate) * (af[band] - f1))))
    return H


def fibre_dispersion(f: np.ndarray, p: LinkParams) -> np.ndarray:
    """Linear fibre response exp(j beta2/2 w^2 L) for the baseband frequencies f."""
    beta2 = -p.dispersion * p.wavelength**2 / (2.0 * np.pi * C_LIGHT)
    w = 2.0 * np.pi * f
    return np.exp(1j * 0.5 * beta2 * w * w * p.length)


def haar_unitary(rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed 2x2 unitary (Mezzadri's QR recipe)."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def iq_coefficients(eps: float, phi: float) -> tuple[complex, complex]:
    """(mu, nu) of the transmitter IQ imbalance x -> mu x + nu conj(x) for I and Q branches
    I' = (1 + eps)(I cos phi - Q sin phi), Q' = (1 - eps)(Q cos phi - I sin phi)."""
    mu = np.cos(phi) + 1j * eps * np.sin(phi)
    nu = eps * np.cos(phi) - 1j * np.sin(phi)
    return complex(mu), complex(nu)


def _streams(seed: int):
    ss = np.random.SeedSequence(seed)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(5)]


def generate(p: LinkParams, seed: int) -> Frame:
    """Draw one periodic frame of ``p.n_sym`` symbols per polarisation."""
    if p.n_sym <= 0:
        raise ValueError("n_sym must be positive")
    rng_bits, rng_jones, rng_phase, rng_awgn, _rng_nl = _streams(seed)
    m = p.bits_per_sym
    N, S, sps = p.n_sym, p.n_samp, p.sps

    bits = rng_bits.integers(0, 2, size=(2, N * m), dtype=np.uint8)
    symbols = modulate(bits, m)

    x = np.zeros((2, S), dtype=np.complex128)
    x[:, ::sps] = symbols
    f = np.fft.fftfreq(S, d=1.0 / p.fs)
    shape = np.sqrt(sps) * rrc_spectrum(f, p.symbol_rate, p.rolloff) if p.tx_rrc else \
        np.where(np.abs(f) <= p.symbol_rate / 2, np.sqrt(sps), 0.0)
    extra = {}
    if p.iq_imbalance is None:
        X = np.fft.fft(x, axis=1) * (shape * fibre_dispersion(f, p))[None, :]
        x = np.fft.ifft(X, axis=1)
    else:
        # the IQ modulator acts on the shaped drive signals, ahead of the fibre
        x = np.fft.ifft(np.fft.fft(x, axis=1) * shape[None, :], axis=1)
        mu, nu = iq_coefficients(*p.iq_imbalance)
        x = mu * x + nu * np.conj(x)
        x = np.fft.ifft(np.fft.fft(x, axis=1) * fibre_dispersion(f, p)[None, :], axis=1)
        extra["iq"] = (mu, nu)

    J = haar_unitary(rng_jones) if p.jones else np.eye(2, dtype=np.complex128)
    x = J @ x

    i = np.arange(S, dtype=np.float64)
    if p.linewidth > 0:
        steps = rng_phase.normal(0.0, np.sqrt(2.0 * np.pi * p.linewidth / p.fs), size=S)
        wiener = np.cumsum(steps)
    else:
        wiener = np.zeros(S)
    phase = 2.0 * np.pi * p.freq_offset * i / p.fs + wiener
    x = x * np.exp(1j * phase)[None, :]

    noise_var = np.zeros(2)
    if p.snr_db is not None:
        snr = 10.0 ** (p.snr_db / 10.0)
        for pol in range(2):
            P = np.mean(np.abs(x[pol]) ** 2)
            noise_var[pol] = sps * P / snr
            n = rng_awgn.standard_normal(S) + 1j * rng_awgn.standard_normal(S)
            x[pol] = x[pol] + np.sqrt(noise_var[pol] / 2.0) * n

    return Frame(params=p, seed=seed, samples=x, bits=bits, ref_words=pack_bits(bits),
                 symbols=symbols, jones=J, phase=phase, noise_var=noise_var, extra=extra)


# ----------------------------------------------------------------------------
# ADC front ends (precision forms of the input)
# ----------------------------------------------------------------------------

def quantise_int8(samples: np.ndarray, clip_sigma: float = 4.0):
    """Mid-tread 8-bit ADC per polarisation and real dimension.

    Step Delta_p = clip_sigma * sigma_p / 127 with sigma_p the RMS per real
    dimension of polarisation p; code = clamp(round(x / Delta_p), -127, 127).
    Returns (int8 [2, S, 2] interleaved I/Q codes, Delta [2]).
    """
    sig = np.sqrt(np.mean(np.abs(samples) ** 2, axis=1) / 2.0)
    delta = clip_sigma * sig / 127.0
    out = np.empty(samples.shape + (2,), dtype=np.int8)
    for p in range(samples.shape[0]):
        out[p, :, 0] = np.clip(np.rint(samples[p].real / delta[p]), -127, 127)
        out[p, :, 1] = np.clip(np.rint(samples[p].imag / delta[p]), -127, 127)
    return out, delta


def to_fp16(samples: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even FP16 I/Q pairs, float16 [2, S, 2]."""
    out = np.empty(samples.shape + (2,), dtype=np.float16)
    out[..., 0] = samples.real.astype(np.float16)
    out[..., 1] = samples.imag.astype(np.float16)
    return out


def to_c64(samples: np.ndarray) -> np.ndarray:
    """complex64 copy laid out as [2, S] interleaved (re, im) float32 pairs."""
    return np.ascontiguousarray(samples.astype(np.complex64))
