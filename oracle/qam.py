"""Gray square-QAM alphabet, hard decisions and (de)mapping, FP64.

TEST INFRASTRUCTURE (see the package docstring).

The paper's receivers decide and demap inside their last kernel (Sec. III-C
for PAM, Sec. IV-D for QAM) but do not state a bit mapping. Reading taken
here: per polarisation, M = L^2 points with L = 2^(m/2) levels per real
dimension at (2l - (L-1)) * a, a = 1/sqrt(2(M-1)/3) (unit average energy);
the first m/2 bits of a symbol (MSB first) are the binary-reflected Gray word
of the in-phase level l_I, the last m/2 that of the quadrature level l_Q. For
QPSK this means bit 0 -> negative, bit 1 -> positive amplitude.

The hard decision is the nearest alphabet point (the maximum-likelihood
decision for circular Gaussian noise). For a square grid it separates into
one nearest-level decision per real dimension, which is what ``decide_levels``
computes; ``tests`` check it against an exhaustive nearest-point search.
"""

from __future__ import annotations

import numpy as np


def n_levels(m: int) -> int:
    if m not in (2, 4, 6, 8):
        raise ValueError(f"bits per symbol must be 2, 4, 6 or 8, got {m}")
    return 1 << (m // 2)


def amp(m: int) -> float:
    """Level spacing half-step a: points at (2l - (L-1)) * a."""
    M = n_levels(m) ** 2
    return 1.0 / np.sqrt(2.0 * (M - 1) / 3.0)


def level_values(m: int) -> np.ndarray:
    L = n_levels(m)
    return (2.0 * np.arange(L) - (L - 1)) * amp(m)


def alphabet(m: int) -> np.ndarray:
    """All M points, index = l_I * L + l_Q."""
    v = level_values(m)
    return (v[:, None] + 1j * v[None, :]).reshape(-1)


def cma_radius(m: int) -> float:
    """R2 = E|s|^4 / E|s|^2 of the unit-energy alphabet (Godard p = 2)."""
    s = alphabet(m)
    return float(np.mean(np.abs(s) ** 4) / np.mean(np.abs(s) ** 2))


def decide_levels(z: np.ndarray, m: int):
    """Nearest-point decision as integer level indices (l_I, l_Q)."""
    L = n_levels(m)
    a = amp(m)

    def one(u):
        return np.clip(np.rint((u / a + (L - 1)) / 2.0), 0, L - 1).astype(np.int64)

    return one(np.real(z)), one(np.imag(z))


def levels_to_symbols(li: np.ndarray, lq: np.ndarray, m: int) -> np.ndarray:
    L = n_levels(m)
    a = amp(m)
    return ((2.0 * li - (L - 1)) + 1j * (2.0 * lq - (L - 1))) * a


def decide(z: np.ndarray, m: int) -> np.ndarray:
    """dec(z): the nearest alphabet point."""
    li, lq = decide_levels(z, m)
    return levels_to_symbols(li, lq, m)


def _level_to_gray(l: np.ndarray) -> np.ndarray:
    return l ^ (l >> 1)


def _gray_to_level(g: np.ndarray, nbits: int) -> np.ndarray:
    out = np.zeros_like(g)
    for k in range(nbits - 1, -1, -1):            # b_k = g_k xor b_{k+1}, MSB first
        prev = (out >> (k + 1)) & 1
        out |= (((g >> k) & 1) ^ prev) << k
    return out


def levels_to_bits(li: np.ndarray, lq: np.ndarray, m: int) -> np.ndarray:
    """(l_I, l_Q) -> uint8 bits [..., m], MSB of each Gray word first."""
    h = m // 2
    gi = _level_to_gray(np.asarray(li, dtype=np.int64))
    gq = _level_to_gray(np.asarray(lq, dtype=np.int64))
    sh = np.arange(h - 1, -1, -1)
    bi = (gi[..., None] >> sh) & 1
    bq = (gq[..., None] >> sh) & 1
    return np.concatenate([bi, bq], axis=-1).astype(np.uint8)


def bits_to_levels(bits: np.ndarray, m: int):
    """uint8 bits [..., m] -> (l_I, l_Q)."""
    h = m // 2
    b = np.asarray(bits, dtype=np.int64)
    w = 1 << np.arange(h - 1, -1, -1)
    gi = (b[..., :h] * w).sum(-1)
    gq = (b[..., h:] * w).sum(-1)
    return _gray_to_level(gi, h), _gray_to_level(gq, h)


def unpack_words(words: np.ndarray, n_bits: int) -> np.ndarray:
    """uint32 words [..., W] -> uint8 bits [..., n_bits]; bit i is bit i%32 of word i//32."""
    w = np.asarray(words, dtype=np.uint64)[..., :, None] >> np.arange(32, dtype=np.uint64)
    return (w & 1).astype(np.uint8).reshape(words.shape[:-1] + (-1,))[..., :n_bits]


def pack_words(bits: np.ndarray) -> np.ndarray:
    """uint8 bits [..., n] -> uint32 words [..., ceil(n/32)] (same layout)."""
    n = bits.shape[-1]
    nw = (n + 31) // 32
    pad = np.zeros(bits.shape[:-1] + (nw * 32,), dtype=np.uint64)
    pad[..., :n] = bits
    pad = pad.reshape(bits.shape[:-1] + (nw, 32))
    return (pad << np.arange(32, dtype=np.uint64)).sum(-1).astype(np.uint32)
