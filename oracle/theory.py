"""Closed forms used to pin the oracle.

TEST INFRASTRUCTURE (see the package docstring).

* ``gray_qam_ber``: exact bit-error ratio of Gray-coded square M-QAM with
  nearest-point decisions over AWGN at a given Es/N0. The I and Q rails are
  independent L-PAM channels (L = sqrt(M)) with noise variance N0/2 per real
  dimension; for each sent level l and decided level l' the probability is a
  difference of Gaussian tails between the decision thresholds, weighted by
  the Hamming distance of the two Gray words (the same quantity as the
  Cho-Yoon 2002 expression, summed term by term).
* ``q_from_ber`` / ``ber_from_q``: Q = 20 log10(sqrt(2) erfcinv(2 BER)), the
  conversion behind the paper's hard-decision FEC thresholds, Q = 8.4 dB for
  6.7 % overhead and 5.7 dB for 20 % overhead (Sec. I, Sec. V-B).
"""

from __future__ import annotations

import numpy as np
from scipy.special import erfc, erfcinv


def _qfunc(x):
    return 0.5 * erfc(np.asarray(x, dtype=np.float64) / np.sqrt(2.0))


def gray_qam_ber(m: int, es_n0_db: float) -> float:
    h = m // 2
    L = 1 << h
    M = L * L
    a = 1.0 / np.sqrt(2.0 * (M - 1) / 3.0)
    sigma = np.sqrt(1.0 / (2.0 * 10.0 ** (es_n0_db / 10.0)))   # per real dimension, Es = 1
    v = (2.0 * np.arange(L) - (L - 1)) * a
    thr = (2.0 * np.arange(1, L) - L) * a                      # L-1 thresholds between levels
    gray = np.arange(L) ^ (np.arange(L) >> 1)
    total = 0.0
    for l in range(L):
        for lp in range(L):
            if lp == l:
                continue
            ham = bin(int(gray[l] ^ gray[lp])).count("1")
            if lp > l:   # lower threshold of region lp above v_l
                p = _qfunc((thr[lp - 1] - v[l]) / sigma) - (_qfunc((thr[lp] - v[l]) / sigma) if lp < L - 1 else 0.0)
            else:
                p = _qfunc((v[l] - thr[lp]) / sigma) - (_qfunc((v[l] - thr[lp - 1]) / sigma) if lp > 0 else 0.0)
            total += p * ham
    return float(total / (L * h))


def q_from_ber(ber: float) -> float:
    return float(20.0 * np.log10(np.sqrt(2.0) * erfcinv(2.0 * ber)))


def ber_from_q(q_db: float) -> float:
    q = 10.0 ** (q_db / 20.0)
    return float(0.5 * erfc(q / np.sqrt(2.0)))
