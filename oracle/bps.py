"""A5 blind phase search, integer unwrap and derotation, FP64.

TEST INFRASTRUCTURE (see the package docstring).

Method: blind phase search (Pfau, Hoffmann, Noe, JLT 2009). The paper has no
carrier-phase estimator of this kind; its nearest relative is the serial
clock-phase unwrap done by one warp (Sec. III-B), which checks each averaged
phase against the previous one for a jump of more than pi. Readings taken:

* test phases theta_b = (b/B - 1/2) pi/2, b = 0..B-1;
* dist[k, b] = |y_k e^{-j theta_b} - dec(y_k e^{-j theta_b})|^2;
* D[k, b] = sum of dist[i, b] over i in [k - W//2, k - W//2 + W) clipped to the
  frame; b*_k = argmin_b D[k, b], ties to the smallest b;
* unwrap in integers: m_k = m_{k-1} + J(b*_{k-1} - b*_k) with J(d) = +1 for
  d > B/2, -1 for d < -B/2, else 0 (a tie |d| = B/2 does not jump); m and the
  last b* carry across frames of a stream, m starts at 0;
* z_k = y_k e^{-j theta_{b*_k}} (-j)^(m_k mod 4).
"""

from __future__ import annotations

import numpy as np

from . import qam

QUARTER_TURNS = np.array([1.0, -1j, -1.0, 1j])  # (-j)^r, r = 0..3


def test_phases(B: int) -> np.ndarray:
    return (np.arange(B) / B - 0.5) * (np.pi / 2.0)


def distances(y: np.ndarray, m: int, B: int, chunk: int = 1 << 15) -> np.ndarray:
    """dist [N, B] for one polarisation."""
    th = test_phases(B)
    rot = np.exp(-1j * th)[None, :]
    out = np.empty((y.shape[0], B))
    for s in range(0, y.shape[0], chunk):
        r = y[s:s + chunk, None] * rot
        out[s:s + chunk] = np.abs(r - qam.decide(r, m)) ** 2
    return out


def window_sums(dist: np.ndarray, W: int, chunk: int = 1 << 14) -> np.ndarray:
    """D[k, b] = sum_{i=k-W//2}^{k-W//2+W-1} dist[i, b], terms outside [0, N) omitted."""
    N, B = dist.shape
    lead = W // 2
    pad = np.zeros((N + W, B))
    pad[lead:lead + N] = dist
    D = np.empty((N, B))
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        win = np.lib.stride_tricks.sliding_window_view(pad[s:e + W - 1], W, axis=0)  # [e-s, B, W]
        D[s:e] = win.sum(axis=-1)
    return D


def unwrap(bstar: np.ndarray, B: int, b_prev=None, m_prev: int = 0) -> np.ndarray:
    prev = np.concatenate([[bstar[0] if b_prev is None else b_prev], bstar[:-1]]).astype(np.int64)
    d = prev - bstar.astype(np.int64)
    J = np.where(d > B / 2, 1, np.where(d < -B / 2, -1, 0))
    return m_prev + np.cumsum(J)


def blind_phase_search(y: np.ndarray, m: int, B: int, W: int, b_prev=None, m_prev: int = 0):
    """One polarisation. Returns (b* int64 [N], m int64 [N], z complex128 [N])."""
    N = y.shape[0]
    if N == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.complex128)
    D = window_sums(distances(y, m, B), W)
    bstar = np.argmin(D, axis=1)
    mk = unwrap(bstar, B, b_prev, m_prev)
    th = test_phases(B)
    z = y * np.exp(-1j * th[bstar]) * QUARTER_TURNS[np.mod(mk, 4)]
    return bstar.astype(np.int64), mk, z
