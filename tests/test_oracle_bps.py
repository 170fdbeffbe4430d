"""Pins for the oracle's A5 blind phase search + unwrap and A6 alignment/counting."""

import itertools

import numpy as np
import pytest

from oracle import bps, decide, qam


def _brute_bps(y, m, B, W):
    """Direct transcription of the BPS definition: exhaustive nearest point, explicit window loops."""
    pts = qam.alphabet(m)
    N = len(y)
    th = [(b / B - 0.5) * np.pi / 2 for b in range(B)]
    dist = [[min(abs(y[i] * np.exp(-1j * th[b]) - s) ** 2 for s in pts) for b in range(B)] for i in range(N)]
    best = []
    for k in range(N):
        D = []
        for b in range(B):
            tot = 0.0
            for i in range(k - W // 2, k - W // 2 + W):
                if 0 <= i < N:
                    tot += dist[i][b]
            D.append(tot)
        best.append(min(range(B), key=lambda b: (D[b], b)))
    return best


@pytest.mark.parametrize("m,B,W", [(2, 4, 4), (4, 4, 4), (4, 5, 3), (2, 8, 2)])
def test_bps_matches_brute_force_on_tiny_inputs(m, B, W):
    rng = np.random.default_rng(B * 10 + W)
    for _ in range(20):
        y = (rng.normal(size=8) + 1j * rng.normal(size=8)) * 0.8
        b, _, _ = bps.blind_phase_search(y, m, B, W)
        assert b.tolist() == _brute_bps(y, m, B, W)


@pytest.mark.parametrize("m,B", [(2, 32), (4, 64), (6, 64)])
def test_bps_grid_phase_is_recovered_exactly(m, B):
    rng = np.random.default_rng(m)
    s = qam.alphabet(m)[rng.integers(0, 2**m, 2000)]
    th = bps.test_phases(B)
    for b0 in (0, 1, B // 2, B - 1):
        b, mk, z = bps.blind_phase_search(s * np.exp(1j * th[b0]), m, B, 64)
        assert np.all(b == b0) and np.all(mk == 0)
        assert np.allclose(z, s, atol=1e-12)


def test_unwrap_counts_quarter_turns_on_a_phase_ramp():
    """A slow ramp across many pi/4 boundaries: m_k counts each crossing exactly."""
    m, B = 2, 32
    rng = np.random.default_rng(9)
    N = 6000
    s = qam.alphabet(m)[rng.integers(0, 4, N)]
    phi = np.linspace(-0.3, 5.0, N)                        # crosses +pi/4 + k pi/2 several times
    b, mk, z = bps.blind_phase_search(s * np.exp(1j * phi), m, B, 16)
    # the unwrapped estimate tracks the ramp within one grid step, away from the edges
    est = bps.test_phases(B)[b] + (np.pi / 2) * mk
    inner = slice(50, N - 50)
    assert np.max(np.abs(est[inner] - phi[inner])) < np.pi / 2 / B
    assert mk[-1] - mk[0] == 3                              # boundaries pi/4, 3pi/4, 5pi/4 lie in (-0.3, 5.0)
    assert np.allclose(z[inner], s[inner] * np.exp(1j * (phi[inner] - est[inner])), atol=1e-12)
    assert np.all(np.abs(np.diff(mk)) <= 1)
    # carried state continues the count across a frame cut
    b1, m1, _ = bps.blind_phase_search((s * np.exp(1j * phi))[:3000], m, B, 16)
    b2, m2, _ = bps.blind_phase_search((s * np.exp(1j * phi))[3000:], m, B, 16, b_prev=int(b1[-1]), m_prev=int(m1[-1]))
    assert m2[-1] == mk[-1]


def test_unwrap_jump_rule():
    B = 8
    seq = np.array([7, 0, 1, 7, 6, 2, 6, 3])
    # d = prev - cur: (7-0)=7>4:+1, (0-1)=-1:0, (1-7)=-6<-4:-1, (7-6)=1:0, (6-2)=4 tie:0, (2-6)=-4 tie:0, (6-3)=3:0
    assert bps.unwrap(seq, B).tolist() == [0, 1, 1, 0, 0, 0, 0, 0]
    assert bps.unwrap(seq, B, b_prev=0, m_prev=5).tolist() == [4, 5, 5, 4, 4, 4, 4, 4]


def test_resolve_finds_a_planted_alignment_and_count_is_exact():
    rng = np.random.default_rng(2)
    m, N = 4, 3000
    bits = rng.integers(0, 2, size=(2, N * m), dtype=np.uint8)
    words = qam.pack_words(bits)
    li, lq = qam.bits_to_levels(bits.reshape(2, N, m), m)
    s = qam.levels_to_symbols(li, lq, m)
    planted = [(1, 3, -5), (0, 2, 7)]                      # (p, r, d) per output
    z = np.zeros((2, N), complex)
    n = np.arange(N)
    for q, (p, r, d) in enumerate(planted):
        t = np.clip(n + d, 0, N - 1)
        z[q] = s[p, t] / decide.QUARTER[r]
    z += 0.02 * (rng.normal(size=z.shape) + 1j * rng.normal(size=z.shape))
    z[0, 700] = 5.0                                         # one planted symbol error
    sync, L = decide.resolve(z, words, m, N, 100, 1100, 16)
    assert [t[:3] for t in sync] == planted and L == 1000
    c = decide.count(z, sync, words, m, N, 100, N - 100)
    # brute force: the planted error flips the bits of symbol 700 of output 0 only
    want = qam.levels_to_bits(li[1, 695], lq[1, 695], m)
    got = qam.levels_to_bits(*qam.decide_levels(np.array([5.0 * decide.QUARTER[3]]), m), m)[0]
    assert c["bit_errors"] == int(np.sum(want != got))
    assert c["symbol_errors"] == int(np.any(want != got))
    assert c["bits"] == 2 * (N - 200) * m and c["symbols"] == 2 * (N - 200)


def test_resolve_tie_goes_to_smallest_tuple():
    m, N = 2, 400
    z = np.full((2, N), (1 + 1j) / np.sqrt(2))              # constant: every (p, r=0, d) matches equally
    words = qam.pack_words(np.ones((2, N * m), np.uint8))
    sync, _ = decide.resolve(z, words, m, N, 20, 300, 4)
    assert [t[:3] for t in sync] == [(0, 0, -4), (0, 0, -4)]
