"""CPU pins of the learned post-equaliser's training labels (the oracle's FP64 reference, which the
GPU label kernel rx_pe_targets is compared with): alignment from the decision stage's (pol, turn,
delay) and the per-block quarter-turn repair after a cycle slip."""

import numpy as np

from oracle import cnn


def _symbols(n, seed=0):
    rng = np.random.default_rng(seed)
    s = (rng.integers(0, 4, (2, n)) * 2 - 3) + 1j * (rng.integers(0, 4, (2, n)) * 2 - 3)
    return s / np.sqrt(10)


def test_aligned_targets_follow_pol_turn_and_delay():
    """Outputs built the way the decision stage describes them (z_q[k] j^r_q = s_p_q[k + d_q]) are
    their own labels; positions without a transmitted symbol are 0."""
    n = 300
    s = _symbols(n)
    pol, rot, dly = [1, 0], [3, 1], [2, -3]
    z = np.zeros((2, n), dtype=np.complex128)
    for q in range(2):
        for k in range(n):
            if 0 <= k + dly[q] < n:
                z[q, k] = s[pol[q], k + dly[q]] / (1j ** rot[q])
    t = cnn.aligned_targets(pol, rot, dly, s, n)
    assert np.allclose(t, z, atol=1e-15)
    assert np.all(t[0, n - 2:] == 0) and np.all(t[1, :3] == 0)


def test_quarter_turn_repair_per_block():
    """Blocks of outputs turned by known quarter turns get labels turned the same way; a tail
    shorter than one block keeps its labels."""
    n, blk = 4096, 1024
    s = _symbols(n, 1)
    turns = [0, 1, 1, 3]
    rng = np.random.default_rng(2)
    z = s.copy()
    for b, r in enumerate(turns):
        z[:, b * blk:(b + 1) * blk] *= 1j ** r
    z += 0.05 * (rng.normal(size=z.shape) + 1j * rng.normal(size=z.shape))
    fixed = cnn.repair_quarter_turns(z, s, blk)
    for b, r in enumerate(turns):
        assert np.allclose(fixed[:, b * blk:(b + 1) * blk], s[:, b * blk:(b + 1) * blk] * (1j ** r))
    z2 = np.concatenate([z, z[:, :100]], 1)
    s2 = np.concatenate([s, s[:, :100]], 1)
    assert np.array_equal(cnn.repair_quarter_turns(z2, s2, blk)[:, n:], s2[:, n:])


def test_quarter_turn_errors_by_explicit_sums():
    rng = np.random.default_rng(3)
    z = rng.normal(size=(2, 50)) + 1j * rng.normal(size=(2, 50))
    t = rng.normal(size=(2, 50)) + 1j * rng.normal(size=(2, 50))
    err = cnn.quarter_turn_errors(z, t, 16)
    assert err.shape == (4, 2, 3)
    for u in range(4):
        for q in range(2):
            for j in range(3):
                want = sum(abs(z[q, i] - t[q, i] * (1j ** u)) ** 2 for i in range(16 * j, 16 * j + 16))
                assert abs(err[u, q, j] - want) < 1e-12
