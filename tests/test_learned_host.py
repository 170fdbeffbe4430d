"""Host-side logic of the learned post-equaliser's training loop (CPU tensors, no GPU):
target alignment from the decision stage's (pol, turn, delay) and the per-block
quarter-turn repair of labels after a cycle slip."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2011_13695_gb300.learned import aligned_targets, repair_quarter_turns  # noqa: E402


def _symbols(n, seed=0):
    rng = np.random.default_rng(seed)
    s = (rng.integers(0, 4, (2, n)) * 2 - 3) + 1j * (rng.integers(0, 4, (2, n)) * 2 - 3)
    return torch.from_numpy((s / np.sqrt(10)).astype(np.complex64))


def test_aligned_targets_follow_pol_turn_and_delay():
    n = 300
    s = _symbols(n)
    stats = {"pol_map": [1, 0], "rotation": [3, 1], "delay": [2, -3]}
    # outputs as the decision stage describes them: z_q[k] j^r_q = s_p_q[k + d_q]
    z = torch.zeros((2, n), dtype=torch.complex64)
    for q in range(2):
        p, r, d = stats["pol_map"][q], stats["rotation"][q], stats["delay"][q]
        for k in range(n):
            if 0 <= k + d < n:
                z[q, k] = s[p, k + d] * (-1j) ** r
    t = aligned_targets(stats, s, n)
    assert torch.equal(t, z)
    assert torch.all(t[0, n - 2:] == 0) and torch.all(t[1, :3] == 0)


def test_quarter_turn_repair_per_block():
    n, blk = 4096, 1024
    s = _symbols(n, 1)
    turns = [0, 1, 1, 3]
    z = s.clone()
    for b, r in enumerate(turns):
        z[:, b * blk:(b + 1) * blk] *= 1j ** r
    z += 0.05 * torch.randn(2, n, dtype=torch.complex64)
    fixed = repair_quarter_turns(z, s, blk)
    for b, r in enumerate(turns):
        assert torch.allclose(fixed[:, b * blk:(b + 1) * blk], s[:, b * blk:(b + 1) * blk] * (1j ** r))
    # a tail shorter than one block keeps its labels
    z2 = torch.cat([z, z[:, :100]], 1)
    s2 = torch.cat([s, s[:, :100]], 1)
    assert torch.equal(repair_quarter_turns(z2, s2, blk)[:, n:], s2[:, n:])
