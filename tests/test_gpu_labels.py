"""GPU: the post-equaliser's training labels (rx_pe_targets) against the oracle's FP64 reference
(oracle.cnn.aligned_targets, repair_quarter_turns): transmitted symbols put in the outputs' frame
by the decision stage's (pol, turn, delay), each whole block turned by its best quarter turn. A
block's choice may differ only where the oracle's error sums of the two turns tie within FP32 reach;
every label is a sign swap of a transmitted symbol, so agreeing labels are equal bit for bit."""

import numpy as np
import pytest

from oracle import cnn

pytestmark = pytest.mark.gpu


def _case(n_sym, n_ref, pol, rot, dly, block, seed, noise=0.08):
    rng = np.random.default_rng(seed)
    lv = np.array([-3.0, -1.0, 1.0, 3.0]) / np.sqrt(10.0)
    s = (lv[rng.integers(0, 4, (2, n_ref))] + 1j * lv[rng.integers(0, 4, (2, n_ref))]).astype(np.complex64)
    base = cnn.aligned_targets(pol, rot, dly, s.astype(np.complex128), n_sym)
    nb = n_sym // block
    turns = rng.integers(0, 4, (2, nb))            # the chain's carrier slips, per block
    z = base.copy()
    for q in range(2):
        for j in range(nb):
            z[q, j * block:(j + 1) * block] *= 1j ** turns[q, j]
    z = z + noise * (rng.normal(size=z.shape) + 1j * rng.normal(size=z.shape))
    return s, z.astype(np.complex64)


@pytest.mark.parametrize("n_sym,n_ref,pol,rot,dly,block,seed", [
    (8192, 8192, [0, 1], [0, 0], [0, 0], 1024, 1),
    (10000, 9990, [1, 0], [3, 1], [5, -16], 1024, 2),     # ragged tail, delays both ways, swapped pols
    (4096, 4100, [0, 0], [2, 3], [-3, 7], 256, 3),
    (777, 800, [1, 1], [1, 2], [16, -1], 1000, 4),        # no whole block: labels unturned
])
def test_labels_match_the_oracle(n_sym, n_ref, pol, rot, dly, block, seed):
    import torch
    from paper_2011_13695_gb300 import build, rx
    build.build()
    s, z = _case(n_sym, n_ref, pol, rot, dly, block, seed)
    zd = torch.from_numpy(np.ascontiguousarray(z)).cuda()
    sd = torch.from_numpy(np.ascontiguousarray(s)).cuda()
    out = torch.full_like(zd, complex(float("nan"), float("nan")))
    rx.rx_pe_targets(zd.data_ptr(), n_sym, sd.data_ptr(), n_ref, pol, rot, dly, block, out.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    z64 = z.astype(np.complex128)
    want = cnn.repair_quarter_turns(z64, cnn.aligned_targets(pol, rot, dly, s.astype(np.complex128), n_sym), block)
    err = cnn.quarter_turn_errors(z64, cnn.aligned_targets(pol, rot, dly, s.astype(np.complex128), n_sym), block)
    nb = n_sym // block
    for q in range(2):
        for j in range(nb):
            sl = slice(j * block, (j + 1) * block)
            if not np.array_equal(got[q, sl], want[q, sl].astype(np.complex64)):
                e = np.sort(err[:, q, j])
                assert e[1] - e[0] <= 1e-5 * e[1], f"block {j} of output {q}: not a near-tie"
    tail = slice(nb * block, n_sym)
    assert np.array_equal(got[:, tail], want[:, tail].astype(np.complex64))


def test_labels_reject_bad_alignment():
    import torch
    from paper_2011_13695_gb300 import build, rx
    build.build()
    t = torch.zeros(64, dtype=torch.complex64, device="cuda")
    for pol, rot in (([2, 0], [0, 0]), ([0, 1], [0, 4])):
        with pytest.raises(rx.RxError) as e:
            rx.rx_pe_targets(t.data_ptr(), 32, t.data_ptr(), 32, pol, rot, [0, 0], 8, t.data_ptr(), None)
        assert e.value.status == rx.RX_EINVAL
