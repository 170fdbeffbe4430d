"""The learned post-equaliser against the plain chain on split-step (nonlinear)
data: trained by the library's own kernels on chain outputs of some frames,
judged by the chain's own decision stage on a frame of another seed."""

from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _frame_on_device(fr):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(fr.samples.astype(np.complex64))).cuda()
    ref = torch.from_numpy(np.ascontiguousarray(fr.ref_words).view(np.int32)).cuda()
    sym = torch.from_numpy(np.ascontiguousarray(fr.symbols.astype(np.complex64))).cuda()
    return x, ref, sym


def test_post_equaliser_gains_over_plain_chain():
    import torch
    from oracle import cnn
    from paper_2011_13695_gb300.learned import PostEqualiser, chain_pairs, decide_stats
    from paper_2011_13695_gb300.receiver import Receiver
    from synth.ssfm import generate_nonlinear
    from synth.workloads import workload

    n = 1 << 18
    w = workload("dp-16qam-32gbd-ssfm", n_sym=n, launch_dbm=4.0, train_frames=2)
    rcv = Receiver(w["rx"], n)
    zs, ts, plain_train = [], [], []
    for seed in w["train_seeds"]:
        x, ref, sym = _frame_on_device(generate_nonlinear(w["link"], w["fibre"], seed, device="cuda"))
        z, t, st = chain_pairs(rcv, x, n, ref, sym)
        assert st["ber"] < 2e-2, st          # the plain chain acquired the frame
        zs.append(z)
        ts.append(t)
    x, ref, sym = _frame_on_device(generate_nonlinear(w["link"], w["fibre"], w["test_seed"], device="cuda"))
    z_test, _, plain = chain_pairs(rcv, x, n, ref, sym)

    pe = PostEqualiser(n, cnn.flatten(cnn.init_params(64, 9, seed=0)).astype(np.float32))
    edge = 1024
    losses = pe.train(zs, ts, edge, n - edge, steps=3000, window=4096, lr=1e-3, lr_final=1e-4, seed=0)
    assert torch.isfinite(losses).all()
    out = pe.forward(z_test)
    learned = decide_stats(rcv, out, n, ref)
    pe.close()
    rcv.close()
    print(f"plain BER {plain['ber']:.3e} EVM {plain['evm']:.4f}; learned BER {learned['ber']:.3e} "
          f"EVM {learned['evm']:.4f}; loss {float(losses[:20].mean()):.4e} -> {float(losses[-20:].mean()):.4e}")
    assert learned["symbols_counted"] == plain["symbols_counted"]
    # the gain at this size is small (a receptive field of 33 symbols against a dispersion memory of
    # about 120); the test asks for no loss in either measure and a lower bit error count
    assert learned["evm"] <= plain["evm"]
    assert learned["bit_errors"] < plain["bit_errors"]
