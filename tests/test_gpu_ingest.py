"""GPU tests of the real-time ingest emulation (rx_ingest_run through the C ABI).

* Continuity: buffers processed one by one on several streams, each joined to its predecessor by the
  overlap step (the previous buffer's last 2N codes), give the stream's KK output: the concatenated
  outputs equal the oracle's KK front end on the whole stream as one frame (same block grid, same
  downshift phase), within the KK parity tolerance (2e-5 relative RMS), also around every buffer
  boundary; only the stream's first N/2 outputs (the start-up transient of the zero carry) differ.
* Drops: buffers arriving faster than one slot can take them are counted as dropped, and
  processed + dropped = delivered.
* Real time: at the paper's 4 GSa/s with 2^22-sample buffers (1.049 ms each) on five streams no
  buffer is dropped and the mean latency stays below five buffer periods.
"""

import numpy as np
import pytest

from oracle import kk
from synth.kk import KKLink, generate_kk
from tests.gpu_util import rel_rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2011_13695_gb300 import build
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    build.build()


def front_end(fr, N=1024):
    from paper_2011_13695_gb300.receiver import KKFrontEnd
    p = fr.link
    return KKFrontEnd(N, p.tone_offset / p.fs, p.rolloff, fr.scale, fr.dc, 1e-6)


@pytest.mark.parametrize("n_streams", [1, 3])
def test_buffers_join_into_the_stream(n_streams):
    N, S, nb = 1024, 16384, 8
    fr = generate_kk(KKLink(bits_per_sym=4, n_sym=nb * S // 4, cspr_db=11.0, snr_db=25.0), seed=3)
    fe = front_end(fr, N)
    # 20 MSa/s: 0.8 ms per buffer, far longer than a buffer takes
    stats, out = fe.ingest(fr.codes, S, 2e7, n_streams, nb, keep_outputs=True)
    fe.close()
    assert stats["buffers"] == nb and stats["processed"] == nb and stats["dropped"] == 0, stats
    p = fr.link
    _, y_o = kk.kk_receive(fr.codes, float(np.float32(fr.scale)), float(np.float32(fr.dc)),
                           float(np.float32(1e-6)), p.tone_offset / p.fs, p.rolloff, N)
    # buffer i holds stream outputs [i S/2 - N/2, (i + 1) S/2 - N/2)
    got = out.astype(np.complex128)[N // 2:]
    ref = y_o[:got.size]
    # the first N/2 outputs of the stream see the zero carry of the first buffer (start-up transient)
    e = rel_rms(got[N // 2:], ref[N // 2:])
    print("stream rel rms %.2e" % e)
    assert e <= 2e-5, e
    # every buffer boundary, sample by sample
    for i in range(1, nb):
        b = i * S // 2 - N // 2
        w = slice(b - 64, b + 64)
        assert rel_rms(got[w], ref[w]) <= 1e-4, i


def test_buffers_are_dropped_when_no_slot_is_free():
    N, S = 1024, 1 << 16
    fr = generate_kk(KKLink(bits_per_sym=4, n_sym=S // 4, cspr_db=11.0), seed=4)
    fe = front_end(fr, N)
    # a buffer every 0.07 ns: one slot cannot keep up
    stats, _ = fe.ingest(fr.codes, S, 1e15, 1, 40)
    fe.close()
    assert stats["buffers"] == 40
    assert stats["processed"] >= 1 and stats["dropped"] >= 1, stats
    assert stats["processed"] + stats["dropped"] == stats["buffers"]


def test_real_time_at_four_gsa_per_second():
    S = 1 << 22
    fr = generate_kk(KKLink(bits_per_sym=4, n_sym=S // 4, cspr_db=11.0, snr_db=20.0), seed=5)
    fe = front_end(fr, 1024)
    stats, _ = fe.ingest(fr.codes, S, 4e9, 5, 30)
    fe.close()
    print(stats)
    assert abs(stats["buffer_period_ms"] - 1.048576) < 1e-9
    assert stats["dropped"] == 0, stats
    assert stats["mean_latency_ms"] < 5 * stats["buffer_period_ms"], stats
