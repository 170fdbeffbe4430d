"""GPU: batched channels in one graph launch (tuned FFT size and LMS CTA size).

Every channel of the batch must give exactly what a single handle with the
same (tuned) configuration gives on the same frame, and two channels are
checked against the FP64 oracle with the tuned FFT size.
"""

import numpy as np
import pytest

from oracle.receiver import Receiver as OracleRx
from oracle.receiver import RxConfig
from synth import generate
from synth.workloads import batch_channels
from tests.gpu_util import rel_rms

pytestmark = pytest.mark.gpu

N_TEST = 1 << 14


@pytest.fixture(scope="module")
def batch_setup():
    import torch
    from paper_2011_13695_gb300 import build, rx
    from paper_2011_13695_gb300.receiver import config_from
    build.build()
    chans = batch_channels(42)
    frames, xs, refs, outs, cfgs = [], [], [], [], []
    for ch in chans:
        link = ch["link"].with_(n_sym=min(ch["link"].n_sym, N_TEST))
        fr = generate(link, ch["seed"])
        frames.append(fr)
        x = np.ascontiguousarray(fr.samples.astype(np.complex64))
        xs.append(torch.from_numpy(x.view(np.float32)).cuda())
        refs.append(torch.from_numpy(fr.ref_words.astype(np.uint32).view(np.int32)).cuda())
        words = (link.n_sym * link.bits_per_sym + 31) // 32
        outs.append(torch.zeros(2 * words, dtype=torch.int32, device="cuda"))
        cfgs.append(config_from(ch["rx"], link.n_sym))
    b = rx.rx_batch_create(cfgs)
    n_sym = [fr.params.n_sym for fr in frames]
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                                  # capture, then a replay
        rx.rx_batch_process(b, [t.data_ptr() for t in xs], n_sym, [t.data_ptr() for t in refs],
                            [t.data_ptr() for t in outs], stream)
    torch.cuda.synchronize()
    yield dict(b=b, chans=chans, frames=frames, xs=xs, refs=refs, outs=outs, n_sym=n_sym)
    rx.rx_batch_destroy(b)


def test_tuner_respects_the_dispersion_memory(batch_setup):
    from paper_2011_13695_gb300 import rx
    b = batch_setup["b"]
    for i, ch in enumerate(batch_setup["chans"]):
        c = rx.rx_batch_config(b, i)
        link = ch["link"]
        mem = (link.dispersion * link.length * link.wavelength ** 2 / 299792458.0 * link.symbol_rate * 1.1
               * 2 * link.symbol_rate)
        assert c.fft_size in (512, 1024, 2048, 4096, 8192)
        assert c.fft_size // 4 >= mem or c.fft_size == 8192
        assert c.lms_threads in (128, 256, 512)


def test_batch_equals_single_handles(batch_setup):
    import torch
    from paper_2011_13695_gb300 import rx
    b = batch_setup["b"]
    for i in range(len(batch_setup["chans"])):
        cfg = rx.rx_batch_config(b, i)
        h = rx.rx_create(cfg)
        N = batch_setup["n_sym"][i]
        out = torch.zeros_like(batch_setup["outs"][i])
        rx.rx_process(h, batch_setup["xs"][i].data_ptr(), N, batch_setup["refs"][i].data_ptr(), out.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
        st = rx.rx_stats(h)
        bst = rx.rx_batch_stats(b, i)
        assert torch.equal(out, batch_setup["outs"][i]), f"channel {i}: bits differ"
        # the batch ran the frame twice (capture + replay): counters are exactly twice a single run
        assert bst["bit_errors"] == 2 * st["bit_errors"] and bst["bits_counted"] == 2 * st["bits_counted"]
        assert bst["fo_code"] == st["fo_code"]
        rx.rx_destroy(h)


@pytest.mark.parametrize("i", [0, 5])
def test_batch_channels_against_the_oracle(batch_setup, i):
    import torch
    from paper_2011_13695_gb300 import rx
    from oracle import qam as oqam
    b = batch_setup["b"]
    cfg = rx.rx_batch_config(b, i)
    ch = batch_setup["chans"][i]
    fr = batch_setup["frames"][i]
    N = batch_setup["n_sym"][i]
    rxs = dict(ch["rx"], fft_size=cfg.fft_size)
    h = rx.rx_batch_handle(b, i)
    nbytes = rx.rx_buffer_bytes(h, rx.RX_BUF_Y)
    yb = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    rx.rx_get_buffer(h, rx.RX_BUF_Y, yb.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    y = yb.cpu().numpy().view(np.complex64).reshape(2, -1)[:, :N]
    x = fr.samples.astype(np.complex64).astype(np.complex128)
    r = OracleRx(RxConfig.from_dict(rxs)).process(x, fr.ref_words)
    if r.fo_margin < 0.01:
        pytest.skip("oracle FO estimate within 1 % of a rounding boundary")
    assert rel_rms(y, r.y) < 1e-4
    bits = batch_setup["outs"][i].cpu().numpy().view(np.uint32).reshape(2, -1)
    want = oqam.pack_words(__import__("oracle.decide", fromlist=["x"]).demap_output(r.z, r.sync, cfg.bits_per_sym))
    assert np.mean(bits != want) < 1e-3
