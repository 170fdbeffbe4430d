"""GPU: batched channels in one graph launch (tuned FFT size and LMS CTA size).

Every channel of the batch must give exactly what a single handle with the
same (tuned) configuration gives on the same frame, and every channel is held
to the single-frame parity rules against the FP64 oracle with the tuned FFT
size (y and z within 1e-4 relative RMS, FO code equal, b* near-ties only,
decisions differing on at most 1e-5 of the symbols, exact bit-error counts).
Frames take each channel's drawn length up to 2^18 symbols per polarisation
(the oracle's time bound); the drawn lengths are 2^16 to 2^20.
"""

import numpy as np
import pytest

from oracle.receiver import Receiver as OracleRx
from oracle.receiver import RxConfig
from synth import generate
from synth.workloads import batch_channels
from tests.gpu_util import COUNTERS, handle_buffers

pytestmark = pytest.mark.gpu

N_MAX = 1 << 18


@pytest.fixture(scope="module")
def batch_setup():
    import torch
    from paper_2011_13695_gb300 import build, rx
    from paper_2011_13695_gb300.receiver import config_from
    build.build()
    chans = batch_channels(42)
    frames, xs, refs, outs, cfgs = [], [], [], [], []
    for ch in chans:
        link = ch["link"].with_(n_sym=min(ch["link"].n_sym, N_MAX))
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
    first = {}
    for r in range(2):                                  # capture (and run), then a replay
        rx.rx_batch_process(b, [t.data_ptr() for t in xs], n_sym, [t.data_ptr() for t in refs],
                            [t.data_ptr() for t in outs], stream)
        torch.cuda.synchronize()
        if r == 0:
            # one frame's counters and every buffer of each channel after the first pass
            for i, ch in enumerate(chans):
                first[i] = dict(stats=rx.rx_batch_stats(b, i), bits=outs[i].cpu().numpy().view(np.uint32).copy(),
                                **handle_buffers(rx.rx_batch_handle(b, i), n_sym[i], ch["rx"]["n_taps"]))
    yield dict(b=b, chans=chans, frames=frames, xs=xs, refs=refs, outs=outs, n_sym=n_sym, first=first)
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


@pytest.mark.parametrize("i", range(16))
def test_batch_channel_against_the_oracle(batch_setup, i, record_property):
    from paper_2011_13695_gb300 import rx
    from tests.test_gpu_parity import check_frame
    b = batch_setup["b"]
    cfg = rx.rx_batch_config(b, i)
    ch = batch_setup["chans"][i]
    fr = batch_setup["frames"][i]
    N = batch_setup["n_sym"][i]
    rxs = dict(ch["rx"], fft_size=cfg.fft_size)
    f = batch_setup["first"][i]
    st = f["stats"]
    g = dict(f, n=N, oracle_input=fr.samples.astype(np.complex64).astype(np.complex128),
             delta={k: st[k] for k in COUNTERS}, bits=f["bits"].reshape(2, -1))
    ocfg = RxConfig.from_dict(rxs)
    r = OracleRx(ocfg).process(g["oracle_input"], fr.ref_words)
    dev = check_frame(g, r, ocfg, fr.ref_words)
    for k, v in dev.items():
        record_property(k, v)
    print(f"\nchannel {i} ({ch['link'].symbol_rate / 1e9:.0f} GBd, m {ch['link'].bits_per_sym}, N {N}, "
          f"T {ch['rx']['n_taps']}, FFT {cfg.fft_size}): y {dev['y_rel_rms']:.2e}, z {dev['z_rel_rms']:.2e}, "
          f"decisions differ {dev['decisions_differ']}")
