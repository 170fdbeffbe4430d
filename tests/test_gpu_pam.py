"""GPU parity of the IM/DD PAM-M chain with FD clock recovery (rx_pam_* through the C ABI) against
the FP64 oracle (``oracle.pam.pam_receive``) on the same seeded 12-bit codes.

Tolerances: the kernels compute the FFTs, the clock products and the corrected samples in FP32 and
the 105-block averages and their phases in FP64. Clock products and extracted samples: 1e-5
relative RMS; averaged phases: 1e-5 rad; winding numbers, output offsets and counts: equal; mean and
mean absolute deviation: within 1e-5 of the outputs' RMS (the outputs' own tolerance); levels: equal except where the oracle's normalised sample lies
within 1e-4 of a decision threshold (every such symbol is checked, and they are at most 1e-5 of the
symbols).
"""

import numpy as np
import pytest

from oracle import pam
from synth.pam import PAMLink, generate_pam
from tests.gpu_util import rel_rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2011_13695_gb300 import build
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    build.build()


def run_gpu(fr, M, N, rolloff=0.5):
    import torch
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.receiver import PAMReceiver
    S = fr.codes.size
    pr = PAMReceiver(N, M, rolloff, fr.scale, fr.dc, S)
    codes = torch.from_numpy(fr.codes.view(np.int16)).cuda()
    y, lev, n_out = pr.process(codes)
    torch.cuda.synchronize()
    n = int(n_out.item())
    J = (S + N // 2 - 1) // (N // 2)
    out = dict(y=y[:n].cpu().numpy().astype(np.float64), levels=lev[:n].cpu().numpy().astype(np.int64),
               c=pr.internal(rx.RX_PAM_CLOCK, J, torch.complex64).cpu().numpy().astype(np.complex128),
               phi=pr.internal(rx.RX_PAM_PHASE, J, torch.float32).cpu().numpy().astype(np.float64),
               w=pr.internal(rx.RX_PAM_WINDING, J, torch.int32).cpu().numpy().astype(np.int64),
               off=pr.internal(rx.RX_PAM_OFFSETS, J + 1, torch.int64).cpu().numpy(),
               stat=pr.internal(rx.RX_PAM_STATS, 2, torch.float64).cpu().numpy())
    pr.close()
    return out


def run_oracle(fr, M, N, rolloff=0.5):
    # the kernels take scale and dc in FP32: the oracle gets the same rounded values
    return pam.pam_receive(fr.codes, float(np.float32(fr.scale)), float(np.float32(fr.dc)), M, rolloff, N)


def check(g, o, M):
    assert rel_rms(g["c"], o["c"]) <= 1e-5, rel_rms(g["c"], o["c"])
    dphi = np.angle(np.exp(1j * (g["phi"] - o["phi"])))
    assert np.max(np.abs(dphi)) <= 1e-5, np.max(np.abs(dphi))
    assert np.array_equal(g["w"], o["w"])
    n = o["y"].size
    assert g["y"].size == n and g["off"][-1] == n
    e = rel_rms(g["y"], o["y"])
    assert e <= 1e-5, e
    mu = np.mean(o["y"])
    mad = np.mean(np.abs(o["y"] - mu))
    rms = np.sqrt(np.mean(o["y"] ** 2))
    # the outputs carry the bias (the DC bin is the largest): their errors scale with their RMS
    assert abs(g["stat"][0] - mu) <= 1e-5 * rms and abs(g["stat"][1] - mad) <= 1e-5 * rms
    diff = np.nonzero(g["levels"] != o["levels"])[0]
    if diff.size:
        t = (o["u"][diff] + (M - 1)) / 2.0
        assert np.all(np.abs(t - np.floor(t) - 0.5) < 5e-5), diff[:10]
    assert diff.size <= max(1, 1e-5 * n)
    return e


# (M, n_samp, ppm, timing, snr, N): several blocks with ragged ends, one-block frames, slips both ways,
# the three FFT sizes
CASES = [
    (4, 1 << 17, 0.0, 0.15, None, 1024),
    (4, (1 << 17) + 300, 25.0, 0.1, 20.0, 1024),
    (2, 100, 0.0, 0.0, 12.0, 1024),
    (8, 3000, -20.0, -0.3, 26.0, 2048),
    (4, 1 << 18, -5.0, 0.4, 18.0, 4096),
]


@pytest.mark.parametrize("M,n_samp,ppm,tau,snr,N", CASES)
def test_matches_oracle(M, n_samp, ppm, tau, snr, N):
    fr = generate_pam(PAMLink(levels=M, n_samp=n_samp, clock_ppm=ppm, timing=tau, snr_db=snr), seed=n_samp % 97)
    g = run_gpu(fr, M, N)
    o = run_oracle(fr, M, N)
    print("y rel rms %.2e" % check(g, o, M))


def test_full_buffer_with_slips():
    """The paper's buffer of 2^22 samples (8192 blocks of 512 valid samples, N = 1024), PAM-4 with a
    25 ppm receiver clock offset (about 52 slips); then the GPU's decisions, away from the buffer
    edges where the 105-block average is one-sided, equal the transmitted symbols."""
    M = 4
    fr = generate_pam(PAMLink(levels=M, n_samp=1 << 22, clock_ppm=25.0, timing=0.2), seed=8)
    g = run_gpu(fr, M, 1024)
    o = run_oracle(fr, M, 1024)
    check(g, o, M)
    assert abs(g["w"][-1]) >= 50
    tx = (fr.symbols[fr.first:fr.first + g["levels"].size] + M - 1) // 2
    E = 60 * 256
    assert np.array_equal(g["levels"][E:-E], tx[E:-E])
