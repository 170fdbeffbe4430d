"""The synthetic workloads: link parameters plus receiver settings.

Each entry pairs a :class:`LinkParams` (what the channel does) with the
receiver settings that process it (plain numbers mirroring the fields of the
C ``rx_config`` struct). The paper measured on lab and field captures that do
not exist here; these seeded frames stand in for them.
"""

from __future__ import annotations

import numpy as np

from .channel import LinkParams

# Receiver defaults shared by all workloads (block-LMS schedule, sync, edges).
# CMA steps of 1e-3 drift to delayed or singular solutions on 64QAM; those
# workloads use 3e-4.
RX_DEFAULTS = dict(
    sps=2,
    cma_blocks=64,
    dd_acq_blocks=128,
    seg_blocks=16,
    warmup_blocks=4,
    edge_skip=512,
    sync_len=4096,
    max_delay=16,
    mu_cma=1e-3,
    mu_dd=1e-3,
    fo_grid_hz=100e3,
)



def _rx(link: LinkParams, **kw) -> dict:
    d = dict(RX_DEFAULTS)
    d.update(bits_per_sym=link.bits_per_sym, symbol_rate=link.symbol_rate,
             wavelength=link.wavelength, dispersion=link.dispersion, length=link.length,
             rrc_rolloff=link.rolloff)
    d.update(kw)
    return d


def _qpsk_25g(n_sym=2**14) -> dict:
    link = LinkParams(bits_per_sym=2, symbol_rate=25e9, n_sym=n_sym, length=50e3,
                      linewidth=100e3, freq_offset=200e6, snr_db=14.0)
    return dict(name="dp-qpsk-25gbd", link=link,
                rx=_rx(link, fft_size=1024, n_taps=15, lms_block=64, bps_phases=32, bps_window=64))


def _qam16_32g(n_sym=2**20) -> dict:
    link = LinkParams(bits_per_sym=4, symbol_rate=32e9, n_sym=n_sym, length=80e3,
                      linewidth=100e3, freq_offset=500e6, snr_db=20.0)
    return dict(name="dp-16qam-32gbd", link=link,
                rx=_rx(link, fft_size=4096, n_taps=21, lms_block=128, bps_phases=64, bps_window=64))


def _qam64_48g_stream(n_frames=64, frame_sym=2**18) -> dict:
    link = LinkParams(bits_per_sym=6, symbol_rate=48e9, n_sym=n_frames * frame_sym, length=120e3,
                      linewidth=50e3, freq_offset=1e9, snr_db=24.0)
    return dict(name="dp-64qam-48gbd-stream", link=link, n_frames=n_frames, frame_sym=frame_sym,
                rx=_rx(link, fft_size=4096, n_taps=21, lms_block=128, bps_phases=64, bps_window=64,
                       mu_cma=3e-4))


def _qam16_32g_ssfm(n_sym=2**20, launch_dbm=4.0, train_frames=4) -> dict:
    """Nonlinear link for the learned post-equaliser: 10 x 80 km SSMF simulated by split-step
    Fourier (synth.ssfm), launch power 2..6 dBm; training frames and a test frame of different
    seeds. The SNR comes from the amplifiers' noise (snr_db is unused). After 800 km a 64-block CMA
    acquisition sometimes leaves one output unconverged; this link uses 128 blocks."""
    from .ssfm import FibreLink
    fibre = FibreLink(spans=10, span_km=80.0, launch_dbm=launch_dbm)
    link = LinkParams(bits_per_sym=4, symbol_rate=32e9, n_sym=n_sym, length=fibre.spans * fibre.span_km * 1e3,
                      linewidth=100e3, freq_offset=500e6, snr_db=None)
    return dict(name="dp-16qam-32gbd-ssfm", link=link, fibre=fibre, train_frames=train_frames,
                train_seeds=[1000 + i for i in range(train_frames)], test_seed=2000,
                rx=_rx(link, fft_size=4096, n_taps=21, lms_block=128, bps_phases=64, bps_window=64,
                       cma_blocks=128))


def batch_channels(seed: int = 42, n_channels: int = 16) -> list[dict]:
    """Seeded per-channel draws of the 16-channel batch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for ch in range(n_channels):
        rs = float(rng.choice([16e9, 32e9, 48e9, 64e9]))
        m = int(rng.choice([2, 4, 6]))
        n_sym = int(2 ** rng.integers(16, 21))
        length = float(rng.integers(10, 201)) * 1e3
        taps = int(2 * rng.integers(5, 16) + 1)          # odd, 11..31
        snr = float(rng.uniform(12.0, 24.0))
        link = LinkParams(bits_per_sym=m, symbol_rate=rs, n_sym=n_sym, length=length,
                          linewidth=100e3, freq_offset=float(rng.uniform(-1e9, 1e9)), snr_db=snr)
        out.append(dict(name=f"ch{ch}", link=link, seed=seed * 1000 + ch,
                        rx=_rx(link, fft_size=0, n_taps=taps, lms_block=128,
                               bps_phases=64, bps_window=64, mu_cma=3e-4 if m == 6 else 1e-3)))
    return out


WORKLOADS = {
    "dp-qpsk-25gbd": _qpsk_25g,
    "dp-16qam-32gbd": _qam16_32g,
    "dp-64qam-48gbd-stream": _qam64_48g_stream,
    "dp-16qam-32gbd-ssfm": _qam16_32g_ssfm,
}


def workload(name: str, **kw) -> dict:
    return WORKLOADS[name](**kw)
