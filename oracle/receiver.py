"""The whole chain A0-A6 in FP64, single frame or stream of frames.

TEST INFRASTRUCTURE (see the package docstring).

Stage order (the reading taken here): the
frequency offset is *estimated* on the CMA acquisition output, because the
4th-power statistic needs dispersion removed and polarisations separated; it
is *corrected* on the compensated samples the DD-LMS reads (and in the
acquired taps). So: A0 -> A1 -> A2 CMA (first frame) -> A3 estimate (first
frame) -> A3 derotation -> A2 DD acquisition (first frame) -> A4 -> A5 -> A6.

Stream mode (frames of one continuous signal, state carried between them as
the paper's overlap kernel and events carry it between buffers, Sec. II-C/D):
the dispersion stage carries N_fft/2 input samples and delays its output by
N_fft/4 samples; the equaliser keeps H = c + 2 ceil(c/2) samples of the
previous frame's compensated output and delays its symbols by ceil(c/2), so
that every tap it needs has already arrived; the equaliser taps, the FO code,
the unwrap state (m, last b*) and the alignment found on the first frame carry
over. The receiver's symbol latency is lat = N_fft/8 + ceil(c/2); the counted
window of each frame is [E', N - E'), E' = max(E, lat + max_delay). The FO
derotation of a compensated sample is indexed by the input sample it belongs
to (stream position of the frame start - N_fft/4 + its index).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import bps as _bps
from . import cdc as _cdc
from . import decide as _dec
from . import mimo as _mimo
from . import qam


@dataclass
class RxConfig:
    bits_per_sym: int
    symbol_rate: float
    wavelength: float = 1550e-9
    dispersion: float = 17e-6
    length: float = 0.0
    sps: int = 2
    fft_size: int = 1024
    n_taps: int = 15
    lms_block: int = 64
    cma_blocks: int = 64
    dd_acq_blocks: int = 128
    seg_blocks: int = 16
    warmup_blocks: int = 4
    bps_phases: int = 32
    bps_window: int = 64
    edge_skip: int = 512
    sync_len: int = 4096
    max_delay: int = 16
    mu_cma: float = 1e-3
    mu_dd: float = 1e-3
    fo_grid_hz: float = 100e3
    rrc_rolloff: float = 0.1

    @classmethod
    def from_dict(cls, d: dict) -> "RxConfig":
        names = cls.__dataclass_fields__.keys()
        return cls(**{k: v for k, v in d.items() if k in names})

    @property
    def fs(self) -> float:
        return self.sps * self.symbol_rate

    @property
    def c(self) -> int:
        return (self.n_taps - 1) // 2

    @property
    def d4(self) -> int:
        return (self.c + 1) // 2

    @property
    def hist(self) -> int:
        return self.c + 2 * self.d4

    @property
    def stream_latency(self) -> int:
        return self.fft_size // 8 + self.d4


@dataclass
class FrameResult:
    scale: np.ndarray = None
    dd_margin: np.ndarray = None    # smallest A4 decision margin per segment and row [nseg, 2]
    cdc: np.ndarray = None          # A1 output [2, S]
    taps_cma: np.ndarray = None
    y_acq: np.ndarray = None        # CMA outputs while adapting [2, N_acq]
    y_foe: np.ndarray = None        # fixed-tap outputs the FO estimate uses
    taps_foe: np.ndarray = None     # CMA taps after the FO correction
    rho: float = 0.0
    reran: bool = False
    fo_code: int = 0
    fo_w: float = 0.0
    fo_margin: float = 0.5
    taps_init: np.ndarray = None
    y: np.ndarray = None            # A4 output P1 [2, N]
    taps_final: np.ndarray = None
    bstar: np.ndarray = None        # [2, N]
    m: np.ndarray = None            # [2, N]
    z: np.ndarray = None            # A5 output P2 [2, N]
    sync: list = None
    sync_len: int = 0
    bits_out: np.ndarray = None     # uint8 [2, N*m]
    counts: dict = field(default_factory=dict)


def _count_window(cfg: RxConfig, n_sym: int, lat: int):
    E = max(cfg.edge_skip, lat + cfg.max_delay) if lat else cfg.edge_skip
    lo, hi = E, n_sym - E
    return lo, max(hi, lo)


class Receiver:
    """Stateful FP64 receiver; ``stream=False`` treats each call as its own frame."""

    def __init__(self, cfg: RxConfig, stream: bool = False):
        if cfg.sps != 2:
            raise ValueError("sps must be 2")
        self.cfg = cfg
        self.stream = stream
        self.H = _cdc.cdc_response(cfg.fft_size, cfg.fs, cfg.dispersion, cfg.length, cfg.wavelength,
                                   cfg.symbol_rate, cfg.rrc_rolloff, cfg.sps)
        self.m = cfg.bits_per_sym
        self.R2 = qam.cma_radius(self.m)
        self.reset()

    def reset(self):
        cfg = self.cfg
        self.frame = 0
        self.scale = None
        self.tail = np.zeros((2, cfg.fft_size // 2), dtype=np.complex128)
        self.hist = np.zeros((2, cfg.hist), dtype=np.complex128)
        self.taps = None
        self.fo_code = 0
        self.b_prev = [None, None]
        self.m_prev = [0, 0]
        self.sync = None

    def process(self, x: np.ndarray, ref_words=None) -> FrameResult:
        if not self.stream:
            self.reset()
        cfg, m = self.cfg, self.m
        S = x.shape[1]
        if S % 2:
            raise ValueError("frames hold whole symbols (even sample count)")
        N = S // 2
        r = FrameResult()
        first = self.frame == 0
        L_b = cfg.lms_block
        n_cma = min(cfg.cma_blocks, N // L_b)

        # A0
        if first:
            self.scale = _cdc.power_scale(x, 2 * n_cma * L_b)
        r.scale = self.scale
        xs = x * self.scale[:, None]
        off = cfg.hist - 2 * cfg.d4 if self.stream else 0
        lat = cfg.stream_latency if self.stream else 0

        # A1
        if self.stream:
            r.cdc, self.tail = _cdc.overlap_save_stream(xs, self.H, self.tail)
            buf = np.concatenate([self.hist, r.cdc], axis=1)
            g0 = self.frame * S - cfg.fft_size // 4 - cfg.hist
        else:
            r.cdc = _cdc.overlap_save(xs, self.H)
            buf, g0 = r.cdc, 0

        # A2 CMA and A3 FO estimate (first frame only)
        if first:
            h, r.y_acq, r.rho, r.reran = _mimo.cma_acquire(buf, cfg.n_taps, L_b, n_cma, cfg.mu_cma, self.R2, off)
            r.taps_cma = h
            if n_cma > 0:
                r.y_foe = _mimo.foe_window(buf, h, n_cma * L_b, cfg.n_taps, off)
                r.fo_code, r.fo_w, r.fo_margin = _mimo.foe_code(r.y_foe, cfg.symbol_rate, cfg.fo_grid_hz, L_b)
            self.fo_code = r.fo_code
            self.taps = _mimo.fo_correct_taps(h, self.fo_code, cfg.fo_grid_hz, cfg.fs)
            r.taps_foe = self.taps.copy()
        r.fo_code = self.fo_code

        # A3 derotation of the compensated samples (fused into the equaliser's load on the GPU)
        xd = _mimo.derotate(buf, self.fo_code, cfg.fo_grid_hz, cfg.fs, g0)

        # A2 DD acquisition (first frame only)
        if first:
            n_dd = min(cfg.dd_acq_blocks, N // L_b) if n_cma > 0 else 0
            if n_dd > 0:
                _, self.taps = _mimo.dd_lms(xd, self.taps, n_dd * L_b, L_b, n_dd, 0, m, cfg.mu_dd, off)
        r.taps_init = self.taps.copy()

        # A4
        diag = {}
        r.y, r.taps_final = _mimo.dd_lms(xd, self.taps, N, L_b, cfg.seg_blocks, cfg.warmup_blocks,
                                         m, cfg.mu_dd, off, diag)
        r.dd_margin = diag.get("margin")
        self.taps = r.taps_final

        # A5
        r.bstar = np.zeros((2, N), np.int64)
        r.m = np.zeros((2, N), np.int64)
        r.z = np.zeros((2, N), np.complex128)
        for q in range(2):
            bq, mq, zq = _bps.blind_phase_search(r.y[q], m, cfg.bps_phases, cfg.bps_window,
                                                 self.b_prev[q], self.m_prev[q])
            r.bstar[q], r.m[q], r.z[q] = bq, mq, zq
            if N:
                self.b_prev[q], self.m_prev[q] = int(bq[-1]), int(mq[-1])

        # A6
        lo, hi = _count_window(cfg, N, lat)
        if ref_words is not None:
            if self.sync is None and hi > lo:
                self.sync, r.sync_len = _dec.resolve(r.z, ref_words, m, N, lo, min(lo + cfg.sync_len, hi),
                                                     cfg.max_delay, lat)
            r.sync = self.sync
            if self.sync is not None:
                r.counts = _dec.count(r.z, self.sync, ref_words, m, N, lo, hi, lat)
        r.bits_out = _dec.demap_output(r.z, r.sync, m)

        if self.stream:
            self.hist = r.cdc[:, S - cfg.hist:].copy() if S >= cfg.hist else \
                np.concatenate([self.hist, r.cdc], axis=1)[:, -cfg.hist:]
        self.frame += 1
        return r


def receive(x: np.ndarray, cfg: RxConfig, ref_words=None) -> FrameResult:
    """Single-frame convenience wrapper."""
    return Receiver(cfg, stream=False).process(x, ref_words)
