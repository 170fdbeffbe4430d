"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and the
FP64 oracle on the same seeded frame, and compare them."""

from __future__ import annotations

import numpy as np


def rel_rms(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.sum(np.abs(b) ** 2)
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2) / den)) if den > 0 else float(np.sqrt(np.sum(np.abs(a) ** 2)))


def device_input(samples: np.ndarray, fmt: int = 0):
    """Host samples -> (torch device tensor, the values the oracle should see, input_scale)."""
    import torch
    from synth.channel import quantise_int8, to_fp16
    if fmt == 0:
        c = np.ascontiguousarray(samples.astype(np.complex64))
        return torch.from_numpy(c.view(np.float32)).cuda(), c.astype(np.complex128), 1.0
    if fmt == 1:
        h = to_fp16(samples)
        vals = h[..., 0].astype(np.float64) + 1j * h[..., 1].astype(np.float64)
        return torch.from_numpy(np.ascontiguousarray(h).view(np.int16)).cuda(), vals, 1.0
    codes, delta = quantise_int8(samples)
    # one step for both polarisations: the power normalisation removes any common scale
    step = float(delta[0])
    vals = (codes[..., 0].astype(np.float64) + 1j * codes[..., 1].astype(np.float64)) * np.float64(np.float32(step))
    return torch.from_numpy(np.ascontiguousarray(codes)).cuda(), vals, step


def stream_inputs(samples: np.ndarray, fmt: int, n_frames: int):
    """A stream's samples quantised once over the whole stream (one int8 step, as a digitiser has),
    then cut into frames: [(device tensor, oracle values, input_scale)] per frame."""
    import torch
    from synth.channel import quantise_int8, to_fp16
    S = samples.shape[1] // n_frames
    if fmt == 0:
        c = np.ascontiguousarray(samples.astype(np.complex64))
        return [(torch.from_numpy(np.ascontiguousarray(c[:, f * S:(f + 1) * S]).view(np.float32)).cuda(),
                 c[:, f * S:(f + 1) * S].astype(np.complex128), 1.0) for f in range(n_frames)]
    if fmt == 1:
        h = to_fp16(samples)
        vals = h[..., 0].astype(np.float64) + 1j * h[..., 1].astype(np.float64)
        return [(torch.from_numpy(np.ascontiguousarray(h[:, f * S:(f + 1) * S]).view(np.int16)).cuda(),
                 vals[:, f * S:(f + 1) * S], 1.0) for f in range(n_frames)]
    codes, delta = quantise_int8(samples)
    step = float(delta[0])
    vals = (codes[..., 0].astype(np.float64) + 1j * codes[..., 1].astype(np.float64)) * np.float64(np.float32(step))
    return [(torch.from_numpy(np.ascontiguousarray(codes[:, f * S:(f + 1) * S])).cuda(), vals[:, f * S:(f + 1) * S],
             step) for f in range(n_frames)]


DEFAULT_BUFFERS = ("y", "z", "bstar", "m", "cdc", "taps_cma", "taps_init", "taps_last", "y_foe", "scale")


def handle_buffers(h: int, N: int, T: int, streaming: bool = False, buffers=DEFAULT_BUFFERS) -> dict:
    """The parity export of any librx handle (a single handle or a batch channel's) after a frame of N
    symbols, as host arrays shaped the way the oracle's FrameResult holds them."""
    import torch
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.receiver import _BUF_LAYOUT
    names = {"y": rx.RX_BUF_Y, "z": rx.RX_BUF_Z, "bstar": rx.RX_BUF_BSTAR, "m": rx.RX_BUF_M, "cdc": rx.RX_BUF_CDC,
             "taps_cma": rx.RX_BUF_TAPS_CMA, "taps_init": rx.RX_BUF_TAPS_INIT, "taps_last": rx.RX_BUF_TAPS_LAST,
             "y_foe": rx.RX_BUF_Y_FOE, "scale": rx.RX_BUF_SCALE, "y_acq": rx.RX_BUF_Y_ACQ}
    hist = (T - 1) // 2 + 2 * (((T - 1) // 2 + 1) // 2)
    res = {}
    for b in buffers:
        which = names[b]
        nbytes = rx.rx_buffer_bytes(h, which)
        dt = _BUF_LAYOUT[which]
        esz = torch.tensor([], dtype=dt).element_size()
        buf = torch.empty(nbytes // esz, dtype=dt, device="cuda")
        rx.rx_get_buffer(h, which, buf.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
        torch.cuda.current_stream().synchronize()
        t = buf.cpu().numpy()
        if b in ("y", "z", "bstar", "m"):
            t = t.reshape(2, -1)[:, :N]
        elif b == "cdc":
            t = t.reshape(2, -1)
            t = t[:, hist:hist + 2 * N] if streaming else t[:, :2 * N]
        elif b.startswith("taps"):
            t = t.reshape(2, 2, T)
        elif b == "y_foe":
            t = t.reshape(2, -1)
        res[b] = t
    return res


COUNTERS = ("bits_counted", "bit_errors", "symbols_counted", "symbol_errors", "evm_num", "evm_den")


def run_gpu_frames(rx_settings: dict, frames: list, refs: list | None = None, fmt: int = 0, streaming=False,
                   buffers=DEFAULT_BUFFERS, inputs=None):
    """Process frames (host complex128 [2, S] each) through librx; returns per-frame dicts.
    ``inputs``: device inputs already made (``stream_inputs``) instead of quantising each frame alone."""
    import torch
    from paper_2011_13695_gb300.receiver import Receiver
    n_max = max(f.shape[1] // 2 for f in frames)
    if inputs is None:
        inputs = [device_input(f, fmt) for f in frames]
    scale = inputs[0][2]
    rcv = Receiver(rx_settings, n_max, input_format=fmt, input_scale=scale, streaming=streaming)
    out = []
    T = rx_settings["n_taps"]
    for i, (x, vals, _) in enumerate(inputs):
        N = frames[i].shape[1] // 2
        ref = torch.from_numpy(refs[i].astype(np.int32).view(np.int32)).cuda() if refs is not None else None
        words = rcv.words(N)
        bits = torch.zeros(2 * words, dtype=torch.int32, device="cuda")
        before = rcv.stats()
        rcv.process(x, N, ref, bits)
        st = rcv.stats()
        res = dict(stats=st, oracle_input=vals, n=N)
        res["delta"] = {k: st[k] - before[k] for k in COUNTERS}
        res["bits"] = bits.cpu().numpy().view(np.uint32).reshape(2, words)
        res.update(handle_buffers(rcv.h, N, T, streaming, buffers))
        out.append(res)
    rcv.close()
    return out


def kernel_precision_bits(z: np.ndarray, sync, m: int) -> np.ndarray:
    """Packed output bits [2, words] of complex64 symbols z decided the way the decision kernel does:
    each output's exact quarter turn, then the level rint(fma(u, 1/(2a), (L-1)/2)) in FP32 (a NaN
    input clamps to level 0), then Gray bits. Near a decision boundary the FP32 rule and an FP64 one
    can differ, so checks of the kernel's own demapping take its precision."""
    from oracle import qam as oqam
    L = 1 << (m // 2)
    M = L * L
    h = np.float64(np.float32(0.5 * np.sqrt(2.0 * (M - 1) / 3.0)))
    hl = 0.5 * (L - 1)

    def level(u):
        v = (u.astype(np.float64) * h + hl).astype(np.float32)     # exact product, one FP32 rounding
        v = np.where(np.isnan(v), 0.0, np.rint(v))
        return np.clip(v, 0, L - 1).astype(np.int64)

    rows = []
    for q in range(2):
        r = sync[q][1] if sync is not None else 0
        zr = z[q].astype(np.complex64) * np.complex64(1j ** r)
        rows.append(oqam.levels_to_bits(level(zr.real), level(zr.imag), m).reshape(-1))
    return oqam.pack_words(np.stack(rows))
