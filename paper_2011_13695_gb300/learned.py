"""Learned post-equaliser: a handle over the rx_pe_* C ABI and the training
loop that drives it.

The network (four 1-D convolutions 4->64->64->64->4, kernel 9, ReLU between,
residual output z + f(z)) maps the carrier-recovered symbols z of both
polarisations to corrected symbols. Its forward pass, MSE loss, backward pass
and Adam update, and the training labels, all run in librx's kernels (BF16
weights and activations, FP32 accumulation and master weights); this module
only slices sequences, picks learning rates and counts steps. The paper has no
learned equaliser.
"""

from __future__ import annotations

import numpy as np
import torch

from . import rx


def he_init(channels: int = 64, kernel: int = 9, seed: int = 0, out_scale: float = 0.1) -> np.ndarray:
    """Initial parameters in the flat layout of rx_pe (per layer: W [out][in][k], then b [out]):
    He-normal weights (std sqrt(2 / (in * k))), zero biases, the last layer scaled by ``out_scale``
    so that the network starts close to the identity z -> z."""
    rng = np.random.default_rng(seed)
    dims = [(4, channels), (channels, channels), (channels, channels), (channels, 4)]
    parts = []
    for li, (cin, cout) in enumerate(dims):
        W = rng.normal(0.0, np.sqrt(2.0 / (cin * kernel)), size=(cout, cin, kernel))
        if li == len(dims) - 1:
            W *= out_scale
        parts += [W.ravel(), np.zeros(cout)]
    return np.concatenate(parts).astype(np.float32)


class PostEqualiser:
    """One rx_pe handle on the current CUDA device."""

    def __init__(self, max_len: int, params: np.ndarray | None = None, channels: int = 64, kernel: int = 9):
        self.n_params = rx.rx_pe_param_count(channels, kernel)
        if self.n_params < 0:
            raise ValueError(f"unsupported post-equaliser shape channels={channels} kernel={kernel}")
        if params is not None:
            params = np.ascontiguousarray(params, dtype=np.float32)
            if params.size != self.n_params:
                raise ValueError(f"expected {self.n_params} parameters, got {params.size}")
        self.max_len = max_len
        self.h = rx.rx_pe_create(max_len, params, channels, kernel)

    def close(self) -> None:
        if self.h:
            rx.rx_pe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        rx.rx_pe_params(self.h, out)
        return out

    @staticmethod
    def _seq(z: torch.Tensor) -> tuple[int, int]:
        if z.dtype != torch.complex64 or z.dim() != 2 or z.shape[0] != 2 or not z.is_contiguous() or not z.is_cuda:
            raise ValueError("sequences are contiguous complex64 CUDA tensors of shape [2, T]")
        return z.data_ptr(), z.shape[1]

    def forward(self, z: torch.Tensor, out: torch.Tensor | None = None,
                stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        pz, T = self._seq(z)
        out = torch.empty_like(z) if out is None else out
        s = stream or torch.cuda.current_stream()
        rx.rx_pe_forward(self.h, pz, T, self._seq(out)[0], s.cuda_stream)
        return out

    def error_word(self) -> int:
        """RX_ERR_* bits raised by the post-equaliser's kernels (synchronises)."""
        return rx.rx_pe_error_word(self.h)

    def gradients(self, z: torch.Tensor, target: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
        pz, T = self._seq(z)
        grads = torch.empty(self.n_params, dtype=torch.float32, device=z.device)
        loss = torch.empty(1, dtype=torch.float32, device=z.device)
        rx.rx_pe_gradients(self.h, pz, self._seq(target)[0], T, grads.data_ptr(), loss.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
        return grads, loss

    def train_step(self, z: torch.Tensor, target: torch.Tensor, lr: float, loss_ptr: int | None = None,
                   stream: torch.cuda.Stream | None = None) -> None:
        pz, T = self._seq(z)
        s = stream or torch.cuda.current_stream()
        rx.rx_pe_train_step(self.h, pz, self._seq(target)[0], T, lr, loss_ptr, s.cuda_stream)

    def train(self, z, target, lo: int, hi: int, steps: int, window: int,
              lr: float = 1e-3, seed: int = 0, lr_final: float | None = None) -> torch.Tensor:
        """``steps`` Adam steps, each on a contiguous slice [o, o + window) of one (z, target) pair with
        o drawn uniformly from [lo, hi - window]; ``z`` and ``target`` are tensors or equally long lists of
        tensors (one pair drawn uniformly per step). The learning rate decays geometrically to
        ``lr_final`` when given. Returns the per-step losses (device tensor)."""
        zs_all = z if isinstance(z, (list, tuple)) else [z]
        ts_all = target if isinstance(target, (list, tuple)) else [target]
        if len(zs_all) != len(ts_all) or not zs_all:
            raise ValueError("z and target lists differ in length")
        if hi - lo < window or window > self.max_len or any(hi > a.shape[1] for a in zs_all):
            raise ValueError("training range shorter than one window, window above max_len, or range past the end")
        rng = np.random.default_rng(seed)
        which = rng.integers(0, len(zs_all), size=steps)
        offs = rng.integers(lo, hi - window + 1, size=steps)
        losses = torch.zeros(steps, dtype=torch.float32, device=zs_all[0].device)
        ratio = 1.0 if lr_final is None else (lr_final / lr) ** (1.0 / max(steps - 1, 1))
        lrs = [lr * ratio ** i for i in range(steps)]
        # one library call for the whole schedule: the windows are read in place (each pair contiguous
        # [2][n], polarisation 1 n samples on)
        zc = [a.contiguous() for a in zs_all]
        tc = [a.contiguous() for a in ts_all]
        for a in zc + tc:
            if a.dtype != torch.complex64 or a.dim() != 2 or a.shape[0] != 2:
                raise ValueError("z and target must be complex64 [2, n] tensors")
        if any(a.shape[1] != b.shape[1] for a, b in zip(zc, tc)):
            raise ValueError("each target must be as long as its z")
        rx.rx_pe_train_steps(self.h, [a.data_ptr() for a in zc], [a.data_ptr() for a in tc],
                             [a.shape[1] for a in zc], window, which, offs, lrs, losses.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
        return losses


def chain_pairs(rcv, x: torch.Tensor, n_sym: int, ref: torch.Tensor, symbols: torch.Tensor, block: int = 1024):
    """Run the plain chain on one single frame and return (z, target, stats): the carrier-recovered
    symbols, their training labels (rx_pe_targets: the transmitted symbols put in z's frame by the
    alignment the decision stage found, each block of ``block`` symbols turned by the quarter turn
    that best matches z) and the chain's statistics for this frame alone. ``rcv`` is a
    :class:`receiver.Receiver`; ``ref`` the packed transmitted bits on the device; ``symbols`` the
    transmitted symbols (contiguous complex64 [2, n_ref]) on the device."""
    before = rcv.stats()
    rcv.process(x, n_sym, ref, None)
    st = rcv.stats()
    z = rcv.symbols(n_sym)
    target = torch.empty_like(z)
    rx.rx_pe_targets(z.data_ptr(), n_sym, symbols.data_ptr(), symbols.shape[1], st["pol_map"], st["rotation"],
                     st["delay"], block, target.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return z, target, stats_delta(before, st)


def stats_delta(before: dict, after: dict) -> dict:
    """Counters accumulated between two rx_stats snapshots, with BER and EVM recomputed."""
    d = {k: after[k] - before[k] for k in ("bits_counted", "bit_errors", "symbols_counted", "symbol_errors",
                                           "evm_num", "evm_den")}
    d["ber"] = d["bit_errors"] / d["bits_counted"] if d["bits_counted"] else float("nan")
    d["evm"] = float(np.sqrt(d["evm_num"] / d["evm_den"])) if d["evm_den"] else float("nan")
    for k in ("pol_map", "rotation", "delay", "sync_matches", "sync_len"):
        d[k] = after[k]
    return d


def decide_stats(rcv, z: torch.Tensor, n_sym: int, ref: torch.Tensor) -> dict:
    """Stage A6 on symbols z (e.g. the post-equaliser's output) through ``rcv``; its counts alone."""
    before = rcv.stats()
    rcv.decide(z, n_sym, ref, None)
    return stats_delta(before, rcv.stats())
