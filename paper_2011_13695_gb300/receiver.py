"""Handle wrapper over the librx C ABI for torch device buffers (marshalling only)."""

from __future__ import annotations

import torch

from . import rx

# workload keys -> rx_config fields
_RENAME = {"symbol_rate": "symbol_rate_hz", "wavelength": "wavelength_m", "dispersion": "dispersion_s_per_m2",
           "length": "length_m"}

_BUF_LAYOUT = {
    rx.RX_BUF_Y: torch.complex64, rx.RX_BUF_Z: torch.complex64, rx.RX_BUF_CDC: torch.complex64,
    rx.RX_BUF_TAPS_CMA: torch.complex64, rx.RX_BUF_TAPS_INIT: torch.complex64, rx.RX_BUF_TAPS_LAST: torch.complex64,
    rx.RX_BUF_Y_ACQ: torch.complex64, rx.RX_BUF_Y_FOE: torch.complex64, rx.RX_BUF_BSTAR: torch.uint8,
    rx.RX_BUF_M: torch.int32, rx.RX_BUF_SCALE: torch.float32,
}


def config_from(rx_settings: dict, max_symbols: int, input_format: int = rx.RX_IN_C64, input_scale: float = 1.0,
                streaming: bool = False) -> rx.rx_config:
    kw = {_RENAME.get(k, k): v for k, v in rx_settings.items()}
    kw.update(input_format=input_format, input_scale=input_scale, streaming=1 if streaming else 0,
              max_symbols=max_symbols)
    kw.setdefault("sps", 2)
    return rx.make_config(**kw)


class Receiver:
    """One librx handle on the current CUDA device."""

    def __init__(self, rx_settings: dict, max_symbols: int, input_format: int = rx.RX_IN_C64,
                 input_scale: float = 1.0, streaming: bool = False):
        self.cfg = config_from(rx_settings, max_symbols, input_format, input_scale, streaming)
        self.m = self.cfg.bits_per_sym
        self.h = rx.rx_create(self.cfg)

    def close(self):
        if self.h:
            rx.rx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def words(self, n_sym: int) -> int:
        return (n_sym * self.m + 31) // 32

    def process(self, x: torch.Tensor, n_sym: int, ref: torch.Tensor | None = None,
                out: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None) -> None:
        s = stream or torch.cuda.current_stream()
        rx.rx_process(self.h, x.data_ptr(), n_sym, ref.data_ptr() if ref is not None else None,
                      out.data_ptr() if out is not None else None, s.cuda_stream)

    def process_host(self, x_host, n_sym: int, ref_host=None, out_host=None, stream=None) -> None:
        s = stream or torch.cuda.current_stream()
        rx.rx_process_host(self.h, x_host.data_ptr(), n_sym, ref_host.data_ptr() if ref_host is not None else None,
                           out_host.data_ptr() if out_host is not None else None, s.cuda_stream)

    def stats(self) -> dict:
        return rx.rx_stats(self.h)

    def reset(self) -> None:
        rx.rx_reset(self.h)

    def buffer(self, which: int) -> torch.Tensor:
        nbytes = rx.rx_buffer_bytes(self.h, which)
        dt = _BUF_LAYOUT[which]
        esz = torch.tensor([], dtype=dt).element_size()
        t = torch.empty(nbytes // esz, dtype=dt, device="cuda")
        rx.rx_get_buffer(self.h, which, t.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
        torch.cuda.current_stream().synchronize()
        return t

    def decide(self, z: torch.Tensor, n_sym: int, ref: torch.Tensor | None = None,
               out: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None) -> None:
        """Stage A6 alone on caller-supplied symbols z (complex64 [2, n_sym], contiguous)."""
        s = stream or torch.cuda.current_stream()
        rx.rx_decide(self.h, z.data_ptr(), n_sym, ref.data_ptr() if ref is not None else None,
                     out.data_ptr() if out is not None else None, s.cuda_stream)

    def symbols(self, n_sym: int) -> torch.Tensor:
        """Carrier-recovered symbols z of the last single frame, complex64 [2, n_sym]."""
        z = self.buffer(rx.RX_BUF_Z).view(2, -1)
        return z[:, :n_sym].contiguous()


def dd_lms_wl(x: torch.Tensor, taps: torch.Tensor, n_sym: int, block_len: int, seg_blocks: int, warmup_blocks: int,
              bits_per_sym: int, mu: float, mu_conj: float, y: torch.Tensor | None = None,
              taps_out: torch.Tensor | None = None, threads: int = 0,
              stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """Widely-linear segmented DD-LMS (rx_dd_lms_wl) on device tensors: x complex64 [2, x_len] at
    2 samples/symbol, taps complex64 [2, 4, T] (h_q0, h_q1, g_q0, g_q1 per output row). Returns y
    complex64 [2, n_sym]; ``taps_out`` (complex64 [2, 4, T]) receives the last segment's final taps."""
    for t in (x, taps) + ((y,) if y is not None else ()) + ((taps_out,) if taps_out is not None else ()):
        if t.dtype != torch.complex64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("dd_lms_wl takes contiguous complex64 CUDA tensors")
    if x.dim() != 2 or x.shape[0] != 2 or taps.dim() != 3 or tuple(taps.shape[:2]) != (2, 4):
        raise ValueError("x must be [2, x_len] and taps [2, 4, T]")
    if y is None:
        y = torch.empty((2, n_sym), dtype=torch.complex64, device=x.device)
    elif tuple(y.shape) != (2, n_sym):
        raise ValueError("y must be [2, n_sym]")
    if taps_out is not None and taps_out.shape != taps.shape:
        raise ValueError("taps_out must have the shape of taps")
    s = stream or torch.cuda.current_stream()
    rx.rx_dd_lms_wl(x.data_ptr(), x.shape[1], taps.shape[2], taps.data_ptr(), n_sym, block_len, seg_blocks,
                    warmup_blocks, bits_per_sym, mu, mu_conj, y.data_ptr(),
                    taps_out.data_ptr() if taps_out is not None else None, threads, s.cuda_stream)
    return y


class KKFrontEnd:
    """Kramers-Kronig self-coherent front end (rx_kk_*) on torch device tensors: 12-bit codes in 16-bit
    words (any 2-byte dtype; the bits are read as uint16) at 4 samples/symbol in, the downshifted field
    at 4 samples/symbol and the matched-filtered signal at 2 samples/symbol out (complex64)."""

    def __init__(self, fft_size: int, tone_over_fs: float, rrc_rolloff: float, code_scale: float, dc_offset: float,
                 min_intensity: float = 1e-6):
        self.k = rx.rx_kk_create(fft_size, tone_over_fs, rrc_rolloff, code_scale, dc_offset, min_intensity)

    def close(self):
        if self.k:
            rx.rx_kk_destroy(self.k)
            self.k = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def process(self, codes: torch.Tensor, field: torch.Tensor | None = None, out: torch.Tensor | None = None,
                stream: torch.cuda.Stream | None = None, first_sample: int = 0):
        if not codes.is_cuda or not codes.is_contiguous() or codes.element_size() != 2 or codes.dim() != 1:
            raise ValueError("codes must be a contiguous 1-D CUDA tensor of 16-bit words")
        S = codes.shape[0]
        if field is None:
            field = torch.empty(S, dtype=torch.complex64, device=codes.device)
        if out is None:
            out = torch.empty(S // 2, dtype=torch.complex64, device=codes.device)
        for t, n in ((field, S), (out, S // 2)):
            if t.dtype != torch.complex64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError("field and out must be contiguous complex64 CUDA tensors of S and S/2 samples")
        s = stream or torch.cuda.current_stream()
        rx.rx_kk_process(self.k, codes.data_ptr(), S, first_sample, field.data_ptr(), out.data_ptr(), s.cuda_stream)
        return field, out

    def ingest(self, source, buffer_samples: int, sample_rate_hz: float, n_streams: int, n_buffers: int,
               keep_outputs: bool = False):
        """Real-time ingest emulation over host codes ``source`` (numpy uint16); returns (stats, outputs
        complex64 [n_buffers * buffer_samples / 2] or None)."""
        import numpy as np
        src = np.ascontiguousarray(source, dtype=np.uint16)
        out = np.zeros(n_buffers * buffer_samples // 2, dtype=np.complex64) if keep_outputs else None
        stats = rx.rx_ingest_run(self.k, src, buffer_samples, sample_rate_hz, n_streams, n_buffers, out)
        return stats, out


    def equalise(self, y: torch.Tensor, n_sym: int, taps: torch.Tensor, block_len: int, seg_blocks: int,
                 warmup_blocks: int, bits_per_sym: int, mu: float, mu_conj: float,
                 out: torch.Tensor | None = None, bits: torch.Tensor | None = None,
                 taps_out: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None):
        """Step 9 (rx_kk_equalise): widely-linear DD-LMS of the front end's output y (complex64, 2
        samples/symbol), decisions and Gray demapping. taps: complex64 [2, T] (h, then g). Returns
        (equalised symbols complex64 [n_sym], decided bits int32 [ceil(n_sym m / 32)])."""
        if y.dtype != torch.complex64 or not y.is_cuda or not y.is_contiguous() or y.dim() != 1:
            raise ValueError("y must be a contiguous 1-D complex64 CUDA tensor")
        if taps.dtype != torch.complex64 or not taps.is_cuda or not taps.is_contiguous() or taps.dim() != 2 \
                or taps.shape[0] != 2:
            raise ValueError("taps must be a contiguous complex64 CUDA tensor [2, T]")
        out = torch.empty(n_sym, dtype=torch.complex64, device=y.device) if out is None else out
        words = (n_sym * bits_per_sym + 31) // 32
        bits = torch.empty(words, dtype=torch.int32, device=y.device) if bits is None else bits
        s = stream or torch.cuda.current_stream()
        rx.rx_kk_equalise(self.k, y.data_ptr(), y.shape[0], taps.shape[1], taps.data_ptr(), n_sym, block_len,
                          seg_blocks, warmup_blocks, bits_per_sym, mu, mu_conj, out.data_ptr(), bits.data_ptr(),
                          taps_out.data_ptr() if taps_out is not None else None, s.cuda_stream)
        return out, bits

class PAMReceiver:
    """IM/DD PAM-M chain with FD clock recovery (rx_pam_*) on torch device tensors: 12-bit codes in
    16-bit words (any 2-byte dtype) at 2 samples/symbol in; extracted samples (float32), level
    indices (uint8) and their count out."""

    def __init__(self, fft_size: int, levels: int, rrc_rolloff: float, code_scale: float, dc_offset: float,
                 max_samples: int):
        self.max_samples = max_samples
        self.fft_size = fft_size
        self.p = rx.rx_pam_create(fft_size, levels, rrc_rolloff, code_scale, dc_offset, max_samples)
        self.n_out = torch.zeros(1, dtype=torch.int64, device="cuda")

    def close(self):
        if self.p:
            rx.rx_pam_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def capacity(self, n_samples: int) -> int:
        return n_samples // 2 + n_samples // (self.fft_size // 2) + 1

    def process(self, codes: torch.Tensor, y: torch.Tensor | None = None, levels: torch.Tensor | None = None,
                stream: torch.cuda.Stream | None = None):
        """Returns (y, levels, n_out device tensor); the first n_out entries are valid."""
        if not codes.is_cuda or not codes.is_contiguous() or codes.element_size() != 2 or codes.dim() != 1:
            raise ValueError("codes must be a contiguous 1-D CUDA tensor of 16-bit words")
        S = codes.shape[0]
        cap = self.capacity(S)
        if y is None:
            y = torch.empty(cap, dtype=torch.float32, device=codes.device)
        if levels is None:
            levels = torch.empty(cap, dtype=torch.uint8, device=codes.device)
        if y.numel() < cap or levels.numel() < cap or y.dtype != torch.float32 or levels.dtype != torch.uint8:
            raise ValueError("y (float32) and levels (uint8) need room for capacity(n_samples) outputs")
        s = stream or torch.cuda.current_stream()
        rx.rx_pam_process(self.p, codes.data_ptr(), S, y.data_ptr(), levels.data_ptr(), self.n_out.data_ptr(),
                          s.cuda_stream)
        return y, levels, self.n_out

    def internal(self, which: int, count: int, dtype) -> torch.Tensor:
        t = torch.empty(count, dtype=dtype, device="cuda")
        rx.rx_pam_get(self.p, which, t.data_ptr(), t.numel() * t.element_size(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.current_stream().synchronize()
        return t
