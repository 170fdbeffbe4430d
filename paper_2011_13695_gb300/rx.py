"""ctypes binding of librx (include/rx.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the receiver: all of it runs in the CUDA library. Device
buffers are passed as integer device addresses (e.g. ``tensor.data_ptr()``)
and streams as ``torch.cuda.Stream.cuda_stream``. The library is loaded from
the package directory; if it is missing, :func:`lib` raises instead of
falling back to anything else.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librx.so")

RX_OK, RX_EINVAL, RX_ENOMEM, RX_ECUDA, RX_ETIMEOUT, RX_ESTATE = 0, -1, -2, -3, -4, -5
RX_IN_C64, RX_IN_F16, RX_IN_I8 = 0, 1, 2
RX_ERR_NONFINITE, RX_ERR_SYNC_LOST, RX_ERR_SINGULAR, RX_ERR_TIMEOUT = 0x1, 0x2, 0x4, 0x8
(RX_BUF_CDC, RX_BUF_Y, RX_BUF_Z, RX_BUF_BSTAR, RX_BUF_M, RX_BUF_TAPS_CMA, RX_BUF_TAPS_INIT, RX_BUF_TAPS_LAST,
 RX_BUF_Y_ACQ, RX_BUF_Y_FOE, RX_BUF_SCALE) = range(11)

EXPORTS = ("rx_create", "rx_process", "rx_process_host", "rx_stats", "rx_buffer_bytes", "rx_get_buffer",
           "rx_reset", "rx_state_size", "rx_state_get", "rx_state_set", "rx_set_timing", "rx_stage_count",
           "rx_stage_name", "rx_stage_times", "rx_launch_count", "rx_destroy", "rx_strerror",
           "rx_batch_create", "rx_batch_config", "rx_batch_handle", "rx_batch_process", "rx_batch_stats",
           "rx_batch_launch_count", "rx_batch_destroy", "rx_carrier_recovery_static",
           "rx_decide", "rx_pe_param_count", "rx_pe_create", "rx_pe_params", "rx_pe_forward",
           "rx_pe_error_word", "rx_pe_gradients", "rx_pe_train_step", "rx_pe_train_steps", "rx_pe_destroy", "rx_dd_lms_wl",
           "rx_kk_create", "rx_kk_process", "rx_kk_destroy", "rx_ingest_run", "rx_pam_create", "rx_pam_process",
           "rx_pam_get", "rx_pam_destroy", "rx_fp32_fma_rate", "rx_pe_targets", "rx_kk_equalise")
RX_PAM_CLOCK, RX_PAM_PHASE, RX_PAM_WINDING, RX_PAM_OFFSETS, RX_PAM_STATS = range(5)
RX_STATIC_MAX_SYMBOLS = 262144


class rx_config(C.Structure):
    _fields_ = [
        ("bits_per_sym", C.c_int32), ("sps", C.c_int32),
        ("symbol_rate_hz", C.c_double), ("wavelength_m", C.c_double),
        ("dispersion_s_per_m2", C.c_double), ("length_m", C.c_double), ("rrc_rolloff", C.c_double),
        ("fft_size", C.c_int32), ("n_taps", C.c_int32), ("lms_block", C.c_int32), ("cma_blocks", C.c_int32),
        ("dd_acq_blocks", C.c_int32), ("seg_blocks", C.c_int32), ("warmup_blocks", C.c_int32),
        ("bps_phases", C.c_int32), ("bps_window", C.c_int32), ("edge_skip", C.c_int32), ("sync_len", C.c_int32),
        ("max_delay", C.c_int32), ("mu_cma", C.c_float), ("mu_dd", C.c_float), ("fo_grid_hz", C.c_double),
        ("input_format", C.c_int32), ("input_scale", C.c_float), ("streaming", C.c_int32),
        ("max_symbols", C.c_int64), ("lms_threads", C.c_int32),
    ]


class rx_ingest_stats(C.Structure):
    _fields_ = [("buffers", C.c_uint64), ("processed", C.c_uint64), ("dropped", C.c_uint64), ("pad0", C.c_uint64),
                ("buffer_period_ms", C.c_double), ("mean_latency_ms", C.c_double), ("max_latency_ms", C.c_double),
                ("wall_s", C.c_double)]


class rx_stats_t(C.Structure):
    _fields_ = [
        ("frames", C.c_uint64), ("symbols_processed", C.c_uint64), ("bits_processed", C.c_uint64),
        ("bits_counted", C.c_uint64), ("bit_errors", C.c_uint64), ("symbols_counted", C.c_uint64),
        ("symbol_errors", C.c_uint64), ("evm_num", C.c_double), ("evm_den", C.c_double), ("ber", C.c_double),
        ("evm", C.c_double), ("q_db", C.c_double), ("fo_code", C.c_int32), ("fo_hz", C.c_double),
        ("pol_map", C.c_int32 * 2), ("rotation", C.c_int32 * 2), ("delay", C.c_int32 * 2),
        ("sync_matches", C.c_int32 * 2), ("sync_len", C.c_int32), ("cma_reran", C.c_int32),
        ("cma_rho", C.c_float), ("latency_symbols", C.c_int32), ("error_word", C.c_uint32),
    ]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


_lib = None


def lib() -> C.CDLL:
    """Load librx.so (built by ``paper_2011_13695_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librx.so is not built ({LIB_PATH}); run paper_2011_13695_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
        sig = {
            "rx_create": (i32, [C.POINTER(rx_config), C.POINTER(vp)]),
            "rx_process": (i32, [vp, vp, i64, vp, vp, vp]),
            "rx_process_host": (i32, [vp, vp, i64, vp, vp, vp]),
            "rx_stats": (i32, [vp, C.POINTER(rx_stats_t)]),
            "rx_buffer_bytes": (i32, [vp, i32, C.POINTER(i64)]),
            "rx_get_buffer": (i32, [vp, i32, vp, i64, vp]),
            "rx_reset": (i32, [vp]),
            "rx_state_size": (i32, [vp, C.POINTER(C.c_size_t)]),
            "rx_state_get": (i32, [vp, vp, C.c_size_t]),
            "rx_state_set": (i32, [vp, vp, C.c_size_t]),
            "rx_set_timing": (i32, [vp, i32]),
            "rx_stage_count": (i32, []),
            "rx_stage_name": (C.c_char_p, [i32]),
            "rx_stage_times": (i32, [vp, C.POINTER(C.c_double), C.POINTER(i64), i32]),
            "rx_launch_count": (u64, [vp]),
            "rx_destroy": (None, [vp]),
            "rx_strerror": (C.c_char_p, [i32]),
            "rx_batch_create": (i32, [C.POINTER(rx_config), i32, C.POINTER(vp)]),
            "rx_batch_config": (i32, [vp, i32, C.POINTER(rx_config)]),
            "rx_batch_handle": (vp, [vp, i32]),
            "rx_batch_process": (i32, [vp, C.POINTER(vp), C.POINTER(i64), C.POINTER(vp), C.POINTER(vp), vp]),
            "rx_batch_stats": (i32, [vp, i32, C.POINTER(rx_stats_t)]),
            "rx_batch_launch_count": (u64, [vp]),
            "rx_batch_destroy": (None, [vp]),
            "rx_carrier_recovery_static": (i32, [vp, i64, i32, i32, i32, vp, vp]),
            "rx_decide": (i32, [vp, vp, i64, vp, vp, vp]),
            "rx_pe_param_count": (i64, [i32, i32]),
            "rx_pe_create": (i32, [i32, i32, i64, vp, C.POINTER(vp)]),
            "rx_pe_params": (i32, [vp, vp]),
            "rx_pe_forward": (i32, [vp, vp, i64, vp, vp]),
            "rx_pe_error_word": (i32, [vp, vp]),
            "rx_pe_gradients": (i32, [vp, vp, vp, i64, vp, vp, vp]),
            "rx_pe_train_step": (i32, [vp, vp, vp, i64, C.c_float, vp, vp]),
            "rx_pe_train_steps": (i32, [vp, vp, vp, vp, i32, i64, i32, vp, vp, vp, vp, vp]),
            "rx_pe_destroy": (None, [vp]),
            "rx_dd_lms_wl": (i32, [vp, i64, i32, vp, i64, i32, i32, i32, i32, C.c_float, C.c_float, vp, vp, i32,
                                   vp]),
            "rx_kk_create": (i32, [i32, C.c_double, C.c_double, C.c_float, C.c_float, C.c_float, C.POINTER(vp)]),
            "rx_kk_process": (i32, [vp, vp, i64, i64, vp, vp, vp]),
            "rx_kk_destroy": (None, [vp]),
            "rx_ingest_run": (i32, [vp, vp, i64, i64, C.c_double, i32, i64, vp, C.POINTER(rx_ingest_stats)]),
            "rx_pam_create": (i32, [i32, i32, C.c_double, C.c_float, C.c_float, i64, C.POINTER(vp)]),
            "rx_pam_process": (i32, [vp, vp, i64, vp, vp, vp, vp]),
            "rx_pam_get": (i32, [vp, i32, vp, i64, vp]),
            "rx_pam_destroy": (None, [vp]),
            "rx_fp32_fma_rate": (i32, [i32, i32, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]),
            "rx_pe_targets": (i32, [vp, i64, vp, i64, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), i32, vp, vp]),
            "rx_kk_equalise": (i32, [vp, vp, i64, i32, vp, i64, i32, i32, i32, i32, C.c_float, C.c_float, vp, vp, vp,
                                     vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class RxError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {lib().rx_strerror(status).decode()} ({status})")
        self.status = status


def _check(status: int, where: str) -> None:
    if status != RX_OK:
        raise RxError(status, where)


def make_config(**kw) -> rx_config:
    """rx_config from keyword fields (missing fields are 0)."""
    cfg = rx_config()
    names = {n for n, _ in rx_config._fields_}
    for k, v in kw.items():
        if k in names:
            setattr(cfg, k, v)
    return cfg


# --- entry points, same names as the C ABI ---------------------------------

def rx_create(cfg: rx_config) -> int:
    h = C.c_void_p()
    _check(lib().rx_create(C.byref(cfg), C.byref(h)), "rx_create")
    return h.value


def rx_process(h: int, d_in: int, n_sym: int, d_ref: int | None, d_out: int | None, stream: int | None) -> None:
    _check(lib().rx_process(h, d_in, n_sym, d_ref or None, d_out or None, stream or None), "rx_process")


def rx_process_host(h: int, h_in: int, n_sym: int, h_ref: int | None, h_out: int | None, stream: int | None) -> None:
    _check(lib().rx_process_host(h, h_in, n_sym, h_ref or None, h_out or None, stream or None), "rx_process_host")


def rx_stats(h: int) -> dict:
    st = rx_stats_t()
    _check(lib().rx_stats(h, C.byref(st)), "rx_stats")
    return st.as_dict()


def rx_buffer_bytes(h: int, which: int) -> int:
    n = C.c_int64()
    _check(lib().rx_buffer_bytes(h, which, C.byref(n)), "rx_buffer_bytes")
    return n.value


def rx_get_buffer(h: int, which: int, d_dst: int, nbytes: int, stream: int | None) -> None:
    _check(lib().rx_get_buffer(h, which, d_dst, nbytes, stream or None), "rx_get_buffer")


def rx_reset(h: int) -> None:
    _check(lib().rx_reset(h), "rx_reset")


def rx_state_size(h: int) -> int:
    n = C.c_size_t()
    _check(lib().rx_state_size(h, C.byref(n)), "rx_state_size")
    return n.value


def rx_state_get(h: int) -> bytes:
    n = rx_state_size(h)
    buf = C.create_string_buffer(n)
    _check(lib().rx_state_get(h, buf, n), "rx_state_get")
    return buf.raw


def rx_state_set(h: int, blob: bytes) -> None:
    buf = C.create_string_buffer(blob, len(blob))
    _check(lib().rx_state_set(h, buf, len(blob)), "rx_state_set")


def rx_set_timing(h: int, enable: bool) -> None:
    _check(lib().rx_set_timing(h, 1 if enable else 0), "rx_set_timing")


def rx_stage_count() -> int:
    return lib().rx_stage_count()


def rx_stage_name(i: int) -> str:
    return lib().rx_stage_name(i).decode()


def rx_stage_times(h: int) -> dict:
    n = rx_stage_count()
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    _check(lib().rx_stage_times(h, ms, cnt, n), "rx_stage_times")
    return {rx_stage_name(i): (ms[i], cnt[i]) for i in range(n)}


def rx_launch_count(h: int) -> int:
    return int(lib().rx_launch_count(h))


def rx_destroy(h: int) -> None:
    lib().rx_destroy(h)


def rx_strerror(status: int) -> str:
    return lib().rx_strerror(status).decode()


def rx_batch_create(cfgs: list) -> int:
    arr = (rx_config * len(cfgs))(*cfgs)
    b = C.c_void_p()
    _check(lib().rx_batch_create(arr, len(cfgs), C.byref(b)), "rx_batch_create")
    return b.value


def rx_batch_config(b: int, i: int) -> rx_config:
    cfg = rx_config()
    _check(lib().rx_batch_config(b, i, C.byref(cfg)), "rx_batch_config")
    return cfg


def rx_batch_handle(b: int, i: int) -> int:
    return lib().rx_batch_handle(b, i)


def rx_batch_process(b: int, d_in: list, n_sym: list, d_ref: list | None, d_out: list | None,
                     stream: int | None) -> None:
    n = len(d_in)
    ins = (C.c_void_p * n)(*d_in)
    ns = (C.c_int64 * n)(*n_sym)
    refs = (C.c_void_p * n)(*d_ref) if d_ref is not None else None
    outs = (C.c_void_p * n)(*d_out) if d_out is not None else None
    _check(lib().rx_batch_process(b, ins, ns, refs, outs, stream or None), "rx_batch_process")


def rx_batch_stats(b: int, i: int) -> dict:
    st = rx_stats_t()
    _check(lib().rx_batch_stats(b, i, C.byref(st)), "rx_batch_stats")
    return st.as_dict()


def rx_batch_launch_count(b: int) -> int:
    return int(lib().rx_batch_launch_count(b))


def rx_batch_destroy(b: int) -> None:
    lib().rx_batch_destroy(b)


def rx_decide(h: int, d_z: int, n_sym: int, d_ref: int | None, d_out: int | None, stream: int | None) -> None:
    _check(lib().rx_decide(h, d_z, n_sym, d_ref or None, d_out or None, stream or None), "rx_decide")


def rx_pe_param_count(channels: int = 64, kernel: int = 9) -> int:
    return int(lib().rx_pe_param_count(channels, kernel))


def rx_pe_create(max_len: int, params=None, channels: int = 64, kernel: int = 9) -> int:
    """params: host float32 array (contiguous) of rx_pe_param_count values, or None for zeros."""
    p = C.c_void_p()
    ptr = params.ctypes.data if params is not None else None
    _check(lib().rx_pe_create(channels, kernel, max_len, ptr, C.byref(p)), "rx_pe_create")
    return p.value


def rx_pe_params(p: int, out) -> None:
    _check(lib().rx_pe_params(p, out.ctypes.data), "rx_pe_params")


def rx_pe_forward(p: int, d_z: int, T: int, d_out: int, stream: int | None) -> None:
    _check(lib().rx_pe_forward(p, d_z, T, d_out, stream or None), "rx_pe_forward")


def rx_pe_error_word(p: int) -> int:
    w = C.c_uint32(0)
    _check(lib().rx_pe_error_word(p, C.byref(w)), "rx_pe_error_word")
    return int(w.value)


def rx_pe_gradients(p: int, d_z: int, d_target: int, T: int, d_grads: int | None, d_loss: int | None,
                    stream: int | None) -> None:
    _check(lib().rx_pe_gradients(p, d_z, d_target, T, d_grads or None, d_loss or None, stream or None),
           "rx_pe_gradients")


def rx_pe_train_step(p: int, d_z: int, d_target: int, T: int, lr: float, d_loss: int | None,
                     stream: int | None) -> None:
    _check(lib().rx_pe_train_step(p, d_z, d_target, T, lr, d_loss or None, stream or None), "rx_pe_train_step")


def rx_pe_train_steps(p: int, d_z: list[int], d_target: list[int], lens: list[int], window: int, which, offs, lrs,
                      d_losses: int | None, stream: int | None) -> None:
    """len(which) Adam steps in one call; see include/rx.h."""
    n = len(d_z)
    steps = len(which)
    if len(d_target) != n or len(lens) != n or len(offs) != steps or len(lrs) != steps:
        raise ValueError("mismatched argument lengths")
    zp = (C.c_void_p * n)(*d_z)
    tp = (C.c_void_p * n)(*d_target)
    ln = (C.c_int64 * n)(*[int(v) for v in lens])
    wh = (C.c_int32 * max(steps, 1))(*[int(v) for v in which])
    of = (C.c_int64 * max(steps, 1))(*[int(v) for v in offs])
    lr = (C.c_float * max(steps, 1))(*[float(v) for v in lrs])
    _check(lib().rx_pe_train_steps(p, zp, tp, ln, n, window, steps, wh, of, lr, d_losses or None, stream or None),
           "rx_pe_train_steps")


def rx_pe_destroy(p: int) -> None:
    lib().rx_pe_destroy(p)


def rx_pe_targets(d_z: int, n_sym: int, d_symbols: int, n_ref: int, pol_map, rotation, delay, block: int,
                  d_target: int, stream: int | None) -> None:
    """Training labels of the post-equaliser on the device; see include/rx.h."""
    arr = lambda v: (C.c_int32 * 2)(*[int(x) for x in v])
    _check(lib().rx_pe_targets(d_z, n_sym, d_symbols, n_ref, arr(pol_map), arr(rotation), arr(delay), block, d_target,
                               stream or None), "rx_pe_targets")


def rx_fp32_fma_rate(packed: bool, iters: int, stream: int | None) -> tuple[float, float]:
    """Measured FP32 FMA throughput (flops/s, ms of the timed launch); see include/rx.h."""
    f, t = C.c_double(), C.c_double()
    _check(lib().rx_fp32_fma_rate(1 if packed else 0, iters, C.byref(f), C.byref(t), stream or None),
           "rx_fp32_fma_rate")
    return f.value, t.value


def rx_carrier_recovery_static(d_y: int, n_sym: int, bits_per_sym: int, bps_phases: int, bps_window: int, d_z: int,
                               stream: int | None) -> None:
    """Carrier recovery with the library's fixed device scratch (no allocation); see include/rx.h."""
    _check(lib().rx_carrier_recovery_static(d_y, n_sym, bits_per_sym, bps_phases, bps_window, d_z, stream or None),
           "rx_carrier_recovery_static")


def rx_dd_lms_wl(d_x: int, x_len: int, n_taps: int, d_taps_in: int, n_sym: int, block_len: int, seg_blocks: int,
                 warmup_blocks: int, bits_per_sym: int, mu: float, mu_conj: float, d_y: int, d_taps_out: int | None,
                 threads: int, stream: int | None) -> None:
    """Widely-linear segmented DD-LMS on caller-owned device buffers; see include/rx.h."""
    _check(lib().rx_dd_lms_wl(d_x, x_len, n_taps, d_taps_in, n_sym, block_len, seg_blocks, warmup_blocks,
                              bits_per_sym, mu, mu_conj, d_y, d_taps_out or None, threads, stream or None),
           "rx_dd_lms_wl")


def rx_kk_create(fft_size: int, tone_over_fs: float, rrc_rolloff: float, code_scale: float, dc_offset: float,
                 min_intensity: float) -> int:
    """Kramers-Kronig front end handle; see include/rx.h."""
    h = C.c_void_p()
    _check(lib().rx_kk_create(fft_size, tone_over_fs, rrc_rolloff, code_scale, dc_offset, min_intensity,
                              C.byref(h)), "rx_kk_create")
    return h.value


def rx_kk_process(k: int, d_codes: int, n_samples: int, first_sample: int, d_field: int, d_out: int,
                  stream: int | None) -> None:
    _check(lib().rx_kk_process(k, d_codes, n_samples, first_sample, d_field, d_out, stream or None), "rx_kk_process")


def rx_kk_equalise(k: int, d_x: int, x_len: int, n_taps: int, d_taps_in: int, n_sym: int, block_len: int,
                   seg_blocks: int, warmup_blocks: int, bits_per_sym: int, mu: float, mu_conj: float, d_y: int,
                   d_bits: int | None, d_taps_out: int | None, stream: int | None) -> None:
    """Step 9 of the KK receiver: widely-linear DD-LMS, decisions and demapping; see include/rx.h."""
    _check(lib().rx_kk_equalise(k, d_x, x_len, n_taps, d_taps_in, n_sym, block_len, seg_blocks, warmup_blocks,
                                bits_per_sym, mu, mu_conj, d_y, d_bits or None, d_taps_out or None, stream or None),
           "rx_kk_equalise")


def rx_ingest_run(k: int, h_source, buffer_samples: int, sample_rate_hz: float, n_streams: int, n_buffers: int,
                  h_out=None) -> dict:
    """h_source: host uint16 array (contiguous); h_out: host complex64 array of n_buffers * buffer_samples / 2
    values, or None. Returns the run's statistics."""
    st = rx_ingest_stats()
    _check(lib().rx_ingest_run(k, h_source.ctypes.data, h_source.size, buffer_samples, sample_rate_hz, n_streams,
                               n_buffers, h_out.ctypes.data if h_out is not None else None, C.byref(st)),
           "rx_ingest_run")
    return {f: getattr(st, f) for f, _ in rx_ingest_stats._fields_ if f != "pad0"}


def rx_kk_destroy(k: int) -> None:
    lib().rx_kk_destroy(k)


def rx_pam_create(fft_size: int, levels: int, rrc_rolloff: float, code_scale: float, dc_offset: float,
                  max_samples: int) -> int:
    """IM/DD PAM chain handle; see include/rx.h."""
    h = C.c_void_p()
    _check(lib().rx_pam_create(fft_size, levels, rrc_rolloff, code_scale, dc_offset, max_samples, C.byref(h)),
           "rx_pam_create")
    return h.value


def rx_pam_process(p: int, d_codes: int, n_samples: int, d_y: int, d_levels: int, d_n_out: int,
                   stream: int | None) -> None:
    _check(lib().rx_pam_process(p, d_codes, n_samples, d_y, d_levels, d_n_out, stream or None), "rx_pam_process")


def rx_pam_get(p: int, which: int, d_dst: int, nbytes: int, stream: int | None) -> None:
    _check(lib().rx_pam_get(p, which, d_dst, nbytes, stream or None), "rx_pam_get")


def rx_pam_destroy(p: int) -> None:
    lib().rx_pam_destroy(p)
