// Widely-linear segmented DD-LMS (Sec. IV-D) as a stand-alone stage on caller-owned buffers.
//
// The paper's TD equaliser is widely linear so that it also compensates the
// transmitter's IQ imbalance. The kernels are the segmented block LMS ones
// (compile-time shapes in k_lms_fast.cuh, the generic one in k_mimo.cu)
// instantiated with conjugate taps: one CTA per (segment, output row), the
// same fixed segment schedule and warm-up as the linear A4 stage,
// the input read straight from the caller's buffer (no frequency-offset
// derotation: the caller hands in the samples the equaliser sees).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/rx.h"
#include "rx_kernels.h"

extern "C" rx_status rx_dd_lms_wl(const float* d_x, int64_t x_len, int32_t n_taps, const float* d_taps_in,
                                  int64_t n_sym, int32_t block_len, int32_t seg_blocks, int32_t warmup_blocks,
                                  int32_t bits_per_sym, float mu, float mu_conj, float* d_y, float* d_taps_out,
                                  int32_t threads, rx_stream_t stream) {
    if (threads != 0 && threads != 128 && threads != 256 && threads != 512 && threads != 1024) return RX_EINVAL;
    if (!d_x || !d_taps_in || !d_y || n_sym < 1 || x_len < 1) return RX_EINVAL;
    if (n_taps < 3 || n_taps > 63 || !(n_taps & 1)) return RX_EINVAL;
    if (block_len < 16 || block_len > 256 || seg_blocks < 1 || warmup_blocks < 0) return RX_EINVAL;
    if (bits_per_sym != 2 && bits_per_sym != 4 && bits_per_sym != 6 && bits_per_sym != 8) return RX_EINVAL;
    const int64_t L_seg = (int64_t)seg_blocks * block_len;
    if ((n_sym + L_seg - 1) / L_seg > 0x7fffffffLL) return RX_EINVAL;
    const int64_t tap_bytes = (int64_t)2 * 4 * n_taps * 2 * (int64_t)sizeof(float);
    if (d_taps_out) {
        const char* a = reinterpret_cast<const char*>(d_taps_in);
        const char* b = reinterpret_cast<const char*>(d_taps_out);
        if (a < b + tap_bytes && b < a + tap_bytes) return RX_EINVAL;
    }
    LmsArgs a{};
    a.x = reinterpret_cast<const float2*>(d_x);
    a.xstride = x_len;
    a.xlen = x_len;
    a.off = 0;
    a.T = n_taps;
    a.Lb = block_len;
    a.n_sym = n_sym;
    a.L_seg = L_seg;
    a.n_wu = warmup_blocks;
    a.cma = 0;
    a.mu = mu;
    a.mu_c = mu_conj;
    a.R2 = 0.0f;
    a.m = bits_per_sym;
    a.derotate = 0;
    a.g0 = 0;
    a.taps_in = reinterpret_cast<const float2*>(d_taps_in);
    a.taps_out = reinterpret_cast<float2*>(d_taps_out);
    a.y = reinterpret_cast<float2*>(d_y);
    a.ystride = n_sym;
    a.run_if = nullptr;
    a.st = nullptr;
    a.exclusive = 0;
    const cudaError_t e = launch_lms_wl(a, threads, (cudaStream_t)stream);
    // invalid value: a thread count the shape cannot use, refused before any launch
    if (e == cudaErrorInvalidValue) return RX_EINVAL;
    return e == cudaSuccess ? RX_OK : RX_ECUDA;
}
