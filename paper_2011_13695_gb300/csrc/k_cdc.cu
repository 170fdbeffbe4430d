// A0 power normalisation and A1 overlap-save FD dispersion compensation.
//
// Paper anchor (Sec. III-A, Sec. II-D Steps 3-4): 1024-point FFT with
// "100 % overlap-save" (N/2 valid samples per block), an FD filter multiplied
// bin by bin, and an overlap kernel that carries one block between buffers
// and converts the ADC integers to float. Here one CTA transforms one block of
// one polarisation entirely on chip: the input conversion and the A0 scale
// are fused into the first FFT pass (read straight from HBM, coalesced), the
// filter H = H_cdc * H_rrc / N is applied as the forward transform's last pass
// writes shared memory, and the inverse transform's last pass writes only the
// kept centre half [N/4, 3N/4) back to HBM. HBM traffic per block: 2x the new
// samples in (neighbouring blocks overlap by half, mostly served by L2) and
// the N/2 valid samples out.
#include <cuda_fp16.h>

#include <algorithm>

#include "rx_fft.cuh"
#include "rx_kernels.h"

namespace {

template <int FMT>
__device__ __forceinline__ float2 load_sample(const void* in, int64_t idx, float sc) {
    if constexpr (FMT == 0) {
        float2 v = __ldg(reinterpret_cast<const float2*>(in) + idx);
        return make_float2(v.x * sc, v.y * sc);
    } else if constexpr (FMT == 1) {
        __half2 h = reinterpret_cast<const __half2*>(in)[idx];
        float2 v = __half22float2(h);
        return make_float2(v.x * sc, v.y * sc);
    } else {
        char2 c = reinterpret_cast<const char2*>(in)[idx];
        return make_float2((float)c.x * sc, (float)c.y * sc);
    }
}

// A0: mean power of the first n_win samples of each polarisation: FP32 sums per thread (a few
// dozen samples each), then pairwise across the warp and the CTA; scale = 1/sqrt(P).
template <int FMT>
__global__ void k_power(const void* in, float in_scale, int64_t S, int64_t n_win, RxDevState* st, int single) {
    const int p = blockIdx.x;
    if (p == 0 && threadIdx.x == 0) {                 // start of the frame (its first frame of a stream)
        if (single) {
            st->b_prev[0] = st->b_prev[1] = -1;
            st->m_prev[0] = st->m_prev[1] = 0;
            st->sync_valid = 0;
        }
        st->fo_code = 0;
        st->nco_inc = 0;
        st->fo_valid = 0;
        st->cma_reran = 0;
        st->cma_rho = 0.0f;
    }
    // eight loads in flight per thread before their sums (same order of additions as one at a time)
    float acc = 0.0f;
    int64_t i = threadIdx.x;
    const int64_t nt = blockDim.x;
    for (; i + 7 * nt < n_win; i += 8 * nt) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = load_sample<FMT>(in, (int64_t)p * S + i + u * nt, in_scale);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += cabs2(v[u]);
    }
    for (; i < n_win; i += nt) acc += cabs2(load_sample<FMT>(in, (int64_t)p * S + i, in_scale));
    __shared__ float red[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            const float P = n_win > 0 ? v / (float)n_win : 0.0f;
            st->scale[p] = P > 0.0f ? rsqrtf(P) : 1.0f;
        }
    }
}

template <int K, int FMT>
__global__ void __launch_bounds__(((1 << K) / 16 < 32) ? 32 : (1 << K) / 16)
    k_cdc(CdcArgs a) {
    constexpr int N = 1 << K;
    constexpr int HOP = N / 2, LEAD = N / 4;
    extern __shared__ float2 sm[];
    const int p = blockIdx.y;
    const int64_t j = a.j0 + blockIdx.x;
    const float sc = a.st->scale[p] * a.in_scale;
    const int64_t S = a.S;
    const void* in = a.in;
    const int64_t pbase = (int64_t)p * S;
    const float2* tail = a.tail ? a.tail + (int64_t)p * HOP : nullptr;
    bool bad = false;

    // block j covers input samples [j*HOP - LEAD, j*HOP - LEAD + N) (single frame)
    // or stream positions [j*HOP - HOP, j*HOP - HOP + N), negative ones from the tail
    const int64_t start = tail ? j * HOP - HOP : j * HOP - LEAD;
    auto load = [&](int idx) -> float2 {
        const int64_t s = start + idx;
        float2 v = make_float2(0.0f, 0.0f);
        if (s >= 0 && s < S) {
            v = load_sample<FMT>(in, pbase + s, sc);
        } else if (s < 0 && tail) {
            v = tail[HOP + s];
        }
        bad |= !isfinite(v.x + v.y);
        return v;
    };
    const float2* __restrict__ H = a.H;
    auto store_h = [&](int idx, float2 v) { sm[fft_pad(idx)] = cmul(v, __ldg(&H[idx])); };
    // a block wholly inside the frame (the common case) loads without bounds checks
    auto load_in = [&](int idx) -> float2 {
        const float2 v = load_sample<FMT>(in, pbase + start + idx, sc);
        bad |= !isfinite(v.x + v.y);
        return v;
    };
    if (start >= 0 && start + N <= S)
        fft_run<K, -1, true, true>(sm, a.tw, load_in, store_h);
    else
        fft_run<K, -1, true, true>(sm, a.tw, load, store_h);
    __syncthreads();
    float2* out = a.out + (int64_t)p * a.ostride + a.obase;
    const int64_t o0 = j * HOP - LEAD;
    auto store_out = [&](int idx, float2 v) {
        if (idx >= LEAD && idx < LEAD + HOP) {
            const int64_t o = o0 + idx;
            if (o < S) out[o] = v;
        }
    };
    SmemLoad sl{sm};
    fft_run<K, +1, false, true>(sm, a.tw, sl, store_out);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&a.st->err_word, 1u);
}

// stream: keep the last HOP scaled input samples for the next frame
template <int FMT>
__global__ void k_tail(const void* in, float in_scale, int64_t S, int hop, float2* tail, const RxDevState* st) {
    const int p = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= hop) return;
    const float sc = st->scale[p] * in_scale;
    tail[(int64_t)p * hop + t] = load_sample<FMT>(in, (int64_t)p * S + S - hop + t, sc);
}

__global__ void k_copy_hist(float2* buf, int64_t stride, int64_t S, int hist) {
    const int p = blockIdx.y;
    const int t = threadIdx.x;
    if (t < hist) buf[(int64_t)p * stride + t] = buf[(int64_t)p * stride + S + t];
}

__global__ void k_fill_twiddles(float2* tw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < RX_FFT_TW_N) {
        double s, c;
        sincospi(-2.0 * (double)i / (double)RX_FFT_TW_N, &s, &c);
        tw[i] = make_float2((float)c, (float)s);
    }
}

// H[k] = exp(+j pi D L lambda^2 f_k^2 / c) * sqrt(2) * RRC(f_k) / N, f_k the signed bin frequency
__global__ void k_fill_filter(float2* H, int nfft, double fs, double dl2c, double rs, double rolloff) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nfft) return;
    const double f = (double)(k < (nfft + 1) / 2 ? k : k - nfft) * fs / (double)nfft;
    const double phase = dl2c * f * f;               // in units of pi radians
    double s, c;
    sincospi(phase - 2.0 * floor(phase * 0.5), &s, &c);
    double g = 1.0 / (double)nfft;
    if (rolloff > 0.0) {
        const double af = fabs(f), lo = (1.0 - rolloff) * rs * 0.5, hi = (1.0 + rolloff) * rs * 0.5;
        double amp = af <= lo ? 1.0 : (af <= hi ? cospi((af - lo) / (2.0 * rolloff * rs)) : 0.0);
        g *= sqrt(2.0) * amp;
    }
    H[k] = make_float2((float)(c * g), (float)(s * g));
}

template <int K, int FMT>
cudaError_t launch_cdc_t(const CdcArgs& a, cudaStream_t s) {
    constexpr int N = 1 << K;
    const int threads = N / 16 < 32 ? 32 : N / 16;
    const size_t smem = sizeof(float2) * fft_smem_elems(N);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_cdc<K, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int64_t hop = N / 2;
    const int64_t total = (a.S + hop - 1) / hop;
    const int64_t n = a.nblk < 0 ? total - a.j0 : std::min(a.nblk, total - a.j0);
    if (n <= 0) return cudaSuccess;
    dim3 grid((unsigned)n, 2);
    k_cdc<K, FMT><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_cdc_f(const CdcArgs& a, cudaStream_t s) {
    switch (a.nfft) {
        case 512: return launch_cdc_t<9, FMT>(a, s);
        case 1024: return launch_cdc_t<10, FMT>(a, s);
        case 2048: return launch_cdc_t<11, FMT>(a, s);
        case 4096: return launch_cdc_t<12, FMT>(a, s);
        case 8192: return launch_cdc_t<13, FMT>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_power(const void* in, int fmt, float in_scale, int64_t S, int64_t n_win, RxDevState* st,
                         int single, cudaStream_t s) {
    if (n_win > S) n_win = S;
    if (fmt == 0) k_power<0><<<2, 1024, 0, s>>>(in, in_scale, S, n_win, st, single);
    else if (fmt == 1) k_power<1><<<2, 1024, 0, s>>>(in, in_scale, S, n_win, st, single);
    else k_power<2><<<2, 1024, 0, s>>>(in, in_scale, S, n_win, st, single);
    return cudaGetLastError();
}

cudaError_t launch_cdc(const CdcArgs& a, cudaStream_t s) {
    if (a.fmt == 0) return launch_cdc_f<0>(a, s);
    if (a.fmt == 1) return launch_cdc_f<1>(a, s);
    return launch_cdc_f<2>(a, s);
}

cudaError_t launch_tail(const void* in, int fmt, float in_scale, int64_t S, int hop, float2* tail,
                        const RxDevState* st, cudaStream_t s) {
    dim3 grid((hop + 255) / 256, 2);
    if (fmt == 0) k_tail<0><<<grid, 256, 0, s>>>(in, in_scale, S, hop, tail, st);
    else if (fmt == 1) k_tail<1><<<grid, 256, 0, s>>>(in, in_scale, S, hop, tail, st);
    else k_tail<2><<<grid, 256, 0, s>>>(in, in_scale, S, hop, tail, st);
    return cudaGetLastError();
}

cudaError_t launch_copy_hist(float2* buf, int64_t stride, int64_t S, int hist, cudaStream_t s) {
    k_copy_hist<<<dim3(1, 2), 128, 0, s>>>(buf, stride, S, hist);
    return cudaGetLastError();
}

cudaError_t launch_fill_twiddles(float2* tw, cudaStream_t s) {
    k_fill_twiddles<<<RX_FFT_TW_N / 256, 256, 0, s>>>(tw);
    return cudaGetLastError();
}

cudaError_t launch_fill_filter(float2* H, int nfft, double fs, double dl2c, double rs, double rolloff,
                               cudaStream_t s) {
    k_fill_filter<<<(nfft + 255) / 256, 256, 0, s>>>(H, nfft, fs, dl2c, rs, rolloff);
    return cudaGetLastError();
}
