// Kramers-Kronig self-coherent front end (Sec. IV, Steps 1-8) and its C entry points.
//
// Two overlap-save passes over the frame at 4 samples/symbol, blocks of N = 2^K
// samples starting N/4 before the N/2 they keep (zero outside the frame), one CTA
// per block, the in-CTA Stockham FFT of rx_fft.cuh:
//   k_kk_phase<K>  Steps 1-5: 12-bit code -> I = max(scale code + dc, i_min) ->
//                  l = ln sqrt(I) -> FFT -> times -j sgn(k) -> IFFT -> phi (two real
//                  blocks per complex transform); for each kept sample
//                  E = sqrt(I) exp(j phi) exp(-j 2 pi (f_t/fs) n) -> field buffer;
//   k_kk_mf<K>     Steps 6-8: FFT of the field block -> times H[k] = 2 RRC(f_k) / N
//                  on the bins |f| < fs/4, written straight into their places in
//                  the N/2-point spectrum -> N/2-point IFFT -> the centre N/4
//                  outputs at 2 samples/symbol.
// The paper runs the front end inside its overlap kernel and the FFTs as library
// calls; here each pass is one kernel whose first FFT pass reads the input
// through the front end and whose last pass writes the kept outputs, so HBM
// sees the codes once, the field once each way and the output once.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/rx.h"
#include "rx_fft.cuh"
#include "rx_kernels.h"

struct rx_kk {
    int K = 10;
    long long inc = 0;           // tone phase per sample, 2^-64 turns
    float scale = 1.0f, dc = 0.0f, i_min = 0.0f;
    float2* tw = nullptr;        // FFT twiddles
    float* H = nullptr;          // [N] 2 RRC(f_k) / N
};

namespace {

struct KkArgs {
    const uint16_t* codes;
    float* field;                // float2 [S]
    float* out;                  // float2 [S/2]
    int64_t S;
    long long g0;                // stream index of sample 0 (downshift phase)
    float scale, dc, i_min;
    long long inc;
    const float2* tw;
    const float* H;
};

// One CTA takes the block pair (2b, 2b + 1): block 2b starts at 2b N/2 - N/4, block 2b + 1 N/2 later,
// so the pair reads a window of 3N/2 samples. Their log-amplitudes are real, and -j sgn(k) maps the
// spectrum of a real sequence to that of a real sequence, so one complex transform of
// z = l_{2b} + j l_{2b+1} gives both phases: phi_{2b} = Re IFFT(-j sgn Z), phi_{2b+1} = Im.
// Each sample's (log-amplitude, amplitude) is computed once into shared memory.
template <int K>
__global__ void __launch_bounds__(((1 << K) / 16 < 32) ? 32 : (1 << K) / 16) k_kk_phase(KkArgs a) {
    constexpr int N = 1 << K, HOP = N / 2, LEAD = N / 4, W = N + HOP;
    constexpr int NT = (N / 16 < 32) ? 32 : N / 16;
    extern __shared__ float2 sm[];
    float2* la = sm + fft_smem_elems(N);                    // [W]: (ln sqrt I, sqrt I), zero outside the frame
    const int64_t start = (int64_t)blockIdx.x * N - LEAD;   // block 2b
    for (int i = 4 * threadIdx.x; i < W; i += 4 * NT) {
        const int64_t s0 = start + i;
        uint16_t c[4] = {0, 0, 0, 0};
        bool v[4];
        if (s0 >= 0 && s0 + 3 < a.S) {                      // start and i are multiples of 4: 8-byte aligned
            const ushort4 q = *reinterpret_cast<const ushort4*>(a.codes + s0);
            c[0] = q.x; c[1] = q.y; c[2] = q.z; c[3] = q.w;
            v[0] = v[1] = v[2] = v[3] = true;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v[u] = s0 + u >= 0 && s0 + u < a.S;
                if (v[u]) c[u] = a.codes[s0 + u];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 r = make_float2(0.0f, 0.0f);
            if (v[u]) {
                const float I = fmaxf(fmaf(a.scale, (float)c[u], a.dc), a.i_min);
                r = make_float2(0.5f * logf(I), sqrtf(I));
            }
            la[i + u] = r;
        }
    }
    __syncthreads();
    auto load = [&](int idx) -> float2 { return make_float2(la[idx].x, la[idx + HOP].x); };
    // -j sgn(k) and the inverse transform's 1/N
    auto store_h = [&](int k, float2 v) {
        constexpr float inv = 1.0f / (float)N;
        float2 r = make_float2(0.0f, 0.0f);
        if (k > 0 && k < N / 2) r = make_float2(v.y * inv, -v.x * inv);
        else if (k > N / 2) r = make_float2(-v.y * inv, v.x * inv);
        sm[fft_pad(k)] = r;
    };
    fft_run<K, -1, true, true>(sm, a.tw, load, store_h);
    __syncthreads();
    float2* field = reinterpret_cast<float2*>(a.field);
    auto store_out = [&](int idx, float2 v) {
        if (idx >= LEAD && idx < LEAD + HOP) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = idx + h * HOP;
                const int64_t n = start + i;
                if (n < a.S) {
                    float sn, cs;
                    sincosf(h ? v.y : v.x, &sn, &cs);
                    const float amp = la[i].y;
                    field[n] = cmul(make_float2(amp * cs, amp * sn), nco_conj(a.inc, a.g0 + n));
                }
            }
        }
    };
    SmemLoad sl{sm};
    fft_run<K, +1, false, true>(sm, a.tw, sl, store_out);
}

template <int K>
__global__ void __launch_bounds__(((1 << K) / 16 < 32) ? 32 : (1 << K) / 16, (K == 10) ? 16 : 1) k_kk_mf(KkArgs a) {
    constexpr int N = 1 << K, HOP = N / 2, LEAD = N / 4;
    extern __shared__ float2 sm[];
    const int64_t start = (int64_t)blockIdx.x * HOP - LEAD;
    const float2* field = reinterpret_cast<const float2*>(a.field);
    auto load = [&](int idx) -> float2 {
        const int64_t s = start + idx;
        return (s >= 0 && s < a.S) ? field[s] : make_float2(0.0f, 0.0f);
    };
    // bins |f| < fs/4 into the N/2-point spectrum: k -> k (k < N/4), k -> k - N/2 (k >= 3N/4)
    const float* __restrict__ H = a.H;
    auto store_h = [&](int k, float2 v) {
        if (k < N / 4) sm[fft_pad(k)] = cscale(v, __ldg(&H[k]));
        else if (k >= 3 * N / 4) sm[fft_pad(k - N / 2)] = cscale(v, __ldg(&H[k]));
    };
    fft_run<K, -1, true, true>(sm, a.tw, load, store_h);
    __syncthreads();
    float2* out = reinterpret_cast<float2*>(a.out);
    const int64_t o0 = (int64_t)blockIdx.x * (HOP / 2) - LEAD / 2;
    const int64_t S2 = a.S / 2;
    auto store_out = [&](int idx, float2 v) {
        if (idx >= LEAD / 2 && idx < LEAD / 2 + HOP / 2) {
            const int64_t m = o0 + idx;
            if (m < S2) out[m] = v;
        }
    };
    SmemLoad sl{sm};
    fft_run<K - 1, +1, false, true>(sm, a.tw, sl, store_out);
}

template <int K>
cudaError_t launch_kk_t(const KkArgs& a, cudaStream_t s) {
    constexpr int N = 1 << K;
    const int threads = N / 16 < 32 ? 32 : N / 16;
    const size_t smem = sizeof(float2) * fft_smem_elems(N);
    const size_t smem_phase = smem + sizeof(float2) * (N + N / 2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_kk_phase<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_phase);
        cudaFuncSetAttribute(k_kk_mf<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int64_t nblk = (a.S + N / 2 - 1) / (N / 2);
    k_kk_phase<K><<<(unsigned)((nblk + 1) / 2), threads, smem_phase, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_kk_mf<K><<<(unsigned)nblk, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_kk(int K, const KkArgs& a, cudaStream_t s) {
    switch (K) {
        case 10: return launch_kk_t<10>(a, s);
        case 11: return launch_kk_t<11>(a, s);
        case 12: return launch_kk_t<12>(a, s);
        case 13: return launch_kk_t<13>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

extern "C" {

rx_status rx_kk_create(int32_t fft_size, double tone_over_fs, double rrc_rolloff, float code_scale, float dc_offset,
                       float min_intensity, rx_kk** out) {
    if (!out) return RX_EINVAL;
    *out = nullptr;
    int K = 0;
    while (K < 14 && (1 << K) < fft_size) ++K;
    if ((1 << K) != fft_size || K < 10 || K > 13) return RX_EINVAL;
    if (!(tone_over_fs > 0.0 && tone_over_fs < 0.5)) return RX_EINVAL;
    if (!(rrc_rolloff > 0.0 && rrc_rolloff <= 1.0)) return RX_EINVAL;
    if (!std::isfinite(code_scale) || code_scale == 0.0f || !std::isfinite(dc_offset)) return RX_EINVAL;
    if (!(min_intensity > 0.0f) || !std::isfinite(min_intensity)) return RX_EINVAL;
    rx_kk* k = new (std::nothrow) rx_kk();
    if (!k) return RX_ENOMEM;
    k->K = K;
    k->inc = std::llrint(std::ldexp(tone_over_fs, 64));
    k->scale = code_scale;
    k->dc = dc_offset;
    k->i_min = min_intensity;
    const int N = 1 << K;
    // H[k] = 2 RRC(f_k) / N, f_k the signed bin frequency in cycles per sample, symbol rate 1/4
    std::vector<float> H(N);
    const double lo = (1.0 - rrc_rolloff) / 8.0, hi = (1.0 + rrc_rolloff) / 8.0;
    for (int i = 0; i < N; ++i) {
        const double f = std::fabs((double)(i < N / 2 ? i : i - N) / (double)N);
        double amp = f <= lo ? 1.0 : (f <= hi ? std::cos(M_PI / (2.0 * rrc_rolloff * 0.25) * (f - lo)) : 0.0);
        H[i] = (float)(2.0 * amp / (double)N);
    }
    if (cudaMalloc(&k->tw, sizeof(float2) * RX_FFT_TW_N) != cudaSuccess ||
        cudaMalloc(&k->H, sizeof(float) * N) != cudaSuccess) {
        if (k->tw) cudaFree(k->tw);
        if (k->H) cudaFree(k->H);
        delete k;
        return RX_ENOMEM;
    }
    if (launch_fill_twiddles(k->tw, 0) != cudaSuccess ||
        cudaMemcpy(k->H, H.data(), sizeof(float) * N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(k->tw);
        cudaFree(k->H);
        delete k;
        return RX_ECUDA;
    }
    *out = k;
    return RX_OK;
}

rx_status rx_kk_process(rx_kk* k, const uint16_t* d_codes, int64_t n_samples, int64_t first_sample, float* d_field,
                        float* d_out, rx_stream_t stream) {
    if (!k || !d_codes || !d_field || !d_out) return RX_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_codes) & 7) return RX_EINVAL;   // the codes are read 4 at a time
    if (n_samples < 2 || (n_samples & 1) || n_samples > ((int64_t)1 << 36)) return RX_EINVAL;
    KkArgs a;
    a.codes = d_codes;
    a.field = d_field;
    a.out = d_out;
    a.S = n_samples;
    a.g0 = first_sample;
    a.scale = k->scale;
    a.dc = k->dc;
    a.i_min = k->i_min;
    a.inc = k->inc;
    a.tw = k->tw;
    a.H = k->H;
    return launch_kk(k->K, a, (cudaStream_t)stream) == cudaSuccess ? RX_OK : RX_ECUDA;
}

void rx_kk_destroy(rx_kk* k) {
    if (!k) return;
    if (k->tw) cudaFree(k->tw);
    if (k->H) cudaFree(k->H);
    delete k;
}

}  // extern "C"

int kk_fft_size(const rx_kk* k) { return 1 << k->K; }
