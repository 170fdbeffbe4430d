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
    float2* eq = nullptr;        // Step 9 taps in the equaliser's row layout: in [4][RX_TMAX], out [4][RX_TMAX]
};

namespace {

// Step 9 taps: caller layout [2][T] (h, then the conjugate taps g) -> row 0 of the equaliser's layout
// [h_0, h_1, g_0, g_1] with the second input polarisation's taps zero, and back
__global__ void k_kk_taps_in(const float2* in, int T, float2* out) {
    const int t = threadIdx.x;
    if (t < 4 * T) {
        const int v = t / (2 * T), p = (t / T) & 1, k = t % T;
        out[t] = p ? make_float2(0.0f, 0.0f) : in[v * T + k];
    }
}

__global__ void k_kk_taps_out(const float2* eq, int T, float2* out) {
    const int t = threadIdx.x;
    if (t < 2 * T) {
        const int v = t / T, k = t % T;
        out[t] = eq[v * 2 * T + k];
    }
}

// Step 9 decisions: Gray bits of the nearest square-QAM point, packed as rx_process packs one
// polarisation (stream bit i in bit i % 32 of word i / 32; the first m/2 bits of a symbol are the
// Gray word of its in-phase level, most significant first). One thread per output word.
__global__ void k_kk_demap(const float2* __restrict__ y, int64_t n_sym, int m, uint32_t* __restrict__ bits,
                           int64_t words) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= words) return;
    const Qam qm = make_qam(m);
    uint32_t word = 0;
    int64_t cur = -1;
    uint32_t sb = 0;
    for (int i = 0; i < 32; ++i) {
        const int64_t b = w * 32 + i;
        const int64_t n = b / m;
        if (n >= n_sym) break;
        if (n != cur) {
            cur = n;
            const float2 v = y[n];
            const int li = qam_level(v.x, qm), lq = qam_level(v.y, qm);
            sb = qam_bits(li, lq, qm);                       // Gray I word in the top h bits, Q below
        }
        const int j = (int)(b - n * m);                      // bit j of the symbol, first transmitted = 0
        word |= ((sb >> (m - 1 - j)) & 1u) << i;
    }
    bits[w] = word;
}

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
        cudaMalloc(&k->H, sizeof(float) * N) != cudaSuccess ||
        cudaMalloc(&k->eq, sizeof(float2) * 8 * RX_TMAX) != cudaSuccess) {
        if (k->tw) cudaFree(k->tw);
        if (k->H) cudaFree(k->H);
        if (k->eq) cudaFree(k->eq);
        delete k;
        return RX_ENOMEM;
    }
    if (launch_fill_twiddles(k->tw, 0) != cudaSuccess ||
        cudaMemcpy(k->H, H.data(), sizeof(float) * N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(k->tw);
        cudaFree(k->H);
        cudaFree(k->eq);
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
    if (k->eq) cudaFree(k->eq);
    delete k;
}

rx_status rx_kk_equalise(rx_kk* k, const float* d_x, int64_t x_len, int32_t n_taps, const float* d_taps_in,
                         int64_t n_sym, int32_t block_len, int32_t seg_blocks, int32_t warmup_blocks,
                         int32_t bits_per_sym, float mu, float mu_conj, float* d_y, uint32_t* d_bits,
                         float* d_taps_out, rx_stream_t stream) {
    if (!k || !d_x || !d_taps_in || !d_y || n_sym < 1 || x_len < 1) return RX_EINVAL;
    if (n_taps < 3 || n_taps > 63 || !(n_taps & 1)) return RX_EINVAL;
    if (block_len < 16 || block_len > 256 || seg_blocks < 1 || warmup_blocks < 0) return RX_EINVAL;
    if (bits_per_sym != 2 && bits_per_sym != 4 && bits_per_sym != 6 && bits_per_sym != 8) return RX_EINVAL;
    const int64_t L_seg = (int64_t)seg_blocks * block_len;
    if ((n_sym + L_seg - 1) / L_seg > 0x7fffffffLL) return RX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float2* eq_in = k->eq;
    float2* eq_out = k->eq + 4 * RX_TMAX;
    k_kk_taps_in<<<1, 256, 0, s>>>(reinterpret_cast<const float2*>(d_taps_in), n_taps, eq_in);
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
    a.taps_in = eq_in;
    a.taps_out = eq_out;
    a.y = reinterpret_cast<float2*>(d_y);
    a.ystride = n_sym;
    a.run_if = nullptr;
    a.st = nullptr;
    a.exclusive = 0;
    a.npol = 1;
    if (launch_lms_wl_generic(a, 256, s) != cudaSuccess) return RX_ECUDA;
    if (d_taps_out) k_kk_taps_out<<<1, 128, 0, s>>>(eq_out, n_taps, reinterpret_cast<float2*>(d_taps_out));
    if (d_bits) {
        const int64_t words = (n_sym * bits_per_sym + 31) / 32;
        k_kk_demap<<<(unsigned)((words + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float2*>(d_y), n_sym,
                                                                    bits_per_sym, d_bits, words);
    }
    return cudaGetLastError() == cudaSuccess ? RX_OK : RX_ECUDA;
}

}  // extern "C"

int kk_fft_size(const rx_kk* k) { return 1 << k->K; }
