// IM/DD PAM-M chain with frequency-domain clock recovery (Sec. III, Steps 1-9) and its C entry points.
//
// At 2 samples/symbol, overlap-save blocks of N = 2^K samples (block j from j N/2 - N/4, zero
// outside the frame); the FFT passes take one CTA per block pair (the two real blocks go through
// one complex transform) and use the in-CTA Stockham FFT of rx_fft.cuh:
//   k_pam_clock<K>    code -> v = scale code + dc -> FFT (two real blocks per complex transform)
//                     -> times sqrt(2) RRC(f) -> each block's clock product
//                     c_j = sum_{k < N/2} X[k] conj(X[k + N/2]) (spectral line one symbol rate
//                     apart; its phase is -2 pi Rs tau for a delay tau);
//   k_pam_window      cbar_j = sum of c_i over |i - j| <= 52 inside the frame (a difference of
//                     FP64 prefix sums over each CTA's tile of products), phi_j = arg cbar_j, the
//                     unwrap step of block j (-1 if phi_j - phi_{j-1} > pi, +1 if < -pi);
//   k_pam_wind        one CTA: winding numbers w_j (integer prefix sum of the steps), each block's
//                     output count N/4 + w_{j+1} - w_j (N/4 for the last block, clipped to the
//                     frame) and offset;
//   k_pam_correct<K>  the FFT again (recomputing is cheaper than a 64 MB spectrum round trip),
//                     split into the pair's spectra, each times sqrt(2) RRC(f) exp(-j phi_j f / Rs)
//                     / N, recombined, one inverse FFT for both blocks; each block's
//                     outputs are the real parts of its samples N/4 + 2 i, written at its offset
//                     (variable rate: 255, 256 or 257 symbols per block), and their sum;
//   k_pam_final, k_pam_deviation   buffer-wise mean from the blocks' sums, then the mean absolute
//                     deviation (fixed-order two-stage reductions: results do not depend on
//                     scheduling);
//   k_pam_decide      u = (y - mean) (M/2) / mad, level index clip(rint((u + M - 1) / 2)).
// The paper estimates, averages and unwraps in separate kernels over five streams, unwraps
// with one warp, and extracts symbols in a kernel of its own; here the unwrap is an exact integer
// scan and the extraction is fused into the correcting inverse transform's last pass.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/rx.h"
#include "rx_fft.cuh"
#include "rx_kernels.h"

struct rx_pam {
    int K = 10;
    int M = 4;
    int64_t max_samples = 0;
    float scale = 1.0f, dc = 0.0f;
    float2* tw = nullptr;        // FFT twiddles
    float* H = nullptr;          // [N] sqrt(2) RRC(f_k)
    float2* c = nullptr;         // [J] clock products
    float* phi = nullptr;        // [J] averaged clock phase
    int* step = nullptr;         // [J] unwrap steps
    int* w = nullptr;            // [J] winding numbers
    long long* off = nullptr;    // [J + 1] output offsets (off[J] = outputs)
    double* part = nullptr;      // [J] per-block output sums, then [kParts] deviation partials
    double* stat = nullptr;      // [2] mean, mean absolute deviation
};

namespace {

constexpr int kAvgHalf = 52;
constexpr int kParts = 1024;      // CTAs of the partial reductions
constexpr int kRedThreads = 256;

struct PamArgs {
    const uint16_t* codes;
    int64_t S;
    int J;
    float scale, dc;
    const float2* tw;
    const float* H;
    float2* c;
    float* phi;
    int* step;
    int* w;
    long long* off;
    float* y;
    uint8_t* levels;
    double* part;
    double* stat;
    long long* n_out;
    int M;
};

// A CTA takes the block pair (2b, 2b + 1), whose real inputs go through one complex transform as
// z = v_{2b} + j v_{2b+1} (block 2b + 1 starts N/2 later). The matched filter is real and even, so
// the filtered spectra split as A[k] = (Z[k] + conj Z[N-k]) / 2 and B[k] = (Z[k] - conj Z[N-k]) / 2j.
template <int K>
__device__ __forceinline__ void pam_pair_spectrum(const PamArgs& a, float2* sm, int64_t start) {
    constexpr int N = 1 << K, HOP = N / 2;
    auto sample = [&](int64_t s) -> float {
        return (s >= 0 && s < a.S) ? fmaf(a.scale, (float)a.codes[s], a.dc) : 0.0f;
    };
    auto load = [&](int idx) -> float2 { return make_float2(sample(start + idx), sample(start + HOP + idx)); };
    const float* __restrict__ H = a.H;
    auto store = [&](int k, float2 v) { sm[fft_pad(k)] = cscale(v, __ldg(&H[k])); };
    fft_run<K, -1, true, true>(sm, a.tw, load, store);
    __syncthreads();
}

template <int K>
__global__ void __launch_bounds__(((1 << K) / 16 < 32) ? 32 : (1 << K) / 16) k_pam_clock(PamArgs a) {
    constexpr int N = 1 << K, HOP = N / 2, LEAD = N / 4;
    constexpr int NT = (N / 16 < 32) ? 32 : N / 16;
    extern __shared__ float2 sm[];
    __shared__ float2 red[2][NT / 32];
    const int j0 = 2 * blockIdx.x;
    pam_pair_spectrum<K>(a, sm, (int64_t)j0 * HOP - LEAD);
    float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
    for (int k = threadIdx.x; k < N / 2; k += NT) {
        const float2 zk = sm[fft_pad(k)], zm = sm[fft_pad((N - k) & (N - 1))];
        const float2 zh = sm[fft_pad(k + N / 2)], zhm = sm[fft_pad(N / 2 - k)];
        // A = (z + conj zm) / 2, B = (z - conj zm) / 2j = ((z.y + zm.y) / 2, (zm.x - z.x) / 2)
        const float2 ak = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 bk = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
        const float2 ah = make_float2(0.5f * (zh.x + zhm.x), 0.5f * (zh.y - zhm.y));
        const float2 bh = make_float2(0.5f * (zh.y + zhm.y), 0.5f * (zhm.x - zh.x));
        acc0 = cmacc(acc0, ak, ah);
        acc1 = cmacc(acc1, bk, bh);
    }
    acc0.x = warp_sum(acc0.x);
    acc0.y = warp_sum(acc0.y);
    acc1.x = warp_sum(acc1.x);
    acc1.y = warp_sum(acc1.y);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = acc0;
        red[1][threadIdx.x >> 5] = acc1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int h = threadIdx.x;
        float2 t = red[h][0];
        for (int i = 1; i < NT / 32; ++i) t = cadd(t, red[h][i]);
        if (j0 + h < a.J) a.c[j0 + h] = t;
    }
}

// 105-block averages, phases and unwrap steps, CTA b for blocks [128 b, 128 b + 128): one warp scans
// the CTA's 233 clock products (the tile, the block before it and 52 on either side; zero outside
// the frame, which clips the window at the frame edges) in FP64, so that each average is a
// difference of two tile-local prefix sums; the steps compare each phase with the one before.
constexpr int kWinTile = 128;
__global__ void __launch_bounds__(kWinTile) k_pam_window(PamArgs a) {
    constexpr int L = kWinTile + 1 + 2 * kAvgHalf;            // 233 products
    constexpr int CH = (L + 31) / 32;                         // per lane
    __shared__ double2 Q[L + 1];                              // Q[m] = sum of the first m products
    __shared__ double ph[kWinTile + 1];
    const int j0 = blockIdx.x * kWinTile;
    const int base = j0 - 1 - kAvgHalf;                       // block of tile product 0
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, m0 = lane * CH;
        double2 loc[CH];
        double2 s = make_double2(0.0, 0.0);
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int m = m0 + u, i = base + m;
            const float2 v = (m < L && i >= 0 && i < a.J) ? a.c[i] : make_float2(0.0f, 0.0f);
            s.x += (double)v.x;
            s.y += (double)v.y;
            loc[u] = s;
        }
        double2 inc = s;
        for (int o = 1; o < 32; o <<= 1) {
            const double nx = __shfl_up_sync(0xffffffffu, inc.x, o), ny = __shfl_up_sync(0xffffffffu, inc.y, o);
            if (lane >= o) {
                inc.x += nx;
                inc.y += ny;
            }
        }
        const double2 ex = make_double2(inc.x - s.x, inc.y - s.y);
        if (lane == 0) Q[0] = make_double2(0.0, 0.0);
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if (m0 + u < L) Q[m0 + u + 1] = make_double2(ex.x + loc[u].x, ex.y + loc[u].y);
    }
    __syncthreads();
    // ph[r] = phase of block j0 - 1 + r, whose window is tile products r .. r + 104
    for (int r = threadIdx.x; r <= kWinTile; r += kWinTile) {
        const int j = j0 - 1 + r;
        if (j >= 0 && j < a.J) {
            const double2 h = Q[r + 2 * kAvgHalf + 1], l = Q[r];
            ph[r] = atan2(h.y - l.y, h.x - l.x);
        }
    }
    __syncthreads();
    const int j = j0 + threadIdx.x;
    if (j < a.J) {
        const double p = ph[threadIdx.x + 1];
        a.phi[j] = (float)p;
        int st = 0;
        if (j > 0) {
            const double d = p - ph[threadIdx.x];
            st = d > M_PI ? -1 : (d < -M_PI ? 1 : 0);
        }
        a.step[j] = st;
    }
}

// One CTA of 1024 threads: winding numbers (integer prefix sum of the steps), output offsets
// j N/4 + w_j - w_0 (w_0 = 0) and the output count.
__global__ void __launch_bounds__(1024) k_pam_wind(PamArgs a, int quarter) {
    __shared__ int ipart[1024];
    const int t = threadIdx.x, J = a.J;
    const int per = (J + 1023) / 1024;
    const int lo = min(J, t * per), hi = min(J, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += a.step[i];
    ipart[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int v = t >= d ? ipart[t - d] : 0;
        __syncthreads();
        ipart[t] += v;
        __syncthreads();
    }
    int w = t > 0 ? ipart[t - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        w += a.step[i];
        a.w[i] = w;
        a.off[i] = (long long)i * quarter + w;
    }
    __syncthreads();
    if (t == 0) {
        // the last block outputs N/4 symbols, clipped to the frame's slots
        const int jl = J - 1;
        const long long n_last = min((long long)quarter, a.S / 2 - (long long)jl * quarter);
        a.off[J] = a.off[jl] + max(n_last, 0LL);
        *a.n_out = a.off[J];
    }
}

// the block pair again: split, each block's ramp exp(-j phi f / Rs) / N, recombined as
// Y = A R_2b + j B R_2b+1 so that one inverse transform gives block 2b's samples as its real part
// and block 2b + 1's as its imaginary part (both spectra stay Hermitian)
template <int K>
__global__ void __launch_bounds__(((1 << K) / 16 < 32) ? 32 : (1 << K) / 16) k_pam_correct(PamArgs a) {
    constexpr int N = 1 << K, HOP = N / 2, LEAD = N / 4;
    constexpr int NT = (N / 16 < 32) ? 32 : N / 16;
    extern __shared__ float2 sm[];
    const int j0 = 2 * blockIdx.x;
    const bool has1 = j0 + 1 < a.J;
    pam_pair_spectrum<K>(a, sm, (int64_t)j0 * HOP - LEAD);
    const float ph0 = a.phi[j0], ph1 = has1 ? a.phi[j0 + 1] : 0.0f;
    constexpr float inv_half = 2.0f / (float)N, inv_n = 1.0f / (float)N;
    for (int k = threadIdx.x; k <= N / 2; k += NT) {
        const int m = (N - k) & (N - 1);
        const float2 zk = sm[fft_pad(k)], zm = sm[fft_pad(m)];
        const float2 ak = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 bk = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
        const float ks = k < N / 2 ? (float)k : 0.0f;
        float s0, c0, s1, c1;
        __sincosf(-ph0 * ks * inv_half, &s0, &c0);    // |argument| <= pi
        __sincosf(-ph1 * ks * inv_half, &s1, &c1);
        const float2 p = cscale(cmul(ak, make_float2(c0, s0)), inv_n);
        const float2 q = cscale(cmul(bk, make_float2(c1, s1)), inv_n);
        sm[fft_pad(k)] = make_float2(p.x - q.y, p.y + q.x);                 // p + j q
        if (m != k) sm[fft_pad(m)] = make_float2(p.x + q.y, q.x - p.y);     // conj p + j conj q
    }
    __syncthreads();
    const long long o0 = a.off[j0], n0 = a.off[j0 + 1] - o0;
    const long long o1 = has1 ? a.off[j0 + 1] : 0, n1 = has1 ? a.off[j0 + 2] - o1 : 0;
    double bsum0 = 0.0, bsum1 = 0.0;                       // the blocks' outputs, for the mean
    auto store_out = [&](int idx, float2 v) {
        const int r = idx - LEAD;
        if (r >= 0 && !(r & 1)) {
            const int i = r >> 1;
            if (i < n0) {
                a.y[o0 + i] = v.x;
                bsum0 += (double)v.x;
            }
            if (i < n1) {
                a.y[o1 + i] = v.y;
                bsum1 += (double)v.y;
            }
        }
    };
    SmemLoad sl{sm};
    fft_run<K, +1, false, true>(sm, a.tw, sl, store_out);
    __shared__ double red[2][NT / 32];
    for (int o = 16; o; o >>= 1) {
        bsum0 += __shfl_xor_sync(0xffffffffu, bsum0, o);
        bsum1 += __shfl_xor_sync(0xffffffffu, bsum1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = bsum0;
        red[1][threadIdx.x >> 5] = bsum1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int h = threadIdx.x;
        double t = 0.0;
        for (int i = 0; i < NT / 32; ++i) t += red[h][i];
        if (j0 + h < a.J) a.part[j0 + h] = t;
    }
}

// sum of |y - mean| over CTA b's contiguous share of the outputs, four outputs per load where the
// share is aligned (the share boundaries are multiples of 4)
__global__ void __launch_bounds__(kRedThreads) k_pam_deviation(PamArgs a) {
    __shared__ double red[kRedThreads / 32];
    const long long n = *a.n_out;
    const long long per = ((n + kParts - 1) / kParts + 3) & ~3LL;
    const long long lo = min(n, (long long)blockIdx.x * per), hi = min(n, lo + per);
    const float mu = (float)a.stat[0];
    double s = 0.0;
    const long long v_hi = lo + ((hi - lo) & ~3LL);
    const float4* y4 = reinterpret_cast<const float4*>(a.y);
    for (long long i = lo + 4 * (long long)threadIdx.x; i < v_hi; i += 4 * kRedThreads) {
        const float4 v = y4[i >> 2];
        s += (double)(fabsf(v.x - mu) + fabsf(v.y - mu)) + (double)(fabsf(v.z - mu) + fabsf(v.w - mu));
    }
    for (long long i = v_hi + threadIdx.x; i < hi; i += kRedThreads) s += (double)fabsf(a.y[i] - mu);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kRedThreads / 32; ++i) t += red[i];
        a.part[a.J + blockIdx.x] = t;
    }
}

// stat[mode] = (sum of count partials from part + first) / outputs: one CTA of 1024 threads, a fixed
// order (strided per-thread sums, then a shuffle and shared-memory tree)
__global__ void __launch_bounds__(1024) k_pam_final(PamArgs a, int mode, int first, int count) {
    __shared__ double red[32];
    const long long n = *a.n_out;
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += 1024) s += a.part[first + i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = red[threadIdx.x];
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) a.stat[mode] = n > 0 ? t / (double)n : 0.0;
    }
}

__global__ void k_pam_decide(PamArgs a) {
    const long long n = *a.n_out;
    const float mu = (float)a.stat[0];
    const float g = a.stat[1] > 0.0 ? (float)(0.5 * a.M / a.stat[1]) : 0.0f;
    const float hm = 0.5f * (float)(a.M - 1), top = (float)(a.M - 1);
    auto level = [&](float y) -> uint8_t {
        const float l = rintf(fmaf(0.5f, (y - mu) * g, hm));
        return (uint8_t)fminf(fmaxf(l, 0.0f), top);
    };
    const long long n4 = n >> 2;
    const float4* y4 = reinterpret_cast<const float4*>(a.y);
    uchar4* l4 = reinterpret_cast<uchar4*>(a.levels);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 v = y4[i];
        l4[i] = make_uchar4(level(v.x), level(v.y), level(v.z), level(v.w));
    }
    for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        a.levels[i] = level(a.y[i]);
}

template <int K>
cudaError_t launch_pam_t(const PamArgs& a, cudaStream_t s) {
    constexpr int N = 1 << K;
    const int threads = N / 16 < 32 ? 32 : N / 16;
    const size_t smem = sizeof(float2) * fft_smem_elems(N);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_pam_clock<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_pam_correct<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int pairs = (a.J + 1) / 2;
    k_pam_clock<K><<<pairs, threads, smem, s>>>(a);
    k_pam_window<<<(a.J + kWinTile - 1) / kWinTile, kWinTile, 0, s>>>(a);
    k_pam_wind<<<1, 1024, 0, s>>>(a, N / 4);
    k_pam_correct<K><<<pairs, threads, smem, s>>>(a);
    k_pam_final<<<1, 1024, 0, s>>>(a, 0, 0, a.J);
    k_pam_deviation<<<kParts, kRedThreads, 0, s>>>(a);
    k_pam_final<<<1, 1024, 0, s>>>(a, 1, a.J, kParts);
    k_pam_decide<<<4 * 152, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pam(int K, const PamArgs& a, cudaStream_t s) {
    switch (K) {
        case 10: return launch_pam_t<10>(a, s);
        case 11: return launch_pam_t<11>(a, s);
        case 12: return launch_pam_t<12>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

extern "C" {

rx_status rx_pam_create(int32_t fft_size, int32_t levels, double rrc_rolloff, float code_scale, float dc_offset,
                        int64_t max_samples, rx_pam** out) {
    if (!out) return RX_EINVAL;
    *out = nullptr;
    int K = 0;
    while (K < 14 && (1 << K) < fft_size) ++K;
    if ((1 << K) != fft_size || K < 10 || K > 12) return RX_EINVAL;
    if (levels != 2 && levels != 4 && levels != 8) return RX_EINVAL;
    if (!(rrc_rolloff > 0.0 && rrc_rolloff <= 1.0)) return RX_EINVAL;
    if (!std::isfinite(code_scale) || code_scale == 0.0f || !std::isfinite(dc_offset)) return RX_EINVAL;
    if (max_samples < 2 || max_samples > ((int64_t)1 << 30)) return RX_EINVAL;
    rx_pam* p = new (std::nothrow) rx_pam();
    if (!p) return RX_ENOMEM;
    p->K = K;
    p->M = levels;
    p->max_samples = max_samples;
    p->scale = code_scale;
    p->dc = dc_offset;
    const int N = 1 << K;
    const int64_t J = (max_samples + N / 2 - 1) / (N / 2);
    // sqrt(2) RRC(f_k), f_k the signed bin frequency in cycles per sample, symbol rate 1/2
    std::vector<float> H(N);
    const double lo = (1.0 - rrc_rolloff) / 4.0, hi = (1.0 + rrc_rolloff) / 4.0;
    for (int i = 0; i < N; ++i) {
        const double f = std::fabs((double)(i < N / 2 ? i : i - N) / (double)N);
        const double amp = f <= lo ? 1.0 : (f <= hi ? std::cos(M_PI / rrc_rolloff * (f - lo)) : 0.0);
        H[i] = (float)(std::sqrt(2.0) * amp);
    }
    bool ok = cudaMalloc(&p->tw, sizeof(float2) * RX_FFT_TW_N) == cudaSuccess &&
              cudaMalloc(&p->H, sizeof(float) * N) == cudaSuccess &&
              cudaMalloc(&p->c, sizeof(float2) * J) == cudaSuccess &&
              cudaMalloc(&p->phi, sizeof(float) * J) == cudaSuccess &&
              cudaMalloc(&p->step, sizeof(int) * J) == cudaSuccess &&
              cudaMalloc(&p->w, sizeof(int) * J) == cudaSuccess &&
              cudaMalloc(&p->off, sizeof(long long) * (J + 1)) == cudaSuccess &&
              cudaMalloc(&p->part, sizeof(double) * (J + kParts)) == cudaSuccess &&
              cudaMalloc(&p->stat, sizeof(double) * 2) == cudaSuccess;
    if (ok)
        ok = launch_fill_twiddles(p->tw, 0) == cudaSuccess &&
             cudaMemcpy(p->H, H.data(), sizeof(float) * N, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        rx_pam_destroy(p);
        return RX_ENOMEM;
    }
    *out = p;
    return RX_OK;
}

rx_status rx_pam_process(rx_pam* p, const uint16_t* d_codes, int64_t n_samples, float* d_y, uint8_t* d_levels,
                         int64_t* d_n_out, rx_stream_t stream) {
    if (!p || !d_codes || !d_y || !d_levels || !d_n_out) return RX_EINVAL;
    // outputs are read four at a time
    if ((reinterpret_cast<uintptr_t>(d_y) & 15) || (reinterpret_cast<uintptr_t>(d_levels) & 3)) return RX_EINVAL;
    if (n_samples < 2 || (n_samples & 1) || n_samples > p->max_samples) return RX_EINVAL;
    const int N = 1 << p->K;
    PamArgs a;
    a.codes = d_codes;
    a.S = n_samples;
    a.J = (int)((n_samples + N / 2 - 1) / (N / 2));
    a.scale = p->scale;
    a.dc = p->dc;
    a.tw = p->tw;
    a.H = p->H;
    a.c = p->c;
    a.phi = p->phi;
    a.step = p->step;
    a.w = p->w;
    a.off = p->off;
    a.y = d_y;
    a.levels = d_levels;
    a.part = p->part;
    a.stat = p->stat;
    a.n_out = reinterpret_cast<long long*>(d_n_out);
    a.M = p->M;
    return launch_pam(p->K, a, (cudaStream_t)stream) == cudaSuccess ? RX_OK : RX_ECUDA;
}

rx_status rx_pam_get(rx_pam* p, int32_t which, void* d_dst, int64_t bytes, rx_stream_t stream) {
    if (!p || !d_dst || bytes < 0) return RX_EINVAL;
    const int64_t J = (p->max_samples + (1 << p->K) / 2 - 1) / ((1 << p->K) / 2);
    const void* src = nullptr;
    int64_t have = 0;
    switch (which) {
        case RX_PAM_CLOCK: src = p->c; have = (int64_t)sizeof(float2) * J; break;
        case RX_PAM_PHASE: src = p->phi; have = (int64_t)sizeof(float) * J; break;
        case RX_PAM_WINDING: src = p->w; have = (int64_t)sizeof(int) * J; break;
        case RX_PAM_OFFSETS: src = p->off; have = (int64_t)sizeof(long long) * (J + 1); break;
        case RX_PAM_STATS: src = p->stat; have = (int64_t)sizeof(double) * 2; break;
        default: return RX_EINVAL;
    }
    if (bytes > have) return RX_EINVAL;
    return cudaMemcpyAsync(d_dst, src, (size_t)bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) == cudaSuccess
               ? RX_OK
               : RX_ECUDA;
}

void rx_pam_destroy(rx_pam* p) {
    if (!p) return;
    void* ptrs[] = {p->tw, p->H, p->c, p->phi, p->step, p->w, p->off, p->part, p->stat};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

}  // extern "C"
