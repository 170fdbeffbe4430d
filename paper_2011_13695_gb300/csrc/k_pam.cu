// IM/DD PAM-M chain with frequency-domain clock recovery (Sec. III, Steps 1-9) and its C entry points.
//
// At 2 samples/symbol, overlap-save blocks of N = 2^K samples (block j from j N/2 - N/4, zero
// outside the frame), one CTA per block, the in-CTA Stockham FFT of rx_fft.cuh:
//   k_pam_clock<K>    code -> v = scale code + dc -> FFT -> times sqrt(2) RRC(f) -> the block's
//                     clock product c_j = sum_{k < N/2} X[k] conj(X[k + N/2]) (spectral line one
//                     symbol rate apart; its phase is -2 pi Rs tau for a delay tau);
//   k_pam_average     cbar_j = sum of c_i over |i - j| <= 52 inside the frame (FP64), phi_j =
//                     arg cbar_j, and the unwrap step of block j: -1 if phi_j - phi_{j-1} > pi,
//                     +1 if < -pi;
//   k_pam_scan        one CTA: winding numbers w_j (integer prefix sum of the steps), each block's
//                     output count N/4 + w_{j+1} - w_j (N/4 for the last block, clipped to the
//                     frame) and output offset;
//   k_pam_correct<K>  the FFT again (recomputing is cheaper than a 64 MB spectrum round trip),
//                     times sqrt(2) RRC(f) exp(-j phi_j f / Rs) / N, inverse FFT; the block's
//                     outputs are the real parts of its samples N/4 + 2 i, written at its offset
//                     (variable rate: 255, 256 or 257 symbols per block);
//   k_pam_partial, k_pam_final   buffer-wise mean, then mean absolute deviation (fixed-order
//                     two-stage reductions, so results do not depend on scheduling);
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
    double* part = nullptr;      // [2][kParts] partial sums
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

template <int K>
__global__ void __launch_bounds__(((1 << K) / 16 < 32) ? 32 : (1 << K) / 16) k_pam_clock(PamArgs a) {
    constexpr int N = 1 << K, HOP = N / 2, LEAD = N / 4;
    constexpr int NT = (N / 16 < 32) ? 32 : N / 16;
    extern __shared__ float2 sm[];
    __shared__ float2 red[NT / 32];
    const int j = blockIdx.x;
    const int64_t start = (int64_t)j * HOP - LEAD;
    auto load = [&](int idx) -> float2 {
        const int64_t s = start + idx;
        return make_float2((s >= 0 && s < a.S) ? fmaf(a.scale, (float)a.codes[s], a.dc) : 0.0f, 0.0f);
    };
    const float* __restrict__ H = a.H;
    auto store = [&](int k, float2 v) { sm[fft_pad(k)] = cscale(v, __ldg(&H[k])); };
    fft_run<K, -1, true, true>(sm, a.tw, load, store);
    __syncthreads();
    float2 acc = make_float2(0.0f, 0.0f);
    for (int k = threadIdx.x; k < N / 2; k += NT) acc = cmacc(acc, sm[fft_pad(k)], sm[fft_pad(k + N / 2)]);
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = red[0];
        for (int i = 1; i < NT / 32; ++i) t = cadd(t, red[i]);
        a.c[j] = t;
    }
}

__global__ void k_pam_average(PamArgs a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.J) return;
    auto avg_phase = [&](int jj) -> double {
        double re = 0.0, im = 0.0;
        const int lo = max(0, jj - kAvgHalf), hi = min(a.J - 1, jj + kAvgHalf);
        for (int i = lo; i <= hi; ++i) {
            const float2 v = a.c[i];
            re += (double)v.x;
            im += (double)v.y;
        }
        return atan2(im, re);
    };
    const double p = avg_phase(j);
    a.phi[j] = (float)p;
    int s = 0;
    if (j > 0) {
        const double d = p - avg_phase(j - 1);
        s = d > M_PI ? -1 : (d < -M_PI ? 1 : 0);
    }
    a.step[j] = s;
}

// one CTA of 1024 threads: w = inclusive prefix sum of the steps, counts, offsets
__global__ void __launch_bounds__(1024) k_pam_scan(PamArgs a) {
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (a.J + 1023) / 1024;
    const int lo = min(a.J, t * per), hi = min(a.J, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += a.step[i];
    part[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = t > 0 ? part[t - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        run += a.step[i];
        a.w[i] = run;
    }
}

__global__ void k_pam_offsets(PamArgs a, int quarter) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > a.J) return;
    const long long w0 = a.w[0];
    const long long slots = a.S / 2;
    if (j < a.J) {
        a.off[j] = (long long)j * quarter + a.w[j] - w0;
    } else {
        // the last block outputs N/4 symbols, clipped to the frame's slots
        const int jl = a.J - 1;
        const long long n_last = min((long long)quarter, slots - (long long)jl * quarter);
        a.off[a.J] = (long long)jl * quarter + a.w[jl] - w0 + max(n_last, 0LL);
        *a.n_out = a.off[a.J];
    }
}

template <int K>
__global__ void __launch_bounds__(((1 << K) / 16 < 32) ? 32 : (1 << K) / 16) k_pam_correct(PamArgs a) {
    constexpr int N = 1 << K, HOP = N / 2, LEAD = N / 4;
    extern __shared__ float2 sm[];
    const int j = blockIdx.x;
    const int64_t start = (int64_t)j * HOP - LEAD;
    auto load = [&](int idx) -> float2 {
        const int64_t s = start + idx;
        return make_float2((s >= 0 && s < a.S) ? fmaf(a.scale, (float)a.codes[s], a.dc) : 0.0f, 0.0f);
    };
    const float* __restrict__ H = a.H;
    const float ph = a.phi[j];
    constexpr float inv_half = 2.0f / (float)N;
    auto store = [&](int k, float2 v) {
        const int ks = k < N / 2 ? k : (k == N / 2 ? 0 : k - N);
        float sn, cs;
        sincosf(-ph * (float)ks * inv_half, &sn, &cs);
        sm[fft_pad(k)] = cscale(cmul(v, make_float2(cs, sn)), __ldg(&H[k]) * (1.0f / (float)N));
    };
    fft_run<K, -1, true, true>(sm, a.tw, load, store);
    __syncthreads();
    const long long o0 = a.off[j];
    const long long n = a.off[j + 1] - o0;
    auto store_out = [&](int idx, float2 v) {
        const int r = idx - LEAD;
        if (r >= 0 && !(r & 1) && (r >> 1) < n) a.y[o0 + (r >> 1)] = v.x;
    };
    SmemLoad sl{sm};
    fft_run<K, +1, false, true>(sm, a.tw, sl, store_out);
}

// stage 1: CTA b sums its contiguous share of the outputs (mode 0: y; mode 1: |y - mean|)
__global__ void __launch_bounds__(kRedThreads) k_pam_partial(PamArgs a, int mode) {
    __shared__ double red[kRedThreads / 32];
    const long long n = *a.n_out;
    const long long per = (n + kParts - 1) / kParts;
    const long long lo = min(n, (long long)blockIdx.x * per), hi = min(n, lo + per);
    const double mu = mode ? a.stat[0] : 0.0;
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kRedThreads) {
        const double v = (double)a.y[i];
        s += mode ? fabs(v - mu) : v;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kRedThreads / 32; ++i) t += red[i];
        a.part[mode * kParts + blockIdx.x] = t;
    }
}

// stage 2: one warp adds the partials in a fixed order
__global__ void k_pam_final(PamArgs a, int mode) {
    const long long n = *a.n_out;
    double s = 0.0;
    for (int i = threadIdx.x; i < kParts; i += 32) s += a.part[mode * kParts + i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) a.stat[mode] = n > 0 ? s / (double)n : 0.0;
}

__global__ void k_pam_decide(PamArgs a) {
    const long long n = *a.n_out;
    const float mu = (float)a.stat[0];
    const float g = a.stat[1] > 0.0 ? (float)(0.5 * a.M / a.stat[1]) : 0.0f;
    const float hm = 0.5f * (float)(a.M - 1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float u = (a.y[i] - mu) * g;
        const float l = rintf(fmaf(0.5f, u, hm));
        a.levels[i] = (uint8_t)fminf(fmaxf(l, 0.0f), (float)(a.M - 1));
    }
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
    k_pam_clock<K><<<a.J, threads, smem, s>>>(a);
    k_pam_average<<<(a.J + 255) / 256, 256, 0, s>>>(a);
    k_pam_scan<<<1, 1024, 0, s>>>(a);
    k_pam_offsets<<<(a.J + 1 + 255) / 256, 256, 0, s>>>(a, N / 4);
    k_pam_correct<K><<<a.J, threads, smem, s>>>(a);
    k_pam_partial<<<kParts, kRedThreads, 0, s>>>(a, 0);
    k_pam_final<<<1, 32, 0, s>>>(a, 0);
    k_pam_partial<<<kParts, kRedThreads, 0, s>>>(a, 1);
    k_pam_final<<<1, 32, 0, s>>>(a, 1);
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
              cudaMalloc(&p->part, sizeof(double) * 2 * kParts) == cudaSuccess &&
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
