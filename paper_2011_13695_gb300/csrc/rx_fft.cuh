// In-CTA complex FFT of N = 2^K points, K in [9, 14], FP32.
//
// Stockham autosort formulation (Stockham 1966; the GPU form of Govindaraju
// et al., SC 2008): every pass reads all N points with the stride N/R,
// twiddles and transforms R of them in registers, and writes them back so
// that the last pass leaves the spectrum in natural order. Radix-16 passes
// come first and one radix-2/4/8 pass last when K is not a multiple of 4.
// N/16 threads take part; each holds 16 points between passes. Shared memory
// holds one padded copy (index i stored at i + i/16) and every pass reads
// all points into registers before any thread overwrites them. A radix-16
// pass reads two twiddles of the table (W^k and W^4k) and forms the other
// thirteen by complex products (at most four roundings deep), instead of
// fifteen scattered table reads. The first
// pass can read through a functor (from global memory) and the last can
// write through one (to global memory), so the transform costs no extra
// global round trip.
#pragma once

#include "rx_dev.cuh"

#define RX_FFT_TW_LOG2 14
#define RX_FFT_TW_N (1 << RX_FFT_TW_LOG2)   // twiddle table: exp(-2 pi i t / 16384)

__host__ __device__ constexpr int fft_pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int fft_smem_elems(int n) { return n + n / 16; }

// multiply by DIR * i
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int DIR>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2* v) {
    float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    float2 s13 = cadd(v[1], v[3]), d13 = mul_i<DIR>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}

template <int DIR>
__device__ __forceinline__ void dft8(float2* v) {
    const float r2 = 0.70710678118654752f;
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft4<DIR>(e);
    dft4<DIR>(o);
    // W8^k = (cos(2 pi k/8), DIR sin(2 pi k/8))
    float2 w1 = make_float2(r2, DIR * r2), w3 = make_float2(-r2, DIR * r2);
    float2 t0 = o[0], t1 = cmul(o[1], w1), t2 = mul_i<DIR>(o[2]), t3 = cmul(o[3], w3);
    v[0] = cadd(e[0], t0); v[4] = csub(e[0], t0);
    v[1] = cadd(e[1], t1); v[5] = csub(e[1], t1);
    v[2] = cadd(e[2], t2); v[6] = csub(e[2], t2);
    v[3] = cadd(e[3], t3); v[7] = csub(e[3], t3);
}

template <int DIR>
__device__ __forceinline__ void dft16(float2* v) {
    // cos and sin of 2 pi k / 16, k = 0..7
    const float C[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f,
                        0.0f, -0.38268343236508978f, -0.70710678118654752f, -0.92387953251128674f};
    const float S[8] = {0.0f, 0.38268343236508978f, 0.70710678118654752f, 0.92387953251128674f,
                        1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f};
    float2 e[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    dft8<DIR>(e);
    dft8<DIR>(o);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float2 t = (k == 0) ? o[0] : cmul(o[k], make_float2(C[k], DIR * S[k]));
        v[k] = cadd(e[k], t);
        v[k + 8] = csub(e[k], t);
    }
}

template <int R, int DIR>
__device__ __forceinline__ void dftR(float2* v) {
    if constexpr (R == 2) dft2<DIR>(v[0], v[1]);
    else if constexpr (R == 4) dft4<DIR>(v);
    else if constexpr (R == 8) dft8<DIR>(v);
    else dft16<DIR>(v);
}

// Twiddle sources: entry t of the table exp(-2 pi i t / RX_FFT_TW_N) from global memory, or from a
// shared copy of every 2^shift-th entry (the only ones an N-point transform reads have t a multiple of
// RX_FFT_TW_N / N).
struct TwGlobal {
    const float2* __restrict__ p;
    __device__ float2 operator()(int t) const { return __ldg(&p[t]); }
};
struct TwShared {
    const float2* p;
    int shift;
    __device__ float2 operator()(int t) const { return p[t >> shift]; }
};

// One Stockham pass. SRC/DST: 0 = shared memory, 1 = functor.
template <int N, int R, int DIR, int SRC, int DST, class Load, class Store, class Tw>
__device__ __forceinline__ void fft_pass(float2* sm, int Ns, const Tw& tw, const Load& load, const Store& store) {
    constexpr int P = N / 16;
    constexpr int BPT = 16 / R;
    const int tid = threadIdx.x;
    float2 v[BPT][R];
    if (tid < P) {
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int j = tid + b * P;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int idx = j + r * (N / R);
                v[b][r] = SRC ? load(idx) : sm[fft_pad(idx)];
            }
        }
    }
    if (!SRC) __syncthreads();
    if (tid < P) {
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int j = tid + b * P;
            const int k = j & (Ns - 1);
            if (Ns > 1) {
                const int step = (RX_FFT_TW_N / (Ns * R)) * k;
                if constexpr (R == 16) {
                    float2 w[16];
                    w[1] = tw(step);
                    w[4] = tw(4 * step);
                    if (DIR > 0) { w[1].y = -w[1].y; w[4].y = -w[4].y; }
                    w[2] = cmul(w[1], w[1]);
                    w[3] = cmul(w[2], w[1]);
                    w[5] = cmul(w[4], w[1]);
                    w[6] = cmul(w[4], w[2]);
                    w[7] = cmul(w[4], w[3]);
                    w[8] = cmul(w[4], w[4]);
#pragma unroll
                    for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
#pragma unroll
                    for (int r = 1; r < 16; ++r) v[b][r] = cmul(v[b][r], w[r]);
                } else {
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        float2 w = tw(step * r);
                        if (DIR > 0) w.y = -w.y;
                        v[b][r] = cmul(v[b][r], w);
                    }
                }
            }
            dftR<R, DIR>(v[b]);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int idx = base + r * Ns;
                if (DST) store(idx, v[b][r]);
                else sm[fft_pad(idx)] = v[b][r];
            }
        }
    }
    if (!DST) __syncthreads();
}

struct SmemLoad {
    const float2* sm;
    __device__ float2 operator()(int i) const { return sm[fft_pad(i)]; }
};
struct SmemStore {
    float2* sm;
    __device__ void operator()(int i, float2 v) const { sm[fft_pad(i)] = v; }
};

// Full transform. FIRST_FROM_FN: the first pass reads load(idx);
// LAST_TO_FN: the last pass writes store(idx, value) (natural order).
// Otherwise data comes from / goes to shared memory. Must be called by all
// threads of the block (blockDim.x >= N/16).
template <int K, int DIR, bool FIRST_FROM_FN, bool LAST_TO_FN, class Load, class Store, class Tw>
__device__ __forceinline__ void fft_run_tw(float2* sm, const Tw& tw, const Load& load, const Store& store) {
    constexpr int N = 1 << K;
    constexpr int NR16 = K / 4;
    constexpr int REM = K % 4;
    constexpr int NPASS = NR16 + (REM ? 1 : 0);
    SmemLoad sl{sm};
    SmemStore ss{sm};
    int Ns = 1;
#pragma unroll
    for (int p = 0; p < NPASS; ++p) {
        const bool first = (p == 0), last = (p == NPASS - 1);
        const bool small = (REM && last);
        if (small) {
            constexpr int R = 1 << (REM ? REM : 1);
            if (first && FIRST_FROM_FN) {
                if (LAST_TO_FN) fft_pass<N, R, DIR, 1, 1>(sm, Ns, tw, load, store);
                else fft_pass<N, R, DIR, 1, 0>(sm, Ns, tw, load, ss);
            } else {
                if (LAST_TO_FN) fft_pass<N, R, DIR, 0, 1>(sm, Ns, tw, sl, store);
                else fft_pass<N, R, DIR, 0, 0>(sm, Ns, tw, sl, ss);
            }
            Ns *= R;
        } else {
            if (first && FIRST_FROM_FN) {
                if (last && LAST_TO_FN) fft_pass<N, 16, DIR, 1, 1>(sm, Ns, tw, load, store);
                else fft_pass<N, 16, DIR, 1, 0>(sm, Ns, tw, load, ss);
            } else {
                if (last && LAST_TO_FN) fft_pass<N, 16, DIR, 0, 1>(sm, Ns, tw, sl, store);
                else fft_pass<N, 16, DIR, 0, 0>(sm, Ns, tw, sl, ss);
            }
            Ns *= 16;
        }
    }
}

template <int K, int DIR, bool FIRST_FROM_FN, bool LAST_TO_FN, class Load, class Store>
__device__ __forceinline__ void fft_run(float2* sm, const float2* __restrict__ tw, const Load& load,
                                        const Store& store) {
    fft_run_tw<K, DIR, FIRST_FROM_FN, LAST_TO_FN>(sm, TwGlobal{tw}, load, store);
}
