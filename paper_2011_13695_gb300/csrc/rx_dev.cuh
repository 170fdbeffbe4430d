// Device-side declarations shared by the librx translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define RX_TMAX 63          // largest tap count
#define RX_MAX_DELAY 64     // largest alignment search half-width
#define RX_BPS_MAXB 64      // largest number of BPS test phases

// State the chain carries on the device between kernels and between frames.
struct RxDevState {
    float scale[2];                   // A0 per-polarisation scale
    int32_t fo_code;                  // A3 quantised frequency offset
    int32_t fo_valid;
    long long nco_inc;                // A3 phase increment per sample, 2^-64 turns (two's complement)
    double fo_w;                      // A3 unquantised estimate [rad/symbol]
    double fo_margin;                 // distance of the estimate to a rounding boundary [grid steps]
    int32_t coarse_bin;               // A3 periodogram peak (signed)
    int32_t cma_reran;
    float cma_rho;
    float pad0;
    float2 taps_cma[4 * RX_TMAX];     // [q][p][k] after CMA
    float2 taps_init[4 * RX_TMAX];    // taps every segment starts from
    float2 taps_last[4 * RX_TMAX];    // final taps of the last segment
    int32_t m_prev[2];                // A5 unwrap carry
    int32_t b_prev[2];                // A5 last b* (-1 = none)
    int32_t sync_valid;
    int32_t sync_p[2], sync_r[2], sync_d[2], sync_match[2];
    int32_t sync_len;
    uint32_t err_word;
    unsigned long long bits, bit_errors, symbols, symbol_errors;
    unsigned long long evm_num_fx, evm_den_fx;   // EVM sums in units of 2^-28 (integer atomics)
};

// -------------------------------------------------------------------------
// complex helpers (float2 = I, Q)
// -------------------------------------------------------------------------
// Programmatic dependent launch. A kernel that lets the stream's next kernel (launched with launch_pdl)
// become resident while it runs calls pdl_trigger; a kernel launched with launch_pdl calls pdl_wait before
// its first access to anything the stream's previous kernel writes or reads: after it, that kernel has
// completed and its writes are visible. Both are no-ops for ordinary launches.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float2 cmac(float2 acc, float2 a, float2 b) {  // acc + a*b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cmacc(float2 acc, float2 a, float2 b) {  // acc + a*conj(b)
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.y, b.x, acc.y);
    acc.y = fmaf(-a.x, b.y, acc.y);
    return acc;
}

// -------------------------------------------------------------------------
// Gray square QAM (unit average energy): L levels per dimension at
// (2l - (L-1)) * a, a = 1 / sqrt(2 (M-1) / 3).
// -------------------------------------------------------------------------
struct Qam {
    int L;        // levels per dimension
    int m;        // bits per symbol
    float a;      // half level spacing
    float half_inv_a;  // 0.5 / a
    float hL;     // (L - 1) / 2
};

// a and 1/(2a) are the FP32 roundings of the FP64 values of 1/sqrt(2(M-1)/3) and sqrt(2(M-1)/3)/2,
// written out for M = 4, 16, 64, 256 so that device code takes no FP64 arithmetic (a small fraction
// of the FP32 rate on this part); other M compute them.
__host__ __device__ inline Qam make_qam(int m) {
    Qam q;
    q.m = m;
    q.L = 1 << (m / 2);
    q.hL = 0.5f * (float)(q.L - 1);
    switch (m) {
        case 2: q.a = 0x1.6a09e6p-1f; q.half_inv_a = 0x1.6a09e6p-1f; break;
        case 4: q.a = 0x1.43d136p-2f; q.half_inv_a = 0x1.94c584p+0f; break;
        case 6: q.a = 0x1.3c0366p-3f; q.half_inv_a = 0x1.9ec474p+1f; break;
        case 8: q.a = 0x1.3a261cp-4f; q.half_inv_a = 0x1.a13a9cp+2f; break;
        default: {
            const int M = q.L * q.L;
            q.a = (float)(1.0 / sqrt(2.0 * (M - 1) / 3.0));
            q.half_inv_a = (float)(0.5 * sqrt(2.0 * (M - 1) / 3.0));
        }
    }
    return q;
}

// nearest level index of one real dimension
__device__ __forceinline__ int qam_level(float u, const Qam& q) {
    float t = rintf(fmaf(u, q.half_inv_a, q.hL));
    t = fminf(fmaxf(t, 0.0f), (float)(q.L - 1));
    return (int)t;
}
__device__ __forceinline__ float qam_value(int l, const Qam& q) {
    return (float)(2 * l - (q.L - 1)) * q.a;
}
__device__ __forceinline__ float2 qam_decide(float2 z, const Qam& q) {
    return make_float2(qam_value(qam_level(z.x, q), q), qam_value(qam_level(z.y, q), q));
}
// Gray bits of the decision, MSB of the I word in bit m-1 of the result
__device__ __forceinline__ uint32_t qam_bits(int li, int lq, const Qam& q) {
    int h = q.m / 2;
    uint32_t gi = (uint32_t)(li ^ (li >> 1));
    uint32_t gq = (uint32_t)(lq ^ (lq >> 1));
    return (gi << h) | gq;
}
// bit-reverse the m bits so that the first transmitted bit sits in bit 0
__device__ __forceinline__ uint32_t msb_first_to_stream(uint32_t v, int m) {
    return __brev(v) >> (32 - m);
}

// -------------------------------------------------------------------------
// 64-bit fixed-point phase accumulator: phase(g) = frac(inc * g) turns,
// returns exp(-j 2 pi phase).
// -------------------------------------------------------------------------
__device__ __forceinline__ float2 nco_conj(long long inc, long long g) {
    unsigned long long ph = (unsigned long long)inc * (unsigned long long)g;
    int top = (int)(ph >> 32);                       // [-2^31, 2^31) = [-0.5, 0.5) turns
    float half_turns = (float)top * 4.656612873077393e-10f;   // 2 * top / 2^32, in [-1, 1)
    float s, c;
    sincospif(half_turns, &s, &c);
    return make_float2(c, -s);
}

// Principal square root of a unit complex number (c, s), arg in (-pi, pi] -> arg / 2 in (-pi/2, pi/2],
// in the cancellation-free form for either sign of c: with v = (1 + |c|) / 2 in [1/2, 1] and
// r = 1 / sqrt(v), the larger component is v r = sqrt(v) and the smaller |s| / (2 sqrt(v)) = |s| r / 2.
__device__ __forceinline__ float2 unit_sqrt(float2 u) {
    const float v = 0.5f * (1.0f + fabsf(u.x));
    const float r = rsqrtf(v);
    if (u.x >= 0.0f) return make_float2(v * r, 0.5f * u.y * r);
    return make_float2(0.5f * fabsf(u.y) * r, copysignf(v * r, u.y));
}

// exp(-j psi) with psi = arg(w) / 4, arg in (-pi, pi]: the conjugate of the principal fourth root of
// w / |w|, as two principal square roots. A zero w takes atan2's signed-zero arguments (0 for
// x = +0, +-pi for x = -0 by the sign of y).
__device__ __forceinline__ float2 quarter_root_conj(float2 w) {
    const float n2 = cabs2(w);
    if (!(n2 > 0.0f)) {
        if (!signbit(w.x)) return make_float2(1.0f, 0.0f);
        return make_float2(0.70710678118654752f, signbit(w.y) ? 0.70710678118654752f : -0.70710678118654752f);
    }
    const float inv = rsqrtf(n2);
    const float2 r = unit_sqrt(unit_sqrt(make_float2(w.x * inv, w.y * inv)));
    return make_float2(r.x, -r.y);
}

#define RX_EVM_FX_SCALE 268435456.0f                // 2^28

// block-wide helpers
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
