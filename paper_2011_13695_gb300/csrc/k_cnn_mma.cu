// The 64 -> 64 convolutions of the learned post-equaliser's forward pass on the
// tensor cores: BF16 x BF16 products, FP32 accumulation (mma.sync m16n8k16).
//
// As a matrix product, out[co][t] = sum_K A[co][K] B[K][t] with K = (k, ci) in
// the order k * 64 + ci: A[co][k*64 + ci] = W[co][ci][k] and
// B[k*64 + ci][t] = x[ci][t + k - 4]. A CTA computes all 64 output channels
// of 128 positions per tile and loops over tiles (one resident wave of CTAs):
// it keeps the layer's BF16 weights in shared memory, in rows of
// (k, ci) padded to 584 entries so that the 8 rows an ldmatrix reads fall in
// distinct banks (copied from a BF16 copy in that order that the weight
// update writes); per tile it stages the input positions t0 - 4 .. t0 + 132
// transposed to [position][channel] (rows of 72 entries), so that the B
// fragment of tap k is an ldmatrix of rows shifted by k, loading the next
// tile into registers while the current one computes. Eight warps take
// 32 x 32 output blocks (2 x 4 mma tiles, 36 K-steps of 16). The epilogue adds
// the bias, applies the ReLU, rounds to BF16 and writes the activation plane.
//
// The same product gives the layer's data gradient in the backward pass:
// din[ci][t] = sum_{k', co} W[co][ci][8 - k'] dout[co][t + k' - 4], i.e. the
// weights' flipped transpose as A (rows ci, K = (k', co)) and the BF16 copy of
// the gradient planes as B; that epilogue multiplies by the forward ReLU's
// derivative (the layer's input activation > 0) and writes FP32 gradient planes
// (and a BF16 copy for the next layer's data gradient).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "rx_cnn.h"

namespace {

constexpr int C = 64;              // channels in and out
constexpr int KW = 9;
constexpr int PAD = KW / 2;
constexpr int TT = 128;            // positions per tile
constexpr int NTHR = 256;          // 8 warps
constexpr int KTOT = C * KW;       // 576
constexpr int WS = KTOT + 8;       // weight row stride (bf16)
constexpr int XR = TT + 2 * PAD;   // staged positions per tile
constexpr int XS = C + 8;          // staged row stride (bf16)
constexpr int OS = TT + 8;         // output tile row stride (bf16), over the staging rows
static_assert(C * OS <= XR * XS, "the output tile fits over the staged input");
constexpr size_t SMEM = sizeof(__nv_bfloat16) * ((size_t)C * WS + (size_t)XR * XS);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int CH = XR / 8;                                 // 16-byte chunks per channel and tile
constexpr int NCH = (C * CH + NTHR - 1) / NTHR;            // chunks per thread

template <int EPI>                             // 0: forward (bias, ReLU, BF16); 1: data gradient (mask, FP32)
__global__ void __launch_bounds__(NTHR, 2) k_conv64_mma(const __nv_bfloat16* __restrict__ x, int64_t Tp, int64_t T,
                                                        const __nv_bfloat16* __restrict__ Wm,
                                                        const float* __restrict__ bias,
                                                        __nv_bfloat16* __restrict__ act_out, int vec,
                                                        const __nv_bfloat16* __restrict__ mask,
                                                        float* __restrict__ gout, __nv_bfloat16* __restrict__ gout16) {
    extern __shared__ float4 smem4[];
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(smem4);      // [C][WS]
    __nv_bfloat16* Xs = Ws + C * WS;                                  // [XR][XS]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;                          // 2 x 4 warps of 32 x 32
    const int g = lane >> 2, tq = lane & 3;

    // weights, once: rows of KTOT BF16 copied into rows of WS
    for (int i = tid; i < C * (KTOT / 8); i += NTHR) {
        const int co = i / (KTOT / 8), u = i - co * (KTOT / 8);
        *reinterpret_cast<uint4*>(Ws + co * WS + 8 * u) = *reinterpret_cast<const uint4*>(Wm + co * KTOT + 8 * u);
    }
    float bco[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    if constexpr (EPI == 0) {
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int h = 0; h < 2; ++h) bco[mi][h] = bias[wm * 32 + mi * 16 + g + 8 * h];
    }

    // ldmatrix row addresses: A rows co0 + (lane % 16), column block (lane / 16) * 8;
    // B^T rows n = (lane / 16) * 8 + lane % 8 of an n-tile pair, column block ((lane / 8) % 2) * 8
    const uint32_t a_base = smem_addr(Ws + (wm * 32 + (lane & 15)) * WS + (lane >> 4) * 8);
    const int bn = (lane >> 4) * 8 + (lane & 7), bk = ((lane >> 3) & 1) * 8;
    const uint32_t b_base = smem_addr(Xs + (wn * 32 + bn) * XS + bk);

    // Staging: chunk i = u * C + ci holds x[ci][t0 + 8u .. t0 + 8u + 8) (padded index); consecutive
    // threads take consecutive channels, so the transposed 2-byte stores Xs[8u + e][ci] of a warp are
    // consecutive. The next tile's chunks are loaded into registers while the current tile computes.
    uint4 pre[NCH];
    auto fetch = [&](int64_t t0) {
#pragma unroll
        for (int r = 0; r < NCH; ++r) {
            const int i = tid + r * NTHR;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (i < C * CH) {
                const int u = i / C, ci = i - u * C;
                const int64_t tp = t0 + 8 * u;
                const __nv_bfloat16* src = x + (int64_t)ci * Tp + tp;
                if (vec && tp + 7 < Tp) {
                    v = __ldg(reinterpret_cast<const uint4*>(src));
                } else {
                    __nv_bfloat16 tmp[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) tmp[e] = tp + e < Tp ? src[e] : __float2bfloat16_rn(0.0f);
                    v = *reinterpret_cast<const uint4*>(tmp);
                }
            }
            pre[r] = v;
        }
    };
    // two neighbouring channels swap halves with one shuffle, so that each stores bf16 pairs
    // (ci, ci + 1) of 4 positions as 32-bit words: the even lane positions 0..3, the odd lane 4..7
    auto stage = [&]() {
#pragma unroll
        for (int r = 0; r < NCH; ++r) {
            const int i = tid + r * NTHR;             // C is even: a pair never straddles the guard
            const int u = i / C, ci = i - u * C;
            const bool odd = ci & 1;
            uint4 mine = pre[r];
            // send the half the partner stores, receive the partner's half of the same positions
            const uint32_t s0 = odd ? mine.x : mine.z, s1 = odd ? mine.y : mine.w;
            const uint32_t r0 = __shfl_xor_sync(0xffffffffu, s0, 1), r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
            if (i < C * CH) {
                // my 4 positions (even lane: e = 0..3 from .x .y; odd lane: e = 4..7 from .z .w)
                const uint32_t m0 = odd ? mine.z : mine.x, m1 = odd ? mine.w : mine.y;
                const __nv_bfloat16* mv = reinterpret_cast<const __nv_bfloat16*>(&m0);
                const __nv_bfloat16* mw = reinterpret_cast<const __nv_bfloat16*>(&m1);
                const __nv_bfloat16* pv = reinterpret_cast<const __nv_bfloat16*>(&r0);
                const __nv_bfloat16* pw = reinterpret_cast<const __nv_bfloat16*>(&r1);
                const __nv_bfloat16 my4[4] = {mv[0], mv[1], mw[0], mw[1]};
                const __nv_bfloat16 pa4[4] = {pv[0], pv[1], pw[0], pw[1]};
                const int e0 = odd ? 4 : 0, c0 = ci & ~1;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    __nv_bfloat162 w;
                    w.x = odd ? pa4[e] : my4[e];      // channel c0
                    w.y = odd ? my4[e] : pa4[e];      // channel c0 + 1
                    *reinterpret_cast<__nv_bfloat162*>(Xs + (8 * u + e0 + e) * XS + c0) = w;
                }
            }
        }
    };

    const int64_t ntiles = (T + TT - 1) / TT;
    if ((int64_t)blockIdx.x < ntiles) fetch((int64_t)blockIdx.x * TT);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t t0 = tile * TT;                 // first output position; staged rows = padded t0 ..
        __syncthreads();                              // previous tile's reads of Xs are done
        stage();
        __syncthreads();
        if (tile + gridDim.x < ntiles) fetch((tile + gridDim.x) * TT);

        float acc[2][4][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.0f;
#pragma unroll 4
        for (int ks = 0; ks < KTOT / 16; ++ks) {
            const int k = ks >> 2, ci0 = (ks & 3) * 16;
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
                ldsm_x4(a_base + (uint32_t)((mi * 16 * WS + ks * 16) * 2), a[mi][0], a[mi][1], a[mi][2], a[mi][3]);
#pragma unroll
            for (int pr = 0; pr < 2; ++pr)
                ldsm_x4(b_base + (uint32_t)(((pr * 16 + k) * XS + ci0) * 2), b[2 * pr][0], b[2 * pr][1],
                        b[2 * pr + 1][0], b[2 * pr + 1][1]);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni][0], b[ni][1]);
        }
        if constexpr (EPI == 1) {
            // data gradient: times the forward ReLU's derivative, FP32 pairs (and BF16 pairs) straight
            // from the fragments
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int ci = wm * 32 + mi * 16 + g + 8 * h;
                        const int64_t t = t0 + wn * 32 + ni * 8 + 2 * tq;
                        const int64_t o = (int64_t)ci * Tp + t + PAD;
                        if (vec && t + 1 < T) {
                            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + o);
                            const float2 v = make_float2(__bfloat162float(mk.x) > 0.0f ? acc[mi][ni][2 * h] : 0.0f,
                                                         __bfloat162float(mk.y) > 0.0f ? acc[mi][ni][2 * h + 1] : 0.0f);
                            *reinterpret_cast<float2*>(gout + o) = v;
                            if (gout16) *reinterpret_cast<__nv_bfloat162*>(gout16 + o) = __floats2bfloat162_rn(v.x, v.y);
                        } else {
#pragma unroll
                            for (int e = 0; e < 2; ++e)
                                if (t + e < T) {
                                    const float v = __bfloat162float(mask[o + e]) > 0.0f ? acc[mi][ni][2 * h + e] : 0.0f;
                                    gout[o + e] = v;
                                    if (gout16) gout16[o + e] = __float2bfloat16_rn(v);
                                }
                        }
                    }
            continue;
        }
        // epilogue: bias, ReLU, BF16 into an output tile Os[co][t] (over Xs once every warp is done),
        // then 8-byte row segments to act_out[co][t0 + PAD + ...]
        __syncthreads();
        __nv_bfloat16* Os = Xs;                       // [C][OS]
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int co = wm * 32 + mi * 16 + g + 8 * h;
                    const int n = wn * 32 + ni * 8 + 2 * tq;
                    __nv_bfloat162 w;
                    w.x = __float2bfloat16_rn(fmaxf(acc[mi][ni][2 * h] + bco[mi][h], 0.0f));
                    w.y = __float2bfloat16_rn(fmaxf(acc[mi][ni][2 * h + 1] + bco[mi][h], 0.0f));
                    *reinterpret_cast<__nv_bfloat162*>(Os + co * OS + n) = w;
                }
        __syncthreads();
        for (int i = tid; i < C * (TT / 4); i += NTHR) {
            const int co = i / (TT / 4), u = i - co * (TT / 4);
            const int64_t t = t0 + 4 * u;
            __nv_bfloat16* dst = act_out + (int64_t)co * Tp + t + PAD;
            const __nv_bfloat16* src = Os + co * OS + 4 * u;
            if (vec && t + 3 < T) {
                *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(src);
            } else {
                for (int e = 0; e < 4; ++e)
                    if (t + e < T) dst[e] = src[e];
            }
        }
    }
}


// Weight gradients of a 64 -> 64 layer on the tensor cores. For tap k, dW[co][ci][k] = sum_t dY[co][t]
// x[ci][t + k - 4] is the product D_k = A B_k with A[co][t] = dY (the BF16 copy of the gradient planes,
// M = 64, K = positions) and B_k[t][ci] = x[ci][t + k - 4] (the layer's input activation, N = 64). A chunk
// of WT positions stages A as rows [co][t] (ldmatrix) and x transposed to [position][channel] like the
// forward, so that tap k's B fragment is an ldmatrix.trans of the rows shifted by k. CTA (r, j) takes taps
// 3 j .. 3 j + 2 and the chunks r, r + gridDim.x, ...; eight warps hold 32 x 16 output blocks of the three
// taps in FP32 fragments and write them to partial row r ([co][ci][k], then the bias gradient, summed by
// tap group 0 from the staged BF16 dY); k_wgrad_sum adds the rows in a fixed order. The next chunk's
// global loads are in flight while the current chunk computes.
constexpr int WT = 128;                                    // positions per chunk
constexpr int WXR = WT + 2 * PAD;                          // staged input positions per chunk
constexpr int WAS = WT + 8;                                // A row stride (bf16)
constexpr size_t WSMEM = sizeof(__nv_bfloat16) * ((size_t)C * WAS + (size_t)WXR * XS);

__global__ void __launch_bounds__(NTHR) k_wgrad64_mma(const __nv_bfloat16* __restrict__ x,
                                                      const __nv_bfloat16* __restrict__ dy16, int64_t Tp,
                                                      int64_t T, float* __restrict__ part, int vec) {
    extern __shared__ float4 smem4[];
    __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem4);      // [C][WAS]: dY of positions t0 + j
    __nv_bfloat16* Xs = As + C * WAS;                                 // [WXR][XS]: x of padded index t0 + r
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;                          // 2 x 4 warps of 32 co x 16 ci
    const int g = lane >> 2, tq = lane & 3;
    const int kt0 = blockIdx.y * 3;                                   // taps of this CTA
    constexpr int64_t ROW = (int64_t)C * C * KW + C;
    float* prow = part + (int64_t)blockIdx.x * ROW;

    // A rows co0 + (lane % 16), column block (lane / 16) * 8 (as the forward's weights)
    const uint32_t a_base = smem_addr(As + (wm * 32 + (lane & 15)) * WAS + (lane >> 4) * 8);
    // B (x4.trans): matrix i = lane / 8 covers positions (i & 1) * 8 + lane % 8 of the k-step and channels
    // (i >> 1) * 8 of the warp's 16
    const uint32_t b_base = smem_addr(Xs + (((lane >> 3) & 1) * 8 + (lane & 7)) * XS + wn * 16 + (lane >> 4) * 8);

    float acc[3][2][2][4];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 2; ++ni)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[k][mi][ni][e] = 0.0f;
    float dbs = 0.0f;                                                 // bias: thread co = tid / 4, quarter tid % 4

    const int64_t nchunk = (T + WT - 1) / WT;
    // Staging, software-pipelined: the next chunk's global loads go to registers while the current chunk
    // computes. Thread item i < C (WT / 8 + 1) of A: row co, 16-byte chunk u of the padded row from t0;
    // item i < C (WXR / 8) of x: 16-byte chunk u of channel ci.
    constexpr int NA = (C * (WT / 8 + 1) + NTHR - 1) / NTHR, NX = (C * (WXR / 8) + NTHR - 1) / NTHR;
    uint4 pa[NA], px[NX];
    auto load16 = [&](const __nv_bfloat16* src, int64_t tp) -> uint4 {
        if (vec && tp + 7 < Tp) return __ldg(reinterpret_cast<const uint4*>(src));
        __nv_bfloat16 tmp[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) tmp[e] = tp + e < Tp ? src[e] : __float2bfloat16_rn(0.0f);
        return *reinterpret_cast<const uint4*>(tmp);
    };
    auto fetch = [&](int64_t t0) {
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            const int i = tid + r * NTHR;
            pa[r] = make_uint4(0u, 0u, 0u, 0u);
            if (i < C * (WT / 8 + 1)) {
                const int co = i / (WT / 8 + 1), u = i - co * (WT / 8 + 1);
                pa[r] = load16(dy16 + (int64_t)co * Tp + t0 + 8 * u, t0 + 8 * u);
            }
        }
#pragma unroll
        for (int r = 0; r < NX; ++r) {
            const int i = tid + r * NTHR;
            px[r] = make_uint4(0u, 0u, 0u, 0u);
            if (i < C * (WXR / 8)) {
                const int u = i / C, ci = i - u * C;
                px[r] = load16(x + (int64_t)ci * Tp + t0 + 8 * u, t0 + 8 * u);
            }
        }
    };
    // A: dY of positions t0 .. t0 + WT (padded t0 + 4 ..): the padded row's 16-byte chunks from t0 stored as
    // two 8-byte halves at their column; x transposed: Xs[r][ci] = x[ci][padded t0 + r]
    auto stage = [&]() {
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            const int i = tid + r * NTHR;
            if (i < C * (WT / 8 + 1)) {
                const int co = i / (WT / 8 + 1), u = i - co * (WT / 8 + 1);
                const int c0 = 8 * u - PAD;                       // column of the chunk's first element
                if (c0 >= 0) *reinterpret_cast<uint2*>(As + co * WAS + c0) = make_uint2(pa[r].x, pa[r].y);
                if (c0 + 4 < WT) *reinterpret_cast<uint2*>(As + co * WAS + c0 + 4) = make_uint2(pa[r].z, pa[r].w);
            }
        }
#pragma unroll
        for (int r = 0; r < NX; ++r) {
            const int i = tid + r * NTHR;
            if (i < C * (WXR / 8)) {
                const int u = i / C, ci = i - u * C;
                const __nv_bfloat16* v = reinterpret_cast<const __nv_bfloat16*>(&px[r]);
#pragma unroll
                for (int e = 0; e < 8; ++e) Xs[(8 * u + e) * XS + ci] = v[e];
            }
        }
    };
    if ((int64_t)blockIdx.x < nchunk) fetch((int64_t)blockIdx.x * WT);
    for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        __syncthreads();                                              // the previous chunk's reads are done
        stage();
        __syncthreads();
        if (ch + gridDim.x < nchunk) fetch((ch + gridDim.x) * WT);
        // the bias gradient from the staged dY: four threads per channel, 32 positions each, pairs of
        // the quarter's 8-element groups in order
        if (blockIdx.y == 0) {
            const int co = tid >> 2, qq = tid & 3;
            const uint4* ar = reinterpret_cast<const uint4*>(As + co * WAS + qq * (WT / 4));
            float sb = 0.0f;
#pragma unroll
            for (int j = 0; j < WT / 32; ++j) {
                const uint4 w4 = ar[j];
                const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&w4);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 f = __bfloat1622float2(h[e]);
                    sb += f.x + f.y;
                }
            }
            sb += __shfl_xor_sync(0xffffffffu, sb, 1);
            sb += __shfl_xor_sync(0xffffffffu, sb, 2);
            dbs += sb;
        }
#pragma unroll 2
        for (int ks = 0; ks < WT / 16; ++ks) {
            uint32_t a[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
                ldsm_x4(a_base + (uint32_t)((mi * 16 * WAS + ks * 16) * 2), a[mi][0], a[mi][1], a[mi][2], a[mi][3]);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                // tap kt0 + k: positions t0 + 16 ks + (0..15) read x at padded t0 + 16 ks + kt0 + k + (0..15)
                uint32_t b[4];
                ldsm_x4_t(b_base + (uint32_t)(((ks * 16 + kt0 + k) * XS) * 2), b[0], b[1], b[2], b[3]);
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    mma_bf16(acc[k][mi][0], a[mi], b[0], b[1]);
                    mma_bf16(acc[k][mi][1], a[mi], b[2], b[3]);
                }
            }
        }
    }
    // the CTA's partial row: D_k fragment (row co, column ci) -> dW[co][ci][k]
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 2; ++ni)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int co = wm * 32 + mi * 16 + g + 8 * h, ci = wn * 16 + ni * 8 + 2 * tq + e;
                        prow[((int64_t)co * C + ci) * KW + kt0 + k] = acc[k][mi][ni][2 * h + e];
                    }
    if (blockIdx.y == 0 && (tid & 3) == 0) prow[(int64_t)C * C * KW + (tid >> 2)] = dbs;
}

}  // namespace

template <int EPI>
int conv64_grid(int64_t T) {
    static int resident = 0;
    if (!resident) {
        int dev = 0, nsm = 152, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_conv64_mma<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_conv64_mma<EPI>, NTHR, SMEM);
        resident = std::max(1, nsm * per);
    }
    const int64_t ntiles = (T + TT - 1) / TT;
    return (int)std::min<int64_t>(ntiles, resident);
}

cudaError_t conv64_mma_fwd(const __nv_bfloat16* x, int64_t Tp, int64_t T, const __nv_bfloat16* Wm, const float* b,
                           __nv_bfloat16* act, cudaStream_t s) {
    // 16-byte staging loads need 16-byte aligned input rows, the 8-byte stores 8-byte aligned output rows
    const int vec = ((uintptr_t)x % 16 == 0) && ((uintptr_t)act % 16 == 0) && (Tp % 8 == 0);
    k_conv64_mma<0><<<conv64_grid<0>(T), NTHR, SMEM, s>>>(x, Tp, T, Wm, b, act, vec, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t conv64_mma_dgrad(const __nv_bfloat16* dout, int64_t Tp, int64_t T, const __nv_bfloat16* Wd,
                             const __nv_bfloat16* mask, float* din, __nv_bfloat16* din16, cudaStream_t s) {
    // 16-byte staging loads; the epilogue's pairs need even element offsets (8- and 4-byte aligned)
    const int vec = ((uintptr_t)dout % 16 == 0) && ((uintptr_t)din % 16 == 0) && ((uintptr_t)mask % 16 == 0) &&
                    (!din16 || (uintptr_t)din16 % 16 == 0) && (Tp % 8 == 0);
    k_conv64_mma<1><<<conv64_grid<1>(T), NTHR, SMEM, s>>>(dout, Tp, T, Wd, nullptr, nullptr, vec, mask, din, din16);
    return cudaGetLastError();
}

cudaError_t conv64_mma_wgrad_parts(const __nv_bfloat16* x, const __nv_bfloat16* dy16, int64_t Tp, int64_t T,
                                   float* part, int max_rows, int* nrow, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_wgrad64_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WSMEM);
        attr = true;
    }
    const int64_t nchunk = (T + WT - 1) / WT;
    const int rows = (int)std::min<int64_t>(std::max<int64_t>(nchunk, 1), max_rows);
    const int vec = ((uintptr_t)x % 16 == 0) && ((uintptr_t)dy16 % 16 == 0) && (Tp % 8 == 0);
    k_wgrad64_mma<<<dim3((unsigned)rows, KW / 3), NTHR, WSMEM, s>>>(x, dy16, Tp, T, part, vec);
    *nrow = rows;
    return cudaGetLastError();
}
