// A9 learned post-equaliser: a 4-layer 1-D CNN on the carrier-recovered
// symbols (4 real channels I_x, Q_x, I_y, Q_y), out = z + f(z),
// f = conv(C->4) relu conv(C->C) relu conv(C->C) relu conv(4->C), kernel K = 9,
// "same" zero padding. Weights and activations are BF16, products and sums
// FP32, master weights FP32 (Adam). The paper has no learned equaliser.
//
// Layout: activations [C][T + 8] with the 4 zero columns of the padding on
// each side stored, so a convolution reads x[c][t + k] with no bounds checks.
// One CTA computes 128 positions (64 in the 4-input-channel layers) of all
// output channels: 8 output channels x 4 (2) positions per thread (positions
// strided by 32 so a warp's loads hit distinct banks), input channels staged
// in chunks of 16 (FP32 in shared memory), weights staged as [ci][k][co] so 8
// output channels come from two 128-bit broadcast loads; the 4-output layer
// (k_conv_out4) splits each position's input channels over four lanes. The
// backward pass on the data reuses the same kernel with transposed, flipped
// weights W'[ci][co][k] = W[co][ci][K-1-k] and the ReLU mask fused into its
// store; the weight gradient sums dY[co][t] x[ci][t + k - 4] over a chunk of
// positions per thread with a 9-register sliding window and adds the chunk's
// result to FP32 accumulators.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "rx_cnn.h"

namespace {

constexpr int KW = 9;          // kernel width
constexpr int PAD = KW / 2;
constexpr int CT = 256;        // threads per CTA
constexpr int CC = 16;         // input channels per staged chunk

__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld(const float* p) { return *p; }

// EPI 0: bias + ReLU -> BF16 activations; 1: bias + residual -> float2 symbols (COUT = 4);
// EPI 2: ReLU mask of `mask` -> FP32 gradient (no bias) and, when act_out is given, its BF16 copy
template <typename Tin, int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(CT) k_conv(const Tin* __restrict__ x, int64_t Tp, int64_t T,
                                             const float* __restrict__ W, const float* __restrict__ bias,
                                             __nv_bfloat16* __restrict__ act_out, const __nv_bfloat16* __restrict__ mask,
                                             float* __restrict__ grad_out, const float2* __restrict__ zres,
                                             float2* __restrict__ sym_out, int64_t zs) {
    constexpr int CO_T = COUT >= 8 ? 8 : COUT;       // output channels per thread
    constexpr int NG = COUT / CO_T;                   // output-channel groups
    constexpr int TPG = CT / NG;                      // threads per group
    // positions per thread: fewer for the 4-channel layers, so that a 16384-position window gives 256 CTAs
    constexpr int PPT = COUT <= 4 ? 1 : CIN <= 4 ? 2 : 4;
    constexpr int TT = TPG * PPT;                     // positions per CTA
    constexpr int XW = TT + 2 * PAD;
    constexpr int CCH = CIN < (TT >= 1024 ? CC / 2 : CC) ? CIN : (TT >= 1024 ? CC / 2 : CC);   // static smem < 48 KB
    __shared__ float xs[CCH][XW];
    __shared__ __align__(16) float ws[CCH][KW][COUT];
    const int tid = threadIdx.x;
    const int g = tid / TPG, lt = tid - g * TPG;
    const int64_t t0 = (int64_t)blockIdx.x * TT;      // first output position (unpadded index)
    float acc[CO_T][PPT];
#pragma unroll
    for (int c = 0; c < CO_T; ++c)
#pragma unroll
        for (int j = 0; j < PPT; ++j) acc[c][j] = 0.0f;
    for (int c0 = 0; c0 < CIN; c0 += CCH) {
        // stage x[c0 .. c0+CCH)[t0 - 4 .. t0 + TT + 4) (padded index t0 .. t0 + XW), eight loads per thread
        // in flight at a time (the latency of this part's L2 is long)
        for (int i0 = 0; i0 < CCH * XW; i0 += 8 * CT) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int i = i0 + e * CT + tid;
                const int ci = i / XW, u = i - ci * XW;
                const int64_t tp = t0 + u;
                v[e] = (i < CCH * XW && tp < Tp) ? ld(x + (int64_t)(c0 + ci) * Tp + tp) : 0.0f;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int i = i0 + e * CT + tid;
                if (i < CCH * XW) xs[i / XW][i - (i / XW) * XW] = v[e];
            }
        }
        for (int i = tid; i < CCH * KW * COUT; i += CT) {
            const int co = i / (CCH * KW), r = i - co * CCH * KW, ci = r / KW, k = r - ci * KW;
            ws[ci][k][co] = W[((int64_t)co * CIN + c0 + ci) * KW + k];
        }
        __syncthreads();
#pragma unroll 1
        for (int ci = 0; ci < CCH; ++ci) {
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                float w[CO_T];
#pragma unroll
                for (int c = 0; c < CO_T; ++c) w[c] = ws[ci][k][g * CO_T + c];
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const float xv = xs[ci][lt + j * (TT / PPT) + k];
#pragma unroll
                    for (int c = 0; c < CO_T; ++c) acc[c][j] = fmaf(w[c], xv, acc[c][j]);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const int64_t t = t0 + lt + j * (TT / PPT);   // unpadded output position
        if (t >= T) continue;
#pragma unroll
        for (int c = 0; c < CO_T; ++c) {
            const int co = g * CO_T + c;
            if (EPI == 0) {
                const float v = fmaxf(acc[c][j] + bias[co], 0.0f);
                act_out[(int64_t)co * Tp + t + PAD] = __float2bfloat16_rn(v);
            } else if (EPI == 2) {
                const bool on = __bfloat162float(mask[(int64_t)co * Tp + t + PAD]) > 0.0f;
                grad_out[(int64_t)co * Tp + t + PAD] = on ? acc[c][j] : 0.0f;
                if (act_out) act_out[(int64_t)co * Tp + t + PAD] = __float2bfloat16_rn(on ? acc[c][j] : 0.0f);
            }
        }
        if (EPI == 1) {
            // channels (I_x, Q_x, I_y, Q_y) -> symbols of pol 0 and 1
            const float2 z0 = zres[t], z1 = zres[zs + t];     // the residual's polarisations zs apart
            sym_out[t] = make_float2(z0.x + acc[0][j] + bias[0], z0.y + acc[1][j] + bias[1]);
            sym_out[T + t] = make_float2(z1.x + acc[2][j] + bias[2], z1.y + acc[3][j] + bias[3]);
        }
    }
}

// The C -> 4 layer (bias + residual into the symbols): four output channels leave too few products per
// position to fill CTAs with positions alone, so each position's input channels are split over four
// lanes (lane bits 3-4: channels s, s + 4, s + 8, ..., whose rows fall in distinct shared-memory banks)
// and two shuffles add the four partial sums; 64 positions per CTA, all input channels staged at once.
// With a target (training), the epilogue also forms the loss gradient d3 and adds the loss, as k_mse
// does from the stored output.
template <int CIN>
__global__ void __launch_bounds__(CT) k_conv_out4(const __nv_bfloat16* __restrict__ x, int64_t Tp, int64_t T,
                                                  const float* __restrict__ W, const float* __restrict__ bias,
                                                  const float2* __restrict__ zres, float2* __restrict__ sym_out,
                                                  int64_t zs, const float2* __restrict__ tgt, int64_t ts,
                                                  float* __restrict__ d3, float* __restrict__ loss) {
    constexpr int CS = 4;                             // lanes per position
    constexpr int TT = CT / CS;                       // positions per CTA
    constexpr int XW = TT + 2 * PAD;                  // 72: rows s and s + 1 are 8 banks apart
    static_assert(CIN % CS == 0 && (CS * XW) % 32 == 0, "channel split");
    __shared__ float xs[CIN][XW];
    __shared__ __align__(16) float ws[CIN][KW][4];
    const int tid = threadIdx.x, lane = tid & 31;
    const int sp = lane >> 3;                         // channel split
    const int p = 8 * (tid >> 5) + (lane & 7);        // tile position
    const int64_t t0 = (int64_t)blockIdx.x * TT;
    for (int i0 = 0; i0 < CIN * XW; i0 += 8 * CT) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int i = i0 + e * CT + tid;
            const int ci = i / XW, u = i - ci * XW;
            const int64_t tp = t0 + u;
            v[e] = (i < CIN * XW && tp < Tp) ? __bfloat162float(x[(int64_t)ci * Tp + tp]) : 0.0f;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int i = i0 + e * CT + tid;
            if (i < CIN * XW) xs[i / XW][i - (i / XW) * XW] = v[e];
        }
    }
    for (int i = tid; i < CIN * KW * 4; i += CT) {
        const int co = i / (CIN * KW), r = i - co * CIN * KW, ci = r / KW, k = r - ci * KW;
        ws[ci][k][co] = W[((int64_t)co * CIN + ci) * KW + k];
    }
    __syncthreads();
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 2
    for (int j = 0; j < CIN / CS; ++j) {
        const int ci = sp + CS * j;
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            const float4 w = *reinterpret_cast<const float4*>(&ws[ci][k][0]);
            const float xv = xs[ci][p + k];
            acc[0] = fmaf(w.x, xv, acc[0]);
            acc[1] = fmaf(w.y, xv, acc[1]);
            acc[2] = fmaf(w.z, xv, acc[2]);
            acc[3] = fmaf(w.w, xv, acc[3]);
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 8);
        acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 16);
    }
    const int64_t t = t0 + p;
    float l = 0.0f;
    if (sp == 0 && t < T) {
        // channels (I_x, Q_x, I_y, Q_y) -> symbols of pol 0 and 1
        const float2 z0 = zres[t], z1 = zres[zs + t];
        const float2 a = make_float2(z0.x + acc[0] + bias[0], z0.y + acc[1] + bias[1]);
        const float2 b = make_float2(z1.x + acc[2] + bias[2], z1.y + acc[3] + bias[3]);
        sym_out[t] = a;
        sym_out[T + t] = b;
        if (tgt) {
            const float inv = 1.0f / (4.0f * (float)T);
            const float2 ta = tgt[t], tb = tgt[ts + t];
            const float e[4] = {a.x - ta.x, a.y - ta.y, b.x - tb.x, b.y - tb.y};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                d3[(int64_t)c * Tp + t + PAD] = 2.0f * e[c] * inv;
                l += e[c] * e[c] * inv;
            }
        }
    }
    if (tgt) {                                        // uniform over the grid
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (lane == 0 && loss) atomicAdd(loss, l);
    }
}

// Weight gradients dW[co][ci][k] = sum_t dY[co][t] x[ci][t + k - 4], db[co] = sum_t dY[co][t]: CTA
// (x, y, z) sums the 256-position chunks x, x + gridDim.x, ... of its (co, ci) tile and writes its partial
// to row x of part ([row][co][ci][k], then [row][COUT][co] for the biases); k_wgrad_sum adds the rows in
// order. A tile of fewer than 256 (co, ci) pairs splits each chunk's positions over PS threads per pair,
// whose sums are added in split order at the end. No atomics: every run gives the same sums.
template <typename Tin, int CIN, int COUT>
__global__ void __launch_bounds__(CT) k_conv_wgrad(const Tin* __restrict__ x, const float* __restrict__ dy,
                                                   int64_t Tp, int64_t T, float* __restrict__ part) {
    constexpr int TC = 256;                           // positions per chunk (static smem < 48 KB)
    constexpr int CO_TILE = COUT < 16 ? COUT : 16;
    constexpr int CI_TILE = CIN < 16 ? CIN : 16;
    constexpr int NP = CO_TILE * CI_TILE;             // (co, ci) pairs of the tile
    constexpr int PS = CT / NP;                       // threads per pair
    constexpr int TS = TC / PS;                       // positions per thread and chunk
    constexpr int64_t ROW = (int64_t)COUT * CIN * KW + COUT;
    constexpr int DYS = TC + 1, XWC = TC + 2 * PAD, XSS = XWC + 1;   // row strides: rows in distinct banks
    static_assert(CT % NP == 0 && TC % PS == 0, "pairs x splits = threads");
    __shared__ float dys[CO_TILE][DYS];
    __shared__ float xs[CI_TILE][XSS];
    __shared__ float red[PS > 1 ? PS - 1 : 1][NP][KW + 1];
    const int co0 = blockIdx.y * CO_TILE, ci0 = blockIdx.z * CI_TILE;
    const int tid = threadIdx.x;
    const int pi = tid % NP, sp = tid / NP;
    const int co = pi / CI_TILE, ci = pi % CI_TILE;
    const int u0 = sp * TS;
    float acc[KW];
#pragma unroll
    for (int k = 0; k < KW; ++k) acc[k] = 0.0f;
    float dbs = 0.0f;
    const int64_t nchunk = (T + TC - 1) / TC;
    for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const int64_t t0 = ch * TC;                   // unpadded
        __syncthreads();                              // the previous chunk's reads are done
        // staging with eight loads per thread in flight at a time
        for (int i0 = 0; i0 < CO_TILE * TC; i0 += 8 * CT) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int i = i0 + e * CT + tid;
                const int c = i / TC, u = i - c * TC;
                const int64_t t = t0 + u;
                v[e] = (i < CO_TILE * TC && t < T) ? dy[(int64_t)(co0 + c) * Tp + t + PAD] : 0.0f;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int i = i0 + e * CT + tid;
                if (i < CO_TILE * TC) dys[i / TC][i - (i / TC) * TC] = v[e];
            }
        }
        for (int i0 = 0; i0 < CI_TILE * XWC; i0 += 8 * CT) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int i = i0 + e * CT + tid;
                const int c = i / XWC, u = i - c * XWC;
                const int64_t tp = t0 + u;            // padded index of position t0 + u - 4
                v[e] = (i < CI_TILE * XWC && tp < Tp) ? ld(x + (int64_t)(ci0 + c) * Tp + tp) : 0.0f;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int i = i0 + e * CT + tid;
                if (i < CI_TILE * XWC) xs[i / XWC][i - (i / XWC) * XWC] = v[e];
            }
        }
        __syncthreads();
        float win[KW];
#pragma unroll
        for (int k = 0; k < KW; ++k) win[k] = xs[ci][u0 + k];
        for (int u = u0; u < u0 + TS; ++u) {
            const float d = dys[co][u];
#pragma unroll
            for (int k = 0; k < KW; ++k) acc[k] = fmaf(d, win[k], acc[k]);
            dbs += d;
#pragma unroll
            for (int k = 0; k < KW - 1; ++k) win[k] = win[k + 1];
            if (u + 1 < u0 + TS) win[KW - 1] = xs[ci][u + KW];   // window of position u + 1
        }
    }
    if (PS > 1) {
        if (sp > 0) {
#pragma unroll
            for (int k = 0; k < KW; ++k) red[sp - 1][pi][k] = acc[k];
            red[sp - 1][pi][KW] = dbs;
        }
        __syncthreads();
        if (sp == 0)
            for (int r = 0; r < PS - 1; ++r) {
#pragma unroll
                for (int k = 0; k < KW; ++k) acc[k] += red[r][pi][k];
                dbs += red[r][pi][KW];
            }
    }
    if (sp == 0) {
        float* row = part + (int64_t)blockIdx.x * ROW;
#pragma unroll
        for (int k = 0; k < KW; ++k) row[((int64_t)(co0 + co) * CIN + ci0 + ci) * KW + k] = acc[k];
        if (ci == 0 && blockIdx.z == 0) row[(int64_t)COUT * CIN * KW + co0 + co] = dbs;
    }
}

// dW = the sum of the nrow partial rows in order, then db likewise; every row's load is issued before
// the first add (one memory latency per thread instead of nrow)
__global__ void k_wgrad_sum(const float* __restrict__ part, int64_t nw, int64_t nb, int nrow, float* __restrict__ dW,
                            float* __restrict__ db) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw + nb) return;
    const int64_t row = nw + nb;
    float v[CNN_WG_SPLIT];
#pragma unroll
    for (int r = 0; r < CNN_WG_SPLIT; ++r) v[r] = r < nrow ? part[(int64_t)r * row + i] : 0.0f;
    float s = 0.0f;
#pragma unroll
    for (int r = 0; r < CNN_WG_SPLIT; ++r)
        if (r < nrow) s += v[r];
    if (i < nw) dW[i] = s;
    else db[i - nw] = s;
}

__global__ void k_to_channels(const float2* __restrict__ z, int64_t zs, int64_t T, int64_t Tp,
                              __nv_bfloat16* __restrict__ x0) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const float2 a = z[t], b = z[zs + t];
    x0[0 * Tp + t + PAD] = __float2bfloat16_rn(a.x);
    x0[1 * Tp + t + PAD] = __float2bfloat16_rn(a.y);
    x0[2 * Tp + t + PAD] = __float2bfloat16_rn(b.x);
    x0[3 * Tp + t + PAD] = __float2bfloat16_rn(b.y);
}

// d3[c][t] = 2 (out - target) / (4 T); loss += sum (out - target)^2 / (4 T)
__global__ void k_mse(const float2* __restrict__ out, const float2* __restrict__ tgt, int64_t ts, int64_t T, int64_t Tp,
                      float* __restrict__ d3, float* __restrict__ loss) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (t < T) {
        const float inv = 1.0f / (4.0f * (float)T);
        const float2 a = out[t], b = out[T + t], ta = tgt[t], tb = tgt[ts + t];
        const float e[4] = {a.x - ta.x, a.y - ta.y, b.x - tb.x, b.y - tb.y};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            d3[(int64_t)c * Tp + t + PAD] = 2.0f * e[c] * inv;
            l += e[c] * e[c] * inv;
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// W'[ci][co][k] = bf16(W[co][ci][K-1-k]) and the forward weights as BF16-rounded FP32, for parameter i
// of value w
__device__ __forceinline__ void weight_copies(int64_t i, float w, float* __restrict__ fwd, const int* offs,
                                              const int* cins, const int* couts, float* __restrict__ bwd,
                                              __nv_bfloat16* __restrict__ wtc, __nv_bfloat16* __restrict__ wtd) {
    const __nv_bfloat16 vb = __float2bfloat16_rn(w);
    const float v = __bfloat162float(vb);
    fwd[i] = v;
    // locate the layer and, for weights, the transposed position and the tensor-core copy in (k, ci)
    // order (rows of 9 * cin, the input layer's padded to 48)
    for (int l = 0; l < 4; ++l) {
        const int64_t wo = offs[2 * l], nw = (int64_t)couts[l] * cins[l] * KW;
        if (i >= wo && i < wo + nw) {
            const int64_t r = i - wo;
            const int co = (int)(r / (cins[l] * KW)), ci = (int)((r / KW) % cins[l]), k = (int)(r % KW);
            bwd[wo + ((int64_t)ci * couts[l] + co) * KW + (KW - 1 - k)] = v;
            const int C = cins[1];
            const int row = l == 0 ? 48 : cins[l] * KW;
            wtc[wtc_offset(C, l) + (int64_t)co * row + k * cins[l] + ci] = vb;
            if (l == 1 || l == 2)                     // the data gradient's flipped transpose, (k, co) order
                wtd[(int64_t)(l - 1) * C * C * KW + (int64_t)ci * (KW * C) + (KW - 1 - k) * C + co] = vb;
        }
    }
}

__global__ void k_weights(const float* __restrict__ master, int64_t n, float* __restrict__ fwd, const int* offs,
                          const int* cins, const int* couts, float* __restrict__ bwd, __nv_bfloat16* __restrict__ wtc,
                          __nv_bfloat16* __restrict__ wtd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    weight_copies(i, master[i], fwd, offs, cins, couts, bwd, wtc, wtd);
}

// one Adam step of parameter i, then (with B's copies given) the weight copies of the new value
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2, float* __restrict__ fwd,
                       const int* offs, const int* cins, const int* couts, float* __restrict__ bwd,
                       __nv_bfloat16* __restrict__ wtc, __nv_bfloat16* __restrict__ wtd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pn = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pn;
    if (fwd) weight_copies(i, pn, fwd, offs, cins, couts, bwd, wtc, wtd);
}

template <typename Tin, int CIN, int COUT, int EPI>
cudaError_t conv_t(const Tin* x, int64_t Tp, int64_t T, const float* W, const float* b, __nv_bfloat16* act,
                   const __nv_bfloat16* mask, float* grad, const float2* zres, float2* sym, cudaStream_t s, int64_t zs = 0) {
    constexpr int CO_T = COUT >= 8 ? 8 : COUT;
    constexpr int TT = (CT / (COUT / CO_T)) * (COUT <= 4 ? 1 : CIN <= 4 ? 2 : 4);   // k_conv's positions per CTA
    k_conv<Tin, CIN, COUT, EPI><<<(unsigned)((T + TT - 1) / TT), CT, 0, s>>>(x, Tp, T, W, b, act, mask, grad, zres, sym, zs);
    return cudaGetLastError();
}

template <typename Tin, int CIN, int COUT>
cudaError_t wgrad_t(const Tin* x, const float* dy, int64_t Tp, int64_t T, float* part, float* dW, float* db,
                    cudaStream_t s) {
    constexpr int CO_TILE = COUT < 16 ? COUT : 16;
    constexpr int CI_TILE = CIN < 16 ? CIN : 16;
    const int64_t nchunk = (T + 255) / 256;
    const int nrow = (int)std::min<int64_t>(std::max<int64_t>(nchunk, 1), CNN_WG_SPLIT);
    dim3 grid((unsigned)nrow, COUT / CO_TILE, CIN / CI_TILE);
    k_conv_wgrad<Tin, CIN, COUT><<<grid, CT, 0, s>>>(x, dy, Tp, T, part);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    const int64_t nw = (int64_t)COUT * CIN * KW, nb = COUT;
    k_wgrad_sum<<<(unsigned)((nw + nb + 255) / 256), 256, 0, s>>>(part, nw, nb, nrow, dW, db);
    return cudaGetLastError();
}

// the hidden layers' weight gradients: partial rows on the tensor cores, then the rows in order
cudaError_t wgrad64_t(const __nv_bfloat16* x, const __nv_bfloat16* dy16, int64_t Tp, int64_t T, float* part, float* dW,
                      float* db, cudaStream_t s) {
    int nrow = 0;
    cudaError_t e = conv64_mma_wgrad_parts(x, dy16, Tp, T, part, CNN_WG_SPLIT, &nrow, s);
    if (e) return e;
    const int64_t nw = (int64_t)64 * 64 * KW, nb = 64;
    k_wgrad_sum<<<(unsigned)((nw + nb + 255) / 256), 256, 0, s>>>(part, nw, nb, nrow, dW, db);
    return cudaGetLastError();
}

}  // namespace

// forward of the 4 layers; act[0] holds the input channels, act[1..3] the hidden activations
cudaError_t cnn_forward(const CnnBufs& B, const float2* z, int64_t zs, int64_t T, float2* out, cudaStream_t s,
                        const float2* tgt, int64_t ts, float* loss) {
    const int64_t Tp = T + 2 * PAD;
    const int C = B.C;
    if (C != 64) return cudaErrorInvalidValue;
    k_to_channels<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(z, zs, T, Tp, B.act[0]);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    const float* W = B.wfwd;
    e = conv_t<__nv_bfloat16, 4, 64, 0>(B.act[0], Tp, T, W + B.off[0], W + B.off[1], B.act[1], nullptr, nullptr, nullptr,
                                        nullptr, s);
    if (e) return e;
    e = conv64_mma_fwd(B.act[1], Tp, T, B.wtc + wtc_offset(C, 1), W + B.off[3], B.act[2], s);
    if (e) return e;
    e = conv64_mma_fwd(B.act[2], Tp, T, B.wtc + wtc_offset(C, 2), W + B.off[5], B.act[3], s);
    if (e) return e;
    k_conv_out4<64><<<(unsigned)((T + CT / 4 - 1) / (CT / 4)), CT, 0, s>>>(B.act[3], Tp, T, W + B.off[6], W + B.off[7],
                                                                            z, out, zs, tgt, ts, B.d[3], loss);
    return cudaGetLastError();
}

// loss gradient and all parameter gradients (every entry of B.grad written) for the last forward
cudaError_t cnn_backward(const CnnBufs& B, const float2* out, const float2* tgt, int64_t ts, int64_t T, float* loss,
                         cudaStream_t s) {
    const int64_t Tp = T + 2 * PAD;
    cudaError_t e = cudaSuccess;
    if (tgt) {                                        // else the forward formed d[3] and the loss
        k_mse<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(out, tgt, ts, T, Tp, B.d[3], loss);
        if ((e = cudaGetLastError())) return e;
    }
    float* G = B.grad;
    const float* Wb = B.wbwd;
    // layer 3: weights, then data (masked by act[3] > 0) -> d[2]
    if ((e = wgrad_t<__nv_bfloat16, 64, 4>(B.act[3], B.d[3], Tp, T, B.wpart, G + B.off[6], G + B.off[7], s))) return e;
    // (and the BF16 copy of d[2]: the hidden layers' data gradients on the tensor cores read it)
    if ((e = conv_t<float, 4, 64, 2>(B.d[3], Tp, T, Wb + B.off[6], nullptr, B.d16[2], B.act[3], B.d[2], nullptr,
                                     nullptr, s)))
        return e;
    if ((e = wgrad64_t(B.act[2], B.d16[2], Tp, T, B.wpart, G + B.off[4], G + B.off[5], s))) return e;
    const int64_t lw = (int64_t)64 * 64 * KW;
    if ((e = conv64_mma_dgrad(B.d16[2], Tp, T, B.wtd + lw, B.act[2], B.d[1], B.d16[1], s))) return e;
    if ((e = wgrad64_t(B.act[1], B.d16[1], Tp, T, B.wpart, G + B.off[2], G + B.off[3], s))) return e;
    if ((e = conv64_mma_dgrad(B.d16[1], Tp, T, B.wtd, B.act[1], B.d[0], nullptr, s))) return e;
    return wgrad_t<__nv_bfloat16, 4, 64>(B.act[0], B.d[0], Tp, T, B.wpart, G + B.off[0], G + B.off[1], s);
}

// the padding columns of every activation/gradient plane for a sequence of length T
__global__ void k_zero_pads(CnnBufs B, int64_t T) {
    const int64_t Tp = T + 2 * PAD;
    const int c = blockIdx.x;                         // channel
    const int u = threadIdx.x;                        // 0 .. 2*PAD-1
    if (u >= 2 * PAD) return;
    const int64_t col = u < PAD ? u : T + u;          // [0, PAD) and [T + PAD, Tp)
    for (int buf = 0; buf < 4; ++buf) {
        const int nch = buf == 0 ? 4 : B.C;
        if (c < nch) B.act[buf][(int64_t)c * Tp + col] = __float2bfloat16_rn(0.0f);
        const int ndch = buf == 3 ? 4 : B.C;
        if (c < ndch) B.d[buf][(int64_t)c * Tp + col] = 0.0f;
        if ((buf == 1 || buf == 2) && c < B.C) B.d16[buf][(int64_t)c * Tp + col] = __float2bfloat16_rn(0.0f);
    }
}

cudaError_t cnn_zero_pads(const CnnBufs& B, int64_t T, cudaStream_t s) {
    k_zero_pads<<<B.C, 32, 0, s>>>(B, T);
    return cudaGetLastError();
}

cudaError_t cnn_prepare_weights(const CnnBufs& B, cudaStream_t s) {
    k_weights<<<(unsigned)((B.nparam + 255) / 256), 256, 0, s>>>(B.master, B.nparam, B.wfwd, B.offs_dev, B.cin_dev,
                                                                 B.cout_dev, B.wbwd, B.wtc, B.wtd);
    return cudaGetLastError();
}

cudaError_t cnn_adam(const CnnBufs& B, float lr, int step, cudaStream_t s, bool copies) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<(unsigned)((B.nparam + 255) / 256), 256, 0, s>>>(B.master, B.grad, B.m, B.v, B.nparam, lr, b1, b2, eps,
                                                              c1, c2, copies ? B.wfwd : nullptr, B.offs_dev, B.cin_dev,
                                                              B.cout_dev, B.wbwd, B.wtc, B.wtd);
    return cudaGetLastError();
}
