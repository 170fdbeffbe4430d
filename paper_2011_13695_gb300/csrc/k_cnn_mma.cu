// The 64 -> 64 convolutions of the learned post-equaliser's forward pass on the
// tensor cores: BF16 x BF16 products, FP32 accumulation (mma.sync m16n8k16).
//
// As a matrix product, out[co][t] = sum_K A[co][K] B[K][t] with K = (k, ci) in
// the order k * 64 + ci: A[co][k*64 + ci] = W[co][ci][k] and
// B[k*64 + ci][t] = x[ci][t + k - 4]. A CTA computes all 64 output channels
// of 128 positions per tile and loops over tiles (one resident wave of CTAs):
// it converts the layer's weights to BF16 in shared memory once, in rows of
// (k, ci) padded to 584 entries so that the 8 rows an ldmatrix reads fall in
// distinct banks; per tile it stages the input positions t0 - 4 .. t0 + 132
// transposed to [position][channel] (rows of 72 entries), so that the B
// fragment of tap k is an ldmatrix of rows shifted by k. Eight warps take
// 32 x 32 output blocks (2 x 4 mma tiles, 36 K-steps of 16). The epilogue adds
// the bias, applies the ReLU, rounds to BF16 and writes the activation plane.
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
constexpr size_t SMEM = sizeof(__nv_bfloat16) * ((size_t)C * WS + (size_t)XR * XS);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
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

__global__ void __launch_bounds__(NTHR, 2) k_conv64_mma(const __nv_bfloat16* __restrict__ x, int64_t Tp, int64_t T,
                                                        const float* __restrict__ W, const float* __restrict__ bias,
                                                        __nv_bfloat16* __restrict__ act_out, int vec) {
    extern __shared__ float4 smem4[];
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(smem4);      // [C][WS]
    __nv_bfloat16* Xs = Ws + C * WS;                                  // [XR][XS]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;                          // 2 x 4 warps of 32 x 32
    const int g = lane >> 2, tq = lane & 3;

    // weights, once: Ws[co][k * 64 + ci] = W[co][ci][k] (W holds BF16-rounded values)
    for (int i = tid; i < C * KTOT; i += NTHR) {
        const int co = i / KTOT, r = i - co * KTOT, ci = r / KW, k = r - ci * KW;
        Ws[co * WS + k * C + ci] = __float2bfloat16_rn(W[i]);
    }
    float bco[2][2];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int h = 0; h < 2; ++h) bco[mi][h] = bias[wm * 32 + mi * 16 + g + 8 * h];

    // ldmatrix row addresses: A rows co0 + (lane % 16), column block (lane / 16) * 8;
    // B^T rows n = (lane / 16) * 8 + lane % 8 of an n-tile pair, column block ((lane / 8) % 2) * 8
    const uint32_t a_base = smem_addr(Ws + (wm * 32 + (lane & 15)) * WS + (lane >> 4) * 8);
    const int bn = (lane >> 4) * 8 + (lane & 7), bk = ((lane >> 3) & 1) * 8;
    const uint32_t b_base = smem_addr(Xs + (wn * 32 + bn) * XS + bk);

    const int64_t ntiles = (T + TT - 1) / TT;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t t0 = tile * TT;                 // first output position; staged rows = padded t0 ..
        __syncthreads();                              // previous tile's reads of Xs are done
        // stage x[ci][t0 + r] (padded index) transposed into Xs[r][ci], r < XR, zero past Tp
        if (vec) {
            constexpr int CH = XR / 8;                // 16-byte chunks per channel
            for (int i = tid; i < C * CH; i += NTHR) {
                const int ci = i / CH, u = i - ci * CH;
                const int64_t tp = t0 + 8 * u;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (tp + 7 < Tp) v = *reinterpret_cast<const uint4*>(x + (int64_t)ci * Tp + tp);
                else {
                    __nv_bfloat16 tmp[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) tmp[e] = tp + e < Tp ? x[(int64_t)ci * Tp + tp + e] : __float2bfloat16_rn(0.0f);
                    v = *reinterpret_cast<const uint4*>(tmp);
                }
                const __nv_bfloat16* e8 = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
                for (int e = 0; e < 8; ++e) Xs[(8 * u + e) * XS + ci] = e8[e];
            }
        } else {
            for (int i = tid; i < C * XR; i += NTHR) {
                const int ci = i / XR, r = i - ci * XR;
                const int64_t tp = t0 + r;
                Xs[r * XS + ci] = tp < Tp ? x[(int64_t)ci * Tp + tp] : __float2bfloat16_rn(0.0f);
            }
        }
        __syncthreads();

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
        // epilogue: bias, ReLU, BF16 -> act_out[co][t + PAD]
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int h = e >> 1;
                    const int co = wm * 32 + mi * 16 + g + 8 * h;
                    const int64_t t = t0 + wn * 32 + ni * 8 + 2 * tq + (e & 1);
                    if (t < T) {
                        const float v = fmaxf(acc[mi][ni][e] + bco[mi][h], 0.0f);
                        act_out[(int64_t)co * Tp + t + PAD] = __float2bfloat16_rn(v);
                    }
                }
    }
}

}  // namespace

cudaError_t conv64_mma_fwd(const __nv_bfloat16* x, int64_t Tp, int64_t T, const float* W, const float* b,
                           __nv_bfloat16* act, cudaStream_t s) {
    static int resident = 0;
    if (!resident) {
        int dev = 0, nsm = 152, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_conv64_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_conv64_mma, NTHR, SMEM);
        resident = std::max(1, nsm * per);
    }
    const int64_t ntiles = (T + TT - 1) / TT;
    const int grid = (int)std::min<int64_t>(ntiles, resident);
    // 16-byte staging loads need 16-byte aligned rows
    const int vec = ((uintptr_t)x % 16 == 0) && (Tp % 8 == 0);
    k_conv64_mma<<<grid, NTHR, SMEM, s>>>(x, Tp, T, W, b, act, vec);
    return cudaGetLastError();
}
