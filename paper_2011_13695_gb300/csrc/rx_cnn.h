// Device buffers and launchers of the learned post-equaliser (k_cnn.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

// the weight gradients sum their positions in CNN_WG_SPLIT interleaved shares (one CTA each), then the
// shares in a fixed order: the same sums on every run
#define CNN_WG_SPLIT 48

struct CnnBufs {
    int C = 64;                     // hidden channels
    int64_t nparam = 0;
    int64_t off[8] = {0};           // parameter offsets: W0, b0, W1, b1, W2, b2, W3, b3
    int64_t Tmax = 0;
    float* master = nullptr;        // FP32 master parameters (oracle order)
    float* m = nullptr;             // Adam moments
    float* v = nullptr;
    float* grad = nullptr;          // FP32 gradients of the last backward
    float* wpart = nullptr;         // [CNN_WG_SPLIT][C * C * 9 + C] per-CTA weight-gradient partials
    float* wfwd = nullptr;          // BF16-rounded parameters as used by the forward
    float* wbwd = nullptr;          // transposed, flipped BF16-rounded weights for the data gradient
    // BF16 weights in (k, ci) order for the tensor cores: layers 1, 2 as [64][9 * 64], layer 3 as
    // [4][9 * 64], then layer 0 as [64][48] (9 * 4 entries, the rest zero)
    __nv_bfloat16* wtc = nullptr;
    // BF16 weights of the hidden layers' data gradient in (k, co) order: layer l (1, 2) at (l - 1) 64 x 576,
    // row ci, entry k x 64 + co = W_l[co][ci][8 - k] (the flipped transpose)
    __nv_bfloat16* wtd = nullptr;
    __nv_bfloat16* d16[3] = {nullptr, nullptr, nullptr};            // BF16 copies of d[1], d[2] ([C][Tp])
    int* offs_dev = nullptr;        // off[] on the device (int)
    int* cin_dev = nullptr;
    int* cout_dev = nullptr;
    __nv_bfloat16* act[4] = {nullptr, nullptr, nullptr, nullptr};   // [4][Tp], [C][Tp] x 3
    float* d[4] = {nullptr, nullptr, nullptr, nullptr};             // [C][Tp] x 3, [4][Tp]
    float2* out = nullptr;          // [2][Tmax] forward output used by training
    float* loss = nullptr;          // [1]
    unsigned int* err = nullptr;    // [1] error word (RX_ERR_* bits) of the tensor-core kernels
};

// z, tgt: the two polarisations zs / ts complex samples apart (T for contiguous sequences). With a target,
// the forward also forms the loss gradient and adds the loss, and the backward is then called without one.
cudaError_t cnn_forward(const CnnBufs& B, const float2* z, int64_t zs, int64_t T, float2* out, cudaStream_t s,
                        const float2* tgt = nullptr, int64_t ts = 0, float* loss = nullptr);
cudaError_t cnn_backward(const CnnBufs& B, const float2* out, const float2* tgt, int64_t ts, int64_t T, float* loss,
                         cudaStream_t s);
cudaError_t cnn_prepare_weights(const CnnBufs& B, cudaStream_t s);
// one Adam step; with copies, also the weight copies of cnn_prepare_weights for the new values
cudaError_t cnn_adam(const CnnBufs& B, float lr, int step, cudaStream_t s, bool copies = false);
cudaError_t cnn_zero_pads(const CnnBufs& B, int64_t T, cudaStream_t s);
// the inference forward on the tcgen05 tensor cores (k_cnn_tc.cu); act[1..3] hold planar activations
cudaError_t cnn_infer_tc(const CnnBufs& B, const float2* z, int64_t T, float2* out, cudaStream_t s);
// element offsets in wtc
__host__ __device__ inline int64_t wtc_offset(int C, int layer) {
    const int64_t lw = (int64_t)C * C * 9;
    return layer == 1 ? 0 : layer == 2 ? lw : layer == 3 ? 2 * lw : 2 * lw + 4 * (int64_t)C * 9;
}
__host__ __device__ inline int64_t wtc_elems(int C) { return wtc_offset(C, 0) + (int64_t)C * 48; }
// one 64 -> 64 forward convolution (bias, ReLU, BF16 out) on the tensor cores (k_cnn_mma.cu);
// Wm: the layer's BF16 weights as [co][k * 64 + ci]
cudaError_t conv64_mma_fwd(const __nv_bfloat16* x, int64_t Tp, int64_t T, const __nv_bfloat16* Wm, const float* b,
                           __nv_bfloat16* act, cudaStream_t s);
// the data gradient of a 64 -> 64 layer on the tensor cores: din[ci][t] = (sum_{k, co} Wd[ci][k * 64 + co]
// dout[co][t + k - 4]) x (mask[ci][t] > 0), FP32 into din and (nullable) BF16 into din16; dout BF16 planes
// the partial rows of a 64 -> 64 layer's weight and bias gradients on the tensor cores (at most max_rows
// rows of C * C * 9 + C floats in part; *nrow = rows written); x: the layer's input activation planes,
// dy16: the BF16 copy of the gradient planes
cudaError_t conv64_mma_wgrad_parts(const __nv_bfloat16* x, const __nv_bfloat16* dy16, int64_t Tp, int64_t T,
                                   float* part, int max_rows, int* nrow, cudaStream_t s);
cudaError_t conv64_mma_dgrad(const __nv_bfloat16* dout, int64_t Tp, int64_t T, const __nv_bfloat16* Wd,
                             const __nv_bfloat16* mask, float* din, __nv_bfloat16* din16, cudaStream_t s);
