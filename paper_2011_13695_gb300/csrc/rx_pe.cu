// C ABI of the learned post-equaliser (rx_pe_*): allocation at create,
// forward, gradients and Adam training steps on caller-owned device buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "../../include/rx.h"
#include "rx_cnn.h"

struct rx_pe {
    CnnBufs B;
    int step = 0;
    cudaStream_t last = nullptr;
};

namespace {

constexpr int KW = 9;

int64_t count_params(int C, int64_t* off) {
    const int cin[4] = {4, C, C, C}, cout[4] = {C, C, C, 4};
    int64_t o = 0;
    for (int l = 0; l < 4; ++l) {
        if (off) off[2 * l] = o;
        o += (int64_t)cout[l] * cin[l] * KW;
        if (off) off[2 * l + 1] = o;
        o += cout[l];
    }
    return o;
}

void pe_free(rx_pe* p) {
    CnnBufs& B = p->B;
    void* ptrs[] = {B.master, B.m, B.v, B.grad, B.wfwd, B.wbwd, B.wtc, B.offs_dev, B.cin_dev, B.cout_dev, B.out, B.loss,
                    B.act[0], B.act[1], B.act[2], B.act[3], B.d[0], B.d[1], B.d[2], B.d[3], B.err};
    for (void* q : ptrs)
        if (q) cudaFree(q);
}

}  // namespace

extern "C" {

int64_t rx_pe_param_count(int32_t channels, int32_t kernel) {
    if (channels != 64 || kernel != KW) return -1;
    return count_params(channels, nullptr);
}

rx_status rx_pe_create(int32_t channels, int32_t kernel, int64_t max_len, const float* h_params, rx_pe** out) {
    if (!out || channels != 64 || kernel != KW || max_len < 1 || max_len > ((int64_t)1 << 24)) return RX_EINVAL;
    *out = nullptr;
    rx_pe* p = new (std::nothrow) rx_pe();
    if (!p) return RX_ENOMEM;
    CnnBufs& B = p->B;
    B.C = channels;
    B.Tmax = max_len;
    B.nparam = count_params(channels, B.off);
    const int64_t Tp = max_len + 2 * (KW / 2);
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(cudaMalloc(&B.master, sizeof(float) * B.nparam));
    A(cudaMalloc(&B.m, sizeof(float) * B.nparam));
    A(cudaMalloc(&B.v, sizeof(float) * B.nparam));
    A(cudaMalloc(&B.grad, sizeof(float) * B.nparam));
    A(cudaMalloc(&B.wfwd, sizeof(float) * B.nparam));
    A(cudaMalloc(&B.wbwd, sizeof(float) * B.nparam));
    A(cudaMalloc(&B.wtc, sizeof(__nv_bfloat16) * (size_t)wtc_elems(channels)));
    A(cudaMalloc(&B.err, sizeof(unsigned int)));
    A(cudaMalloc(&B.offs_dev, sizeof(int) * 8));
    A(cudaMalloc(&B.cin_dev, sizeof(int) * 4));
    A(cudaMalloc(&B.cout_dev, sizeof(int) * 4));
    A(cudaMalloc(&B.out, sizeof(float2) * 2 * max_len));
    A(cudaMalloc(&B.loss, sizeof(float)));
    for (int l = 0; l < 4; ++l) {
        const int ach = l == 0 ? 4 : channels, dch = l == 3 ? 4 : channels;
        A(cudaMalloc(&B.act[l], sizeof(__nv_bfloat16) * ach * Tp));
        A(cudaMalloc(&B.d[l], sizeof(float) * dch * Tp));
    }
    if (e != cudaSuccess) {
        pe_free(p);
        delete p;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? RX_ENOMEM : RX_ECUDA;
    }
    int offs[8], cin[4] = {4, channels, channels, channels}, cout[4] = {channels, channels, channels, 4};
    for (int i = 0; i < 8; ++i) offs[i] = (int)B.off[i];
    A(cudaMemcpy(B.offs_dev, offs, sizeof(offs), cudaMemcpyHostToDevice));
    A(cudaMemcpy(B.cin_dev, cin, sizeof(cin), cudaMemcpyHostToDevice));
    A(cudaMemcpy(B.cout_dev, cout, sizeof(cout), cudaMemcpyHostToDevice));
    if (h_params) A(cudaMemcpy(B.master, h_params, sizeof(float) * B.nparam, cudaMemcpyHostToDevice));
    else A(cudaMemset(B.master, 0, sizeof(float) * B.nparam));
    A(cudaMemset(B.m, 0, sizeof(float) * B.nparam));
    A(cudaMemset(B.v, 0, sizeof(float) * B.nparam));
    A(cudaMemset(B.wtc, 0, sizeof(__nv_bfloat16) * (size_t)wtc_elems(channels)));   // the input layer's K padding
    A(cudaMemset(B.err, 0, sizeof(unsigned int)));
    A(cnn_prepare_weights(B, 0));
    A(cudaDeviceSynchronize());
    if (e != cudaSuccess) {
        pe_free(p);
        delete p;
        return RX_ECUDA;
    }
    *out = p;
    return RX_OK;
}

rx_status rx_pe_params(rx_pe* p, float* h_params) {
    if (!p || !h_params) return RX_EINVAL;
    if (p->last && cudaStreamSynchronize(p->last) != cudaSuccess) return RX_ECUDA;
    if (cudaMemcpy(h_params, p->B.master, sizeof(float) * p->B.nparam, cudaMemcpyDeviceToHost) != cudaSuccess)
        return RX_ECUDA;
    return RX_OK;
}

rx_status rx_pe_forward(rx_pe* p, const float* d_z, int64_t T, float* d_out, rx_stream_t stream) {
    if (!p || !d_z || !d_out || T < 1 || T > p->B.Tmax) return RX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    p->last = s;
    if (cnn_infer_tc(p->B, (const float2*)d_z, T, (float2*)d_out, s) != cudaSuccess) return RX_ECUDA;
    return RX_OK;
}

rx_status rx_pe_error_word(rx_pe* p, uint32_t* out) {
    if (!p || !out) return RX_EINVAL;
    if (p->last && cudaStreamSynchronize(p->last) != cudaSuccess) return RX_ECUDA;
    unsigned int w = 0;
    if (cudaMemcpy(&w, p->B.err, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return RX_ECUDA;
    *out = w;
    return RX_OK;
}

rx_status rx_pe_gradients(rx_pe* p, const float* d_z, const float* d_target, int64_t T, float* d_grads,
                          float* d_loss, rx_stream_t stream) {
    if (!p || !d_z || !d_target || T < 1 || T > p->B.Tmax) return RX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    p->last = s;
    CnnBufs& B = p->B;
    if (cnn_zero_pads(B, T, s) != cudaSuccess) return RX_ECUDA;
    if (cnn_forward(B, (const float2*)d_z, T, B.out, s) != cudaSuccess) return RX_ECUDA;
    if (cudaMemsetAsync(B.loss, 0, sizeof(float), s) != cudaSuccess) return RX_ECUDA;
    if (cnn_backward(B, B.out, (const float2*)d_target, T, B.loss, s) != cudaSuccess) return RX_ECUDA;
    if (d_grads && cudaMemcpyAsync(d_grads, B.grad, sizeof(float) * B.nparam, cudaMemcpyDeviceToDevice, s))
        return RX_ECUDA;
    if (d_loss && cudaMemcpyAsync(d_loss, B.loss, sizeof(float), cudaMemcpyDeviceToDevice, s)) return RX_ECUDA;
    return RX_OK;
}

rx_status rx_pe_train_step(rx_pe* p, const float* d_z, const float* d_target, int64_t T, float lr, float* d_loss,
                           rx_stream_t stream) {
    rx_status r = rx_pe_gradients(p, d_z, d_target, T, nullptr, d_loss, stream);
    if (r != RX_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    p->step += 1;
    if (cnn_adam(p->B, lr, p->step, s) != cudaSuccess) return RX_ECUDA;
    if (cnn_prepare_weights(p->B, s) != cudaSuccess) return RX_ECUDA;
    return RX_OK;
}

void rx_pe_destroy(rx_pe* p) {
    if (!p) return;
    if (p->last) cudaStreamSynchronize(p->last);
    pe_free(p);
    delete p;
}

}  // extern "C"
