// C ABI of the learned post-equaliser (rx_pe_*): allocation at create,
// forward, gradients and Adam training steps on caller-owned device buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "../../include/rx.h"
#include "rx_cnn.h"
#include "rx_dev.cuh"

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
    void* ptrs[] = {B.master, B.m, B.v, B.grad, B.wpart, B.wfwd, B.wbwd, B.wtc, B.offs_dev, B.cin_dev, B.cout_dev, B.out, B.loss,
                    B.act[0], B.act[1], B.act[2], B.act[3], B.d[0], B.d[1], B.d[2], B.d[3], B.err, B.wtd,
                    B.d16[1], B.d16[2]};
    for (void* q : ptrs)
        if (q) cudaFree(q);
}

// Training labels (rx_pe_targets): CTA (j, q) owns symbols [j block, (j + 1) block) of output q.
__global__ void k_pe_targets(const float2* __restrict__ z, int64_t n_sym, const float2* __restrict__ s,
                             int64_t n_ref, int p0, int p1, int r0, int r1, int64_t d0, int64_t d1, int block,
                             float2* __restrict__ out) {
    __shared__ float4 wsum[32];
    __shared__ int best_s;
    const int q = blockIdx.y;
    const int p = q ? p1 : p0, r = q ? r1 : r0;
    const int64_t d = q ? d1 : d0;
    const int64_t lo = (int64_t)blockIdx.x * block, hi = min(n_sym, lo + block);
    const bool whole = hi - lo == block;
    const float2* sp = s + (int64_t)p * n_ref;
    const float2* zq = z + (int64_t)q * n_sym;
    auto label = [&](int64_t n) -> float2 {             // s_p[n + d] (-j)^r, 0 outside the reference
        const int64_t i = n + d;
        if (i < 0 || i >= n_ref) return make_float2(0.0f, 0.0f);
        const float2 v = sp[i];
        switch (r) {
            case 1: return make_float2(v.y, -v.x);
            case 2: return make_float2(-v.x, -v.y);
            case 3: return make_float2(-v.y, v.x);
            default: return v;
        }
    };
    int best = 0;
    if (whole) {
        // sum |z - t u|^2 over the block for u = 1, j, -1, -j: per thread, then the warps in a fixed order
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t n = lo + threadIdx.x; n < hi; n += blockDim.x) {
            const float2 t = label(n), zz = zq[n];
            const float a0 = zz.x - t.x, b0 = zz.y - t.y;     // u = 1:  t
            const float a1 = zz.x + t.y, b1 = zz.y - t.x;     // u = j:  (-t.y, t.x)
            const float a2 = zz.x + t.x, b2 = zz.y + t.y;     // u = -1: -t
            const float a3 = zz.x - t.y, b3 = zz.y + t.x;     // u = -j: (t.y, -t.x)
            e.x += fmaf(a0, a0, b0 * b0);
            e.y += fmaf(a1, a1, b1 * b1);
            e.z += fmaf(a2, a2, b2 * b2);
            e.w += fmaf(a3, a3, b3 * b3);
        }
        e.x = warp_sum(e.x);
        e.y = warp_sum(e.y);
        e.z = warp_sum(e.z);
        e.w = warp_sum(e.w);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) wsum[w] = e;
        __syncthreads();
        if (threadIdx.x == 0) {
            float4 t = wsum[0];
            for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
                t.x += wsum[k].x; t.y += wsum[k].y; t.z += wsum[k].z; t.w += wsum[k].w;
            }
            const float v[4] = {t.x, t.y, t.z, t.w};
            int b = 0;
            for (int u = 1; u < 4; ++u)
                if (v[u] < v[b]) b = u;                        // first minimum
            best_s = b;
        }
        __syncthreads();
        best = best_s;
    }
    for (int64_t n = lo + threadIdx.x; n < hi; n += blockDim.x) {
        float2 t = label(n);
        switch (best) {                                        // t j^best
            case 1: t = make_float2(-t.y, t.x); break;
            case 2: t = make_float2(-t.x, -t.y); break;
            case 3: t = make_float2(t.y, -t.x); break;
            default: break;
        }
        out[(int64_t)q * n_sym + n] = t;
    }
}

}  // namespace

extern "C" {

rx_status rx_pe_targets(const float* d_z, int64_t n_sym, const float* d_symbols, int64_t n_ref,
                        const int32_t* h_pol_map, const int32_t* h_rotation, const int32_t* h_delay, int32_t block,
                        float* d_target, rx_stream_t stream) {
    if (!d_z || !d_symbols || !d_target || !h_pol_map || !h_rotation || !h_delay) return RX_EINVAL;
    if (n_sym < 1 || n_ref < 1 || block < 1) return RX_EINVAL;
    for (int q = 0; q < 2; ++q)
        if (h_pol_map[q] < 0 || h_pol_map[q] > 1 || h_rotation[q] < 0 || h_rotation[q] > 3) return RX_EINVAL;
    const int64_t nb = (n_sym + block - 1) / block;
    if (nb > 0x7fffffff) return RX_EINVAL;
    k_pe_targets<<<dim3((unsigned)nb, 2), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float2*>(d_z), n_sym, reinterpret_cast<const float2*>(d_symbols), n_ref, h_pol_map[0],
        h_pol_map[1], h_rotation[0], h_rotation[1], h_delay[0], h_delay[1], block, reinterpret_cast<float2*>(d_target));
    return cudaGetLastError() == cudaSuccess ? RX_OK : RX_ECUDA;
}

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
    A(cudaMalloc(&B.wpart, sizeof(float) * CNN_WG_SPLIT * ((size_t)channels * channels * 9 + channels)));
    A(cudaMalloc(&B.wfwd, sizeof(float) * B.nparam));
    A(cudaMalloc(&B.wbwd, sizeof(float) * B.nparam));
    A(cudaMalloc(&B.wtc, sizeof(__nv_bfloat16) * (size_t)wtc_elems(channels)));
    A(cudaMalloc(&B.wtd, sizeof(__nv_bfloat16) * 2 * (size_t)channels * channels * 9));
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
        if (l == 1 || l == 2) A(cudaMalloc(&B.d16[l], sizeof(__nv_bfloat16) * channels * Tp));
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
    if (cnn_forward(B, (const float2*)d_z, T, T, B.out, s) != cudaSuccess) return RX_ECUDA;
    if (cudaMemsetAsync(B.loss, 0, sizeof(float), s) != cudaSuccess) return RX_ECUDA;
    if (cnn_backward(B, B.out, (const float2*)d_target, T, T, B.loss, s) != cudaSuccess) return RX_ECUDA;
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
    if (cnn_adam(p->B, lr, p->step, s, true) != cudaSuccess) return RX_ECUDA;
    return RX_OK;
}

rx_status rx_pe_train_steps(rx_pe* p, const float* const* d_z, const float* const* d_target, const int64_t* len,
                            int32_t npairs, int64_t window, int32_t steps, const int32_t* which, const int64_t* offs,
                            const float* lrs, float* d_losses, rx_stream_t stream) {
    if (!p || !d_z || !d_target || !len || npairs < 1 || window < 1 || window > p->B.Tmax || steps < 0 ||
        (steps > 0 && (!which || !offs || !lrs)))
        return RX_EINVAL;
    for (int32_t i = 0; i < steps; ++i) {
        const int32_t k = which[i];
        if (k < 0 || k >= npairs || !d_z[k] || !d_target[k] || offs[i] < 0 || offs[i] + window > len[k])
            return RX_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    p->last = s;
    CnnBufs& B = p->B;
    if (cnn_zero_pads(B, window, s) != cudaSuccess) return RX_ECUDA;   // the pad columns of this length
    if (d_losses && steps > 0 && cudaMemsetAsync(d_losses, 0, sizeof(float) * (size_t)steps, s) != cudaSuccess)
        return RX_ECUDA;
    for (int32_t i = 0; i < steps; ++i) {
        const int32_t k = which[i];
        const float2* z = reinterpret_cast<const float2*>(d_z[k]) + offs[i];
        const float2* t = reinterpret_cast<const float2*>(d_target[k]) + offs[i];
        // the loss accumulates straight into its slot of d_losses (zeroed above), else into B.loss; the
        // forward's output layer forms the loss gradient
        float* loss = d_losses ? d_losses + i : B.loss;
        if (!d_losses && cudaMemsetAsync(B.loss, 0, sizeof(float), s) != cudaSuccess) return RX_ECUDA;
        if (cnn_forward(B, z, len[k], window, B.out, s, t, len[k], loss) != cudaSuccess) return RX_ECUDA;
        if (cnn_backward(B, B.out, nullptr, 0, window, nullptr, s) != cudaSuccess) return RX_ECUDA;
        p->step += 1;
        // the Adam step and the weight copies of the new values in one launch
        if (cnn_adam(B, lrs[i], p->step, s, true) != cudaSuccess) return RX_ECUDA;
    }
    return RX_OK;
}

void rx_pe_destroy(rx_pe* p) {
    if (!p) return;
    if (p->last) cudaStreamSynchronize(p->last);
    pe_free(p);
    delete p;
}

}  // extern "C"
