// Batched multi-channel processing: one CUDA graph launch for many channels,
// with a tuner that picks each channel's FD block size and DD-LMS CTA size.
//
// The paper keeps a GPU busy by running five buffers in five streams with
// events ordering the dependent kernels (Sec. II-C, Sec. III). Here every
// channel's chain is captured once, each on its own forked stream, into one
// graph; a batch is then a single cudaGraphLaunch whose branches run
// concurrently and whose stage order is the graph's edges (no device-side
// waiting). Channels are independent, so nothing is exchanged between them.
//
// Tuner: for a channel with fft_size == 0 every N in 512..8192 whose quarter
// block covers the dispersion memory (N/4 >= D L lambda^2 / c * Rs (1 + rolloff)
// * fs samples, the largest N when none does) is timed on the channel's frame
// length with CUDA events, and the fastest kept; lms_threads == 0 times the
// segmented DD-LMS with 128, 256 and 512 threads per CTA. Results are cached
// per (symbol rate, format, taps, D*L, frame length) for the process.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/rx.h"
#include "rx_fft.cuh"
#include "rx_kernels.h"

struct rx_batch {
    int n = 0;
    std::vector<rx_handle*> h;
    std::vector<rx_config> cfg;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;        // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;      // buffers the graph was captured with
    cudaStream_t last = nullptr;
    uint64_t launches = 0;
};

namespace {

constexpr double C_LIGHT = 299792458.0;

using TuneKey = std::tuple<double, int, int, double, int64_t, int>;
std::map<TuneKey, std::pair<int, int>>& tune_cache() {
    static std::map<TuneKey, std::pair<int, int>> m;
    return m;
}
std::mutex& tune_mutex() {
    static std::mutex m;
    return m;
}

double dispersion_memory_samples(const rx_config& c) {
    const double fs = c.sps * c.symbol_rate_hz;
    return std::fabs(c.dispersion_s_per_m2 * c.length_m) * c.wavelength_m * c.wavelength_m / C_LIGHT *
           c.symbol_rate_hz * (1.0 + c.rrc_rolloff) * fs;
}

float time_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

// pick N_fft and DD-LMS threads for one channel; returns false on a CUDA error
bool tune_channel(rx_config& c, int64_t n_sym) {
    const int64_t S = 2 * n_sym;
    TuneKey key{c.symbol_rate_hz, c.bits_per_sym, c.n_taps, c.dispersion_s_per_m2 * c.length_m, n_sym,
                c.fft_size * 16 + (c.lms_threads ? 1 : 0)};
    {
        std::lock_guard<std::mutex> g(tune_mutex());
        auto it = tune_cache().find(key);
        if (it != tune_cache().end()) {
            if (!c.fft_size) c.fft_size = it->second.first;
            if (!c.lms_threads) c.lms_threads = it->second.second;
            return true;
        }
    }
    float2 *in = nullptr, *out = nullptr, *H = nullptr, *tw = nullptr, *taps = nullptr;
    RxDevState* st = nullptr;
    cudaEvent_t e0, e1;
    bool ok = cudaMalloc(&in, sizeof(float2) * 2 * S) == cudaSuccess &&
              cudaMalloc(&out, sizeof(float2) * 2 * (S + 64)) == cudaSuccess &&
              cudaMalloc(&H, sizeof(float2) * 8192) == cudaSuccess &&
              cudaMalloc(&tw, sizeof(float2) * RX_FFT_TW_N) == cudaSuccess &&
              cudaMalloc(&taps, sizeof(float2) * 4 * RX_TMAX) == cudaSuccess &&
              cudaMalloc(&st, sizeof(RxDevState)) == cudaSuccess;
    ok = ok && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (ok) {
        cudaMemset(in, 0, sizeof(float2) * 2 * S);
        cudaMemset(H, 0, sizeof(float2) * 8192);
        cudaMemset(taps, 0, sizeof(float2) * 4 * RX_TMAX);
        cudaMemset(st, 0, sizeof(RxDevState));
        launch_fill_twiddles(tw, 0);
    }
    int best_n = c.fft_size ? c.fft_size : 8192;
    if (ok && !c.fft_size) {
        const double mem = dispersion_memory_samples(c);
        float best = 1e30f;
        bool any = false;
        for (int nfft = 512; nfft <= 8192; nfft *= 2) {
            if (nfft / 4 < mem && nfft != 8192) continue;
            if (any && nfft / 4 < mem) continue;
            CdcArgs a{in, 0, 1.0f, S, nfft, H, tw, nullptr, out, S + 64, 0, st};
            launch_cdc(a, 0);                                   // warm-up (sets attributes)
            cudaEventRecord(e0, 0);
            for (int r = 0; r < 3; ++r) launch_cdc(a, 0);
            cudaEventRecord(e1, 0);
            cudaEventSynchronize(e1);
            const float t = time_ms(e0, e1);
            if (nfft / 4 >= mem || !any) {
                if (t < best) { best = t; best_n = nfft; }
                any = true;
            }
        }
        ok = cudaGetLastError() == cudaSuccess;
    }
    int best_t = c.lms_threads ? c.lms_threads : 256;
    if (ok && !c.lms_threads) {
        float best = 1e30f;
        const int cands[3] = {128, 256, 512};
        for (int i = 0; i < 3; ++i) {
            LmsArgs a{};
            a.x = out;
            a.xstride = S + 64;
            a.xlen = S;
            a.off = 0;
            a.T = c.n_taps;
            a.Lb = c.lms_block;
            a.n_sym = n_sym;
            a.L_seg = (int64_t)c.seg_blocks * c.lms_block;
            a.n_wu = c.warmup_blocks;
            a.cma = 0;
            a.mu = c.mu_dd;
            a.m = c.bits_per_sym;
            a.taps_in = taps;
            a.taps_out = nullptr;
            a.y = in;
            a.ystride = n_sym;
            a.st = st;
            launch_lms(a, cands[i], 0);
            cudaEventRecord(e0, 0);
            for (int r = 0; r < 3; ++r) launch_lms(a, cands[i], 0);
            cudaEventRecord(e1, 0);
            cudaEventSynchronize(e1);
            const float t = time_ms(e0, e1);
            if (t < best) { best = t; best_t = cands[i]; }
        }
        ok = cudaGetLastError() == cudaSuccess;
    }
    cudaFree(in); cudaFree(out); cudaFree(H); cudaFree(tw); cudaFree(taps); cudaFree(st);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    if (!ok) return false;
    if (!c.fft_size) c.fft_size = best_n;
    if (!c.lms_threads) c.lms_threads = best_t;
    std::lock_guard<std::mutex> g(tune_mutex());
    tune_cache()[key] = {c.fft_size, c.lms_threads};
    return true;
}

void batch_free(rx_batch* b) {
    // handles first: rx_destroy waits on the last stream each handle used, one of ours
    for (auto h : b->h) rx_destroy(h);
    b->h.clear();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
}

}  // namespace

extern "C" {

rx_status rx_batch_create(const rx_config* cfgs, int32_t n, rx_batch** out) {
    if (!cfgs || !out || n < 1 || n > 4096) return RX_EINVAL;
    *out = nullptr;
    rx_batch* b = new rx_batch();
    b->n = n;
    for (int i = 0; i < n; ++i) {
        rx_config c = cfgs[i];
        if (c.streaming || c.max_symbols < 1 || c.max_symbols > ((int64_t)1 << 28)) {
            batch_free(b); delete b; return RX_EINVAL;
        }
        if (!tune_channel(c, c.max_symbols)) { batch_free(b); delete b; return RX_ECUDA; }
        rx_handle* h = nullptr;
        rx_status st = rx_create(&c, &h);
        if (st != RX_OK) { batch_free(b); delete b; return st; }
        b->h.push_back(h);
        b->cfg.push_back(c);
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            batch_free(b); delete b; return RX_ECUDA;
        }
        b->streams.push_back(s);
        b->join.push_back(e);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        batch_free(b); delete b; return RX_ECUDA;
    }
    *out = b;
    return RX_OK;
}

rx_status rx_batch_config(rx_batch* b, int32_t i, rx_config* out) {
    if (!b || !out || i < 0 || i >= b->n) return RX_EINVAL;
    *out = b->cfg[i];
    return RX_OK;
}

rx_handle* rx_batch_handle(rx_batch* b, int32_t i) {
    if (!b || i < 0 || i >= b->n) return nullptr;
    return b->h[i];
}

rx_status rx_batch_process(rx_batch* b, const void* const* d_in, const int64_t* n_sym,
                           const uint32_t* const* d_ref, uint32_t* const* d_out, rx_stream_t stream_) {
    if (!b || !d_in || !n_sym) return RX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream_;
    std::vector<const void*> key;
    for (int i = 0; i < b->n; ++i) {
        if (!d_in[i] || n_sym[i] < 1 || n_sym[i] > b->cfg[i].max_symbols) return RX_EINVAL;
        key.push_back(d_in[i]);
        key.push_back((const void*)(intptr_t)n_sym[i]);
        key.push_back(d_ref ? d_ref[i] : nullptr);
        key.push_back(d_out ? d_out[i] : nullptr);
    }
    if (!b->exec || key != b->key) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        // capture on the batch's own stream (the caller's may be the legacy default stream,
        // which cannot be captured); the graph then launches on the caller's stream
        cudaStream_t cap = b->cap;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) return RX_ECUDA;
        rx_status st = RX_OK;
        cudaEventRecord(b->fork, cap);
        for (int i = 0; i < b->n && st == RX_OK; ++i) {
            cudaStreamWaitEvent(b->streams[i], b->fork, 0);
            st = rx_process(b->h[i], d_in[i], n_sym[i], d_ref ? d_ref[i] : nullptr, d_out ? d_out[i] : nullptr,
                            (rx_stream_t)b->streams[i]);
            cudaEventRecord(b->join[i], b->streams[i]);
            cudaStreamWaitEvent(cap, b->join[i], 0);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cap, &g);
        if (st != RX_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (ec != cudaSuccess || !g) return RX_ECUDA;
        b->graph = g;
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) { b->exec = nullptr; return RX_ECUDA; }
        b->key = key;
    }
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return RX_ECUDA;
    b->last = s;
    b->launches += 1;
    return RX_OK;
}

rx_status rx_batch_stats(rx_batch* b, int32_t i, rx_stats_t* out) {
    if (!b || !out || i < 0 || i >= b->n) return RX_EINVAL;
    if (b->last && cudaStreamSynchronize(b->last) != cudaSuccess) return RX_ECUDA;
    rx_status st = rx_stats(b->h[i], out);
    if (st == RX_OK) {
        // the chain was enqueued once (at capture) and replayed `launches` times
        const uint64_t n_sym = b->key.empty() ? 0 : (uint64_t)(intptr_t)b->key[4 * i + 1];
        out->frames = b->launches;
        out->symbols_processed = 2 * n_sym * b->launches;
        out->bits_processed = out->symbols_processed * (uint64_t)b->cfg[i].bits_per_sym;
    }
    return st;
}

uint64_t rx_batch_launch_count(rx_batch* b) { return b ? b->launches : 0; }

void rx_batch_destroy(rx_batch* b) {
    if (!b) return;
    if (b->last) cudaStreamSynchronize(b->last);
    batch_free(b);
    delete b;
}

}  // extern "C"
