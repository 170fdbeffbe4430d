// librx host side: the C ABI of include/rx.h.
//
// rx_create validates the configuration, allocates every buffer the handle
// will ever use and computes the FD filter and FFT twiddles on the device.
// rx_process enqueues the chain on the caller's stream without allocating or
// synchronising; decisions that depend on data (the CMA rerun, the FO code,
// the alignment) stay on the device, so the host never waits for them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rx.h"
#include "rx_fft.cuh"
#include "rx_kernels.h"

namespace {

constexpr double C_LIGHT = 299792458.0;

enum Stage {
    ST_POWER, ST_CDC, ST_CMA, ST_FOE, ST_DDACQ, ST_LMS, ST_BPS, ST_UNWRAP, ST_SYNC, ST_COUNT, ST_STATE, ST_H2D,
    ST_D2H, ST_CDC_REST, ST_N
};
// "cdc" is the part of the FD compensation the acquisition reads (all of it when there is no
// acquisition); "cdc_rest" the remainder, which runs on the handle's side stream beside the acquisition
const char* kStageNames[ST_N] = {"power", "cdc", "cma", "foe", "dd_acq", "lms", "bps",
                                 "unwrap", "sync", "count", "stream_state", "h2d", "d2h", "cdc_rest"};
constexpr int kPool = 64;
// CTA sizes of the block-LMS kernel: the acquisition is one CTA per output row
// and latency-bound, and four warps (eight outputs per lane) carry the least
// per-step overhead; the segments are many CTAs, three of which share an SM.
constexpr int kAcqThreads = 128;
constexpr int kSegThreads = 128;

__global__ void k_state_init(RxDevState* st) {
    st->b_prev[0] = st->b_prev[1] = -1;
    st->scale[0] = st->scale[1] = 1.0f;
}

// start of a decision-only call: forget the carried unwrap state and alignment
__global__ void k_decide_begin(RxDevState* st) {
    st->b_prev[0] = st->b_prev[1] = -1;
    st->m_prev[0] = st->m_prev[1] = 0;
    st->sync_valid = 0;
}

__global__ void k_identity_taps(float2* taps, int T) {
    const int t = threadIdx.x;
    if (t < 4 * T) {
        const int q = t / (2 * T), p = (t / T) & 1, k = t % T;
        taps[t] = make_float2((q == p && k == (T - 1) / 2) ? 1.0f : 0.0f, 0.0f);
    }
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) { int k = 0; while ((1 << k) < v) ++k; return k; }

}  // namespace

struct rx_handle {
    rx_config cfg;
    int dev = 0;
    int m = 2, T = 15, c = 7, d4 = 4, hist = 15, Lb = 64, hop = 512;
    int64_t Nmax = 0, Smax = 0, cap = 0;
    int64_t nacq = 0, nw = 0;
    int kf = 9;
    double fs = 0.0;
    // device memory
    float2* H = nullptr;
    float2* tw = nullptr;
    float2* cdc = nullptr;        // [2][cap]
    float2* tail = nullptr;       // [2][hop]
    float2* y = nullptr;          // [2][Nmax]
    float2* z = nullptr;
    uint8_t* bstar = nullptr;
    int* mq = nullptr;
    int* tiles = nullptr;
    float2* yacq = nullptr;       // [2][nacq]
    float2* yfoe = nullptr;       // [2][nw]
    int* sync_counts = nullptr;
    int* flag = nullptr;
    float2* taps_id = nullptr;
    RxDevState* st = nullptr;
    void* stage_in = nullptr;
    uint32_t* stage_ref = nullptr;
    uint32_t* stage_out = nullptr;
    int64_t in_elem = 8;
    // host bookkeeping
    uint64_t frames = 0, sym_processed = 0;
    bool sync_done = false;
    cudaStream_t last = nullptr;
    cudaStream_t side = nullptr;   // the rest of a frame's FD compensation, beside the acquisition
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_host = nullptr;
    cudaEvent_t ev_chk = nullptr, ev_chk_done = nullptr;   // the rerun's check beside the segments
    // replay of a single frame's launches as one CUDA graph, per entry point (device / host buffers)
    struct FrameGraph {
        bool valid = false, timing = false;
        const void* in = nullptr;
        const void* ref = nullptr;
        void* out = nullptr;
        int64_t n = 0;
        cudaGraphExec_t exec = nullptr;
        uint64_t nl = 0;                // kernels per replay
        int events[ST_N] = {0};         // stage events recorded per replay
    } graph[2];
    cudaStream_t capstream = nullptr;  // graphs are captured here
    bool graphs_ok = true;
    bool capturing = false;
    int graph_misses = 0;               // captures in a row without a replay
    uint64_t launches = 0;
    cudaError_t last_err = cudaSuccess;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev0[ST_N], ev1[ST_N];
    int used[ST_N] = {0};
    double tot_ms[ST_N] = {0};
    int64_t tot_n[ST_N] = {0};
};

namespace {

void timing_flush(rx_handle* h) {
    for (int s = 0; s < ST_N; ++s) {
        for (int i = 0; i < h->used[s]; ++i) {
            float ms = 0.0f;
            cudaEventSynchronize(h->ev1[s][i]);
            if (cudaEventElapsedTime(&ms, h->ev0[s][i], h->ev1[s][i]) == cudaSuccess) {
                h->tot_ms[s] += ms;
                h->tot_n[s] += 1;
            }
        }
        h->used[s] = 0;
    }
}

struct StageScope {
    rx_handle* h;
    int s;
    cudaStream_t st;
    bool on;
    // while a frame is captured into a graph the events must be recorded by the graph itself
    // (an external record), not taken as a capture dependency
    StageScope(rx_handle* h_, int s_, cudaStream_t st_) : h(h_), s(s_), st(st_), on(h_->timing) {
        if (on) {
            if (h->used[s] >= kPool) timing_flush(h);
            cudaEventRecordWithFlags(h->ev0[s][h->used[s]], st, h->capturing ? cudaEventRecordExternal : 0);
        }
    }
    ~StageScope() {
        if (on) {
            cudaEventRecordWithFlags(h->ev1[s][h->used[s]], st, h->capturing ? cudaEventRecordExternal : 0);
            h->used[s] += 1;
        }
    }
};

#define RX_CK(expr)                                   \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) {                      \
            h->last_err = e_;                         \
            return RX_ECUDA;                          \
        }                                             \
    } while (0)

rx_status validate(const rx_config* c) {
    if (!c) return RX_EINVAL;
    if (c->bits_per_sym != 2 && c->bits_per_sym != 4 && c->bits_per_sym != 6 && c->bits_per_sym != 8) return RX_EINVAL;
    if (c->sps != 2) return RX_EINVAL;
    if (!(c->symbol_rate_hz > 0.0) || !std::isfinite(c->symbol_rate_hz)) return RX_EINVAL;
    if (!std::isfinite(c->dispersion_s_per_m2) || !std::isfinite(c->length_m) || !std::isfinite(c->wavelength_m))
        return RX_EINVAL;
    if (!(c->rrc_rolloff >= 0.0 && c->rrc_rolloff <= 1.0)) return RX_EINVAL;
    if (!pow2(c->fft_size) || c->fft_size < 512 || c->fft_size > 8192) return RX_EINVAL;
    if (c->n_taps < 3 || c->n_taps > RX_TMAX || (c->n_taps & 1) == 0) return RX_EINVAL;
    if (c->lms_block < 16 || c->lms_block > 256) return RX_EINVAL;
    if (c->cma_blocks < 0 || c->dd_acq_blocks < 0 || c->seg_blocks < 1) return RX_EINVAL;
    if (c->warmup_blocks < 0 || c->warmup_blocks > c->seg_blocks) return RX_EINVAL;
    if ((int64_t)c->cma_blocks * c->lms_block > 16384) return RX_EINVAL;
    if (c->bps_phases < 2 || c->bps_phases > RX_BPS_MAXB) return RX_EINVAL;
    if (!pow2(c->bps_window) || c->bps_window < 2 || c->bps_window > 64) return RX_EINVAL;
    if (c->edge_skip < 0 || c->sync_len < 1 || c->sync_len > 32768 || c->max_delay < 0 || c->max_delay > RX_MAX_DELAY) return RX_EINVAL;
    if (!(c->mu_cma >= 0.0f) || !(c->mu_dd >= 0.0f)) return RX_EINVAL;
    if (!(c->fo_grid_hz > 0.0)) return RX_EINVAL;
    if (c->input_format < 0 || c->input_format > 2) return RX_EINVAL;
    if (!std::isfinite(c->input_scale)) return RX_EINVAL;
    if (c->max_symbols < 1 || c->max_symbols > (int64_t)1 << 28) return RX_EINVAL;
    if (c->streaming && (c->max_symbols % (c->fft_size / 4)) != 0) return RX_EINVAL;
    if (c->lms_threads != 0 && c->lms_threads != 128 && c->lms_threads != 256 && c->lms_threads != 512 &&
        c->lms_threads != 1024)
        return RX_EINVAL;
    return RX_OK;
}

template <class T>
cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

void free_all(rx_handle* h) {
    void* ptrs[] = {h->H,    h->tw,    h->cdc,   h->tail,     h->y,           h->z,    h->bstar,
                    h->mq,   h->tiles, h->yacq,  h->yfoe,     h->sync_counts, h->flag,
                    h->taps_id, h->st, h->stage_in, h->stage_ref, h->stage_out};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int s = 0; s < ST_N; ++s) {
        for (auto e : h->ev0[s]) cudaEventDestroy(e);
        for (auto e : h->ev1[s]) cudaEventDestroy(e);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_chk) cudaEventDestroy(h->ev_chk);
    if (h->ev_chk_done) cudaEventDestroy(h->ev_chk_done);
    if (h->ev_host) cudaEventDestroy(h->ev_host);
    for (auto& g : h->graph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (h->capstream) cudaStreamDestroy(h->capstream);
    if (h->side) cudaStreamDestroy(h->side);
}

// Single frame with an acquisition: the number of overlap-save blocks whose FD compensation the
// acquisition reads (symbols [0, max(n_cma, n_dd) Lb) plus the filter's reach); those come first,
// the rest can run beside the acquisition. 0: no such split.
int64_t acq_cdc_blocks(const rx_handle* h, int64_t N) {
    const rx_config& c = h->cfg;
    if (c.streaming) return 0;
    const int64_t n_cma = std::min<int64_t>(c.cma_blocks, N / h->Lb);
    if (n_cma <= 0) return 0;
    const int64_t n_dd = std::min<int64_t>(c.dd_acq_blocks, N / h->Lb);
    const int hopc = c.fft_size / 2;
    const int64_t nblk = (2 * N + hopc - 1) / hopc;
    const int64_t acq_sym = std::max(n_cma, n_dd) * h->Lb;
    const int64_t na = std::min<int64_t>(nblk, (2 * acq_sym + h->T + 2 + hopc - 1) / hopc);
    return na < nblk ? na : 0;
}

}  // namespace

extern "C" {

const char* rx_strerror(rx_status s) {
    switch (s) {
        case RX_OK: return "ok";
        case RX_EINVAL: return "invalid argument or configuration";
        case RX_ENOMEM: return "device out of memory";
        case RX_ECUDA: return "CUDA error";
        case RX_ETIMEOUT: return "device wait timed out";
        case RX_ESTATE: return "state does not match this handle";
        default: return "unknown status";
    }
}

int32_t rx_stage_count(void) { return ST_N; }
const char* rx_stage_name(int32_t s) { return (s >= 0 && s < ST_N) ? kStageNames[s] : ""; }

rx_status rx_create(const rx_config* cfg, rx_handle** out) {
    if (!out) return RX_EINVAL;
    *out = nullptr;
    rx_status v = validate(cfg);
    if (v != RX_OK) return v;
    rx_handle* h = new (std::nothrow) rx_handle();
    if (!h) return RX_ENOMEM;
    h->cfg = *cfg;
    cudaGetDevice(&h->dev);
    h->m = cfg->bits_per_sym;
    h->T = cfg->n_taps;
    h->c = (h->T - 1) / 2;
    h->d4 = (h->c + 1) / 2;
    h->hist = h->c + 2 * h->d4;
    h->Lb = cfg->lms_block;
    h->hop = cfg->fft_size / 2;
    h->Nmax = cfg->max_symbols;
    h->Smax = 2 * h->Nmax;
    h->cap = h->hist + h->Smax;
    h->nacq = (int64_t)cfg->cma_blocks * h->Lb;
    h->nw = h->nacq - h->nacq / 2;
    int nf = 512;
    while (nf < 2 * h->nw) nf *= 2;
    h->kf = ilog2(nf);
    h->fs = cfg->sps * cfg->symbol_rate_hz;
    h->in_elem = cfg->input_format == RX_IN_C64 ? 8 : (cfg->input_format == RX_IN_F16 ? 4 : 2);
    const int64_t words = (h->Nmax * h->m + 31) / 32;
    const int64_t ntiles = (h->Nmax + 1023) / 1024;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(dalloc(&h->H, cfg->fft_size));
    A(dalloc(&h->tw, RX_FFT_TW_N));
    A(dalloc(&h->cdc, 2 * h->cap));
    A(dalloc(&h->tail, 2 * h->hop));
    A(dalloc(&h->y, 2 * h->Nmax));
    A(dalloc(&h->z, 2 * h->Nmax));
    A(dalloc(&h->bstar, 2 * h->Nmax));
    A(dalloc(&h->mq, 2 * h->Nmax));
    A(dalloc(&h->tiles, 2 * ntiles + 4));          // per-tile jump sums, then the carry's snapshot
    A(dalloc(&h->yacq, 2 * h->nacq));
    A(dalloc(&h->yfoe, 2 * h->nw));
    A(dalloc(&h->sync_counts, 16 * (2 * RX_MAX_DELAY + 1) + 1));     // the counts, then an arrival ticket
    A(dalloc(&h->flag, 512));           // [0] CMA rerun flag, [1] check counter, [2..] check partials
    A(dalloc(&h->taps_id, 4 * RX_TMAX));
    A(dalloc(&h->st, 1));
    A(cudaMalloc(&h->stage_in, (size_t)(2 * h->Smax * h->in_elem)));
    A(dalloc(&h->stage_ref, 2 * words));
    A(dalloc(&h->stage_out, 2 * words));
    A(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    A(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    A(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    A(cudaEventCreateWithFlags(&h->ev_chk, cudaEventDisableTiming));
    A(cudaEventCreateWithFlags(&h->ev_chk_done, cudaEventDisableTiming));
    A(cudaEventCreateWithFlags(&h->ev_host, cudaEventDisableTiming));
    A(cudaStreamCreateWithFlags(&h->capstream, cudaStreamNonBlocking));
    for (int s = 0; s < ST_N && e == cudaSuccess; ++s) {
        h->ev0[s].resize(kPool);
        h->ev1[s].resize(kPool);
        for (int i = 0; i < kPool; ++i) {
            A(cudaEventCreate(&h->ev0[s][i]));
            A(cudaEventCreate(&h->ev1[s][i]));
        }
    }
    if (e != cudaSuccess) {
        free_all(h);
        delete h;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? RX_ENOMEM : RX_ECUDA;
    }
    cudaStream_t s0 = 0;
    A(cudaMemset(h->st, 0, sizeof(RxDevState)));
    A(cudaMemset(h->cdc, 0, sizeof(float2) * 2 * h->cap));
    A(cudaMemset(h->tail, 0, sizeof(float2) * 2 * h->hop));
    // counters that kernels accumulate into and reset after use must start at zero
    A(cudaMemset(h->sync_counts, 0, sizeof(int) * (16 * (2 * RX_MAX_DELAY + 1) + 1)));
    A(cudaMemset(h->flag, 0, sizeof(int) * 512));
    k_state_init<<<1, 1, 0, s0>>>(h->st);
    k_identity_taps<<<1, 256, 0, s0>>>(h->taps_id, h->T);
    A(cudaGetLastError());
    A(launch_fill_twiddles(h->tw, s0));
    const double dl2c = cfg->dispersion_s_per_m2 * cfg->length_m * cfg->wavelength_m * cfg->wavelength_m / C_LIGHT;
    A(launch_fill_filter(h->H, cfg->fft_size, h->fs, dl2c, cfg->symbol_rate_hz, cfg->rrc_rolloff, s0));
    A(cudaDeviceSynchronize());
    if (e != cudaSuccess) {
        free_all(h);
        delete h;
        return RX_ECUDA;
    }
    *out = h;
    return RX_OK;
}

static rx_status enqueue_frame(rx_handle* h, const void* d_in, int64_t n_sym, const uint32_t* d_ref, uint32_t* d_out,
                               rx_stream_t stream_) {
    if (!h || !d_in || n_sym < 1 || n_sym > h->Nmax) return RX_EINVAL;
    const rx_config& c = h->cfg;
    const bool stream_mode = c.streaming != 0;
    if (stream_mode && (n_sym % (c.fft_size / 4)) != 0) return RX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream_;
    h->last = s;
    const int64_t N = n_sym, S = 2 * n_sym;
    const bool first = !stream_mode || h->frames == 0;
    const int Lb = h->Lb, T = h->T;
    const int64_t n_cma = std::min<int64_t>(c.cma_blocks, N / Lb);
    const int64_t n_dd = n_cma > 0 ? std::min<int64_t>(c.dd_acq_blocks, N / Lb) : 0;
    // acquisition window of this frame (shorter than the configured one for short frames)
    const int64_t nacq_e = n_cma * Lb, nw_e = nacq_e - nacq_e / 2;
    int nf_e = 512;
    while (nf_e < 2 * nw_e) nf_e *= 2;
    const int kf_e = ilog2(nf_e);
    const int64_t obase = stream_mode ? h->hist : 0;
    const int64_t off = stream_mode ? h->hist - 2 * h->d4 : 0;
    const int64_t xlen = obase + S;
    const long long g0 = stream_mode ? (long long)h->frames * S - c.fft_size / 4 - h->hist : 0;
    const int64_t lat = stream_mode ? c.fft_size / 8 + h->d4 : 0;
    RxDevState* st = h->st;
    uint64_t nl = 0;

    // a stream's later frames carry every piece of state; a first frame (every single frame) starts it
    // in the power kernel
    if (first) {
        StageScope sc(h, ST_POWER, s);
        RX_CK(launch_power(d_in, c.input_format, c.input_scale, S, 2 * n_cma * Lb, st, stream_mode ? 0 : 1, s));
        ++nl;
    }
    // A single frame with an acquisition: the FD compensation of the blocks the acquisition reads
    // (symbols [0, max(n_cma, n_dd) Lb) and the filter's reach) comes first on the stream, the rest
    // runs on the side stream meanwhile and joins before the segments.
    const int64_t nblk_a = acq_cdc_blocks(h, N);
    const bool split = nblk_a > 0;
    {
        StageScope sc(h, ST_CDC, s);
        CdcArgs a{d_in, c.input_format, c.input_scale, S, c.fft_size, h->H, h->tw,
                  stream_mode ? h->tail : nullptr, h->cdc, h->cap, obase, st};
        if (split) a.nblk = nblk_a;
        RX_CK(launch_cdc(a, s));
        ++nl;
    }
    // the rest of the compensation forks here but is enqueued after the acquisition's first launch,
    // whose CTAs, each holding a whole SM, are then placed before the side stream fills the GPU
    if (split) RX_CK(cudaEventRecord(h->ev_fork, s));
    bool rest_done = !split;
    auto enqueue_rest = [&]() -> rx_status {
        if (rest_done) return RX_OK;
        rest_done = true;
        RX_CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        {
            StageScope sc(h, ST_CDC_REST, h->side);
            CdcArgs a{d_in, c.input_format, c.input_scale, S, c.fft_size, h->H, h->tw, nullptr, h->cdc, h->cap,
                      obase, st};
            a.j0 = nblk_a;
            RX_CK(launch_cdc(a, h->side));
            ++nl;
        }
        RX_CK(cudaEventRecord(h->ev_join, h->side));
        return RX_OK;
    };
    LmsArgs base{};
    base.x = h->cdc;
    base.xstride = h->cap;
    base.xlen = xlen;
    base.off = off;
    base.T = T;
    base.Lb = Lb;
    base.m = h->m;
    base.g0 = g0;
    base.st = st;
    bool late_check = false;                      // the rerun's check on the side stream (joined before the count)
    if (first) {
        if (n_cma > 0) {
            {
                StageScope sc(h, ST_CMA, s);
                LmsArgs a = base;
                a.n_sym = n_cma * Lb;
                a.L_seg = n_cma * Lb;
                a.n_wu = 0;
                a.cma = 1;
                a.mu = c.mu_cma;
                const Qam q = make_qam(h->m);
                // R2 = E|s|^4 / E|s|^2 of the unit-energy alphabet
                double s4 = 0.0;
                for (int i = 0; i < q.L; ++i)
                    for (int j = 0; j < q.L; ++j) {
                        const double re = (2 * i - (q.L - 1)) * (double)q.a, im = (2 * j - (q.L - 1)) * (double)q.a;
                        s4 += (re * re + im * im) * (re * re + im * im);
                    }
                a.R2 = (float)(s4 / (q.L * q.L));
                a.derotate = 0;
                a.taps_in = h->taps_id;
                a.taps_out = st->taps_cma;
                a.y = h->yacq;
                a.ystride = h->nacq;
                a.exclusive = 1;
                RX_CK(launch_lms(a, kAcqThreads, s));
                if (rx_status r = enqueue_rest(); r != RX_OK) return r;
                // the singularity check (it also rebuilds the rerun's start taps), then the rerun when the
                // check raised the flag
                RX_CK(launch_cma_check(h->yacq, h->nacq, nacq_e, T, st, h->flag, 0, s));
                LmsArgs a2 = a;
                a2.taps_in = st->taps_init;
                a2.run_if = h->flag;
                a2.pdl = 1;                               // resident while the check runs
                RX_CK(launch_lms(a2, kAcqThreads, s));
                // the rerun's own check only raises an error bit: with a side stream it runs there after
                // the DD acquisition's launch, beside the segments, and joins before the count
                if (!split) RX_CK(launch_cma_check(h->yacq, h->nacq, nacq_e, T, st, h->flag, 1, s));
                late_check = split;
                nl += 4;
            }
            {
                StageScope sc(h, ST_FOE, s);
                FoeArgs f{h->cdc, h->cap, xlen, off, T, nacq_e / 2, nw_e, st->taps_cma, h->yfoe, h->tw, Lb,
                          c.symbol_rate_hz / (2.0 * M_PI) / c.fo_grid_hz, c.fo_grid_hz / h->fs, st};
                RX_CK(launch_foe(f, kf_e, s));
                ++nl;
            }
            if (n_dd > 0) {
                StageScope sc(h, ST_DDACQ, s);
                LmsArgs a = base;
                a.n_sym = n_dd * Lb;
                a.L_seg = n_dd * Lb;
                a.n_wu = 0;
                a.cma = 0;
                a.mu = c.mu_dd;
                a.derotate = 1;
                a.taps_in = st->taps_init;
                a.taps_out = st->taps_init;
                a.y = nullptr;
                a.exclusive = 1;
                a.pdl = 1;                                // resident while the FO estimate runs
                RX_CK(launch_lms(a, kAcqThreads, s));
                ++nl;
            }
            if (late_check) {
                RX_CK(cudaEventRecord(h->ev_chk, s));
                RX_CK(cudaStreamWaitEvent(h->side, h->ev_chk, 0));
                RX_CK(launch_cma_check(h->yacq, h->nacq, nacq_e, T, st, h->flag, 1, h->side));
                RX_CK(cudaEventRecord(h->ev_chk_done, h->side));
            }
        } else {
            RX_CK(cudaMemcpyAsync(st->taps_init, h->taps_id, sizeof(float2) * 4 * T, cudaMemcpyDeviceToDevice, s));
            RX_CK(cudaMemcpyAsync(st->taps_cma, h->taps_id, sizeof(float2) * 4 * T, cudaMemcpyDeviceToDevice, s));
        }
    } else {
        RX_CK(cudaMemcpyAsync(st->taps_init, st->taps_last, sizeof(float2) * 4 * T, cudaMemcpyDeviceToDevice, s));
    }
    if (rx_status r = enqueue_rest(); r != RX_OK) return r;
    if (split) RX_CK(cudaStreamWaitEvent(s, h->ev_join, 0));   // the whole frame is compensated
    {
        StageScope sc(h, ST_LMS, s);
        LmsArgs a = base;
        a.n_sym = N;
        a.L_seg = (int64_t)c.seg_blocks * Lb;
        a.n_wu = c.warmup_blocks;
        a.cma = 0;
        a.mu = c.mu_dd;
        a.derotate = 1;
        a.taps_in = st->taps_init;
        a.taps_out = st->taps_last;
        a.y = h->y;
        a.ystride = h->Nmax;
        RX_CK(launch_lms(a, c.lms_threads ? c.lms_threads : kSegThreads, s));
        ++nl;
    }
    {
        StageScope sc(h, ST_BPS, s);
        RX_CK(launch_bps(h->y, h->Nmax, N, c.bps_phases, c.bps_window, h->m, h->bstar, h->Nmax, s));
        ++nl;
    }
    {
        StageScope sc(h, ST_UNWRAP, s);
        int k = 0;
        RX_CK(launch_unwrap(h->y, h->Nmax, h->bstar, h->Nmax, N, c.bps_phases, h->tiles, h->mq, h->Nmax, h->z, h->Nmax,
                            st, s, &k));
        nl += k;
    }
    const int64_t words = (N * h->m + 31) / 32;
    const int64_t E = stream_mode ? std::max<int64_t>(c.edge_skip, lat + c.max_delay) : c.edge_skip;
    const int64_t lo = E, hi = std::max<int64_t>(N - E, lo);
    if (d_ref) {
        if ((!stream_mode || !h->sync_done) && hi > lo) {
            StageScope sc(h, ST_SYNC, s);
            int k = 0;
            RX_CK(launch_sync(h->z, h->Nmax, d_ref, words, N, h->m, lo, std::min<int64_t>(lo + c.sync_len, hi),
                              c.max_delay, lat, h->sync_counts, st, s, &k));
            nl += k;
            h->sync_done = true;
        }
    }
    if (late_check) RX_CK(cudaStreamWaitEvent(s, h->ev_chk_done, 0));
    if (d_ref || d_out) {
        StageScope sc(h, ST_COUNT, s);
        RX_CK(launch_count(h->z, h->Nmax, N, d_ref, words, N, h->m, lo, hi, lat, d_out, words, st, s));
        ++nl;
    }
    if (stream_mode) {
        StageScope sc(h, ST_STATE, s);
        RX_CK(launch_tail(d_in, c.input_format, c.input_scale, S, h->hop, h->tail, st, s));
        RX_CK(launch_copy_hist(h->cdc, h->cap, S, h->hist, s));
        nl += 2;
    }
    h->frames += 1;
    h->sym_processed += 2 * (uint64_t)N;
    h->launches += nl;
    return RX_OK;
}

rx_status rx_decide(rx_handle* h, const float* d_z, int64_t n_sym, const uint32_t* d_ref, uint32_t* d_out,
                    rx_stream_t stream_) {
    if (!h || !d_z || n_sym < 1 || n_sym > h->Nmax || h->cfg.streaming) return RX_EINVAL;
    const rx_config& c = h->cfg;
    cudaStream_t s = (cudaStream_t)stream_;
    h->last = s;
    const int64_t N = n_sym;
    const float2* z = reinterpret_cast<const float2*>(d_z);
    k_decide_begin<<<1, 1, 0, s>>>(h->st);
    RX_CK(cudaGetLastError());
    const int64_t words = (N * h->m + 31) / 32;
    const int64_t lo = c.edge_skip, hi = std::max<int64_t>(N - c.edge_skip, lo);
    int k = 0;
    if (d_ref && hi > lo) {
        StageScope sc(h, ST_SYNC, s);
        RX_CK(launch_sync(z, N, d_ref, words, N, h->m, lo, std::min<int64_t>(lo + c.sync_len, hi), c.max_delay, 0,
                          h->sync_counts, h->st, s, &k));
    }
    if (d_ref || d_out) {
        StageScope sc(h, ST_COUNT, s);
        RX_CK(launch_count(z, N, N, d_ref, words, N, h->m, lo, hi, 0, d_out, words, h->st, s));
        ++k;
    }
    h->launches += k + 1;
    return RX_OK;
}

static rx_status enqueue_host(rx_handle* h, const void* h_in, int64_t n_sym, const uint32_t* h_ref, uint32_t* h_out,
                              rx_stream_t stream_) {
    if (!h || !h_in || n_sym < 1 || n_sym > h->Nmax) return RX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream_;
    const int64_t S = 2 * n_sym;
    const int64_t words = (n_sym * h->m + 31) / 32;
    const int64_t na = acq_cdc_blocks(h, n_sym);
    if (na > 0) {
        // The acquisition needs only the head of each polarisation: that is copied on the caller's
        // stream, the rest of the input and the reference bits on the side stream, where they overlap
        // the acquisition and precede the rest of the FD compensation (and the join before the
        // segments). The side stream waits for the head's copy (and so for the caller's stream, whose
        // previous frame may still read the staging buffers): copies issued together share the link,
        // and the head would then arrive only with the whole frame.
        const int64_t head = std::min<int64_t>(S, na * (h->cfg.fft_size / 2) + h->cfg.fft_size / 4);
        const char* src = static_cast<const char*>(h_in);
        char* dst = static_cast<char*>(h->stage_in);
        const size_t eb = (size_t)h->in_elem;
        {
            StageScope sc(h, ST_H2D, s);
            for (int p = 0; p < 2; ++p)
                RX_CK(cudaMemcpyAsync(dst + p * S * eb, src + p * S * eb, (size_t)head * eb, cudaMemcpyHostToDevice, s));
        }
        RX_CK(cudaEventRecord(h->ev_host, s));
        RX_CK(cudaStreamWaitEvent(h->side, h->ev_host, 0));
        for (int p = 0; p < 2; ++p)
            if (S > head)
                RX_CK(cudaMemcpyAsync(dst + (p * S + head) * eb, src + (p * S + head) * eb, (size_t)(S - head) * eb,
                                      cudaMemcpyHostToDevice, h->side));
        if (h_ref)
            RX_CK(cudaMemcpyAsync(h->stage_ref, h_ref, sizeof(uint32_t) * 2 * words, cudaMemcpyHostToDevice,
                                  h->side));
    } else {
        StageScope sc(h, ST_H2D, s);
        RX_CK(cudaMemcpyAsync(h->stage_in, h_in, (size_t)(2 * S * h->in_elem), cudaMemcpyHostToDevice, s));
        if (h_ref)
            RX_CK(cudaMemcpyAsync(h->stage_ref, h_ref, sizeof(uint32_t) * 2 * words, cudaMemcpyHostToDevice, s));
    }
    rx_status r = enqueue_frame(h, h->stage_in, n_sym, h_ref ? h->stage_ref : nullptr,
                                h_out ? h->stage_out : nullptr, stream_);
    if (r != RX_OK) return r;
    if (h_out) {
        StageScope sc(h, ST_D2H, s);
        RX_CK(cudaMemcpyAsync(h_out, h->stage_out, sizeof(uint32_t) * 2 * words, cudaMemcpyDeviceToHost, s));
    }
    return RX_OK;
}

// Single frames replay their launches as one CUDA graph, captured on the first call with a given set
// of buffers and frame length (and timing on or off): the frame's launches carry no host-side state
// that changes between frames. Streams of frames (each frame's launch arguments change), calls on a
// stream that is itself being captured (the batch) and a handle whose capture failed once run the
// launches directly. With stage timing on, the graph holds the stage events; their times are
// collected before the next replay records them again.
static rx_status run_graph(rx_handle* h, int which, const void* in, int64_t n_sym, const void* ref, void* out,
                           cudaStream_t s, bool& done) {
    done = false;
    if (h->cfg.streaming || !h->graphs_ok) return RX_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return RX_OK;
    rx_handle::FrameGraph& g = h->graph[which];
    if (h->timing) timing_flush(h);                   // stage events of the previous frame, if any
    const bool hit = g.valid && g.timing == h->timing && g.in == in && g.ref == ref && g.out == out && g.n == n_sym;
    if (hit) h->graph_misses = 0;
    if (!hit && ++h->graph_misses > 2) {
        // buffers or lengths change from call to call: capturing would cost more than it saves
        h->graphs_ok = false;
        return RX_OK;
    }
    if (!hit) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = rx_handle::FrameGraph{};
        const uint64_t l0 = h->launches, f0 = h->frames, s0 = h->sym_processed;
        if (cudaStreamBeginCapture(h->capstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            h->graphs_ok = false;
            return RX_OK;
        }
        h->capturing = true;
        rx_status r = which == 0 ? enqueue_frame(h, in, n_sym, static_cast<const uint32_t*>(ref),
                                                 static_cast<uint32_t*>(out), h->capstream)
                                 : enqueue_host(h, in, n_sym, static_cast<const uint32_t*>(ref),
                                                static_cast<uint32_t*>(out), h->capstream);
        h->capturing = false;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(h->capstream, &graph);
        const uint64_t nl_cap = h->launches - l0;     // what one replay adds
        h->launches = l0;
        h->frames = f0;
        h->sym_processed = s0;
        cudaGraphExec_t exec = nullptr;
        const bool ok = r == RX_OK && ec == cudaSuccess && graph &&
                        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            // e.g. pageable host buffers cannot be captured: run this handle's frames directly
            cudaGetLastError();
            for (int st = 0; st < ST_N; ++st) h->used[st] = 0;
            h->graphs_ok = false;
            return RX_OK;
        }
        g.valid = true;
        g.timing = h->timing;
        g.in = in;
        g.ref = ref;
        g.out = out;
        g.n = n_sym;
        g.exec = exec;
        g.nl = nl_cap;
        for (int st = 0; st < ST_N; ++st) g.events[st] = h->used[st];   // stage events each replay records
    }
    RX_CK(cudaGraphLaunch(g.exec, s));
    h->last = s;
    h->frames += 1;
    h->sym_processed += 2 * (uint64_t)n_sym;
    h->launches += g.nl;
    for (int st = 0; st < ST_N; ++st) h->used[st] = g.events[st];
    done = true;
    return RX_OK;
}

rx_status rx_process(rx_handle* h, const void* d_in, int64_t n_sym, const uint32_t* d_ref, uint32_t* d_out,
                     rx_stream_t stream_) {
    if (!h || !d_in || n_sym < 1 || n_sym > h->Nmax) return RX_EINVAL;
    bool done = false;
    rx_status r = run_graph(h, 0, d_in, n_sym, d_ref, d_out, (cudaStream_t)stream_, done);
    if (r != RX_OK || done) return r;
    return enqueue_frame(h, d_in, n_sym, d_ref, d_out, stream_);
}

rx_status rx_process_host(rx_handle* h, const void* h_in, int64_t n_sym, const uint32_t* h_ref, uint32_t* h_out,
                          rx_stream_t stream_) {
    if (!h || !h_in || n_sym < 1 || n_sym > h->Nmax) return RX_EINVAL;
    bool done = false;
    rx_status r = run_graph(h, 1, h_in, n_sym, h_ref, h_out, (cudaStream_t)stream_, done);
    if (r != RX_OK || done) return r;
    return enqueue_host(h, h_in, n_sym, h_ref, h_out, stream_);
}

rx_status rx_stats(rx_handle* h, rx_stats_t* out) {
    if (!h || !out) return RX_EINVAL;
    if (h->last) RX_CK(cudaStreamSynchronize(h->last));
    else RX_CK(cudaDeviceSynchronize());
    RxDevState st;
    RX_CK(cudaMemcpy(&st, h->st, sizeof(st), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->frames = h->frames;
    out->symbols_processed = h->sym_processed;
    out->bits_processed = h->sym_processed * (uint64_t)h->m;
    out->bits_counted = st.bits;
    out->bit_errors = st.bit_errors;
    out->symbols_counted = st.symbols;
    out->symbol_errors = st.symbol_errors;
    out->evm_num = (double)st.evm_num_fx / (double)RX_EVM_FX_SCALE;
    out->evm_den = (double)st.evm_den_fx / (double)RX_EVM_FX_SCALE;
    out->ber = st.bits ? (double)st.bit_errors / (double)st.bits : 0.0;
    out->evm = out->evm_den > 0 ? std::sqrt(out->evm_num / out->evm_den) : 0.0;
    if (st.bits == 0) out->q_db = 0.0;
    else if (st.bit_errors == 0) out->q_db = INFINITY;
    else {
        // Q = 20 log10(sqrt(2) erfcinv(2 BER)), erfcinv by Newton steps on erfc
        const double target = 2.0 * out->ber;
        double x = 1.0;
        for (int i = 0; i < 60; ++i) {
            const double f = std::erfc(x) - target;
            const double df = -2.0 / std::sqrt(M_PI) * std::exp(-x * x);
            const double nx = x - f / df;
            x = nx > 0.0 ? nx : x * 0.5;
        }
        out->q_db = 20.0 * std::log10(std::sqrt(2.0) * x);
    }
    out->fo_code = st.fo_code;
    out->fo_hz = st.fo_code * h->cfg.fo_grid_hz;
    for (int q = 0; q < 2; ++q) {
        out->pol_map[q] = st.sync_p[q];
        out->rotation[q] = st.sync_r[q];
        out->delay[q] = st.sync_d[q];
        out->sync_matches[q] = st.sync_match[q];
    }
    out->sync_len = st.sync_len;
    out->cma_reran = st.cma_reran;
    out->cma_rho = st.cma_rho;
    out->latency_symbols = h->cfg.streaming ? h->cfg.fft_size / 8 + h->d4 : 0;
    out->error_word = st.err_word;
    return RX_OK;
}

rx_status rx_buffer_bytes(rx_handle* h, int32_t which, int64_t* bytes) {
    if (!h || !bytes) return RX_EINVAL;
    const int64_t N = h->Nmax;
    switch (which) {
        case RX_BUF_CDC: *bytes = sizeof(float2) * 2 * h->cap; break;
        case RX_BUF_Y: case RX_BUF_Z: *bytes = sizeof(float2) * 2 * N; break;
        case RX_BUF_BSTAR: *bytes = 2 * N; break;
        case RX_BUF_M: *bytes = sizeof(int) * 2 * N; break;
        case RX_BUF_TAPS_CMA: case RX_BUF_TAPS_INIT: case RX_BUF_TAPS_LAST: *bytes = sizeof(float2) * 4 * h->T; break;
        case RX_BUF_Y_ACQ: *bytes = sizeof(float2) * 2 * h->nacq; break;
        case RX_BUF_Y_FOE: *bytes = sizeof(float2) * 2 * h->nw; break;
        case RX_BUF_SCALE: *bytes = sizeof(float) * 2; break;
        default: return RX_EINVAL;
    }
    return RX_OK;
}

rx_status rx_get_buffer(rx_handle* h, int32_t which, void* d_dst, int64_t bytes, rx_stream_t stream_) {
    int64_t need = 0;
    rx_status r = rx_buffer_bytes(h, which, &need);
    if (r != RX_OK) return r;
    if (!d_dst || bytes != need) return RX_EINVAL;
    const void* src = nullptr;
    switch (which) {
        case RX_BUF_CDC: src = h->cdc; break;
        case RX_BUF_Y: src = h->y; break;
        case RX_BUF_Z: src = h->z; break;
        case RX_BUF_BSTAR: src = h->bstar; break;
        case RX_BUF_M: src = h->mq; break;
        case RX_BUF_TAPS_CMA: src = h->st->taps_cma; break;
        case RX_BUF_TAPS_INIT: src = h->st->taps_init; break;
        case RX_BUF_TAPS_LAST: src = h->st->taps_last; break;
        case RX_BUF_Y_ACQ: src = h->yacq; break;
        case RX_BUF_Y_FOE: src = h->yfoe; break;
        case RX_BUF_SCALE: src = h->st->scale; break;
    }
    RX_CK(cudaMemcpyAsync(d_dst, src, (size_t)bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream_));
    return RX_OK;
}

rx_status rx_reset(rx_handle* h) {
    if (!h) return RX_EINVAL;
    if (h->last) RX_CK(cudaStreamSynchronize(h->last));
    RX_CK(cudaMemset(h->st, 0, sizeof(RxDevState)));
    RX_CK(cudaMemset(h->tail, 0, sizeof(float2) * 2 * h->hop));
    RX_CK(cudaMemset(h->cdc, 0, sizeof(float2) * 2 * h->cap));
    RX_CK(cudaMemset(h->sync_counts, 0, sizeof(int) * (16 * (2 * RX_MAX_DELAY + 1) + 1)));
    RX_CK(cudaMemset(h->flag, 0, sizeof(int) * 512));
    k_state_init<<<1, 1>>>(h->st);
    RX_CK(cudaGetLastError());
    RX_CK(cudaDeviceSynchronize());
    h->frames = 0;
    h->sym_processed = 0;
    h->sync_done = false;
    return RX_OK;
}

// state blob: header, device state, tail, equaliser history
struct BlobHeader {
    uint64_t magic, bytes, frames, sym_processed;
    int32_t sync_done, T, hop, hist;
    double symbol_rate;
};

rx_status rx_state_size(rx_handle* h, size_t* bytes) {
    if (!h || !bytes) return RX_EINVAL;
    *bytes = sizeof(BlobHeader) + sizeof(RxDevState) + sizeof(float2) * 2 * ((size_t)h->hop + h->hist);
    return RX_OK;
}

rx_status rx_state_get(rx_handle* h, void* blob, size_t bytes) {
    size_t need = 0;
    if (rx_state_size(h, &need) != RX_OK || !blob || bytes != need) return RX_EINVAL;
    if (h->last) RX_CK(cudaStreamSynchronize(h->last));
    char* p = (char*)blob;
    BlobHeader hd{0x52584254u, need, h->frames, h->sym_processed, h->sync_done ? 1 : 0, h->T, h->hop, h->hist,
                  h->cfg.symbol_rate_hz};
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    RX_CK(cudaMemcpy(p, h->st, sizeof(RxDevState), cudaMemcpyDeviceToHost));
    p += sizeof(RxDevState);
    RX_CK(cudaMemcpy(p, h->tail, sizeof(float2) * 2 * h->hop, cudaMemcpyDeviceToHost));
    p += sizeof(float2) * 2 * h->hop;
    for (int q = 0; q < 2; ++q) {
        RX_CK(cudaMemcpy(p, h->cdc + q * h->cap, sizeof(float2) * h->hist, cudaMemcpyDeviceToHost));
        p += sizeof(float2) * h->hist;
    }
    return RX_OK;
}

rx_status rx_state_set(rx_handle* h, const void* blob, size_t bytes) {
    size_t need = 0;
    if (rx_state_size(h, &need) != RX_OK || !blob || bytes < sizeof(BlobHeader)) return RX_EINVAL;
    const char* p = (const char*)blob;
    BlobHeader hd;
    std::memcpy(&hd, p, sizeof(hd));
    // a blob of another configuration is a state error, a truncated buffer an argument error
    if (hd.magic != 0x52584254u || hd.bytes != need || hd.T != h->T || hd.hop != h->hop || hd.hist != h->hist ||
        hd.symbol_rate != h->cfg.symbol_rate_hz)
        return RX_ESTATE;
    if (bytes != need) return RX_EINVAL;
    if (h->last) RX_CK(cudaStreamSynchronize(h->last));
    p += sizeof(hd);
    RX_CK(cudaMemcpy(h->st, p, sizeof(RxDevState), cudaMemcpyHostToDevice));
    p += sizeof(RxDevState);
    RX_CK(cudaMemcpy(h->tail, p, sizeof(float2) * 2 * h->hop, cudaMemcpyHostToDevice));
    p += sizeof(float2) * 2 * h->hop;
    for (int q = 0; q < 2; ++q) {
        RX_CK(cudaMemcpy(h->cdc + q * h->cap, p, sizeof(float2) * h->hist, cudaMemcpyHostToDevice));
        p += sizeof(float2) * h->hist;
    }
    h->frames = hd.frames;
    h->sym_processed = hd.sym_processed;
    h->sync_done = hd.sync_done != 0;
    return RX_OK;
}

rx_status rx_set_timing(rx_handle* h, int32_t enable) {
    if (!h) return RX_EINVAL;
    if (h->timing && !enable) timing_flush(h);
    h->timing = enable != 0;
    for (int s = 0; s < ST_N; ++s) {
        h->tot_ms[s] = 0.0;
        h->tot_n[s] = 0;
        h->used[s] = 0;
    }
    return RX_OK;
}

rx_status rx_stage_times(rx_handle* h, double* ms, int64_t* launches, int32_t n) {
    if (!h || n < 0) return RX_EINVAL;
    timing_flush(h);
    for (int s = 0; s < n && s < ST_N; ++s) {
        if (ms) ms[s] = h->tot_ms[s];
        if (launches) launches[s] = h->tot_n[s];
    }
    return RX_OK;
}

uint64_t rx_launch_count(rx_handle* h) { return h ? h->launches : 0; }

void rx_destroy(rx_handle* h) {
    if (!h) return;
    if (h->last) cudaStreamSynchronize(h->last);
    free_all(h);
    delete h;
}

}  // extern "C"
