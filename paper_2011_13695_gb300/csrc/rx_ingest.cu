// Real-time ingest emulation (Sec. II-C/II-D): a digitiser delivers buffers of
// buffer_samples 12-bit samples at a fixed sample rate; each accepted buffer gets
// one of n_streams GPU slots (its own stream), is copied in (standing for the
// digitiser's DMA into GPU memory), joined to its predecessor by the overlap step
// (the previous buffer's last 2N codes are put in front of it, in buffer order,
// ordered by an event chain across the slots), processed by the Kramers-Kronig
// front end and its output copied back to host memory.
//
// Why 2N: the front end is two cascaded overlap-save passes, each needing N/4
// samples of real input on either side of the N/2 outputs a block keeps. The
// joined frame [i S - 2N, (i + 1) S) starts on a block boundary of the stream's
// grid (blocks at multiples of N/2, less N/4), its field is exact on
// [N/2, S + 3N/2) of the frame and its output on [N, S + N): S samples at
// 4 samples/symbol, stream [i S - N, (i + 1) S - N), which continue the
// previous buffer's outputs. A buffer that becomes
// ready while every slot is still busy is dropped (the paper's data loss), and
// the next accepted buffer restarts the overlap chain from zero codes (its
// first N/2 outputs from its first sample on are a start-up transient). Real time holds when the
// mean time a buffer holds its slot stays below the buffer period times the
// number of slots.
//
// Host only: the pacing thread sleeps, then spins, until each buffer's ready
// time; completion times come from host functions queued behind each slot's
// last copy.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/rx.h"
#include "rx_kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;     // slot free again
    uint16_t* codes = nullptr;      // [2N + S]: carry, then the buffer
    float* field = nullptr;         // [2N + S] complex
    float* out = nullptr;           // [(2N + S) / 2] complex
    float* h_out = nullptr;         // pinned [S / 2] complex when the caller wants no outputs
    std::atomic<int64_t> finish_ns{0};
    Clock::time_point ready;
    bool busy = false;
};

void CUDART_CB mark_done(void* p) {
    auto* s = static_cast<Slot*>(p);
    s->finish_ns.store(std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count(),
                       std::memory_order_release);
}

}  // namespace

extern "C" rx_status rx_ingest_run(rx_kk* kk, const uint16_t* h_source, int64_t source_samples,
                                   int64_t buffer_samples, double sample_rate_hz, int32_t n_streams,
                                   int64_t n_buffers, float* h_out, rx_ingest_stats* stats) {
    if (!kk || !h_source || !stats) return RX_EINVAL;
    const int N = kk_fft_size(kk);
    const int64_t HOP = N / 2, CARRY = 2 * (int64_t)N;
    if (buffer_samples < CARRY || buffer_samples % HOP || buffer_samples > ((int64_t)1 << 30)) return RX_EINVAL;
    if (source_samples < buffer_samples || source_samples % buffer_samples) return RX_EINVAL;
    if (!(sample_rate_hz > 0.0) || n_streams < 1 || n_streams > 64 || n_buffers < 1) return RX_EINVAL;
    std::memset(stats, 0, sizeof(*stats));
    const int64_t S = buffer_samples, SP = CARRY + S;
    if (h_out && (uint64_t)n_buffers > ((uint64_t)1 << 40) / (uint64_t)S) return RX_EINVAL;

    // pin the source (the digitiser's memory) and the output for asynchronous copies; either may
    // already be pinned
    auto pin = [](const void* p, size_t bytes, bool* registered) -> bool {
        const cudaError_t e = cudaHostRegister(const_cast<void*>(p), bytes, cudaHostRegisterDefault);
        if (e == cudaSuccess) { *registered = true; return true; }
        cudaGetLastError();
        return e == cudaErrorHostMemoryAlreadyRegistered;
    };
    bool src_reg = false, out_reg = false;
    if (!pin(h_source, sizeof(uint16_t) * source_samples, &src_reg)) return RX_ECUDA;
    if (h_out && !pin(h_out, sizeof(float) * (size_t)S * (size_t)n_buffers, &out_reg)) {
        if (src_reg) cudaHostUnregister(const_cast<uint16_t*>(h_source));
        return RX_ECUDA;
    }
    std::vector<Slot> slots(n_streams);
    uint16_t* carry = nullptr;
    cudaEvent_t chain = nullptr;      // the last overlap step issued
    rx_status st = RX_OK;
    auto fail = [&](rx_status s) { st = s; };
    if (cudaMalloc(&carry, sizeof(uint16_t) * CARRY) != cudaSuccess) fail(RX_ENOMEM);
    if (st == RX_OK && cudaEventCreateWithFlags(&chain, cudaEventDisableTiming) != cudaSuccess) fail(RX_ECUDA);
    for (auto& s : slots) {
        if (st != RX_OK) break;
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) { fail(RX_ECUDA); break; }
        if (cudaMalloc(&s.codes, sizeof(uint16_t) * SP) != cudaSuccess ||
            cudaMalloc(&s.field, 8 * SP) != cudaSuccess || cudaMalloc(&s.out, 4 * SP) != cudaSuccess ||
            (!h_out && cudaMallocHost(&s.h_out, 4 * S) != cudaSuccess)) { fail(RX_ENOMEM); break; }
    }
    int64_t lat_sum_ns = 0, lat_max_ns = 0;
    // the host function behind a completed event runs shortly after it; give up after 10 s
    auto wait_finish = [&](Slot& s) -> bool {
        const auto limit = Clock::now() + std::chrono::seconds(10);
        while (s.finish_ns.load(std::memory_order_acquire) == 0) {
            if (Clock::now() > limit) return false;
            std::this_thread::yield();
        }
        return true;
    };
    auto retire = [&](Slot& s) {
        // the slot's host function has run once its event completed
        const int64_t fin = s.finish_ns.load(std::memory_order_acquire);
        const int64_t rdy = std::chrono::duration_cast<std::chrono::nanoseconds>(s.ready.time_since_epoch()).count();
        const int64_t lat = std::max<int64_t>(0, fin - rdy);
        lat_sum_ns += lat;
        lat_max_ns = std::max(lat_max_ns, lat);
        s.busy = false;
    };
    auto slot_free = [&](Slot& s) -> bool {
        if (!s.busy) return true;
        const cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) return false;
        if (q != cudaSuccess || !wait_finish(s)) { fail(RX_ECUDA); return false; }
        retire(s);
        return true;
    };
    if (st == RX_OK && cudaMemset(carry, 0, sizeof(uint16_t) * CARRY) != cudaSuccess) fail(RX_ECUDA);
    if (st == RX_OK && cudaDeviceSynchronize() != cudaSuccess) fail(RX_ECUDA);

    const double period_s = (double)S / sample_rate_hz;
    const Clock::time_point t0 = Clock::now() + std::chrono::milliseconds(1);
    bool chain_valid = false;         // the carry holds the previous buffer's tail
    bool chain_recorded = false;      // an overlap step has been issued (and may still be pending)
    int64_t next_slot = 0;
    for (int64_t i = 0; i < n_buffers && st == RX_OK; ++i) {
        const Clock::time_point ready =
            t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(period_s * (double)i));
        // the digitiser's clock: the buffer exists from `ready` on
        for (;;) {
            const auto now = Clock::now();
            if (now >= ready) break;
            if (ready - now > std::chrono::microseconds(200)) std::this_thread::sleep_for(ready - now - std::chrono::microseconds(100));
        }
        stats->buffers++;
        // a free slot, in round-robin order from the last one used
        int pick = -1;
        for (int t = 0; t < n_streams && st == RX_OK; ++t) {
            const int c = (int)((next_slot + t) % n_streams);
            if (slot_free(slots[c])) { pick = c; break; }
        }
        if (st != RX_OK) break;
        if (pick < 0) {
            stats->dropped++;
            chain_valid = false;
            continue;
        }
        next_slot = pick + 1;
        Slot& s = slots[pick];
        s.ready = ready;
        s.busy = true;
        s.finish_ns.store(0, std::memory_order_relaxed);
        const uint16_t* src = h_source + (i * S) % source_samples;
        cudaError_t e = cudaMemcpyAsync(s.codes + CARRY, src, sizeof(uint16_t) * S, cudaMemcpyHostToDevice, s.stream);
        // overlap step, in buffer order: the carried tail in front, this buffer's tail into the carry
        // (after a drop the carry restarts from zeros, once the last overlap step issued is done with it)
        if (e == cudaSuccess && chain_recorded) e = cudaStreamWaitEvent(s.stream, chain, 0);
        if (e == cudaSuccess && !chain_valid) e = cudaMemsetAsync(carry, 0, sizeof(uint16_t) * CARRY, s.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.codes, carry, sizeof(uint16_t) * CARRY, cudaMemcpyDeviceToDevice, s.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(carry, s.codes + S, sizeof(uint16_t) * CARRY, cudaMemcpyDeviceToDevice, s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(chain, s.stream);
        if (e != cudaSuccess) { fail(RX_ECUDA); break; }
        chain_valid = chain_recorded = true;
        // the joined buffer starts 2N samples before buffer i in the stream
        const rx_status r = rx_kk_process(kk, s.codes, SP, i * S - CARRY, s.field, s.out, (rx_stream_t)s.stream);
        if (r != RX_OK) { fail(r); break; }
        // outputs N/2 .. N/2 + S/2 (2 samples/symbol) of the joined buffer continue the previous buffer's
        float* dst = h_out ? h_out + (size_t)i * (size_t)S : s.h_out;   // S/2 complex = S floats
        e = cudaMemcpyAsync(dst, s.out + 2 * (N / 2), 4 * S, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
        if (e == cudaSuccess) e = cudaLaunchHostFunc(s.stream, mark_done, &s);
        if (e != cudaSuccess) { fail(RX_ECUDA); break; }
        stats->processed++;
    }
    if (cudaDeviceSynchronize() != cudaSuccess && st == RX_OK) st = RX_ECUDA;
    for (auto& s : slots)
        if (s.busy && st == RX_OK) {
            if (wait_finish(s)) retire(s);
            else st = RX_ECUDA;
        }
    stats->wall_s = std::chrono::duration<double>(Clock::now() - t0).count();
    stats->buffer_period_ms = period_s * 1e3;
    if (stats->processed) stats->mean_latency_ms = (double)lat_sum_ns / (double)stats->processed * 1e-6;
    stats->max_latency_ms = (double)lat_max_ns * 1e-6;
    for (auto& s : slots) {
        if (s.codes) cudaFree(s.codes);
        if (s.field) cudaFree(s.field);
        if (s.out) cudaFree(s.out);
        if (s.h_out) cudaFreeHost(s.h_out);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    if (chain) cudaEventDestroy(chain);
    if (carry) cudaFree(carry);
    if (src_reg) cudaHostUnregister(const_cast<uint16_t*>(h_source));
    if (out_reg) cudaHostUnregister(h_out);
    return st;
}
