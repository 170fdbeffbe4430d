// Carrier recovery (blind phase search + unwrap + derotation) on a frame of
// equalised symbols without any device allocation.
//
// Who needs this: callers that cannot allocate device memory at the moment
// they process data - a real-time ingest thread that must never block inside
// the CUDA allocator (cudaMalloc can synchronise the device and take global
// locks, which breaks a fixed per-buffer time budget), and host frameworks that
// hand this library a fixed memory budget at load time and forbid it to grow.
// Such a caller owns its input and output buffers; the scratch the kernels need
// (the chosen test phase and unwrap count per symbol, the per-tile jump sums
// and the carried unwrap state) lives in one file-scope __device__ array that
// every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/rx.h"
#include "rx_kernels.h"

namespace {

// largest frame the static scratch holds, symbols per polarisation
constexpr int64_t kStaticMaxSym = RX_STATIC_MAX_SYMBOLS;
constexpr int64_t kTiles = (kStaticMaxSym + 1023) / 1024;

struct StaticScratch {
    RxDevState st;                       // carried unwrap state (reset every call)
    int tiles[2 * kTiles + 4];           // per-tile jump sums, then the carried (b*, m) snapshot
    int m[2 * kStaticMaxSym];            // unwrap count per symbol
    uint8_t bstar[2 * kStaticMaxSym];    // chosen test phase per symbol
};

__device__ __align__(256) StaticScratch g_scratch;

// Host code may not use g_scratch's name as a device address; each device's
// address comes from cudaGetSymbolAddress, looked up once per device.
constexpr int kMaxDevices = 64;
StaticScratch* g_addr[kMaxDevices] = {nullptr};
std::mutex g_addr_mutex;

__global__ void k_static_reset(RxDevState* st) {
    st->b_prev[0] = st->b_prev[1] = -1;
    st->m_prev[0] = st->m_prev[1] = 0;
}

}  // namespace

extern "C" rx_status rx_carrier_recovery_static(const float* d_y, int64_t n_sym, int32_t bits_per_sym,
                                                int32_t bps_phases, int32_t bps_window, float* d_z,
                                                rx_stream_t stream_) {
    if (!d_y || !d_z || n_sym < 1) return RX_EINVAL;
    if (n_sym > kStaticMaxSym) return RX_EINVAL;
    if (bits_per_sym != 2 && bits_per_sym != 4 && bits_per_sym != 6 && bits_per_sym != 8) return RX_EINVAL;
    if (bps_phases < 2 || bps_phases > RX_BPS_MAXB) return RX_EINVAL;
    if (bps_window < 2 || bps_window > 64 || (bps_window & (bps_window - 1))) return RX_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RX_ECUDA;
    // the scratch address is the current device's: a stream of another device would get the wrong one
    int sdev = dev;
    if (cudaStreamGetDevice((cudaStream_t)stream_, &sdev) != cudaSuccess) return RX_ECUDA;
    if (sdev != dev) return RX_EINVAL;
    StaticScratch* sc = nullptr;
    {
        std::lock_guard<std::mutex> g(g_addr_mutex);
        if (!g_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return RX_ECUDA;
            g_addr[dev] = static_cast<StaticScratch*>(p);
        }
        sc = g_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream_;
    const float2* y = reinterpret_cast<const float2*>(d_y);
    float2* z = reinterpret_cast<float2*>(d_z);
    k_static_reset<<<1, 1, 0, s>>>(&sc->st);
    if (cudaGetLastError() != cudaSuccess) return RX_ECUDA;
    if (launch_bps(y, n_sym, n_sym, bps_phases, bps_window, bits_per_sym, sc->bstar, n_sym, s) != cudaSuccess)
        return RX_ECUDA;
    if (launch_unwrap(y, n_sym, sc->bstar, n_sym, n_sym, bps_phases, sc->tiles, sc->m, n_sym, z, n_sym, &sc->st, s,
                      nullptr) != cudaSuccess)
        return RX_ECUDA;
    return RX_OK;
}
