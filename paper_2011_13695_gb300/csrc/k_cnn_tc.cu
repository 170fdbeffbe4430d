// Inference forward of the learned post-equaliser on the 5th-generation tensor
// cores (tcgen05.mma, BF16 x BF16 -> FP32 accumulators in tensor memory).
//
// Each layer is a matrix product per tile of output positions, with
//   out[co][t] = sum_{k, ci} W[co][ci][k] x[ci][t + k - 4]
// and one of three operand mappings (details at TcShape below): the input
// layer takes the positions as M (128 per tile) and the weights as N; the
// hidden layers take the weights of two taps stacked as M and 256 positions
// as N; the output layer takes (tap, output channel) weight rows as M and 256
// positions as N.
//
// Activation layout (HBM): the hidden layers' BF16 activations are stored in
// eight channel-chunk planes [C/8][T + 8][8], padded position-major, so that
// a chunk of 8 channels of one position is one 16-byte row. Staged to shared
// memory unchanged (one bulk async copy per plane and tile), this is the
// K-major no-swizzle operand layout of the MMA (core matrices of 8 rows x 16
// bytes, rows 16 bytes apart, 8-row groups 128 bytes apart, K chunks one plane
// apart), and shifting the operand by r positions moves the descriptor's
// start address by 16 r bytes, always 16-byte aligned.
// The input layer (4 -> 64) builds its operand from the FP32 symbols:
// K = (tap, channel) with 4 channels, padded to 48 with zero weights, six
// planes whose row r holds the 8 values of taps 2j, 2j + 1 at position r.
//
// Roles (warp-specialised, one CTA per SM, tiles strided over the grid):
//   epilogue   4 x NPART warps; warp w reads TMEM lane quarter w % 4 over
//              part w / 4 of the accumulator's columns, then bias, ReLU, BF16
//              and 16-byte stores per plane (coalesced), or for the output
//              layer the taps' sum, bias and residual into the symbols;
//   producer   one thread issuing the bulk copies of a stage (hidden, output
//              layers), or four warps building the input layer's planes;
//   last warp  TMEM allocation, and one thread issuing the MMAs of a tile
//              into one of the accumulators and committing them to the
//              stage-free and accumulator-full barriers.
// Every wait is bounded (globaltimer); on a timeout the CTA sets the error
// word, stops all roles, waits for its own copies and MMAs in flight (again
// bounded) and frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/rx.h"
#include "rx_cnn.h"

namespace {

constexpr int KW = 9;
constexpr int PAD = KW / 2;
constexpr uint64_t kTimeoutNs = 500000000ull;  // 0.5 s per wait

enum Mode { IN = 0, HID = 1, OUT = 2 };

// Input layer: A = operand planes built from the symbols (M = 128 positions), B = weights (N = 64
// channels), K = (tap, channel) padded to 48.
// Hidden layers: A = weights of a pair of taps (2m, 2m + 1) stacked as rows, B = activations
// (N = 256 staged positions) shifted by 2m rows, one MMA per (pair, 16 input channels). Row r of A
// sits in TMEM lane r: quarter w = r / 32 holds output channels 16 w .. 16 w + 15, lanes 0-15 of it
// the even tap and lanes 16-31 the odd tap, so one warp holds both halves of its 16 channels.
// D_even[co][j] is the even taps' sum for the output at tile position j, D_odd[co][j] the odd taps'
// sum for position j - 1; the epilogue adds D_even[co][p] + D_odd[co][p + 1] (one shuffle), so a
// tile of 256 columns yields 248 outputs. Tap 9 (the odd half of pair 4) has zero weights.
// Output layer: A = weights with one row per (tap k, output channel co), row 4 k + co (36 of 128
// rows used), B = activations (N = 256 staged positions, unshifted), one MMA per 16 input channels;
// D[4 k + co][j] is tap k's term for the output at staged position j - k + 4, and the epilogue adds
// the nine taps' rows at their shifts, so a tile of 256 staged positions yields 248 outputs.
template <int MODE>
struct TcShape {
    static constexpr int TO = MODE == IN ? 128 : 248;                 // output positions per tile
    static constexpr int MMA_N = MODE == IN ? 64 : 256;
    static constexpr int COUT = MODE == OUT ? 4 : 64;
    // weight planes of 8 K values: input layer 6 (K = 48); hidden layers 5 tap pairs x 8 channel
    // chunks; output layer 8 channel chunks
    static constexpr int NKC = MODE == IN ? 6 : MODE == HID ? 40 : 8;
    static constexpr int NKS = NKC / 2;                               // MMAs of K = 16 per tile
    static constexpr int XROWS = MODE == IN ? 128 : MODE == HID ? 264 : 256;   // staged rows per plane
    static constexpr int WROWS = MODE == IN ? 64 : 128;               // weight rows per plane
    // plane strides are 64 bytes past a multiple of 128 (the two 16-byte K chunks of a row that one
    // MMA reads then fall in different shared-memory banks)
    static constexpr int XPL = (XROWS + 4) * 16;                      // activation plane stride (bytes)
    static constexpr int WPL = (WROWS + 4) * 16;                      // weight plane stride (bytes)
    static constexpr int NPL = MODE == IN ? 6 : 8;                    // activation planes per stage
    static constexpr int STAGE = NPL * XPL;
    static constexpr int S = 3;                                       // pipeline stages
    static constexpr int WB = NKC * WPL;                              // weight bytes: planes [kc][row][8]
    static constexpr int NPW = MODE == IN ? 4 : 1;                    // producer warps
    static constexpr int NPART = MODE == IN ? 2 : 4;                  // epilogue warps per TMEM lane quarter
    static constexpr int NEPI = 4 * NPART;                            // epilogue warps
    static constexpr int NWARP = NEPI + NPW + 1;
    static constexpr int NTHR = 32 * NWARP;
    static constexpr int NACC = MODE == IN ? 8 : 2;                   // accumulators in tensor memory
    static constexpr int TCOLS = NACC * MMA_N;                        // TMEM columns (a power of 2)
    static constexpr int FROWS = 128 + 12;                            // input layer: staged positions
    static constexpr int DROWS = 36, DSTR = 260;                      // output layer: D rows in smem (floats)
    static constexpr int OSTR = 72;                                   // hidden layers: output tile row (bf16)
    // shared memory: weights, stages, then the input layer's staged positions and output tiles, the
    // hidden layers' BF16 output tile or the output layer's D rows, then barriers and small state
    static constexpr int OFF_ST = WB;
    static constexpr int OFF_F = OFF_ST + S * STAGE;
    // input layer: staged positions, then two output tiles [8 planes][128 positions][16 B] that bulk
    // async stores write out
    static constexpr int OB = 8 * 128 * 16;
    static constexpr int AUX = MODE == IN ? FROWS * 8 + 2 * OB : MODE == HID ? TO * OSTR * 2 : DROWS * DSTR * 4;
    static constexpr int OFF_BAR = (OFF_F + AUX + 15) & ~15;
    static constexpr int NBAR = 2 * S + 2 * NACC;
    static constexpr int OFF_MISC = OFF_BAR + 8 * NBAR;               // tmem address, abort flag
    static constexpr int OFF_BIAS = OFF_MISC + 16;
    static constexpr int SMEM = OFF_BIAS + 4 * 64;
    // instruction descriptor (kind::f16): F32 accumulator, BF16 A and B, both K-major, N >> 3, M >> 4
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(MMA_N >> 3) << 17) |
                                      ((uint32_t)(128 >> 4) << 24);
    static_assert(STAGE % 16 == 0 && WB % 16 == 0 && XPL % 128 == 64 && WPL % 128 == 64, "operand strides");
    static_assert(MMA_N % 16 == 0 && MMA_N >= 16 && MMA_N <= 256, "M = 128 needs N a multiple of 16");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the phase of the given parity to complete; false on a timeout (which raises the CTA's
// abort flag) or when another role has raised it
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try(bar, parity)) {
        if (*abort) return false;
        if (gtimer() - t0 > kTimeoutNs) {
            *abort = 1;
            return false;
        }
    }
    return true;
}
// bounded wait used while shutting down (ignores the abort flag)
__device__ __noinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = gtimer();
    while (!mbar_try(bar, parity))
        if (gtimer() - t0 > kTimeoutNs) return;
}

// named barrier ID over the N threads of one role, returning the OR of a predicate
template <int ID, int N>
__device__ __forceinline__ bool bar_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(ID), "n"(N)
        : "memory");
    return r != 0;
}
template <int ID, int N>
__device__ __forceinline__ void bar_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(N) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory operand descriptor, K-major without swizzle: start, leading (K-direction core
// matrix) byte offset, stride (8-row group) byte offset, fixed field 0b001 at bit 46
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive accumulator columns of this warp's 32 lanes, waited for in the same statement so
// that no use of the registers can be scheduled before the load completes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\ttcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=r"(r)
                 : "r"(taddr)
                 : "memory");
    return __uint_as_float(r);
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

struct TcArgs {
    const __nv_bfloat16* x;      // planar input activations [8][Tp][8] (hidden, output layers)
    const float2* z;             // symbols [2][T] (input layer operand, output layer residual)
    const __nv_bfloat16* Wm;     // BF16 weights [co][K] (K = k * CIN + ci; the input layer padded to 48)
    const float* bias;           // [COUT]
    __nv_bfloat16* act;          // planar output activations (input, hidden layers)
    float2* sym;                 // output symbols [2][T] (output layer)
    __nv_bfloat16* pads[3];      // input layer: planar buffers whose padding rows CTA 0 zeroes
    int64_t T, Tp;
    unsigned int* err;           // error word (RX_ERR_TIMEOUT on a stalled wait)
};

template <int MODE>
__global__ void __launch_bounds__(TcShape<MODE>::NTHR, 1) k_conv_tc(TcArgs a) {
    using S = TcShape<MODE>;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t sbase = smem_u32(sm);
    const uint32_t sW = sbase, sSt = sbase + S::OFF_ST;
    const uint32_t bar0 = sbase + S::OFF_BAR;
    auto in_full = [&](int s) { return bar0 + 8u * s; };
    auto in_empty = [&](int s) { return bar0 + 8u * (S::S + s); };
    auto acc_full = [&](int b) { return bar0 + 8u * (2 * S::S + b); };
    auto acc_empty = [&](int b) { return bar0 + 8u * (2 * S::S + S::NACC + b); };
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + S::OFF_MISC);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + S::OFF_MISC + 4);
    float* bias_s = reinterpret_cast<float*>(sm + S::OFF_BIAS);
    const int mma_warp = S::NWARP - 1;
    const int64_t T = a.T, Tp = a.Tp;
    const int64_t ntiles = (T + S::TO - 1) / S::TO;

    // weights, as 16-byte chunks (row, kc) into plane kc. Input layer: row = output channel, chunk kc
    // of its (k, ci) row. Output layer: row 4 k + co holds W[co][8 kc .. 8 kc + 8][k] (rows 36..127
    // zero). Hidden layers: below.
    for (int i = tid; i < S::NKC * S::WROWS; i += S::NTHR) {
        const int r = i / S::NKC, kc = i - r * S::NKC;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if constexpr (MODE == OUT) {
            if (r < S::DROWS)
                v = __ldg(reinterpret_cast<const uint4*>(a.Wm + (int64_t)(r & 3) * 576 + (r >> 2) * 64 + kc * 8));
        } else if constexpr (MODE == HID) {
            // plane kc = 8 m + c: tap pair m, input channels 8 c .. 8 c + 7; row r: channel
            // 16 (r / 32) + r % 16 of tap 2 m + (r / 16) % 2
            const int m = kc >> 3, c = kc & 7;
            const int co = 16 * (r >> 5) + (r & 15), tap = 2 * m + ((r >> 4) & 1);
            if (tap < 9) v = __ldg(reinterpret_cast<const uint4*>(a.Wm + (int64_t)co * 576 + tap * 64 + c * 8));
        } else {
            v = __ldg(reinterpret_cast<const uint4*>(a.Wm + ((int64_t)r * S::NKC + kc) * 8));
        }
        *reinterpret_cast<uint4*>(sm + kc * S::WPL + r * 16) = v;
    }
    // staged rows past a frame's end are read (by outputs past the end, and by the zero weights of
    // tap 9): start every stage from finite values
    if constexpr (MODE != IN)
        for (int i = tid; i < S::S * S::STAGE / 16; i += S::NTHR)
            *reinterpret_cast<uint4*>(sm + S::OFF_ST + 16 * i) = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < S::COUT; i += S::NTHR) bias_s[i] = a.bias[i];
    if (tid == 0) {
        *abort = 0;
        for (int s = 0; s < S::S; ++s) {
            mbar_init(in_full(s), MODE == IN ? 32 * S::NPW : 1);
            mbar_init(in_empty(s), 1);
        }
        for (int b = 0; b < S::NACC; ++b) {
            mbar_init(acc_full(b), 1);
            mbar_init(acc_empty(b), S::NEPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)S::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the input layer's CTA 0 zeroes the padding rows of the three planar activation buffers
    if (MODE == IN && blockIdx.x == 0) {
        for (int i = tid; i < 3 * 8 * 2 * PAD; i += S::NTHR) {
            const int buf = i / (8 * 2 * PAD), r = i - buf * 8 * 2 * PAD, cc = r / (2 * PAD), u = r - cc * 2 * PAD;
            const int64_t row = u < PAD ? u : T + u;           // [0, PAD) and [T + PAD, Tp)
            __nv_bfloat16* pb = buf == 0 ? a.pads[0] : buf == 1 ? a.pads[1] : a.pads[2];
            if (pb) *reinterpret_cast<uint4*>(pb + ((int64_t)cc * Tp + row) * 8) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    fence_async_smem();                                       // weights written by threads, read by the MMA
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < S::NEPI) {
        // ---- epilogue ----
        int it = 0;
        float2 zcur = make_float2(0.0f, 0.0f);            // output layer: residual of the current tile
        if (MODE == OUT && (tid & 255) < S::TO) {
            const int64_t t = (int64_t)blockIdx.x * S::TO + (tid & 255);
            if (t < T) zcur = a.z[(int64_t)(tid >> 8) * T + t];
        }
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int ab = it % S::NACC;
            const uint32_t aph = (uint32_t)((it / S::NACC) & 1);
            const int64_t t0 = tile * S::TO;
            if constexpr (MODE == OUT) {
                constexpr int NE = 32 * S::NEPI;
                constexpr int QP = S::MMA_N / 16 / S::NPART;  // 16-column chunks per part
                // this thread's output: tile position p = tid % 256, polarisation tid / 256 (co 2 pol,
                // 2 pol + 1), so that a warp reads 32 consecutive columns of one D row
                const int p = tid & 255, pol = tid >> 8;
                const int64_t t = t0 + p;
                const bool mine = p < S::TO && t < T;
                // the residual of this tile (loaded during the previous one) and of the next
                const float2 zr = zcur;
                {
                    const int64_t tn = t + (int64_t)gridDim.x * S::TO;
                    zcur = (p < S::TO && tn < T) ? a.z[(int64_t)pol * T + tn] : make_float2(0.0f, 0.0f);
                }
                const bool ok = mbar_wait(acc_full(ab), aph, abort);
                // one decision for the epilogue warps (named barrier 2), which also orders the
                // previous tile's reads of the D rows before this tile's writes
                if (bar_or<2, NE>(!ok || *abort)) break;
                tc_after();
                float* Ds = reinterpret_cast<float*>(sm + S::OFF_F);     // [36][DSTR]
                const int quarter = warp & 3, part = warp >> 2;
                if (quarter < 2) {                            // the 36 used rows are in quarters 0, 1
                    const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(ab * S::MMA_N);
                    const int row = 32 * quarter + lane;
#pragma unroll
                    for (int qq = 0; qq < QP; ++qq) {
                        const int q = QP * part + qq;
                        float v[16];
                        tmem_ld16(tl + 16 * q, v);
                        if (row < S::DROWS) {
                            float4* dst = reinterpret_cast<float4*>(Ds + row * S::DSTR + 16 * q);
#pragma unroll
                            for (int e = 0; e < 4; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
                        }
                    }
                }
                tc_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty(ab));
                bar_sync<2, NE>();                            // D rows complete
                if (mine) {
                    float f[2];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int co = 2 * pol + c;
                        float acc = 0.0f;
#pragma unroll
                        for (int k = 0; k < 9; ++k) acc += Ds[(4 * k + co) * S::DSTR + p + k];
                        f[c] = acc;
                    }
                    a.sym[(int64_t)pol * T + t] =
                        make_float2(zr.x + f[0] + bias_s[2 * pol], zr.y + f[1] + bias_s[2 * pol + 1]);
                }
            } else if constexpr (MODE == HID) {
                constexpr int NE = 32 * S::NEPI;
                const bool ok = mbar_wait(acc_full(ab), aph, abort);
                // one decision for the epilogue warps, also ordering the previous tile's reads
                // of the output tile before this tile's writes
                if (bar_or<2, NE>(!ok || *abort)) break;
                tc_after();
                __nv_bfloat16* Os = reinterpret_cast<__nv_bfloat16*>(sm + S::OFF_F);   // [TO][OSTR]
                // warp w reads lane quarter w % 4 (channels 16 (w % 4) ..) over column part w / 4
                constexpr int QP = S::MMA_N / 16 / S::NPART;  // 16-column chunks per part
                const int quarter = warp & 3, part = warp >> 2;
                const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(ab * S::MMA_N);
                const bool even = lane < 16;
                const int co = 16 * quarter + (lane & 15);
                const float bco = bias_s[co];
                // D_even of the column before this part (the even lanes' first output needs it)
                float prev = part ? tmem_ld1(tl + 16 * QP * part - 1) : 0.0f;
#pragma unroll 2
                for (int qq = 0; qq < QP; ++qq) {
                    const int q = QP * part + qq;             // 16-column chunk
                    float v[16];
                    tmem_ld16(tl + 16 * q, v);
                    // outputs p = 16 q - 1 + i (even lanes) and 16 q + 7 + i (odd lanes), i < 8, each
                    // D_even[p] + D_odd[p + 1]; the partner lane (xor 16) supplies the other half
                    float x[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = __shfl_xor_sync(0xffffffffu, even ? v[7 + i] : v[i], 16);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float de = even ? (i == 0 ? prev : v[i - 1]) : x[i];
                        const float dod = even ? x[i] : v[8 + i];
                        const int pp = even ? 16 * q - 1 + i : 16 * q + 7 + i;
                        if (pp >= 0 && pp < S::TO)
                            Os[pp * S::OSTR + co] = __float2bfloat16_rn(fmaxf(de + dod + bco, 0.0f));
                    }
                    prev = v[15];
                }
                tc_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty(ab));
                bar_sync<2, NE>();                            // output tile complete
                // 16-byte rows (8 channels of one position) to the planes; a warp covers two planes
                // x 16 consecutive positions
                constexpr int PSTEP = 16 * (NE / 128);        // positions per pass of all threads
                const int cc = (tid >> 4) & 7, poff = 16 * (tid >> 7);
#pragma unroll 4
                for (int r = 0; r < (S::TO + PSTEP - 1) / PSTEP; ++r) {
                    const int pp = PSTEP * r + poff + (tid & 15);
                    const int64_t t = t0 + pp;
                    if (pp < S::TO && t < T)
                        *reinterpret_cast<uint4*>(a.act + ((int64_t)cc * Tp + t + PAD) * 8) =
                            *reinterpret_cast<const uint4*>(Os + pp * S::OSTR + 8 * cc);
                }
            } else {
                // warp w: positions of lane quarter w % 4, channels of part w / 4; the tile goes through
                // one of two shared-memory output tiles and leaves by bulk async stores (one per plane)
                constexpr int NE = 32 * S::NEPI;
                constexpr int CP = S::MMA_N / S::NPART;       // channels per part
                const int quarter = warp & 3, part = warp >> 2;
                const int pl = 32 * quarter + lane;           // this thread's tile position
                const int ob = it & 1;
                const uint32_t obase = sbase + S::OFF_F + S::FROWS * 8 + ob * S::OB;
                // the stores that read this output tile two tiles ago are done with it
                if (tid == 0 && it >= 2) bulk_wait_read<1>();
                const bool ok = mbar_wait(acc_full(ab), aph, abort);
                if (bar_or<2, NE>(!ok || *abort)) break;  // uniform; also orders the tile's reuse
                tc_after();
                const uint32_t tl =
                    tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(ab * S::MMA_N + CP * part);
                float v[CP];
#pragma unroll
                for (int q = 0; q < CP / 16; ++q) tmem_ld16(tl + 16 * q, v + 16 * q);
                tc_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty(ab));
                unsigned char* otile = sm + S::OFF_F + S::FROWS * 8 + ob * S::OB;
#pragma unroll
                for (int c8 = 0; c8 < CP / 8; ++c8) {
                    const int cc = (CP / 8) * part + c8;
                    float w[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) w[e] = fmaxf(v[8 * c8 + e] + bias_s[8 * cc + e], 0.0f);
                    uint4 o;
                    o.x = pack_bf16(w[0], w[1]);
                    o.y = pack_bf16(w[2], w[3]);
                    o.z = pack_bf16(w[4], w[5]);
                    o.w = pack_bf16(w[6], w[7]);
                    *reinterpret_cast<uint4*>(otile + (cc * 128 + pl) * 16) = o;
                }
                fence_async_smem();                           // written by threads, read by the copies
                bar_sync<2, NE>();
                if (tid == 0) {
                    const int n = (int)min((int64_t)128, T - t0);   // positions of this tile in the frame
                    for (int cc = 0; cc < 8; ++cc)
                        bulk_s2g(a.act + ((int64_t)cc * Tp + t0 + PAD) * 8, obase + cc * 128 * 16, (uint32_t)(n * 16));
                    bulk_commit();
                }
            }
        }
        if (MODE == IN && tid == 0) bulk_wait_all();          // the output tiles are written out
    } else if (warp < S::NEPI + S::NPW) {
        // ---- producer ----
        int it = 0, issued = 0;
        if constexpr (MODE == IN) {
            const int r = tid - 32 * S::NEPI;                 // 0 .. 127
            unsigned char* F = sm + S::OFF_F;                 // [FROWS][4] BF16: position t0 - 4 + u
            // this thread's staged positions u = r, r + 128 of a tile, loaded two tiles ahead into one of
            // two register sets used alternately and kept as loaded (converted only when written), so
            // that each load has two tiles' time to arrive
            float2 za[2][2], zb[2][2];
            auto zload = [&](int64_t tile, float2 (&zz)[2][2]) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int u = r + 128 * h;
                    const int64_t tt = tile * S::TO - PAD + u;
                    zz[h][0] = zz[h][1] = make_float2(0.0f, 0.0f);
                    if (u < S::FROWS && tile < ntiles && tt >= 0 && tt < T) {
                        zz[h][0] = a.z[tt];
                        zz[h][1] = a.z[T + tt];
                    }
                }
            };
            // one tile: planes from zz, then zz reloaded for the tile two steps later; false = stop
            auto produce = [&](int64_t tile, float2 (&zz)[2][2]) -> bool {
                const int s = it % S::S;
                bool ok = true;
                if (r == 0) ok = mbar_wait(in_empty(s), (uint32_t)(((it / S::S) & 1) ^ 1), abort);
                // one decision for the 128 producer threads; also orders the previous tile's reads of F
                if (bar_or<1, 128>(!ok || *abort)) return false;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (r + 128 * h < S::FROWS)
                        *reinterpret_cast<uint2*>(F + 8 * (r + 128 * h)) =
                            make_uint2(pack_bf16(zz[h][0].x, zz[h][0].y), pack_bf16(zz[h][1].x, zz[h][1].y));
                zload(tile + 2 * (int64_t)gridDim.x, zz);
                asm volatile("bar.sync 1, 128;" ::: "memory");
                unsigned char* st = sm + S::OFF_ST + s * S::STAGE;
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    const uint2 lo = *reinterpret_cast<const uint2*>(F + 8 * (r + 2 * j));
                    const uint2 hi = *reinterpret_cast<const uint2*>(F + 8 * (r + 2 * j + 1));
                    *reinterpret_cast<uint4*>(st + j * S::XPL + 16 * r) = make_uint4(lo.x, lo.y, hi.x, hi.y);
                }
                fence_async_smem();
                mbar_arrive(in_full(s));
                ++it;
                return true;
            };
            zload(blockIdx.x, za);
            zload(blockIdx.x + gridDim.x, zb);
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += 2 * (int64_t)gridDim.x) {
                if (!produce(tile, za)) break;
                if (tile + gridDim.x < ntiles && !produce(tile + gridDim.x, zb)) break;
            }
        } else {
            if (lane == 0) {
                for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                    const int s = it % S::S;
                    if (!mbar_wait(in_empty(s), (uint32_t)(((it / S::S) & 1) ^ 1), abort)) break;
                    const int64_t t0 = tile * S::TO;          // staged row u = padded position t0 + u
                    const int rows = (int)min((int64_t)S::XROWS, Tp - t0);
                    mbar_arrive_tx(in_full(s), (uint32_t)(8 * rows * 16));
                    for (int cc = 0; cc < 8; ++cc)
                        bulk_g2s(sSt + s * S::STAGE + cc * S::XPL, a.x + ((int64_t)cc * Tp + t0) * 8,
                                 (uint32_t)(rows * 16), in_full(s));
                    issued = it + 1;
                }
                // copies still in flight after an abort land before the CTA exits
                if (*abort)
                    for (int i = max(0, issued - S::S); i < issued; ++i)
                        mbar_drain(in_full(i % S::S), (uint32_t)((i / S::S) & 1));
            }
        }
    } else if (lane == 0) {
        // ---- MMA issue ----
        int it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it % S::S, ab = it % S::NACC;
            if (!mbar_wait(in_full(s), (uint32_t)((it / S::S) & 1), abort)) break;
            if (!mbar_wait(acc_empty(ab), (uint32_t)(((it / S::NACC) & 1) ^ 1), abort)) break;
            tc_after();
            const uint32_t d = tmem + (uint32_t)(ab * S::MMA_N);
            const uint32_t st = sSt + s * S::STAGE;
#pragma unroll 4
            for (int ks = 0; ks < S::NKS; ++ks) {
                uint64_t ad, bd;
                if constexpr (MODE == IN) {
                    ad = sdesc(st + 2 * ks * S::XPL, S::XPL, 128);
                    bd = sdesc(sW + 2 * ks * S::WPL, S::WPL, 128);
                } else if constexpr (MODE == HID) {
                    const int m = ks >> 2, j = ks & 3;        // tap pair, 16-channel group
                    ad = sdesc(sW + (8 * m + 2 * j) * S::WPL, S::WPL, 128);
                    bd = sdesc(st + 2 * j * S::XPL + 32 * m, S::XPL, 128);   // rows shifted by 2 m
                } else {                                      // weights as A, positions as B
                    ad = sdesc(sW + 2 * ks * S::WPL, S::WPL, 128);
                    bd = sdesc(st + 2 * ks * S::XPL, S::XPL, 128);
                }
                mma_ss(d, ad, bd, S::IDESC, ks > 0 ? 1u : 0u);
            }
            mma_commit(in_empty(s));
            mma_commit(acc_full(ab));
        }
        // the last MMAs (and the stage-free arrivals they signal) complete before the CTA exits and
        // its tensor memory is freed
        for (int i = max(0, it - S::S); i < it; ++i) mbar_drain(in_empty(i % S::S), (uint32_t)((i / S::S) & 1));
    }

    tc_before();
    __syncthreads();
    if (*abort && tid == 0) atomicOr(a.err, RX_ERR_TIMEOUT);
    if (warp == mma_warp) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::TCOLS)
                     : "memory");
    }
}

template <int MODE>
cudaError_t launch_tc(const TcArgs& a, cudaStream_t s) {
    using S = TcShape<MODE>;
    static int resident = 0;
    if (!resident) {
        int dev = 0, nsm = 152, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        if (e) return e;
        // the whole unified L1 / shared memory as shared memory, so that the CTAs that fit are resident
        e = cudaFuncSetAttribute(k_conv_tc<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e) return e;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_conv_tc<MODE>, S::NTHR, S::SMEM);
        resident = std::max(1, nsm * std::max(1, per));
    }
    const int64_t ntiles = (a.T + S::TO - 1) / S::TO;
    if (ntiles <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(ntiles, resident);
    k_conv_tc<MODE><<<grid, S::NTHR, S::SMEM, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// the inference forward on the tensor cores: symbols -> act[1] -> act[2] -> act[3] (planar) -> out
cudaError_t cnn_infer_tc(const CnnBufs& B, const float2* z, int64_t T, float2* out, cudaStream_t s) {
    if (B.C != 64) return cudaErrorInvalidValue;
    const int64_t Tp = T + 2 * PAD;
    const float* Wf = B.wfwd;
    TcArgs a{};
    a.T = T;
    a.Tp = Tp;
    a.z = z;
    a.err = B.err;
    // layer 0: 4 -> 64 from the symbols; also zeroes the padding rows of the three planar buffers
    a.Wm = B.wtc + wtc_offset(B.C, 0);
    a.bias = Wf + B.off[1];
    a.act = B.act[1];
    a.pads[0] = B.act[1];
    a.pads[1] = B.act[2];
    a.pads[2] = B.act[3];
    cudaError_t e = launch_tc<IN>(a, s);
    if (e) return e;
    a.pads[0] = a.pads[1] = a.pads[2] = nullptr;
    // layers 1, 2: 64 -> 64
    a.x = B.act[1];
    a.Wm = B.wtc + wtc_offset(B.C, 1);
    a.bias = Wf + B.off[3];
    a.act = B.act[2];
    if ((e = launch_tc<HID>(a, s))) return e;
    a.x = B.act[2];
    a.Wm = B.wtc + wtc_offset(B.C, 2);
    a.bias = Wf + B.off[5];
    a.act = B.act[3];
    if ((e = launch_tc<HID>(a, s))) return e;
    // layer 3: 64 -> 4, bias and the residual into the output symbols
    a.x = B.act[3];
    a.Wm = B.wtc + wtc_offset(B.C, 3);
    a.bias = Wf + B.off[7];
    a.act = nullptr;
    a.sym = out;
    return launch_tc<OUT>(a, s);
}
