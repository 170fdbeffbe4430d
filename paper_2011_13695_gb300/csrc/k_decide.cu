// A6 alignment, Gray hard demapping, bit/symbol error and EVM counting.
//
// Paper anchor: decisions are demapped on the GPU and the bits go to host
// memory (Sec. II-D Step 6); quality is a Q-factor derived from the BER of
// each 21 ms section (Sec. V-D). A blind receiver must first find which
// transmitted polarisation, quarter turn and symbol delay each output
// carries: 16 CTAs (output q, tx pol p, turn r) count decision matches for
// every delay in [-D, D] over the sync window (a warp ballot + popcount per
// delay), and the last CTA to finish picks the best (p, r, d) with ties to
// the smallest tuple. Counting then runs one thread per output symbol: the
// decided levels become Gray bits, 32 symbols of a warp assemble m output
// words with warp-wide ORs, errors are the popcount of the XOR with the
// reference bits, integer counters accumulate with 64-bit atomics, EVM sums
// as FP32 partials turned into fixed-point integer atomics.
#include <algorithm>

#include "rx_kernels.h"

namespace {

// rotate by j^r (exact)
__device__ __forceinline__ float2 quarter(float2 v, int r) {
    switch (r & 3) {
        case 1: return make_float2(-v.y, v.x);
        case 2: return make_float2(-v.x, -v.y);
        case 3: return make_float2(v.y, -v.x);
        default: return v;
    }
}

__device__ __forceinline__ int gray_to_level(uint32_t g) {
    return (int)(g ^ (g >> 1) ^ (g >> 2) ^ (g >> 3));
}

// m stream bits of symbol t (bit 0 = first transmitted bit)
__device__ __forceinline__ uint32_t ref_symbol_bits(const uint32_t* ref, int64_t t, int m) {
    const int64_t b0 = t * m;
    const int64_t w = b0 >> 5;
    const int off = (int)(b0 & 31);
    uint64_t v = ref[w];
    if (off + m > 32) v |= (uint64_t)ref[w + 1] << 32;
    return (uint32_t)(v >> off) & ((1u << m) - 1u);
}

// stream bits -> (l_I, l_Q)
__device__ __forceinline__ void bits_to_levels(uint32_t sbits, int m, int& li, int& lq) {
    const uint32_t msb = __brev(sbits) >> (32 - m);
    const int h = m / 2;
    li = gray_to_level(msb >> h);
    lq = gray_to_level(msb & ((1u << h) - 1u));
}

// One warp per output q (warps 0 and 1 of the last CTA): the (p, r, d) with most matches, ties to
// the smallest tuple (p, then r, then d). The warp then zeroes the counts it read for the next sync.
__device__ void sync_pick(int* counts, int D, int64_t len, RxDevState* st, int q, int lane) {
    const int nd = 2 * D + 1, ntup = 8 * nd;
    int* cq = counts + (int64_t)q * ntup;             // tuple index t = (p * 4 + r) * nd + (d + D)
    int bv = -1, bt = 0;
    for (int t = lane; t < ntup; t += 32) {
        const int v = __ldcg(&cq[t]);
        if (v > bv) { bv = v; bt = t; }               // t increases along the lane's scan
    }
    for (int o = 16; o > 0; o >>= 1) {
        const int ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
        if (ov > bv || (ov == bv && ot < bt)) { bv = ov; bt = ot; }
    }
    __syncwarp();
    for (int t = lane; t < ntup; t += 32) cq[t] = 0;
    if (lane == 0) {
        const int pr = bt / nd;
        st->sync_p[q] = pr >> 2;
        st->sync_r[q] = pr & 3;
        st->sync_d[q] = bt - pr * nd - D;
        st->sync_match[q] = bv;
        if (10LL * bv < 9LL * len) atomicOr(&st->err_word, 2u);
        if (q == 0) st->sync_len = (int)len;
    }
}

// blockIdx.x: (output q, tx pol p, turn r); blockIdx.y: slice of the sync window. Match counts of
// the slice for every delay are added into counts; the last CTA to arrive (a ticket after the
// counts, zero between launches) picks the alignment and zeroes the counts and the ticket.
__global__ void __launch_bounds__(256) k_sync(const float2* __restrict__ z, int64_t zstride,
                                              const uint32_t* __restrict__ ref, int64_t refstride, int64_t n_ref,
                                              int m, int64_t lo, int64_t hi, int D, int64_t lat, int64_t slice,
                                              int64_t len, int* counts, unsigned* ticket, RxDevState* st) {
    const int q = blockIdx.x >> 3, p = (blockIdx.x >> 2) & 1, r = blockIdx.x & 3;
    const int64_t s0 = lo + (int64_t)blockIdx.y * slice;
    const int64_t s1 = min(hi, s0 + slice);
    extern __shared__ int16_t txl[];                  // tx levels for t in [s0 - lat - D, s1 - lat + D)
    __shared__ int cnt[2 * RX_MAX_DELAY + 1];
    __shared__ bool s_last;
    for (int i = threadIdx.x; i < 2 * D + 1; i += blockDim.x) cnt[i] = 0;
    if (s0 < s1) {
        const int64_t t0 = s0 - lat - D;
        const int64_t nt = (s1 - s0) + 2 * D;
        const uint32_t* rp = ref + (int64_t)p * refstride;
        for (int64_t i = threadIdx.x; i < nt; i += blockDim.x) {
            const int64_t t = t0 + i;
            int16_t v = -1;
            if (t >= 0 && t < n_ref) {
                int li, lq;
                bits_to_levels(ref_symbol_bits(rp, t, m), m, li, lq);
                v = (int16_t)(li | (lq << 8));
            }
            txl[i] = v;
        }
        __syncthreads();
        const Qam qm = make_qam(m);
        const int lane = threadIdx.x & 31;
        const int nd = 2 * D + 1;
        // lane j of a warp keeps the warp's matches of delays 32 k + j - D (k < 5) in registers
        int creg[(2 * RX_MAX_DELAY + 32) / 32] = {0};
        for (int64_t base = s0 + (threadIdx.x & ~31); base < s1; base += blockDim.x) {
            const int64_t n = base + lane;
            int16_t mine = -2;
            if (n < s1) {
                const float2 v = quarter(z[(int64_t)q * zstride + n], r);
                mine = (int16_t)(qam_level(v.x, qm) | (qam_level(v.y, qm) << 8));
            }
            const int16_t* tx = txl + (n - s0);
#pragma unroll
            for (int k = 0; k < (2 * RX_MAX_DELAY + 32) / 32; ++k) {
                if (32 * k >= nd) break;
                int c = 0;
#pragma unroll 8
                for (int j = 0; j < 32; ++j) {
                    const int di = 32 * k + j;
                    if (di >= nd) break;
                    const bool hit = (n < s1) && (tx[di] == mine);
                    const int pc = __popc(__ballot_sync(0xffffffffu, hit));
                    c = lane == j ? pc : c;
                }
                creg[k] += c;
            }
        }
#pragma unroll
        for (int k = 0; k < (2 * RX_MAX_DELAY + 32) / 32; ++k)
            if (32 * k + lane < nd && creg[k]) atomicAdd(&cnt[32 * k + lane], creg[k]);
        __syncthreads();
        for (int i = threadIdx.x; i < 2 * D + 1; i += blockDim.x)
            if (cnt[i]) atomicAdd(&counts[blockIdx.x * (2 * D + 1) + i], cnt[i]);
    }
    // arrival: this CTA's additions ordered before its ticket
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned done = atomicAdd(ticket, 1u);
        s_last = done == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < 64) sync_pick(counts, D, len, st, threadIdx.x >> 5, threadIdx.x & 31);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->sync_valid = 1;
        *ticket = 0u;
    }
}

// Grid-stride over groups of four consecutive symbols of one output
// polarisation (M bits per symbol); counters stay in registers until one
// block-wide reduction and one set of atomics per CTA. Two tables in shared
// memory, built per CTA with the same arithmetic as the direct forms: the
// decision's stream bits by its levels (li + 16 lq), and the reference
// symbol's ideal point and energy by its M stream bits. A thread's four
// decisions form one 4M-bit chunk of the output stream; a warp's 32 chunks
// are 4M whole words, each gathered by one lane with shuffles. The
// reference bits of the four symbols are one funnel of two words, compared
// with the chunk in one XOR. I is the index type: 32-bit when every index of
// the launch fits, else 64-bit.
template <int M, typename I>
__global__ void __launch_bounds__(256) k_count(const float2* __restrict__ z, I zstride, I N,
                                               const uint32_t* __restrict__ ref, I refstride, I n_ref,
                                               I lo, I hi, I lat, uint32_t* __restrict__ out, I outstride,
                                               RxDevState* st, int vec) {
    constexpr int C = 4 * M;                          // chunk bits
    constexpr uint32_t MASK = (1u << M) - 1u;
    __shared__ float4 s_pt[1 << M];                   // reference bits -> (s.x, s.y, |s|^2, 0)
    __shared__ uint32_t s_bits[256];                  // li + 16 lq -> decision stream bits
    const int q = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const bool have_sync = ref != nullptr && st->sync_valid;
    const int r = have_sync ? st->sync_r[q] : 0;
    const int p = have_sync ? st->sync_p[q] : 0, d = have_sync ? st->sync_d[q] : 0;
    const Qam qm = make_qam(M);
    {
        const int i = threadIdx.x;                    // launched with 256 threads
        const int li = i & 15, lq = i >> 4;
        s_bits[i] = (li < qm.L && lq < qm.L) ? msb_first_to_stream(qam_bits(li, lq, qm), M) : 0u;
        if (i < (1 << M)) {
            int ti, tq;
            bits_to_levels((uint32_t)i, M, ti, tq);
            const float2 sp = make_float2(qam_value(ti, qm), qam_value(tq, qm));
            s_pt[i] = make_float4(sp.x, sp.y, cabs2(sp), 0.0f);
        }
    }
    __syncthreads();
    const I nwords = (N * M + 31) / 32;
    const I nrw = (n_ref * M + 31) / 32;
    const uint32_t* refp = have_sync ? ref + (I)p * refstride : nullptr;
    // counted symbols: n in [lo, hi) with reference index t = n + d - lat in [0, n_ref)
    const I c0 = max(max(lo, lat - (I)d), (I)0);
    const I c1 = min(min(hi, N), n_ref + lat - (I)d);
    uint32_t errs = 0, serr = 0, cnt = 0;
    // EVM sums: FP32 per thread (a handful of symbols each), per warp and per CTA, then fixed point
    // (FP64 arithmetic, atomics included, runs at a small fraction of the FP32 rate on this part)
    float en = 0.0f, ed = 0.0f;
    const float2* zq = z + (I)q * zstride;
    uint32_t* oq = out ? out + (I)q * outstride : nullptr;
    const I G = (N + 3) / 4;
    const I step = (I)gridDim.x * blockDim.x;
    for (I g = (I)blockIdx.x * blockDim.x + threadIdx.x; g - lane < G; g += step) {
        const I n0 = 4 * g;
        float2 v[4];
        if (vec && n0 + 3 < N) {
            const float4 a = *reinterpret_cast<const float4*>(zq + n0);
            const float4 b = *reinterpret_cast<const float4*>(zq + n0 + 2);
            v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
            v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = n0 + k < N ? zq[n0 + k] : make_float2(0.0f, 0.0f);
        }
        uint32_t chunk = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = quarter(v[k], r);
            const uint32_t sb = s_bits[qam_level(v[k].x, qm) | (qam_level(v[k].y, qm) << 4)];
            if (n0 + k < N) chunk |= sb << (k * M);
        }
        if (oq) {
            // lane w < C assembles word w of the warp's C words: bits [32 w, 32 w + 32) of the 32 chunks
            const int a = (lane * 32) / C, off = (lane * 32) % C;
            uint32_t word = __shfl_sync(0xffffffffu, chunk, a < 32 ? a : 31) >> off;
#pragma unroll
            for (int k = 1; k <= (32 + C - 1) / C; ++k) {
                const int src = a + k;
                const uint32_t part = __shfl_sync(0xffffffffu, chunk, src < 32 ? src : 31);
                const int sh = k * C - off;
                if (src < 32 && sh < 32) word |= part << sh;
            }
            const I wi = (g - lane) * (C / 4) / 8 + lane;   // (g - lane) 4M / 32 whole words before the warp
            if (lane < C && wi < nwords) oq[wi] = word;
        }
        if (have_sync && n0 + 3 >= c0 && n0 < c1) {
            const I bit0 = (n0 + (I)d - lat) * M;
            const I w0 = bit0 >> 5;                   // floor, also below zero
            const int off = (int)(bit0 & 31);
            const uint32_t wl = (w0 >= 0 && w0 < nrw) ? __ldg(&refp[w0]) : 0u;
            uint32_t rb4 = wl >> off;
            if (off + C > 32) {
                const uint32_t wh = (w0 + 1 >= 0 && w0 + 1 < nrw) ? __ldg(&refp[w0 + 1]) : 0u;
                rb4 |= wh << (32 - off);
            }
            const uint32_t x = rb4 ^ chunk;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (n0 + k >= c0 && n0 + k < c1) {
                    const uint32_t e = __popc((x >> (k * M)) & MASK);
                    errs += e;
                    serr += e ? 1u : 0u;
                    cnt += 1;
                    const float4 sp = s_pt[(rb4 >> (k * M)) & MASK];
                    en += cabs2(csub(v[k], make_float2(sp.x, sp.y)));
                    ed += sp.z;
                }
            }
        }
    }
    if (!have_sync) return;
    __shared__ unsigned int ri[3][8];
    __shared__ float rd[2][8];
    errs = __reduce_add_sync(0xffffffffu, errs);
    serr = __reduce_add_sync(0xffffffffu, serr);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    en = warp_sum(en);
    ed = warp_sum(ed);
    const int w = threadIdx.x >> 5;
    if (lane == 0) {
        ri[0][w] = errs; ri[1][w] = serr; ri[2][w] = cnt;
        rd[0][w] = en; rd[1][w] = ed;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0, c = 0;
        float x = 0.0f, y = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += ri[0][i]; b += ri[1][i]; c += ri[2][i]; x += rd[0][i]; y += rd[1][i];
        }
        if (c) {
            atomicAdd(&st->bit_errors, a);
            atomicAdd(&st->symbol_errors, b);
            atomicAdd(&st->symbols, c);
            atomicAdd(&st->bits, c * (unsigned long long)M);
            // EVM sums as fixed point: integer atomics, exact and in no particular order
            atomicAdd(&st->evm_num_fx, __float2ull_rn(x * RX_EVM_FX_SCALE));
            atomicAdd(&st->evm_den_fx, __float2ull_rn(y * RX_EVM_FX_SCALE));
        }
    }
}

template <int M, typename I>
cudaError_t count_m(dim3 grid, const float2* z, I zstride, I N, const uint32_t* ref, I refstride, I n_ref, I lo,
                    I hi, I lat, uint32_t* out, I outstride, RxDevState* st, int vec, cudaStream_t s) {
    k_count<M, I><<<grid, 256, 0, s>>>(z, zstride, N, ref, refstride, n_ref, lo, hi, lat, out, outstride, st, vec);
    return cudaGetLastError();
}

template <typename I>
cudaError_t count_i(int m, dim3 grid, const float2* z, I zstride, I N, const uint32_t* ref, I refstride, I n_ref,
                    I lo, I hi, I lat, uint32_t* out, I outstride, RxDevState* st, int vec, cudaStream_t s) {
    switch (m) {
        case 2: return count_m<2, I>(grid, z, zstride, N, ref, refstride, n_ref, lo, hi, lat, out, outstride, st, vec, s);
        case 4: return count_m<4, I>(grid, z, zstride, N, ref, refstride, n_ref, lo, hi, lat, out, outstride, st, vec, s);
        case 6: return count_m<6, I>(grid, z, zstride, N, ref, refstride, n_ref, lo, hi, lat, out, outstride, st, vec, s);
        case 8: return count_m<8, I>(grid, z, zstride, N, ref, refstride, n_ref, lo, hi, lat, out, outstride, st, vec, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_sync(const float2* z, int64_t zstride, const uint32_t* ref, int64_t refstride, int64_t n_ref,
                        int m, int64_t lo, int64_t hi, int max_delay, int64_t lat, int* counts, RxDevState* st,
                        cudaStream_t s, int* nlaunch) {
    // 16 (q, p, r) combinations x up to 16 slices of at least 256 symbols
    const int64_t len = hi - lo;
    const int nsl = (int)std::max<int64_t>(1, std::min<int64_t>(16, len / 256));
    const int64_t slice = (len + nsl - 1) / nsl;
    const size_t smem = sizeof(int16_t) * (size_t)(slice + 2 * max_delay);
    static size_t attr = 0;
    if (smem > 48 * 1024 && smem > attr) {
        cudaFuncSetAttribute(k_sync, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    // the arrival ticket sits after the largest count table
    unsigned* ticket = reinterpret_cast<unsigned*>(counts + 16 * (2 * RX_MAX_DELAY + 1));
    k_sync<<<dim3(16, nsl), 256, smem, s>>>(z, zstride, ref, refstride, n_ref, m, lo, hi, max_delay, lat, slice,
                                           len, counts, ticket, st);
    if (nlaunch) *nlaunch += 1;
    return cudaGetLastError();
}

cudaError_t launch_count(const float2* z, int64_t zstride, int64_t N, const uint32_t* ref, int64_t refstride,
                         int64_t n_ref, int m, int64_t lo, int64_t hi, int64_t lat, uint32_t* out,
                         int64_t outstride, RxDevState* st, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    // one resident wave: SMs x resident CTAs per SM, split between the two outputs
    static int resident = 0;
    if (!resident) {
        int dev = 0, nsm = 152, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_count<8, int64_t>, 256, 0);
        resident = std::max(1, nsm * per);
    }
    const int64_t want = (N + 1023) / 1024;           // four symbols per thread
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(want, resident / 2)), 2);
    // 16-byte loads of four symbols when both rows are aligned for them
    const int vec = ((uintptr_t)z % 16) == 0 && (zstride % 2) == 0;
    // 32-bit indices when the largest of them (bit positions of both outputs and references, element
    // offsets of the second rows, the grid-stride walk past N) stays below 2^31
    const int64_t lim = (int64_t)1 << 30;
    const bool narrow = N < lim / 16 && n_ref < lim / 16 && zstride < lim && refstride < lim && outstride < lim &&
                        lat < lim && lo < lim && hi < lim;
    if (narrow)
        return count_i<int>(m, grid, z, (int)zstride, (int)N, ref, (int)refstride, (int)n_ref, (int)lo, (int)hi,
                            (int)lat, out, (int)outstride, st, vec, s);
    return count_i<int64_t>(m, grid, z, zstride, N, ref, refstride, n_ref, lo, hi, lat, out, outstride, st, vec, s);
}
