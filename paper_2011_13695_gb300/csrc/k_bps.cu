// A5 blind phase search (Pfau, Hoffmann, Noe 2009), integer unwrap, derotation.
//
// Test phases theta_b = (b/B - 1/2) pi/2. For symbol k and phase b,
// dist = |y_k e^{-j theta_b} - dec(.)|^2 and D[k, b] is its sum over the window
// [k - W/2, k + W/2) clipped to the frame; b*_k = argmin_b D (first minimum).
//
// Layout, B <= 32: one thread per test phase and strip of LEN consecutive
// symbols (32 threads per strip), strips of one polarisation side by side in
// a CTA. The strip's symbols (with a W/2 halo on each side) are staged in
// shared memory as (x, y, y, -x) and read as 16-byte broadcasts, so that the
// rotation, rounding and error of both dimensions are packed FP32x2
// instructions (each component the same FMA or add as the scalar form, so
// the results are bit-identical to it). Each thread keeps the last W
// distances of its phase in registers (a ring indexed at compile time), slides
// the window sum by one add and one subtract per symbol and re-forms it as a
// direct sum of the ring every W symbols, which bounds the rounding drift to
// that of a W-term sum. B > 32 (k_bps2): one warp per strip, each lane holding
// phases l and l + 32, the packed instructions running over the phase pair
// (symbols staged as (x, x, y, y)); the same operations per component, so the
// two layouts give the same bits. The minimum over phases is one warp-wide min reduction
// of a key per lane: the (non-negative) sum's bit pattern with its low six
// bits replaced by the phase index, so one reduction gives both the least sum
// and its phase; sums that agree to within 64 units in the last place
// (7.6e-6 relative, below the FP32 sums' own rounding of ~64 terms) count as
// a tie, which goes to the smallest b. The decision per real
// dimension is evaluated in level units: v = r / (2a) + (L-1)/2, the nearest
// level is rint(clamp(v, 0, L-1)), computed with a saturating multiply and
// the 1.5 * 2^23 rounding constant, so the distance costs only FMA-pipe
// instructions.
//
// The paper's phase unwrap (Sec. III-B) is a single warp walking the blocks
// in order; here the unwrap is exact integer arithmetic on b*, so it becomes
// a three-step scan: per-tile jump sums, a scan of the tile sums with the
// carried count, then per-tile prefixes that also write z.
#include <algorithm>

#include "rx_kernels.h"

namespace {

constexpr int BPS_THREADS = 128;

// distance of one symbol to the nearest point after rotation, in level units. The symbol is staged
// as (x, y, y, -x), so that the rotation of both components is two packed FMAs (per component the
// same fmaf as the scalar form: vI = fma(x, c, fma(y, s, hL)), vQ = fma(y, c, fma(-x, s, hL))),
// and the rounding and the error of both dimensions take one packed instruction each.
__device__ __forceinline__ float bps_dist(float4 v, float2 cc, float2 ss, float2 hh, float invLm1, float2 ll) {
    const float2 MAGIC = make_float2(12582912.0f, 12582912.0f);   // 1.5 * 2^23: x + MAGIC - MAGIC = rint(x)
    const float2 r = __ffma2_rn(make_float2(v.x, v.y), cc, __ffma2_rn(make_float2(v.z, v.w), ss, hh));
    const float2 w = make_float2(__saturatef(r.x * invLm1), __saturatef(r.y * invLm1));
    const float2 t = __fadd2_rn(__ffma2_rn(w, ll, MAGIC), make_float2(-MAGIC.x, -MAGIC.y));
    const float2 e = __ffma2_rn(t, make_float2(-1.0f, -1.0f), r);   // r - t, exactly rounded once
    return fmaf(e.x, e.x, e.y * e.y);
}

// publish one window's warp minimum: the least key (sum bits >> 6, phase) as unsigned integers, the
// order of the sums, which are not negative
__device__ __forceinline__ void bps_publish(float D, unsigned int* slot, int lane, unsigned int b) {
    const unsigned int key = (__float_as_uint(D) & ~63u) | b;
    const unsigned int mn = __reduce_min_sync(0xffffffffu, key);
    if (lane == 0) *slot = mn;
}

// the windows of one strip for one test phase: the ring of distances, the sliding sum, the published
// minima and the picks (EDGE: the strip's span holds symbols outside the frame, NaN, guarded to 0)
template <int W, int GS, bool EDGE>
__device__ __forceinline__ void bps_strip(const float4* __restrict__ yl, float2 cc, float2 ss, float2 hh, float invLm1,
                                          float2 ll, float pen, int nc, int LEN, int64_t s0, int64_t N,
                                          unsigned int (*slots)[W], unsigned int* myslots, int b, int lane, int q,
                                          uint8_t* __restrict__ bstar, int64_t bstride) {
    constexpr int NW = GS / 32;
    // the last W distances of this thread's phase, in registers (indices fixed at compile time)
    float ring[W];
    float D = pen;
#pragma unroll
    for (int u = 0; u < W; ++u) {
        float d = bps_dist(yl[u], cc, ss, hh, invLm1, ll);
        if (EDGE) d = fmaxf(d, 0.0f);
        ring[u] = d;
        D += d;
    }
    bps_publish(D, &myslots[0], lane, (unsigned)b);   // window of local output 0
    for (int ch = 0; ch <= nc; ++ch) {
        if (ch > 0) {
            const float4* yc = yl + ch * W;
#pragma unroll
            for (int u = 0; u < W; ++u) {
                float d = bps_dist(yc[u], cc, ss, hh, invLm1, ll);
                if (EDGE) d = fmaxf(d, 0.0f);
                const float old = ring[u];
                ring[u] = d;
                D = (D + d) - old;
                // window of local output (ch - 1) W + u + 1 is complete; its slot is (u + 1) % W
                bps_publish(EDGE ? fmaxf(D, 0.0f) : D, &myslots[(u + 1) & (W - 1)], lane, (unsigned)b);
            }
            float t = pen;                            // re-form the sum directly from the ring
#pragma unroll
            for (int r = 0; r < W; ++r) t += ring[r];
            D = t;
        }
        __syncthreads();
        for (int slot = b; slot < W; slot += GS) {
            const int kl = slot == 0 ? ch * W : (ch - 1) * W + slot;
            if (kl >= 0 && kl < LEN && s0 + kl < N) {
                const unsigned int k0 = slots[0][slot];
                const int r = (int)((NW == 2 ? min(k0, slots[NW - 1][slot]) : k0) & 63u);
                bstar[(int64_t)q * bstride + s0 + kl] = (uint8_t)r;
            }
        }
        __syncthreads();
    }
}

template <int W, int GS>
__global__ void __launch_bounds__(BPS_THREADS, 5) k_bps(const float2* __restrict__ y, int64_t ystride, int64_t N,
                                                      int B, float cI0, float hL, float invLm1, float Lm1, int LEN,
                                                      uint8_t* __restrict__ bstar, int64_t bstride) {
    constexpr int NSTRIP = BPS_THREADS / GS;
    constexpr int NW = GS / 32;
    pdl_trigger();                                    // the unwrap may become resident now
    pdl_wait();                                       // launched programmatically: y is complete after this
    extern __shared__ float4 smem_v[];
    float4* ys = smem_v;                              // [NSTRIP][LEN + W]: (x, y, y, -x)
    __shared__ unsigned int slots[NSTRIP][NW][W];     // per output slot: the warp's least key
    const int tid = threadIdx.x;
    const int sl = tid / GS;                          // strip within the CTA
    const int b = tid % GS;
    const int lane = tid & 31, wip = b >> 5;          // warp within the strip
    const int q = blockIdx.y;
    const int64_t s0 = ((int64_t)blockIdx.x * NSTRIP + sl) * LEN;
    const int span = LEN + W;
    const float2* yq = y + (int64_t)q * ystride;
    const float4* yl = ys + sl * span;

    // stage y[s0 - W/2, s0 + LEN + W/2); symbols outside [0, N) are NaN, whose
    // distance fmaxf(NaN, 0) turns into 0: they contribute nothing to any window
    const float qnan = __int_as_float(0x7fc00000);
    for (int t = tid; t < NSTRIP * span; t += BPS_THREADS) {
        const int st = t / span, u = t - st * span;
        const int64_t i = ((int64_t)blockIdx.x * NSTRIP + st) * LEN - W / 2 + u;
        const float2 v = (i >= 0 && i < N) ? yq[i] : make_float2(qnan, qnan);
        ys[st * span + u] = make_float4(v.x, v.y, v.y, -v.x);
    }
    __syncthreads();
    // a CTA whose staged spans hold no symbol outside the frame needs no NaN guard: its distances are
    // sums of squares, and the guard is left out of its loop
    const bool edge = (int64_t)blockIdx.x * NSTRIP * LEN < W / 2 ||
                      ((int64_t)blockIdx.x + 1) * NSTRIP * LEN + W / 2 > N;

    // rotation by e^{-j theta_b} folded with 1/(2a); phases b >= B never win (penalty)
    float sn, cs;
    sincospif((float)(2 * b - B) / (float)(4 * B), &sn, &cs);   // theta_b / pi = (b/B - 1/2) / 2
    const float2 cc = make_float2(cs * cI0, cs * cI0), ss = make_float2(sn * cI0, sn * cI0);
    const float2 hh = make_float2(hL, hL), ll = make_float2(Lm1, Lm1);
    const float pen = b < B ? 0.0f : 3.0e38f;
    const int nc = LEN / W;
    unsigned int* myslots = &slots[sl][wip][0];

    if (edge)
        bps_strip<W, GS, true>(yl, cc, ss, hh, invLm1, ll, pen, nc, LEN, s0, N, slots[sl], myslots, b, lane, q, bstar,
                               bstride);
    else
        bps_strip<W, GS, false>(yl, cc, ss, hh, invLm1, ll, pen, nc, LEN, s0, N, slots[sl], myslots, b, lane, q, bstar,
                                bstride);
}

// ---------------------------------------------------------------------------
// Phase pairs: one warp per strip, lane l holding test phases l and l + 32 (B > 32). The rotation,
// rounding and error of a dimension are packed over the two phases, as are the distance and the
// window sums, so that every component is the same FMA or add as the scalar form above and the
// results are bit-identical to it; the minimum over the 64 keys is one in-lane min and one warp
// reduction, and the strip needs no block barrier.
// ---------------------------------------------------------------------------
// W = 64: half of the ring (32 pairs) in registers and half in shared memory, so that 166 registers
// give six CTAs of two warps per SM (12 warps). On a 2^20-symbol frame in the chain this takes 0.133 ms
// against 0.138 ms for the one-phase-per-thread form; the whole ring in registers (8 warps per SM), the
// first window folded into the chunk loop, and a rolled loop over a ring wholly in shared memory were
// each slower.
constexpr int BPS2_STRIPS = 2;                        // strips (warps) per CTA
constexpr int BPS2_MINB = 6;                          // CTAs per SM the registers are sized for
constexpr int BPS2_WR64 = 32;                         // W = 64: ring entries in registers

__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

struct Bps2Phase {
    float2 c, s, ns;                                  // cos, sin, -sin of the two phases, times 1/(2a)
    float2 hh, ll;                                    // (L-1)/2, L-1
    float invLm1;
    float2 pen;                                       // 0, or a penalty for phases >= B
};

// distances of one symbol, staged as (x, x, y, y), to the nearest point after the two rotations:
// per phase vI = fma(x, c, fma(y, s, hL)), vQ = fma(y, c, fma(x, -s, hL)) and
// d = fma(eI, eI, eQ * eQ), the operations of bps_dist
__device__ __forceinline__ float2 bps_dist2(float4 v, const Bps2Phase& p) {
    const float2 MAGIC = make_float2(12582912.0f, 12582912.0f);
    const float2 NMAGIC = make_float2(-12582912.0f, -12582912.0f);
    const float2 NONE = make_float2(-1.0f, -1.0f);
    const float2 xx = make_float2(v.x, v.y), yy = make_float2(v.z, v.w);
    const float2 rI = __ffma2_rn(xx, p.c, __ffma2_rn(yy, p.s, p.hh));
    const float2 rQ = __ffma2_rn(yy, p.c, __ffma2_rn(xx, p.ns, p.hh));
    const float2 wI = make_float2(__saturatef(rI.x * p.invLm1), __saturatef(rI.y * p.invLm1));
    const float2 wQ = make_float2(__saturatef(rQ.x * p.invLm1), __saturatef(rQ.y * p.invLm1));
    const float2 tI = __fadd2_rn(__ffma2_rn(wI, p.ll, MAGIC), NMAGIC);
    const float2 tQ = __fadd2_rn(__ffma2_rn(wQ, p.ll, MAGIC), NMAGIC);
    const float2 eI = __ffma2_rn(tI, NONE, rI), eQ = __ffma2_rn(tQ, NONE, rQ);
    return __ffma2_rn(eI, eI, __fmul2_rn(eQ, eQ));
}

// the least key of the warp's 64 (phase l: D.x, phase l + 32: D.y), as bps_publish
__device__ __forceinline__ void bps_publish2(float2 D, unsigned int* slot, int lane) {
    const unsigned int klo = (__float_as_uint(D.x) & ~63u) | (unsigned)lane;
    const unsigned int khi = (__float_as_uint(D.y) & ~63u) | (unsigned)(lane + 32);
    const unsigned int mn = __reduce_min_sync(0xffffffffu, min(klo, khi));
    if (lane == 0) *slot = mn;
}

// the NaN guard of the CTAs whose spans reach past the frame (as in bps_strip)
template <bool EDGE>
__device__ __forceinline__ float2 guard2(float2 d) {
    return EDGE ? make_float2(fmaxf(d.x, 0.0f), fmaxf(d.y, 0.0f)) : d;
}

// the windows of one strip: the ring of W distance pairs (the first WR in registers, indices fixed
// at compile time, the rest in this lane's column of rs), the sliding sums, and the sum of the
// current chunk, which equals the re-formed window sum of bps_strip (the same terms in the same
// order) at the chunk's end
template <int W, int WR, bool EDGE>
__device__ __forceinline__ void bps2_strip(const float4* __restrict__ yl, const Bps2Phase& p, int nc, int LEN,
                                           int64_t s0, int64_t N, unsigned int* slots, float2* rs, int lane,
                                           uint8_t* __restrict__ bq) {
    float2 ring[WR > 0 ? WR : 1];
    float2* rl = rs + lane;                           // entry u >= WR at rl[(u - WR) * 32]
    float2 D = p.pen;
#pragma unroll
    for (int u = 0; u < W; ++u) {
        const float2 d = guard2<EDGE>(bps_dist2(yl[u], p));
        if (u < WR) ring[u < WR ? u : 0] = d;
        else rl[(u - WR) * 32] = d;
        D = __fadd2_rn(D, d);
    }
    bps_publish2(D, &slots[0], lane);
    for (int ch = 0; ch <= nc; ++ch) {
        if (ch > 0) {
            const float4* yc = yl + ch * W;
            float2 C = p.pen;
#pragma unroll
            for (int u = 0; u < W; ++u) {
                const float2 d = guard2<EDGE>(bps_dist2(yc[u], p));
                const float2 old = u < WR ? ring[u < WR ? u : 0] : rl[(u - WR) * 32];
                D = sub2_rn(__fadd2_rn(D, d), old);
                if (u < WR) ring[u < WR ? u : 0] = d;
                else rl[(u - WR) * 32] = d;
                C = __fadd2_rn(C, d);
                bps_publish2(guard2<EDGE>(D), &slots[(u + 1) & (W - 1)], lane);
            }
            D = C;
        }
        __syncwarp();
        for (int slot = lane; slot < W; slot += 32) {
            const int kl = slot == 0 ? ch * W : (ch - 1) * W + slot;
            if (kl >= 0 && kl < LEN && s0 + kl < N) bq[s0 + kl] = (uint8_t)(slots[slot] & 63u);
        }
        __syncwarp();
    }
}

// distance pairs of the ring kept in registers (the rest in shared memory)
template <int W>
__host__ __device__ constexpr int bps2_wr() {
    return W <= 32 ? W : BPS2_WR64;
}

template <int W>
__global__ void __launch_bounds__(32 * BPS2_STRIPS, BPS2_MINB) k_bps2(const float2* __restrict__ y, int64_t ystride,
                                                                      int64_t N, int B, float cI0, float hL,
                                                                      float invLm1, float Lm1, int LEN,
                                                                      uint8_t* __restrict__ bstar, int64_t bstride) {
    constexpr int WR = bps2_wr<W>();
    pdl_trigger();                                    // the unwrap may become resident now
    pdl_wait();                                       // launched programmatically: y is complete after this
    extern __shared__ float4 smem_v[];
    const int span = LEN + W;
    float4* ys = smem_v;                              // [BPS2_STRIPS][LEN + W]: (x, x, y, y)
    float2* rs = reinterpret_cast<float2*>(ys + BPS2_STRIPS * span);   // [BPS2_STRIPS][W - WR][32]
    __shared__ unsigned int slots[BPS2_STRIPS][W];
    const int tid = threadIdx.x, sl = tid >> 5, lane = tid & 31;
    const int q = blockIdx.y;
    const int64_t s0 = ((int64_t)blockIdx.x * BPS2_STRIPS + sl) * LEN;
    const float2* yq = y + (int64_t)q * ystride;

    const float qnan = __int_as_float(0x7fc00000);
    for (int t = tid; t < BPS2_STRIPS * span; t += 32 * BPS2_STRIPS) {
        const int st = t / span, u = t - st * span;
        const int64_t i = ((int64_t)blockIdx.x * BPS2_STRIPS + st) * LEN - W / 2 + u;
        const float2 v = (i >= 0 && i < N) ? yq[i] : make_float2(qnan, qnan);
        ys[st * span + u] = make_float4(v.x, v.x, v.y, v.y);
    }
    __syncthreads();
    const bool edge = (int64_t)blockIdx.x * BPS2_STRIPS * LEN < W / 2 ||
                      ((int64_t)blockIdx.x + 1) * BPS2_STRIPS * LEN + W / 2 > N;

    Bps2Phase p;
    float s1, c1, s2, c2;
    sincospif((float)(2 * lane - B) / (float)(4 * B), &s1, &c1);
    sincospif((float)(2 * (lane + 32) - B) / (float)(4 * B), &s2, &c2);
    p.c = make_float2(c1 * cI0, c2 * cI0);
    p.s = make_float2(s1 * cI0, s2 * cI0);
    p.ns = make_float2(-p.s.x, -p.s.y);
    p.hh = make_float2(hL, hL);
    p.ll = make_float2(Lm1, Lm1);
    p.invLm1 = invLm1;
    p.pen = make_float2(lane < B ? 0.0f : 3.0e38f, lane + 32 < B ? 0.0f : 3.0e38f);
    const int nc = LEN / W;
    const float4* yl = ys + sl * span;
    float2* rsw = rs + sl * (W - WR) * 32;
    uint8_t* bq = bstar + (int64_t)q * bstride;
    if (edge)
        bps2_strip<W, WR, true>(yl, p, nc, LEN, s0, N, slots[sl], rsw, lane, bq);
    else
        bps2_strip<W, WR, false>(yl, p, nc, LEN, s0, N, slots[sl], rsw, lane, bq);
}

// dynamic shared memory of k_bps2<W> for strips of LEN symbols
template <int W>
size_t bps2_smem(int LEN) {
    return sizeof(float4) * BPS2_STRIPS * (LEN + W) + sizeof(float2) * BPS2_STRIPS * (W - bps2_wr<W>()) * 32;
}

template <int W, int GS>
cudaError_t bps_t(const float2* y, int64_t ystride, int64_t N, int B, int m, uint8_t* bstar, int64_t bstride,
                  cudaStream_t s) {
    const Qam qm = make_qam(m);
    constexpr int NSTRIP = BPS_THREADS / GS;
    // symbols per strip, a multiple of W: the least of (waves of CTAs) x (LEN + W), the time model of a
    // launch whose CTAs each take LEN + W symbols' work, over 4 W .. 16 W (ties to the shorter strip)
    static int slots = 0;
    if (!slots) {
        int dev = 0, nsm = 152, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bps<W, GS>, BPS_THREADS,
                                                      sizeof(float4) * NSTRIP * (8 * W + W));
        slots = std::max(1, nsm * std::max(1, per));
    }
    int LEN = 8 * W;
    int64_t best = -1;
    for (int len = 4 * W; len <= 16 * W && len <= 1024; len += W) {
        const int64_t ctas = 2 * (((N + len - 1) / len + NSTRIP - 1) / NSTRIP);
        const int64_t cost = ((ctas + slots - 1) / slots) * (len + W);
        if (best < 0 || cost < best) { best = cost; LEN = len; }
    }
    const int64_t nstrip = (N + LEN - 1) / LEN;
    dim3 grid((unsigned)((nstrip + NSTRIP - 1) / NSTRIP), 2);
    const size_t smem = sizeof(float4) * NSTRIP * (LEN + W);
    // opt in once for the largest strip (1024 symbols): the static slots come on top of the dynamic
    // part, so no size near the 48 KB default is left to chance
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_bps<W, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float4) * NSTRIP * (1024 + W)));
        attr = true;
    }
    const float Lm1 = (float)(qm.L - 1);
    return launch_pdl(k_bps<W, GS>, grid, dim3(BPS_THREADS), smem, s, y, ystride, N, B, qm.half_inv_a, qm.hL,
                      1.0f / Lm1, Lm1, LEN, bstar, bstride);
}

template <int W>
cudaError_t bps2_t(const float2* y, int64_t ystride, int64_t N, int B, int m, uint8_t* bstar, int64_t bstride,
                   cudaStream_t s) {
    const Qam qm = make_qam(m);
    // strip length: the wave model of bps_t
    static int slots = 0;
    if (!slots) {
        int dev = 0, nsm = 152, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bps2<W>, 32 * BPS2_STRIPS, bps2_smem<W>(8 * W));
        slots = std::max(1, nsm * std::max(1, per));
    }
    int LEN = 8 * W;
    int64_t best = -1;
    for (int len = 4 * W; len <= 16 * W && len <= 1024; len += W) {
        const int64_t ctas = 2 * (((N + len - 1) / len + BPS2_STRIPS - 1) / BPS2_STRIPS);
        const int64_t cost = ((ctas + slots - 1) / slots) * (len + W);
        if (best < 0 || cost < best) { best = cost; LEN = len; }
    }
    const int64_t nstrip = (N + LEN - 1) / LEN;
    dim3 grid((unsigned)((nstrip + BPS2_STRIPS - 1) / BPS2_STRIPS), 2);
    const size_t smem = bps2_smem<W>(LEN);
    static bool attr = false;                         // as in bps_t
    if (!attr) {
        cudaFuncSetAttribute(k_bps2<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bps2_smem<W>(1024));
        attr = true;
    }
    const float Lm1 = (float)(qm.L - 1);
    return launch_pdl(k_bps2<W>, grid, dim3(32 * BPS2_STRIPS), smem, s, y, ystride, N, B, qm.half_inv_a, qm.hL,
                      1.0f / Lm1, Lm1, LEN, bstar, bstride);
}

template <int W>
cudaError_t bps_w(const float2* y, int64_t ystride, int64_t N, int B, int m, uint8_t* bstar, int64_t bstride,
                  cudaStream_t s) {
    if (B <= 32) return bps_t<W, 32>(y, ystride, N, B, m, bstar, bstride, s);
    return bps2_t<W>(y, ystride, N, B, m, bstar, bstride, s);
}

// ---------------------------------------------------------------------------
// unwrap: m_k = m_{k-1} + J(b*_{k-1} - b*_k), J(d) = +1 (d > B/2), -1 (d < -B/2), 0
// ---------------------------------------------------------------------------
constexpr int UT = 1024;          // symbols per tile
constexpr int UTHR = 256;         // 4 symbols per thread

__device__ __forceinline__ int jump(int prev, int cur, int B) {
    const int d = prev - cur;
    return (2 * d > B) ? 1 : ((2 * d < -B) ? -1 : 0);
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* red, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += n;
    }
    if (lane == 31) red[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += n;
        }
        red[lane] = t;
    }
    __syncthreads();
    const int before = (w > 0 ? red[w - 1] : 0) + x - v;
    if (total) *total = red[(blockDim.x >> 5) - 1];
    return before;
}

// the 4 b* of symbols k0 .. k0 + 3 (zero past N) and the b* before k0 (the carried one at k0 = 0);
// one 32-bit load when the row is 4-byte aligned and the group is whole
__device__ __forceinline__ void load_b4(const uint8_t* bq, int64_t k0, int64_t N, int bprev_carry, bool vec,
                                        int bs[4], int& prev) {
    if (vec && k0 + 3 < N) {
        const uchar4 v = *reinterpret_cast<const uchar4*>(bq + k0);
        bs[0] = v.x; bs[1] = v.y; bs[2] = v.z; bs[3] = v.w;
    } else {
        for (int u = 0; u < 4; ++u) bs[u] = k0 + u < N ? bq[k0 + u] : 0;
    }
    if (k0 > 0) prev = bq[k0 - 1];
    else prev = bprev_carry >= 0 ? bprev_carry : bs[0];
}

// Pass 1: the jump sum of every tile; the first tile also copies the carried (b*, m) of its
// polarisation after the sums (snap[q] = {b_prev, m_prev}), where pass 2 reads it while its last
// tile writes the new carry.
__global__ void k_unwrap_sums(const uint8_t* __restrict__ bstar, int64_t bstride, int64_t N, int B,
                              const RxDevState* st, int* tile_sums, int ntiles, int vec) {
    pdl_trigger();
    pdl_wait();                                       // launched programmatically: b* is complete after this
    __shared__ int red[32];
    const int q = blockIdx.y;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        tile_sums[2 * ntiles + 2 * q] = st->b_prev[q];
        tile_sums[2 * ntiles + 2 * q + 1] = st->m_prev[q];
    }
    const uint8_t* bq = bstar + (int64_t)q * bstride;
    const int64_t k0 = (int64_t)blockIdx.x * UT + threadIdx.x * 4;
    int sum = 0;
    if (k0 < N) {
        int bs[4], prev;
        load_b4(bq, k0, N, st->b_prev[q], vec != 0, bs, prev);
        for (int u = 0; u < 4; ++u) {
            if (k0 + u < N) sum += jump(prev, bs[u], B);
            prev = bs[u];
        }
    }
    int total;
    block_exclusive_scan(sum, red, &total);
    if (threadIdx.x == 0) tile_sums[q * ntiles + blockIdx.x] = total;
}

// Pass 2: the tile's base count (the carried m plus the sums of the tiles before it, integers in
// any order), the scan within the tile, the derotation; the thread holding symbol N - 1 writes the
// carry for the next frame.
__global__ void k_unwrap_apply(const float2* __restrict__ y, int64_t ystride, const uint8_t* __restrict__ bstar,
                               int64_t bstride, int64_t N, int B, const int* tile_sums, int ntiles,
                               RxDevState* st, int* m_out, int64_t mstride, float2* z, int64_t zstride,
                               int vec) {
    pdl_trigger();
    pdl_wait();                                       // launched programmatically: the tile sums are complete
    __shared__ int red[32];
    __shared__ int s_base[UTHR / 32];
    __shared__ float2 rot[RX_BPS_MAXB];
    const int q = blockIdx.y;
    if (threadIdx.x < B) {
        float s, c;
        sincospif(-((float)threadIdx.x / (float)B - 0.5f) * 0.5f, &s, &c);   // e^{-j theta_b}
        rot[threadIdx.x] = make_float2(c, s);
    }
    const int* snap = tile_sums + 2 * ntiles + 2 * q;
    int before = 0;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += blockDim.x) before += tile_sums[q * ntiles + i];
    before = __reduce_add_sync(0xffffffffu, before);
    if ((threadIdx.x & 31) == 0) s_base[threadIdx.x >> 5] = before;
    const uint8_t* bq = bstar + (int64_t)q * bstride;
    const int64_t k0 = (int64_t)blockIdx.x * UT + threadIdx.x * 4;
    int J[4] = {0, 0, 0, 0}, bs[4] = {0, 0, 0, 0};
    int sum = 0;
    if (k0 < N) {
        int prev;
        load_b4(bq, k0, N, snap[0], vec != 0, bs, prev);
        for (int u = 0; u < 4; ++u) {
            if (k0 + u < N) J[u] = jump(prev, bs[u], B);
            prev = bs[u];
            sum += J[u];
        }
    }
    int m = block_exclusive_scan(sum, red, nullptr);  // its barriers also publish s_base
    int base = snap[1];
    for (int w = 0; w < UTHR / 32; ++w) base += s_base[w];
    m += base;
    __syncthreads();
    if (k0 >= N) return;
    const float2* yq = y + (int64_t)q * ystride + k0;
    float2* zq = z + (int64_t)q * zstride + k0;
    int* mq = m_out + (int64_t)q * mstride + k0;
    const bool whole = vec && k0 + 3 < N;
    float2 v[4];
    if (whole) {
        const float4 a = *reinterpret_cast<const float4*>(yq);
        const float4 b = *reinterpret_cast<const float4*>(yq + 2);
        v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
        v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
    } else {
        for (int u = 0; u < 4; ++u) v[u] = k0 + u < N ? yq[u] : make_float2(0.0f, 0.0f);
    }
    int mm[4];
    for (int u = 0; u < 4; ++u) {
        m += J[u];
        mm[u] = m;
        float2 w = cmul(v[u], rot[bs[u]]);
        switch (m & 3) {                              // (-j)^(m mod 4)
            case 1: w = make_float2(w.y, -w.x); break;
            case 2: w = make_float2(-w.x, -w.y); break;
            case 3: w = make_float2(-w.y, w.x); break;
            default: break;
        }
        v[u] = w;
    }
    if (N - 1 - k0 < 4) {                             // the frame's last symbol: the next frame's carry
        const int u = (int)(N - 1 - k0);
        st->b_prev[q] = bs[u];
        st->m_prev[q] = mm[u];
    }
    if (whole) {
        *reinterpret_cast<int4*>(mq) = make_int4(mm[0], mm[1], mm[2], mm[3]);
        *reinterpret_cast<float4*>(zq) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        *reinterpret_cast<float4*>(zq + 2) = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    } else {
        for (int u = 0; u < 4; ++u)
            if (k0 + u < N) {
                mq[u] = mm[u];
                zq[u] = v[u];
            }
    }
}

}  // namespace

cudaError_t launch_bps(const float2* y, int64_t ystride, int64_t N, int B, int W, int m, uint8_t* bstar,
                       int64_t bstride, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    switch (W) {
        case 2: return bps_w<2>(y, ystride, N, B, m, bstar, bstride, s);
        case 4: return bps_w<4>(y, ystride, N, B, m, bstar, bstride, s);
        case 8: return bps_w<8>(y, ystride, N, B, m, bstar, bstride, s);
        case 16: return bps_w<16>(y, ystride, N, B, m, bstar, bstride, s);
        case 32: return bps_w<32>(y, ystride, N, B, m, bstar, bstride, s);
        case 64: return bps_w<64>(y, ystride, N, B, m, bstar, bstride, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_unwrap(const float2* y, int64_t ystride, const uint8_t* bstar, int64_t bstride, int64_t N, int B,
                          int* tile_sums, int* m_out, int64_t mstride, float2* z, int64_t zstride, RxDevState* st,
                          cudaStream_t s, int* nlaunch) {
    if (N <= 0) return cudaSuccess;
    const int ntiles = (int)((N + UT - 1) / UT);
    // 4-symbol vector accesses when every row is aligned for them
    auto al = [](const void* p, int64_t stride_bytes, int a) {
        return ((uintptr_t)p % a) == 0 && (stride_bytes % a) == 0;
    };
    const int vec = al(bstar, bstride, 4) && al(y, ystride * 8, 16) && al(z, zstride * 8, 16) &&
                    al(m_out, mstride * 4, 16);
    cudaError_t e = launch_pdl(k_unwrap_sums, dim3(ntiles, 2), dim3(UTHR), 0, s, bstar, bstride, N, B,
                               (const RxDevState*)st, tile_sums, ntiles, vec);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_unwrap_apply, dim3(ntiles, 2), dim3(UTHR), 0, s, y, ystride, bstar, bstride, N, B,
                   (const int*)tile_sums, ntiles, st, m_out, mstride, z, zstride, vec);
    if (nlaunch) *nlaunch += 2;
    return e;
}
