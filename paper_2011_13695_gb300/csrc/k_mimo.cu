// A2 CMA / DD acquisition, A3 frequency-offset estimate, A4 segmented DD-LMS.
//
// The paper's adaptive equaliser (Sec. IV-D) is a serial 4-tap TD DD-LMS in
// one kernel that exchanges data with warp shuffles and decides/demaps as it
// goes. Here the equaliser is the 2x2 butterfly FIR at 2 samples/symbol with
// block updates:
//   y_q[n] = sum_p sum_k h_qp[k] x_p[2n + c - k],   c = (T-1)/2
//   h_qp[k] += mu * sum_{n in block} e_q[n] conj(x_p[2n + c - k])
// with e = y (R2 - |y|^2) (CMA, Godard) or e = dec(y e^{-j psi}) e^{j psi} - y
// (DD, psi = arg(-sum y^4)/4 per block). The two output rows q are
// independent recursions (each has its own taps, error and phase), so one CTA
// runs one row of one segment: grid (segments, 2). The serial recursion along
// a row is broken by a fixed segment schedule: segments of seg_blocks blocks,
// started from common taps and warmed up on the warmup_blocks blocks before.
// Per block a CTA stages the block's input window (both polarisations, FO
// derotation by the 64-bit phase accumulator fused into the load, the next
// window prefetched into registers while the current one is used) in shared
// memory, computes the outputs (P lanes per output, xor-shuffle combine), the
// block phase (fixed-order reduction, so results do not depend on
// scheduling), the errors and the tap gradients (fixed-order partial sums),
// then updates the row's taps in shared memory. All per-thread index
// arithmetic is done once per kernel.
//
// The widely-linear form (WL = true; the paper's equaliser is widely linear,
// Sec. IV-D) adds conjugate taps g_qp: y_q[n] += sum_p sum_k g_qp[k]
// conj(x_p[2n + c - k]) and g_qp[k] += mu_c * sum_n e_q[n] x_p[2n + c - k].
// A row's taps are then [h_q0, h_q1, g_q0, g_q1] (4T); the flattened term
// index u = v 2T + p T + k (v = 1: conjugate) carries the same lane split.
#include <cooperative_groups.h>

#include "rx_fft.cuh"
#include "rx_kernels.h"

namespace {

template <int NT>
struct LmsCtx {
    static constexpr int PF = (2 * (2 * 256 + RX_TMAX) + NT - 1) / NT;   // prefetch registers per thread
    float2* taps;    // row q: [p][k], 2T
    float2* xs0;     // staging double buffer, each [2][XS]
    float2* xs1;
    float2* ys;      // [Lb]
    float2* es;      // [Lb]
    float2* part;    // [G][2T]
    float2* rot;     // e^{-j psi}
    float2* tab;     // NCO derotation of window offset jj: exp(-j 2 pi frac(inc jj)), jj < 2 Lb + T - 1
    int XS, G, logP, logR;
    // output lanes: polarisation-0 taps [ka0, ka1), polarisation-1 taps [kb0, kb1); widely linear:
    // conjugate taps of polarisation 0 [kc0, kc1) and of polarisation 1 [kd0, kd1)
    int ka0, ka1, kb0, kb1, kc0, kc1, kd0, kd1;
    // gradient thread: tap index (-1: idle), group, staging offset of its tap, conjugate tap
    int gt, gg, gx, gconj;
    float2 pf[PF];
};

// Window of the block starting at symbol n0 with L symbols: buffer indices
// i = off + 2 n0 - c + j, j < 2L + T - 1 (zero outside [0, xlen)).
template <int NT>
__device__ __forceinline__ void lms_prefetch(const LmsArgs& a, LmsCtx<NT>& s, int64_t n0, int L) {
    const int c = (a.T - 1) >> 1;
    const int XW = 2 * L + a.T - 1;
    const int64_t i0 = a.off + 2 * n0 - c;
#pragma unroll
    for (int r = 0; r < LmsCtx<NT>::PF; ++r) {
        const int t = threadIdx.x + r * NT;
        float2 v = make_float2(0.0f, 0.0f);
        if (t < 2 * XW) {
            const int p = t >= XW ? 1 : 0, jj = t - p * XW;
            const int64_t i = i0 + jj;
            if (i >= 0 && i < a.xlen && p < a.npol) v = a.x[(int64_t)p * a.xstride + i];
        }
        s.pf[r] = v;
    }
}

template <int NT>
__device__ __forceinline__ void lms_commit(const LmsArgs& a, LmsCtx<NT>& s, float2* xs, int64_t n0, int L,
                                           long long inc) {
    const int c = (a.T - 1) >> 1;
    const int XW = 2 * L + a.T - 1;
    const long long g0 = a.g0 + a.off + 2 * n0 - c;
    // exp(-j 2 pi frac(inc (g0 + jj))) = exp(-j 2 pi frac(inc g0)) exp(-j 2 pi frac(inc jj)) (mod one turn)
    const float2 base = inc ? nco_conj(inc, g0) : make_float2(1.0f, 0.0f);
#pragma unroll
    for (int r = 0; r < LmsCtx<NT>::PF; ++r) {
        const int t = threadIdx.x + r * NT;
        if (t < 2 * XW) {
            const int p = t >= XW ? 1 : 0, jj = t - p * XW;
            float2 v = s.pf[r];
            if (inc) v = cmul(v, cmul(base, s.tab[jj]));
            xs[p * s.XS + jj] = v;
        }
    }
}

// one block of row q: outputs, (DD) phase and errors, gradient, tap update
template <int NT, bool WL>
__device__ __forceinline__ void lms_block(const LmsArgs& a, LmsCtx<NT>& s, const float2* __restrict__ xs,
                                          int64_t n0, int L, bool store, const Qam& qm, int q) {
    const int tid = threadIdx.x;
    const int T = a.T;
    const int NTAP = (WL ? 4 : 2) * T;
    const int P = 1 << s.logP;
    {
        const int ostep = NT >> s.logP;
        const float2* h0 = s.taps;
        const float2* h1 = s.taps + T;
        for (int ob = (tid >> 5) << (5 - s.logP); ob < L; ob += ostep) {
            const int n = ob + ((tid & 31) >> s.logP);
            const bool valid = n < L;
            const int nn = valid ? n : 0;
            const float2* x0 = xs + 2 * nn + T - 1;
            const float2* x1 = x0 + s.XS;
            float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
            const int a1 = valid ? s.ka1 : s.ka0, b1 = valid ? s.kb1 : s.kb0;
            int k = s.ka0;
            for (; k + 1 < a1; k += 2) {
                acc0 = cmac(acc0, h0[k], x0[-k]);
                acc1 = cmac(acc1, h0[k + 1], x0[-k - 1]);
            }
            if (k < a1) acc0 = cmac(acc0, h0[k], x0[-k]);
            k = s.kb0;
            for (; k + 1 < b1; k += 2) {
                acc0 = cmac(acc0, h1[k], x1[-k]);
                acc1 = cmac(acc1, h1[k + 1], x1[-k - 1]);
            }
            if (k < b1) acc0 = cmac(acc0, h1[k], x1[-k]);
            if constexpr (WL) {
                const float2* g0 = s.taps + 2 * T;
                const float2* g1 = s.taps + 3 * T;
                const int c1 = valid ? s.kc1 : s.kc0, d1 = valid ? s.kd1 : s.kd0;
                k = s.kc0;
                for (; k + 1 < c1; k += 2) {
                    acc0 = cmacc(acc0, g0[k], x0[-k]);
                    acc1 = cmacc(acc1, g0[k + 1], x0[-k - 1]);
                }
                if (k < c1) acc0 = cmacc(acc0, g0[k], x0[-k]);
                k = s.kd0;
                for (; k + 1 < d1; k += 2) {
                    acc0 = cmacc(acc0, g1[k], x1[-k]);
                    acc1 = cmacc(acc1, g1[k + 1], x1[-k - 1]);
                }
                if (k < d1) acc0 = cmacc(acc0, g1[k], x1[-k]);
            }
            float2 acc = cadd(acc0, acc1);
            for (int w = 1; w < P; w <<= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, w);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, w);
            }
            if (valid && (tid & (P - 1)) == 0) {
                s.ys[n] = acc;
                if (a.cma) s.es[n] = cscale(acc, a.R2 - cabs2(acc));
                if (store) a.y[(int64_t)q * a.ystride + n0 + n] = acc;
            }
        }
    }
    __syncthreads();
    if (!a.cma) {
        if (tid < 32) {
            float2 acc = make_float2(0.0f, 0.0f);
            for (int n = tid; n < L; n += 32) {
                const float2 y = s.ys[n];
                const float2 y2 = cmul(y, y);
                acc = cadd(acc, cmul(y2, y2));
            }
            acc.x = warp_sum(acc.x);
            acc.y = warp_sum(acc.y);
            if (tid == 0) s.rot[0] = quarter_root_conj(make_float2(-acc.x, -acc.y));
        }
        __syncthreads();
        const float2 r = s.rot[0];
        for (int o = tid; o < L; o += NT) {
            const float2 y = s.ys[o];
            const float2 d = qam_decide(cmul(y, r), qm);
            s.es[o] = csub(cmulc(d, r), y);
        }
        __syncthreads();
    }
    if (s.gt >= 0) {
        const float2* xp = xs + s.gx;
        float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
        const int G = s.G;
        int n = s.gg;
        if (WL && s.gconj) {
            // conjugate tap: e x
            for (; n + G < L; n += 2 * G) {
                acc0 = cmac(acc0, s.es[n], xp[2 * n]);
                acc1 = cmac(acc1, s.es[n + G], xp[2 * (n + G)]);
            }
            if (n < L) acc0 = cmac(acc0, s.es[n], xp[2 * n]);
        } else {
            for (; n + G < L; n += 2 * G) {
                acc0 = cmacc(acc0, s.es[n], xp[2 * n]);
                acc1 = cmacc(acc1, s.es[n + G], xp[2 * (n + G)]);
            }
            if (n < L) acc0 = cmacc(acc0, s.es[n], xp[2 * n]);
        }
        s.part[s.gg * NTAP + s.gt] = cadd(acc0, acc1);
    }
    __syncthreads();
    {
        // R lanes per tap add every R-th group partial, then combine with xor-shuffles
        const int logR = s.logR, R = 1 << logR;
        const int t = tid >> logR, r = tid & (R - 1);
        float2 acc = make_float2(0.0f, 0.0f);
        if (t < NTAP) {
            for (int g = r; g < s.G; g += R) acc = cadd(acc, s.part[g * NTAP + t]);
        }
        for (int w = 1; w < R; w <<= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, w);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, w);
        }
        if (t < NTAP && r == 0) {
            const float mu = (WL && t >= 2 * T) ? a.mu_c : a.mu;
            s.taps[t] = make_float2(fmaf(mu, acc.x, s.taps[t].x), fmaf(mu, acc.y, s.taps[t].y));
        }
    }
}

template <int NT, bool WL>
__global__ void __launch_bounds__(NT) k_lms(LmsArgs a) {
    extern __shared__ float2 smem[];
    if (a.run_if && *a.run_if == 0) return;
    const int T = a.T, Lb = a.Lb;
    const int NTAP = (WL ? 4 : 2) * T;   // taps of one row
    const int q = blockIdx.y;
    const int tid = threadIdx.x;
    LmsCtx<NT> s;
    s.XS = 2 * Lb + T;
    s.G = max(1, NT / NTAP);
    int logP = 0;
    while (logP < 4 && ((Lb << (logP + 1)) <= NT)) ++logP;
    s.logP = logP;
    int logR = 0;
    while (logR < 3 && (1 << (logR + 1)) <= s.G && (NTAP << (logR + 1)) <= NT) ++logR;
    s.logR = logR;
    s.taps = smem;
    s.xs0 = s.taps + NTAP;
    s.xs1 = s.xs0 + 2 * s.XS;
    s.ys = s.xs1 + 2 * s.XS;
    s.es = s.ys + Lb;
    s.part = s.es + Lb;
    s.rot = s.part + s.G * NTAP;
    s.tab = s.rot + 1;
    {
        // output lane j of a group takes the flattened terms u in [j cs, (j + 1) cs),
        // u = v 2T + p T + k (v = 1: conjugate taps, widely linear only)
        const int P = 1 << logP, j = tid & (P - 1);
        const int cs = (NTAP + P - 1) >> logP;
        const int u0 = min(NTAP, j * cs), u1 = min(NTAP, u0 + cs);
        s.ka0 = min(u0, T);
        s.ka1 = min(u1, T);
        s.kb0 = min(max(u0, T), 2 * T) - T;
        s.kb1 = min(max(u1, T), 2 * T) - T;
        s.kc0 = min(max(u0, 2 * T), 3 * T) - 2 * T;
        s.kc1 = min(max(u1, 2 * T), 3 * T) - 2 * T;
        s.kd0 = max(u0, 3 * T) - 3 * T;
        s.kd1 = max(u1, 3 * T) - 3 * T;
        const int g = tid / NTAP, t = tid - g * NTAP;
        s.gt = g < s.G ? t : -1;
        s.gg = g;
        const int v = t >= 2 * T ? 1 : 0, t2 = t - v * 2 * T;
        const int p = t2 >= T ? 1 : 0, k = t2 - p * T;
        s.gx = p * s.XS + T - 1 - k;
        s.gconj = v;
    }
    const Qam qm = make_qam(a.m);

    const int64_t seg = blockIdx.x;
    const int64_t nseg = gridDim.x;
    const long long inc = a.derotate ? a.st->nco_inc : 0;
    for (int t = tid; t < NTAP; t += NT) s.taps[t] = a.taps_in[q * NTAP + t];
    if (inc)
        for (int jj = tid; jj < 2 * Lb + T - 1; jj += NT) s.tab[jj] = nco_conj(inc, jj);
    __syncthreads();
    const int64_t start = seg * a.L_seg;
    const int64_t end = min(a.n_sym, start + a.L_seg);
    const int nwarm = seg > 0 ? a.n_wu : 0;
    const int nmain = (int)((end - start + Lb - 1) / Lb);
    const int nblk = nwarm + nmain;
    auto blk_n0 = [&](int b) -> int64_t {
        return b < nwarm ? start - (int64_t)(nwarm - b) * Lb : start + (int64_t)(b - nwarm) * Lb;
    };
    auto blk_L = [&](int b) -> int {
        return b < nwarm ? Lb : (int)min((int64_t)Lb, end - blk_n0(b));
    };
    if (nblk > 0) {
        lms_prefetch(a, s, blk_n0(0), blk_L(0));
        lms_commit(a, s, s.xs0, blk_n0(0), blk_L(0), inc);
    }
    __syncthreads();
    for (int b = 0; b < nblk; ++b) {
        const int64_t n0 = blk_n0(b);
        const int L = blk_L(b);
        if (b + 1 < nblk) lms_prefetch(a, s, blk_n0(b + 1), blk_L(b + 1));
        lms_block<NT, WL>(a, s, (b & 1) ? s.xs1 : s.xs0, n0, L, b >= nwarm && a.y != nullptr, qm, q);
        if (b + 1 < nblk) lms_commit(a, s, (b & 1) ? s.xs0 : s.xs1, blk_n0(b + 1), blk_L(b + 1), inc);
        __syncthreads();
    }
    if (seg == nseg - 1 && a.taps_out) {
        for (int t = tid; t < NTAP; t += NT) a.taps_out[q * NTAP + t] = s.taps[t];
    }
}

// ---------------------------------------------------------------------------
// A3 on the fixed CMA taps, in one launch: a cluster of FOE_CL CTAs, CTA r on output row
// q = r / (FOE_CL / 2) and one contiguous share of the window. Each CTA stages its share's input
// samples in shared memory (every load in flight at once: the latency of this part's L2 is long), writes
// its outputs y to yw and v = y^4 into the shared memory of its row's leader (rank q FOE_CL / 2) through
// distributed shared memory. Each leader transforms its row's v (N points, zero padded; the last pass
// writes P_q[k] = |V_q[k]|^2 into its own and, where room allows, the other leader's shared memory),
// finds the first maximum of P_0 + P_1 (both leaders add in the same order), and forms its row's
// per-block sums sum_n v_n e^{-j 2 pi kappa n / N}, which equal sum_n (y_n e^{-j w_c n})^4 for
// w_c = 2 pi kappa / (4 N); the phasor is an entry of the FFT twiddle table. Leader 1 writes its sums into
// leader 0's shared memory; leader 0 then takes the phases, their unwrap, the least-squares slope, the
// code and the corrected taps. Every CTA arrives at the cluster barrier first thing and waits on it
// before its first access to another CTA's shared memory, then passes the same three cluster barriers;
// after the third no CTA touches another's shared memory, so the others may exit.
constexpr int FOE_CL = 8;            // CTAs per cluster: four per output row
constexpr int FOE_NBMAX = 1024;      // window blocks of the fine stage, at most

template <int K>
struct FoeShape {
    static constexpr int N = 1 << K;
    static constexpr int NTH = N / 16 > 512 ? N / 16 : 512;
    static constexpr int FB = fft_smem_elems(N);                // FFT working copy (float2)
    static constexpr bool TWS = K <= 13;                        // twiddles and the other periodogram in shared memory
    static constexpr int TWN = TWS ? N : 0;                     // entries t = i RX_FFT_TW_N / N, i < N
    static constexpr int PCN = TWS ? N / 2 : 0;                 // the other leader's P (N floats)
    static constexpr size_t SMEM = sizeof(float2) * (FB + N / 2 + 2 * FOE_NBMAX + TWN + PCN);
    // staged samples per thread: 2 (2 ceil(N / 8) + RX_TMAX - 1) at most over NTH threads
    static constexpr int XPER = (2 * (2 * (N / 8 + 1) + RX_TMAX) + NTH - 1) / NTH;
};

template <int K>
__global__ void __cluster_dims__(FOE_CL, 1, 1) __launch_bounds__(FoeShape<K>::NTH, 1) k_foe(FoeArgs a) {
    namespace cg = cooperative_groups;
    using S = FoeShape<K>;
    constexpr int N = S::N, NTH = S::NTH, HALF = FOE_CL / 2;
    constexpr int TWSHIFT = RX_FFT_TW_LOG2 - K;
    extern __shared__ float2 fsm[];
    float2* fbuf = fsm;                               // window samples, then the FFT working copy, then P_q
    float2* vbuf = fsm + S::FB;                       // [N / 2] v of this row (leaders)
    float2* asum = vbuf + N / 2;                      // [2][FOE_NBMAX] per-block sums (leader 0)
    float2* tws = asum + 2 * FOE_NBMAX;               // [N] twiddle entries (leaders, K <= 13)
    float* Pc = reinterpret_cast<float*>(tws + S::TWN);   // [N] the other leader's P (leaders, K <= 13)
    __shared__ float2 s_taps[2 * RX_TMAX];
    __shared__ float bv[32];
    __shared__ int bi[32];
    __shared__ int s_kappa;
    __shared__ float s_wf;
    cg::cluster_group cl = cg::this_cluster();
    cl.barrier_arrive();                              // this CTA has started
    pdl_trigger();                                    // the DD acquisition may become resident now
    const int rank = (int)cl.block_rank();
    const int q = rank / HALF, part = rank % HALF;
    const bool leader = part == 0;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int T = a.T, c = (T - 1) / 2;
    const int64_t nw = a.nw;

    // 0. stage this CTA's input samples (both polarisations, zero outside the buffer), the row's taps
    //    and, in the leaders, the transform's twiddles
    const int64_t chunk = (nw + HALF - 1) / HALF;
    const int64_t i0 = min(nw, part * chunk), i1 = min(nw, i0 + chunk);
    const int span = i1 > i0 ? (int)(2 * (i1 - i0 - 1) + T) : 0;   // samples of the share's outputs
    const int64_t lo = a.off + 2 * (a.n0 + i0) + c - (T - 1);      // buffer index of sample 0 of the span
    {
        float2 xv[S::XPER];
#pragma unroll
        for (int j = 0; j < S::XPER; ++j) {
            const int t = tid + j * NTH;
            const int p = t >= span ? 1 : 0;
            const int64_t g = lo + (t - p * span);
            xv[j] = (t < 2 * span && g >= 0 && g < a.xlen) ? __ldg(a.x + (int64_t)p * a.xstride + g)
                                                            : make_float2(0.0f, 0.0f);
        }
        if (S::TWS && leader) {
            constexpr int TPER = S::TWN / NTH > 0 ? S::TWN / NTH : 1;
            float2 tv[TPER];
#pragma unroll
            for (int j = 0; j < TPER; ++j) {
                const int i = tid + j * NTH;
                tv[j] = i < S::TWN ? __ldg(&a.tw[i << TWSHIFT]) : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int j = 0; j < TPER; ++j)
                if (tid + j * NTH < S::TWN) tws[tid + j * NTH] = tv[j];
        }
#pragma unroll
        for (int j = 0; j < S::XPER; ++j)
            if (tid + j * NTH < 2 * span) fbuf[tid + j * NTH] = xv[j];
    }
    // the samples and twiddles above were complete before the stream's previous kernel (the CMA rerun)
    // started; its taps, and everything else it writes or reads, only after its completion: this launch
    // is programmatic, so its staging overlaps the rerun
    pdl_wait();
    for (int t = tid; t < 2 * T; t += NTH) s_taps[t] = a.taps[q * 2 * T + t];
    __syncthreads();

    // 1. this CTA's share of row q's outputs, two per thread in one pass over the taps
    cl.barrier_wait();                                // every CTA of the cluster has started
    float2* vlead = cl.map_shared_rank(vbuf, q * HALF);
    for (int64_t i = i0 + tid; i < i1; i += 2 * NTH) {
        const bool two = i + NTH < i1;
        const int u0 = 2 * (int)(i - i0) + T - 1;      // span index of tap 0's sample
        const int u1 = two ? u0 + 2 * NTH : u0;
        float2 a0 = make_float2(0.0f, 0.0f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll 3
        for (int k = 0; k < T; ++k) {
            const float2 h0 = s_taps[k], h1 = s_taps[T + k];
            a0 = cmac(a0, h0, fbuf[u0 - k]);
            b0 = cmac(b0, h1, fbuf[span + u0 - k]);
            a1 = cmac(a1, h0, fbuf[u1 - k]);
            b1 = cmac(b1, h1, fbuf[span + u1 - k]);
        }
        const float2 y0 = cadd(a0, b0);
        a.yw[(int64_t)q * nw + i] = y0;
        const float2 z0 = cmul(y0, y0);
        vlead[i] = cmul(z0, z0);
        if (two) {
            const float2 y1 = cadd(a1, b1);
            a.yw[(int64_t)q * nw + i + NTH] = y1;
            const float2 z1 = cmul(y1, y1);
            vlead[i + NTH] = cmul(z1, z1);
        }
    }
    cl.sync();                                        // #1: every v in its leader (and the spans read)

    // 2. leaders: P_q = |FFT_N(v_q)|^2, left in the FFT buffer as floats by the last pass (whose reads
    //    all precede its writes), and copied into the other leader
    float* P = reinterpret_cast<float*>(fbuf);
    if (leader) {
        auto load = [&](int i) -> float2 { return i < nw ? vbuf[i] : make_float2(0.0f, 0.0f); };
        if constexpr (S::TWS) {
            float* Pr = cl.map_shared_rank(Pc, q ? 0 : HALF);
            auto store = [&](int i, float2 v) {
                const float e = cabs2(v);
                P[i] = e;
                Pr[i] = e;
            };
            fft_run_tw<K, -1, true, true>(fbuf, TwShared{tws, TWSHIFT}, load, store);
        } else {
            auto store = [&](int i, float2 v) { P[i] = cabs2(v); };
            fft_run<K, -1, true, true>(fbuf, a.tw, load, store);
        }
    }
    cl.sync();                                        // #2: both periodograms complete

    const int nb = min((int)(nw / a.Lb), FOE_NBMAX);
    if (leader) {
        // 3. first maximum of P_0 + P_1 (a + b == b + a: both leaders find the same bin); the other
        //    leader's bins from the local copy, else across the cluster, all in flight together
        const float* Pp = S::TWS ? Pc : cl.map_shared_rank(P, q ? 0 : HALF);
        constexpr int PER = N / NTH;
        float pv[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) pv[u] = Pp[tid + u * NTH];
        float best = -1.0f;
        int besti = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const float v = P[tid + u * NTH] + pv[u];
            if (v > best) { best = v; besti = tid + u * NTH; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
            if (ov > best || (ov == best && oi < besti)) { best = ov; besti = oi; }
        }
        if (lane == 0) { bv[w] = best; bi[w] = besti; }
        __syncthreads();
        if (tid == 0) {
            float b = -1.0f;
            int idx = 0;
            for (int k = 0; k < NTH / 32; ++k)
                if (bv[k] > b || (bv[k] == b && bi[k] < idx)) { b = bv[k]; idx = bi[k]; }
            s_kappa = idx < N / 2 ? idx : idx - N;
        }
        __syncthreads();
        // 4. this row's per-block sums, one warp per block (|kappa n| < N nw / 2 <= 2^26: the phase
        //    index kappa n mod N is exact in 32 bits; e^{-j 2 pi t / N} is twiddle entry t RX_FFT_TW_N / N),
        //    into leader 0's shared memory
        const int kappa = s_kappa;
        float2* adst = cl.map_shared_rank(asum, 0) + q * FOE_NBMAX;
        for (int j = w; j < nb; j += NTH / 32) {
            float ax = 0.0f, ay = 0.0f;
            for (int n = j * a.Lb + lane; n < (j + 1) * a.Lb; n += 32) {
                const int t = (kappa * n) & (N - 1);
                const float2 ph = S::TWS ? tws[t] : __ldg(&a.tw[t << TWSHIFT]);
                const float2 v = cmul(vbuf[n], ph);
                ax += v.x;
                ay += v.y;
            }
            ax = warp_sum(ax);
            ay = warp_sum(ay);
            if (lane == 0) adst[j] = make_float2(ax, ay);
        }
    }
    cl.sync();                                        // #3: both rows' sums in leader 0
    if (rank != 0) return;

    // 5. leader 0: phi_j = arg(a_0j + a_1j), unwrapped in sequence (a prefix sum of the steps brought
    //    into [-pi, pi]), then the least-squares slope against the block centres, by warp 0
    float* s_ph = reinterpret_cast<float*>(vbuf);     // vbuf is no longer read
    for (int j = tid; j < nb; j += NTH) {
        const float2 s0 = asum[j], s1 = asum[FOE_NBMAX + j];
        s_ph[j] = atan2f(s0.y + s1.y, s0.x + s1.x);
    }
    __syncthreads();
    const float PIf = 3.14159265358979f;
    if (w == 0 && nb >= 2) {
        const float ph0 = s_ph[0];
        float carry = 0.0f, prev_raw = 0.0f, sx = 0.0f, sy = 0.0f;
        for (int base = 0; base < nb; base += 32) {
            const int j = base + lane;
            const float ph = j < nb ? s_ph[j] : 0.0f;
            float prv = __shfl_up_sync(0xffffffffu, ph, 1);
            if (lane == 0) prv = prev_raw;
            float st_ = 0.0f;
            if (j > 0 && j < nb) {
                st_ = ph - prv;
                if (st_ > PIf) st_ -= 2.0f * PIf;
                else if (st_ < -PIf) st_ += 2.0f * PIf;
            }
            for (int o = 1; o < 32; o <<= 1) {
                const float v = __shfl_up_sync(0xffffffffu, st_, o);
                if (lane >= o) st_ += v;
            }
            const float u = ph0 + carry + st_;
            prev_raw = __shfl_sync(0xffffffffu, ph, 31);
            carry = __shfl_sync(0xffffffffu, carry + st_, 31);
            __syncwarp();
            if (j < nb) s_ph[j] = u;                  // in place: the chunk's raw phases were read above
            __syncwarp();
        }
        for (int j = lane; j < nb; j += 32) { sx += (float)j; sy += s_ph[j]; }
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        const float mj = sx / nb, mu = sy / nb;
        float sjj = 0.0f, sju = 0.0f;
        for (int j = lane; j < nb; j += 32) {
            const float dj = (float)j - mj;
            sjj = fmaf(dj, dj, sjj);
            sju = fmaf(dj, s_ph[j] - mu, sju);
        }
        sjj = warp_sum(sjj);
        sju = warp_sum(sju);
        if (lane == 0) s_wf = sju / (sjj * (float)a.Lb) / 4.0f;   // slope per symbol, / 4 for the 4th power
    }
    __syncthreads();
    // 6. the code: w_c = 2 pi kappa / (4 N) is kappa (pi / 2^(K+1)), the same rounding; the few FP64
    //    steps use host-side scales instead of divisions
    RxDevState* st = a.st;
    if (tid == 0) {
        const double PI = 3.14159265358979323846;
        const int kappa = s_kappa;
        const double wc = (double)kappa * ldexp(PI, -(K + 1));
        const double wh = wc + (nb >= 2 ? (double)s_wf : 0.0);
        const double u = wh * a.u_scale;
        const double code = rint(u);
        st->fo_code = (int)code;
        st->fo_w = wh;
        st->coarse_bin = kappa;
        st->fo_margin = fabs(fabs(u - floor(u)) - 0.5);
        st->fo_valid = 1;
        st->nco_inc = llrint(ldexp(code * a.f_scale, 64));   // turns per sample, |F| < 0.5
    }
    __syncthreads();
    // taps_init = taps_cma * exp(-j 2 pi code grid (k - c) / fs): the phase accumulator at k - c
    const long long inc = st->nco_inc;
    for (int t = tid; t < 4 * T; t += NTH) {
        const int k = t % T;
        st->taps_init[t] = cmul(st->taps_cma[t], nco_conj(inc, (long long)(k - c)));
    }
}

// max over |d| <= c of |rho_d| between the two CMA outputs (second half of
// y_acq). CTA (i, ch): lag d = i - c for i < 2c + 1, the two energies for
// i = 2c + 1, over chunk ch of CMA_CHUNKS; FP32 sums (a threshold test at 0.5
// needs no more precision) stored in flag[2 ...]; the CTA that finishes last
// (a counter in flag[1], reset by it) adds the chunks in a fixed order.
constexpr int CMA_CHUNKS = 4;

__global__ void __launch_bounds__(256) k_cma_check(const float2* __restrict__ yacq, int64_t ystride, int64_t nacq,
                                                   int T, RxDevState* st, int* flag, int pass) {
    pdl_trigger();                                    // the rerun (pass 0) may become resident now
    if (pass == 1 && *flag == 0) return;
    const int64_t h0 = nacq / 2;
    const int L = (int)(nacq - h0);
    const float2* y0 = yacq + h0;
    const float2* y1 = yacq + ystride + h0;
    const int maxlag = (T - 1) / 2, nlag = 2 * maxlag + 1;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    const int ch = blockIdx.y;
    float* part = reinterpret_cast<float*>(flag + 2);          // [nlag + 1][CMA_CHUNKS][2]
    __shared__ float s_x[32], s_y[32];
    __shared__ bool s_last;
    float sx = 0.0f, sy = 0.0f;
    const int clen = (L + CMA_CHUNKS - 1) / CMA_CHUNKS;
    const int c0 = ch * clen, c1 = min(L, c0 + clen);
    if ((int)blockIdx.x < nlag) {
        const int d = (int)blockIdx.x - maxlag;
        const int a0 = max(c0, d < 0 ? -d : 0), a1 = min(c1, L - (d > 0 ? d : 0));
#pragma unroll 4
        for (int n = a0 + tid; n < a1; n += blockDim.x) {
            const float2 v = cmulc(y0[n], y1[n + d]);
            sx += v.x;
            sy += v.y;
        }
    } else {
#pragma unroll 4
        for (int n = c0 + tid; n < c1; n += blockDim.x) {
            sx += cabs2(y0[n]);
            sy += cabs2(y1[n]);
        }
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) { s_x[w] = sx; s_y[w] = sy; }
    __syncthreads();
    if (tid == 0) {
        float ax = 0.0f, ay = 0.0f;
        for (int k = 0; k < nw; ++k) { ax += s_x[k]; ay += s_y[k]; }
        float* pp = part + ((int)blockIdx.x * CMA_CHUNKS + ch) * 2;
        pp[0] = ax;
        pp[1] = ay;
        __threadfence();
        const unsigned done = atomicAdd(reinterpret_cast<unsigned*>(flag + 1), 1u);
        s_last = done == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // last CTA: every partial into shared memory with one parallel load (L2, not L1), then per lag (one
    // lane each of warp 0) the sums over chunks in a fixed order, and the maximum over lags
    __threadfence();
    __shared__ float s_p[(RX_TMAX + 1) * CMA_CHUNKS * 2];
    __shared__ float s_best;
    const int np = (nlag + 1) * CMA_CHUNKS * 2;
    for (int i = tid; i < np; i += blockDim.x) s_p[i] = __ldcg(&part[i]);
    __syncthreads();
    if (w == 0) {
        auto total = [&](int i, int comp) {
            float v = 0.0f;
            for (int c = 0; c < CMA_CHUNKS; ++c) v += s_p[(i * CMA_CHUNKS + c) * 2 + comp];
            return v;
        };
        const float den = sqrtf(total(nlag, 0)) * sqrtf(total(nlag, 1));
        float best = 0.0f;
        for (int k = lane; k < nlag; k += 32) {
            const float rx = total(k, 0), ry = total(k, 1);
            best = fmaxf(best, den > 0.0f ? sqrtf(rx * rx + ry * ry) / den : 0.0f);
        }
        for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) s_best = best;
    }
    __syncthreads();
    const float best = s_best;
    const bool corr = best > 0.5f;
    if (tid == 0) {
        flag[1] = 0;
        if (pass == 0) {
            *flag = corr ? 1 : 0;
            st->cma_rho = best;
            st->cma_reran = corr ? 1 : 0;
        } else if (corr) {
            atomicOr(&st->err_word, 4u);
        }
    }
    // the rerun's start: the second row rebuilt from the first (h_yy[k] = conj h_xx[T-1-k],
    // h_yx[k] = -conj h_xy[T-1-k]), the first row kept; one thread per tap
    if (pass == 0 && corr && tid < T) {
        const int k = tid;
        const float2 hxx = st->taps_cma[0 * T + (T - 1 - k)];
        const float2 hxy = st->taps_cma[1 * T + (T - 1 - k)];
        st->taps_init[0 * T + k] = st->taps_cma[0 * T + k];
        st->taps_init[1 * T + k] = st->taps_cma[1 * T + k];
        st->taps_init[3 * T + k] = make_float2(hxx.x, -hxx.y);
        st->taps_init[2 * T + k] = make_float2(-hxy.x, hxy.y);
    }
}

}  // namespace

int64_t lms_smem_bytes(int T, int Lb, int threads, bool wl) {
    const int XS = 2 * Lb + T;
    const int NTAP = (wl ? 4 : 2) * T;
    const int G = threads / NTAP > 1 ? threads / NTAP : 1;
    return (int64_t)sizeof(float2) * (NTAP + 4 * XS + 2 * Lb + G * NTAP + 1 + (2 * Lb + T - 1));
}

size_t lms_launch_smem(size_t need, int exclusive) {
    if (!exclusive) return need;
    static size_t optin = 0;
    if (!optin) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        optin = v > 0 ? (size_t)v : need;
    }
    return need > optin ? need : optin;
}

template <int NT, bool WL = false>
static cudaError_t launch_lms_t(const LmsArgs& a, cudaStream_t s) {
    const int64_t nseg = (a.n_sym + a.L_seg - 1) / a.L_seg;
    if (nseg <= 0) return cudaSuccess;
    const size_t smem = lms_launch_smem((size_t)lms_smem_bytes(a.T, a.Lb, NT, WL), a.exclusive);
    static size_t attr = 0;
    if (smem > 48 * 1024 && smem > attr) {
        cudaFuncSetAttribute(k_lms<NT, WL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    k_lms<NT, WL><<<dim3((unsigned)nseg, a.npol == 1 ? 1 : 2), NT, smem, s>>>(a);
    return cudaGetLastError();
}

bool lms_fast_a(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err);
bool lms_fast_b(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err);
bool lms_fast_c(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err);
bool lms_tile_a(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err);
bool lms_tile_b(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err);
bool lms_tile_c(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err);

// The register-tiled kernel (k_lms_tile.cuh) for its shapes at 128 or 256 threads, the compile-time
// shapes of k_lms_fast.cuh next (512 threads included), this file's generic kernel every other shape.
cudaError_t launch_lms(const LmsArgs& a, int threads, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    if (lms_tile_a(a, threads, s, &err) || lms_tile_b(a, threads, s, &err) || lms_tile_c(a, threads, s, &err))
        return err;
    if (lms_fast_b(a, threads, s, &err) || lms_fast_a(a, threads, s, &err) || lms_fast_c(a, threads, s, &err))
        return err;
    switch (threads) {
        case 128: return launch_lms_t<128>(a, s);
        case 512: return launch_lms_t<512>(a, s);
        case 1024: return launch_lms_t<1024>(a, s);
        default: return launch_lms_t<256>(a, s);
    }
}

cudaError_t launch_lms_wl_generic(const LmsArgs& a, int threads, cudaStream_t s) {
    if (threads < 4 * a.T) return cudaErrorInvalidValue;
    switch (threads) {
        case 256: return launch_lms_t<256, true>(a, s);
        case 512: return launch_lms_t<512, true>(a, s);
        case 1024: return launch_lms_t<1024, true>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

bool lms_fast_wl(const LmsArgs& a, int threads, cudaStream_t s, cudaError_t* err);

// widely-linear segmented DD-LMS: the compile-time shapes (k_lms_fast_wl.cu) first, this file's generic
// kernel otherwise (threads >= 4T); threads 0 takes 128 for the compile-time shapes, else 256
cudaError_t launch_lms_wl(const LmsArgs& a, int threads, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    if (lms_fast_wl(a, threads ? threads : 128, s, &err)) return err;
    if (!threads) threads = 256;
    if (threads < 4 * a.T) return cudaErrorInvalidValue;
    switch (threads) {
        case 256: return launch_lms_t<256, true>(a, s);
        case 512: return launch_lms_t<512, true>(a, s);
        case 1024: return launch_lms_t<1024, true>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int K>
static cudaError_t foe_t(const FoeArgs& a, cudaStream_t s) {
    using S = FoeShape<K>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_foe<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        attr = true;
    }
    // a programmatic dependent of the stream's previous kernel (the kernel waits before reading its outputs)
    return launch_pdl(k_foe<K>, dim3(FOE_CL), dim3(S::NTH), S::SMEM, s, a);
}

cudaError_t launch_foe(const FoeArgs& a, int kf, cudaStream_t s) {
    if (a.nw < 1 || a.T < 1 || a.T > RX_TMAX || a.Lb < 1 || 2 * a.nw > ((int64_t)1 << kf)) return cudaErrorInvalidValue;
    switch (kf) {
        case 9: return foe_t<9>(a, s);
        case 10: return foe_t<10>(a, s);
        case 11: return foe_t<11>(a, s);
        case 12: return foe_t<12>(a, s);
        case 13: return foe_t<13>(a, s);
        case 14: return foe_t<14>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cma_check(const float2* yacq, int64_t ystride, int64_t nacq, int T, RxDevState* st, int* flag,
                             int pass, cudaStream_t s) {
    const int nlag = 2 * ((T - 1) / 2) + 1;                 // lags |d| <= c, then the energies
    k_cma_check<<<dim3(nlag + 1, CMA_CHUNKS), 256, 0, s>>>(yacq, ystride, nacq, T, st, flag, pass);
    return cudaGetLastError();
}

