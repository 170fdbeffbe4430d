// Block LMS (A2 CMA / DD acquisition, A4 segments) as a register-tiled kernel:
// the same recursion and segment schedule as k_lms_fast.cuh and the generic
// kernel in k_mimo.cu (Sec. IV-D's adaptive equaliser with block updates):
//   y[n] = sum_p sum_k h_p[k] x_p[2n + c - k]                       (taps of the block's start)
//   e[n] = y (R2 - |y|^2)  (CMA)   or   dec(y e^{-j psi}) e^{j psi} - y,  psi = arg(-sum y^4) / 4  (DD)
//   h_p[k] += mu sum_n e[n] conj(x_p[2n + c - k])
// for one output row q per CTA (blockIdx.y) and one segment per CTA (blockIdx.x).
//
// Why another mapping: the acquisition is a serial chain of block steps on one
// CTA, so its speed is the latency of one step. Here every lane holds a tile
// of OPL consecutive outputs x IM taps of one (polarisation, tap parity, tap
// half) class, and the same OPL + IM - 1 samples in registers feed both the
// tile's output products and its gradient products (one 16-byte shared-memory
// load per two samples, no per-term loads). Per block step:
//   1. outputs: each lane forms its tile's partial outputs with packed FP32x2
//      FMAs (tap components staged as (hx, hx, hy, hy)); the eight classes of
//      one output subset sit in lanes differing in bits 0-2, which a
//      reduce-scatter by shuffles sums, leaving each output in one or two lanes;
//   2. errors: CMA locally; DD takes the block phase from a warp sum of y^4,
//      one barrier and the per-warp partials in a fixed order;
//   3. the errors go through a warp-private shared-memory row (no barrier) to
//      the lanes of their output subset, which form their tile's gradient
//      partials from the samples still in registers; a reduce-scatter over the
//      four output subsets (lane bits 3-4) leaves a quarter of the class's
//      partials per lane, written per warp;
//   4. barrier; one thread per tap component adds the warps' partials in a
//      fixed order and updates its tap (held in a register) and the staged
//      copy; barrier.
// Windows are split by sample parity (tap k reads parity k % 2) into three
// rotating buffers: a block's window is copied asynchronously (cp.async) two
// steps ahead, and one step ahead each thread waits for its own copies.
// The FO derotation of the input (phase 2 pi F g of input sample g, F turns
// per sample) is linear in g, so it moves exactly onto the taps and outputs:
// y[n] = e^{-j 2 pi F (g0 + 2n + c)} sum_k (h_k e^{+j 2 pi F k}) x[2n + c - k].
// The kernel keeps the taps in that rotating frame, multiplies each output by
// the NCO phasor of its centre sample and each error by the conjugate before
// the gradient, and stages raw samples; the final taps are rotated back.
#pragma once

#include "rx_kernels.h"

template <int NT, int T, int LB>
struct LmsTileShape {
    static constexpr int NW = NT / 32;
    static constexpr int OPL = LB / (NW * 4);              // outputs per lane
    static constexpr int C = (T - 1) / 2;
    static constexpr int NE = C + 1, NO = C;                // taps of even / odd index
    static constexpr int up_even(int v) { return v + (v & 1); }
    static constexpr int G0 = up_even((NE + 1) / 2);        // even taps of group 0 (group 1: the rest)
    static constexpr int G1 = up_even((NO + 1) / 2);        // odd taps of group 0
    static constexpr int IM = G0 > G1 ? G0 : G1;            // tap slots per lane (even)
    static constexpr int R = OPL + IM;                      // sample registers (OPL + IM - 1 used; even)
    static constexpr int PADL = 2 * IM + 2;                 // zero pad below logical index 0
    // origin of the parity-r array for an extra shift xo (even) of the odd-parity arrays: makes every
    // lane's first sample 16-byte aligned
    static constexpr int org2(int r, int xo) { return PADL + ((PADL + C - r + 1) & 1) + (r ? xo : 0); }
    static constexpr int PS0 = PADL + 1 + 6 + LB + C + 4;   // least length of one parity array (float2)
    // 16-byte bank group (of 8) of the first sample load of lane class (p, r, ig) for a parity-array
    // stride ps: the eight classes of one output subset form one quarter-warp of a 16-byte load
    static constexpr int group(int ps, int xo, int p, int r, int ig) {
        const int i0 = ig ? (r ? G1 : G0) : 0;
        return (((2 * p + r) * ps + org2(r, xo) + C - r - i0 - IM + 1) / 2 % 8 + 8) % 8;
    }
    // quarter-warp conflicts of the sample loads (the largest number of classes sharing a group)
    static constexpr int conflicts(int ps, int xo) {
        int worst = 0;
        for (int g = 0; g < 8; ++g) {
            int n = 0;
            for (int c = 0; c < 8; ++c) n += group(ps, xo, c >> 2, (c >> 1) & 1, c & 1) == g ? 1 : 0;
            worst = n > worst ? n : worst;
        }
        return worst;
    }
    static constexpr int pick(bool want_xo) {             // the least-conflict (stride, shift), smallest first
        int bps = PS0 + (PS0 & 1), bxo = 0, bw = 99;
        for (int xo = 0; xo <= 6; xo += 2)
            for (int ps = PS0 + (PS0 & 1); ps < PS0 + 34; ps += 2) {
                const int c = conflicts(ps, xo);
                if (c < bw) { bw = c; bps = ps; bxo = xo; }
            }
        return want_xo ? bxo : bps;
    }
    static constexpr int PS = pick(false);                  // parity-array stride (float2, even)
    static constexpr int XO = pick(true);                   // extra origin shift of the odd-parity arrays
    static constexpr int org(int r) { return org2(r, XO); }
    static constexpr int ESP = LB + LB / 8;                 // error row: one pad slot per eight outputs
    static constexpr int XW = 2 * LB + T - 1;               // window samples per polarisation
    static constexpr int KS = (2 * XW + NT - 1) / NT;       // window samples staged per thread
    static constexpr int TS = IM + 1;                       // staged tap row stride (float4, odd)
    static constexpr int NUPD = 8 * 2 * IM;                 // tap-component update threads
    // shared memory in float4 units
    static constexpr int WIN4 = 3 * 4 * PS / 2;             // three windows x 4 parity arrays
    static constexpr int TAP4 = 8 * TS;
    static constexpr int ES4 = ESP;
    static constexpr int NPART = OPL == 8 ? NW * 4 : NW;    // gradient partials per tap component
    static constexpr int PART4 = (NPART * 8 * 2 * IM + 3) / 4;
    static constexpr int YTS = 88;                          // transposition stride per output subset (float2):
                                                            // = 8 mod 16, two subsets' 8-byte stores fill the 32 banks
    static constexpr int YT4 = OPL == 8 ? NW * 4 * YTS / 2 : 0;
    static constexpr int YP4 = (NW + 1) / 2;
    static constexpr int NBT = 256;                         // blocks of one CTA with a phasor slot
    static constexpr int PH4 = NBT / 2;                     // block phasors (float2)
    static constexpr int SMEM4 = WIN4 + TAP4 + ES4 + PART4 + YP4 + YT4 + PH4;
    static_assert(NT % 32 == 0 && LB % (NW * 4) == 0, "LB must be a multiple of 4 x warps");
    static_assert(OPL == 2 || OPL == 4 || OPL == 8, "2, 4 or 8 outputs per lane");
    static_assert(T % 2 == 1 && T >= 3, "odd tap count");
    static_assert(NUPD <= NT, "one thread per tap component");
    static_assert(NT <= 256, "the DD block phase's fixed-point sum holds NT <= 256 terms");
    static_assert(PS % 2 == 0, "16-byte aligned parity arrays");
};

// fixed-point scale of the DD block phase's sum of y^4, and the bound of one term (|y^4| < 64)
constexpr float kPhaseFx = 65536.0f;
constexpr float kPhaseLim = 4194304.0f;

// One halving level of a reduce-scatter: lanes with (lane & mask) keep the upper half of v[0, N),
// the others the lower half; each adds its partner's copy of the half it keeps.
template <int N, int M>
__device__ __forceinline__ void rs_level(float (&v)[M], int mask, int lane) {
    const bool up = (lane & mask) != 0;
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const float send = up ? v[i] : v[i + N / 2];
        const float keep = up ? v[i + N / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
}

// 128-thread CTAs (the segments' shape) keep to 128 registers so that four share an SM
template <int NT, int T, int LB>
__global__ void __launch_bounds__(NT, NT == 128 ? 4 : 1) k_lms_tile(LmsArgs a) {
    using S = LmsTileShape<NT, T, LB>;
    constexpr int NW = S::NW, OPL = S::OPL, IM = S::IM, R = S::R, PS = S::PS;
    extern __shared__ float4 smem4[];
    pdl_trigger();                                                  // the next kernel may become resident
    float2* win = reinterpret_cast<float2*>(smem4);                 // [3 buffers][p][parity][PS]
    float4* tapx = smem4 + S::WIN4;                                 // [class][TS]: (hx, hx, hy, hy)
    float4* es = tapx + S::TAP4;                                    // [ESP]: (ex, ex, ey, ey), padded
    float* part = reinterpret_cast<float*>(es + S::ES4);            // [warp][class][2 IM]
    int2* ypart = reinterpret_cast<int2*>(es + S::ES4 + S::PART4);       // [NW] block phase partials
    float2* ytr = reinterpret_cast<float2*>(es + S::ES4 + S::PART4 + S::YP4);   // [warp][subset][YTS] (OPL == 8)
    float2* bph = reinterpret_cast<float2*>(es + S::ES4 + S::PART4 + S::YP4 + S::YT4);   // [NBT]
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int q = blockIdx.y;
    const Qam qm = make_qam(a.m);
    // lane class: b0 tap group, b1 tap parity, b2 polarisation; bits 3-4 the output subset
    const int ig = lane & 1, r = (lane >> 1) & 1, p = (lane >> 2) & 1, cls = lane & 7, ns = lane >> 3;
    const int Gr = r ? S::G1 : S::G0;
    const int i0 = ig ? Gr : 0;

    // zero both windows (pads stay zero), the staged taps and the derotation tables
    for (int i = tid; i < S::WIN4; i += NT) smem4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = tid; i < S::TAP4; i += NT) tapx[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();

    const int64_t seg = blockIdx.x, nseg = gridDim.x;
    const int64_t start = seg * a.L_seg;
    const int64_t end = min(a.n_sym, start + a.L_seg);
    const int nwarm = seg > 0 ? a.n_wu : 0;
    const int nmain = (int)((end - start + LB - 1) / LB);
    const int nblk = nwarm + nmain;
    const int64_t nfirst = start - (int64_t)nwarm * LB;            // block b starts at symbol nfirst + b LB
    const float2* const xp0 = a.x;
    const float2* const xp1 = a.x + a.xstride;
    // input-sample index of the centre tap's sample of output n of block 0: the frame of its phasor
    const long long gout0 = a.g0 + a.off + 2 * nfirst + S::C;
    // every window the CTA will read, requested into L2 (128-byte lines)
    if (nblk > 0) {
        const int64_t lo = max(a.off + 2 * nfirst - (int64_t)S::C, (int64_t)0);
        const int64_t hi = min(a.off + 2 * (nfirst + (int64_t)nblk * LB) - (int64_t)S::C + T, a.xlen);
        const int64_t l0 = (lo * 8) >> 7, l1 = (hi * 8 + 127) >> 7;
        for (int64_t l = l0 + tid; l < l1; l += NT) {
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const char* adr = reinterpret_cast<const char*>(pp ? xp1 : xp0) + (l << 7);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(adr));
            }
        }
    }

    // Window staging by asynchronous copies (cp.async, 8 bytes per sample, zero fill outside the buffer):
    // thread tid stages window positions s = tid + k NT of the two polarisations (s < 2 XW), into the
    // parity arrays of one of three window buffers; a block's copies are issued two steps ahead, the
    // thread waits for its own copies one step ahead, and the barriers of that step make them visible.
    // Slots and relative global offsets are the same for every block.
    const int64_t gstart = a.off + 2 * nfirst - S::C;                  // window start of block 0
    const uint32_t win_sa = (uint32_t)__cvta_generic_to_shared(win);
    // window position k of this thread: polarisation, position in the window, shared slot in buffer 0
    auto spos = [&](int k, int& pp, int& jj) -> bool {
        const int sidx = tid + k * NT;
        pp = sidx >= S::XW ? 1 : 0;
        jj = sidx - pp * S::XW;
        return sidx < 2 * S::XW;
    };
    auto sslot = [&](int pp, int jj) -> uint32_t {
        const int par = jj & 1;
        return win_sa + 8u * (uint32_t)((2 * pp + par) * PS + S::org(par) + (jj >> 1));
    };
    // per window position k of this thread: its shared slot in buffer 0 and its sample offset from
    // xp0 (the polarisation's row plus the position; the launch keeps it below 2^31)
    uint32_t kslot[S::KS];
    int ksrc[S::KS];
#pragma unroll
    for (int k = 0; k < S::KS; ++k) {
        int pp, jj;
        const bool in = spos(k, pp, jj);
        kslot[k] = in ? sslot(pp, jj) : 0u;
        ksrc[k] = in ? (int)(pp * a.xstride) + jj : -1;
    }
    auto issue = [&](int blk) {                                        // copies of block blk's window
        const int64_t g0b = gstart + 2LL * LB * blk;
        const bool fast = g0b >= 0 && g0b + S::XW <= a.xlen;          // whole window inside the buffer
        const uint32_t boff = 8u * (uint32_t)((blk % 3) * 4 * PS);
        const float2* src = xp0 + g0b;
        if (fast) {
#pragma unroll
            for (int k = 0; k < S::KS; ++k) {
                if (ksrc[k] < 0) continue;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(kslot[k] + boff),
                             "l"(src + ksrc[k])
                             : "memory");
            }
        } else {
#pragma unroll
            for (int k = 0; k < S::KS; ++k) {
                int pp, jj;
                if (!spos(k, pp, jj)) continue;
                const bool ok = g0b + jj >= 0 && g0b + jj < a.xlen;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(kslot[k] + boff),
                             "l"(ok ? src + ksrc[k] : xp0), "r"(ok ? 8 : 0)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    auto land = [&]() {                                               // own copies of the next block complete
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    };

    // the first two windows' copies are issued before the wait: the samples were complete before the
    // stream's previous kernel started (a programmatic launch follows a kernel that does not write them)
    if (nblk > 0) {
        issue(0);
        if (nblk > 1) issue(1);
        else asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    pdl_wait();                                                     // (programmatic launches) inputs ready
    if (a.run_if && *a.run_if == 0) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");         // no copy outlives the CTA
        return;
    }
    const long long inc = a.derotate ? a.st->nco_inc : 0;

    // tap-component update role: thread u < NUPD owns component f of slot t of class c
    const bool upd = tid < S::NUPD;
    const int uc = tid / (2 * IM), uf = tid % (2 * IM), ut = uf >> 1;
    const int ur = (uc >> 1) & 1, uig = uc & 1, up = (uc >> 2) & 1;
    const int uG = ur ? S::G1 : S::G0, uN = ur ? S::NO : S::NE;
    const int uI = uig ? max(uN - uG, 0) : min(uG, uN);
    const bool ureal = upd && ut < uI;
    const int uk = 2 * ((uig ? uG : 0) + ut) + ur;                  // tap index of the owned slot
    float hreg = 0.0f;
    if (ureal) {
        float2 h = a.taps_in[q * 2 * T + up * T + uk];
        if (inc) {                                                  // rotating frame: h'_k = h_k e^{+j 2 pi F k}
            const float2 ph = nco_conj(inc, uk);
            h = cmul(h, make_float2(ph.x, -ph.y));
        }
        hreg = (uf & 1) ? h.y : h.x;
        float* dst = reinterpret_cast<float*>(tapx + uc * S::TS + ut) + ((uf & 1) ? 2 : 0);
        dst[0] = hreg;
        dst[1] = hreg;
    }

    // the phasor of output n of block b is e^{-j 2 pi F (gout0 + 2 n)} e^{-j 2 pi F 2 LB b}: the first
    // factor per lane in registers, the second per block in a table (nblk <= NBT)
    if (inc)
        for (int i = tid; i < nblk; i += NT) bph[i] = nco_conj(inc, 2LL * LB * i);

    __syncthreads();                                                // tables and taps staged
    if (nblk > 0) land();
    __syncthreads();

    // first output of the lane's tile within a block, and its first sample (logical parity index)
    const int nl0 = w * (4 * OPL) + ns * OPL;
    const int lbase = nl0 + S::C - r - i0 - IM + 1;
    const int soff = (2 * p + r) * PS + S::org(r) + lbase;         // even: 16-byte aligned
    // the output the lane holds after the reduce-scatter, and whether it is that output's owner
    int jst, comp = 0;
    bool owner;
    if constexpr (OPL == 2) { jst = (lane >> 2) & 1; comp = (lane >> 1) & 1; owner = (lane & 3) == 0; }
    else if constexpr (OPL == 4) { jst = 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1); comp = lane & 1; owner = comp == 0; }
    else { jst = lane & 7; owner = true; }
    const int nown = nl0 + jst;                                     // local index of the held output
    const float2 pown = inc ? nco_conj(inc, gout0 + 2LL * nown) : make_float2(1.0f, 0.0f);

    for (int b = 0; b < nblk; ++b) {
        const int64_t n0 = nfirst + (int64_t)b * LB;
        const int L = b < nwarm ? LB : (int)min((int64_t)LB, end - n0);
        // window of block b + 2 requested now (an empty group past the end keeps the wait count uniform)
        if (b + 2 < nblk) issue(b + 2);
        else asm volatile("cp.async.commit_group;\n" ::: "memory");
        const float2* xs = win + (b % 3) * 4 * PS + soff;

        // 1. the tile's partial outputs
        float2 xr[R];
#pragma unroll
        for (int u = 0; u < R / 2; ++u) {
            const float4 v = reinterpret_cast<const float4*>(xs)[u];
            xr[2 * u] = make_float2(v.x, v.y);
            xr[2 * u + 1] = make_float2(v.z, v.w);
        }
        float2 accA[OPL], accB[OPL];
#pragma unroll
        for (int j = 0; j < OPL; ++j) accA[j] = accB[j] = make_float2(0.0f, 0.0f);
        const float4* tp = tapx + cls * S::TS;
#pragma unroll
        for (int t = 0; t < IM; ++t) {
            const float4 h = tp[t];
            const float2 hx = make_float2(h.x, h.y), hy = make_float2(h.z, h.w);
#pragma unroll
            for (int j = 0; j < OPL; ++j) {
                accA[j] = __ffma2_rn(hx, xr[j + IM - 1 - t], accA[j]);
                accB[j] = __ffma2_rn(hy, xr[j + IM - 1 - t], accB[j]);
            }
        }
        float v[2 * OPL];
#pragma unroll
        for (int j = 0; j < OPL; ++j) {
            v[2 * j] = accA[j].x - accB[j].y;
            v[2 * j + 1] = accA[j].y + accB[j].x;
        }
        // reduce-scatter over the eight classes (lane bits 2, 1, 0): outputs first, then components
        float2 y;
        if constexpr (OPL == 2) {
            rs_level<4>(v, 4, lane);
            rs_level<2>(v, 2, lane);
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
            const float o = __shfl_xor_sync(0xffffffffu, v[0], 2);
            y = comp ? make_float2(o, v[0]) : make_float2(v[0], o);
        } else if constexpr (OPL == 4) {
            rs_level<8>(v, 4, lane);
            rs_level<4>(v, 2, lane);
            rs_level<2>(v, 1, lane);
            const float o = __shfl_xor_sync(0xffffffffu, v[0], 1);
            y = comp ? make_float2(o, v[0]) : make_float2(v[0], o);
        } else {
            // eight outputs per lane: transpose through shared memory (lane (ns, cls) writes its
            // partial of output j at [ns][j][cls], the lane of output j reads the eight classes as
            // four 16-byte loads; strides 10 and YTS keep both sides free of bank conflicts)
            float2* yw = ytr + w * (4 * S::YTS) + ns * S::YTS;
#pragma unroll
            for (int j = 0; j < OPL; ++j) yw[j * 10 + cls] = make_float2(v[2 * j], v[2 * j + 1]);
            __syncwarp();
            const float4* yr = reinterpret_cast<const float4*>(yw + jst * 10);
            const float4 c01 = yr[0], c23 = yr[1], c45 = yr[2], c67 = yr[3];
            y = cadd(cadd(cadd(make_float2(c01.x, c01.y), make_float2(c01.z, c01.w)),
                          cadd(make_float2(c23.x, c23.y), make_float2(c23.z, c23.w))),
                     cadd(cadd(make_float2(c45.x, c45.y), make_float2(c45.z, c45.w)),
                          cadd(make_float2(c67.x, c67.y), make_float2(c67.z, c67.w))));
        }
        // rotating frame: the taps are h_k e^{+j 2 pi F k} and the samples are not derotated, so the
        // output takes the phasor of its centre sample, e^{-j 2 pi F (g0 + 2n + c)}, and the error the
        // conjugate before it meets the samples in the gradient
        float2 phi = make_float2(1.0f, 0.0f);
        if (inc) {
            phi = cmul(pown, bph[b]);
            y = cmul(y, phi);
        }
        const bool valid = nown < L;
        if (b >= nwarm && a.y != nullptr && owner && valid) a.y[(int64_t)q * a.ystride + n0 + nown] = y;

        // 2. errors
        float2 e = make_float2(0.0f, 0.0f);
        if (a.cma) {
            if (valid) e = cscale(y, a.R2 - cabs2(y));
        } else {
            // the block sum of y^4 in 2^-16 fixed point: one integer warp reduction per component (exact and
            // in no particular order) instead of five dependent shuffle levels; each term is held to
            // |y^4| < 64 so that no sum of NT <= 256 terms can overflow, far beyond any equalised symbol
            int2 c4 = make_int2(0, 0);
            if (owner && valid) {
                const float2 y2 = cmul(y, y);
                const float2 y4 = cmul(y2, y2);
                c4.x = __float2int_rn(fminf(fmaxf(y4.x * kPhaseFx, -kPhaseLim), kPhaseLim));
                c4.y = __float2int_rn(fminf(fmaxf(y4.y * kPhaseFx, -kPhaseLim), kPhaseLim));
            }
            c4.x = __reduce_add_sync(0xffffffffu, c4.x);
            c4.y = __reduce_add_sync(0xffffffffu, c4.y);
            if (lane == 0) ypart[w] = c4;
            __syncthreads();
            int2 isum = ypart[0];
#pragma unroll
            for (int k = 1; k < NW; ++k) { isum.x += ypart[k].x; isum.y += ypart[k].y; }
            const float2 sum = make_float2((float)isum.x * (1.0f / kPhaseFx), (float)isum.y * (1.0f / kPhaseFx));
            const float2 rt = quarter_root_conj(make_float2(-sum.x, -sum.y));
            if (valid) {
                const float2 d = qam_decide(cmul(y, rt), qm);
                e = csub(cmulc(d, rt), y);
            }
        }
        // 3. the errors of the warp's outputs to the lanes of their subset, then the gradient partials
        if (inc) e = cmulc(e, phi);
        if (owner) es[nown + nown / 8] = make_float4(e.x, e.x, e.y, e.y);
        __syncwarp();
        float2 gA[IM], gB[IM];
#pragma unroll
        for (int t = 0; t < IM; ++t) gA[t] = gB[t] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < OPL; ++j) {                            // one error live at a time
            const float4 ev = es[nl0 + j + (nl0 + j) / 8];
#pragma unroll
            for (int t = 0; t < IM; ++t) {
                gA[t] = __ffma2_rn(make_float2(ev.x, ev.y), xr[j + IM - 1 - t], gA[t]);
                gB[t] = __ffma2_rn(make_float2(ev.z, ev.w), xr[j + IM - 1 - t], gB[t]);
            }
        }
        float g[2 * IM];
#pragma unroll
        for (int t = 0; t < IM; ++t) {
            g[2 * t] = gA[t].x + gB[t].y;          // Re(e conj x)
            g[2 * t + 1] = gB[t].x - gA[t].y;      // Im(e conj x)
        }
        if constexpr (OPL == 8) {
            float4* pw = reinterpret_cast<float4*>(part + ((w * 4 + ns) * 8 + cls) * 2 * IM);
#pragma unroll
            for (int u = 0; u < IM / 2; ++u) pw[u] = make_float4(g[4 * u], g[4 * u + 1], g[4 * u + 2], g[4 * u + 3]);
        } else {
            rs_level<2 * IM>(g, 16, lane);
            rs_level<IM>(g, 8, lane);
            float* pw = part + (w * 8 + cls) * 2 * IM + ns * (IM / 2);
#pragma unroll
            for (int u = 0; u < IM / 2; ++u) pw[u] = g[u];
        }
        if (b + 1 < nblk) land();                                   // next window in place before the barriers
        __syncthreads();

        // 4. tap update: the warps' partials in a fixed order
        if (ureal) {
            float gs;
            if constexpr (OPL == 8) {                                   // warps x subsets, in a fixed order
                float g0 = part[uc * 2 * IM + uf], g1 = part[(8 + uc) * 2 * IM + uf];
#pragma unroll
                for (int k = 2; k < S::NPART; k += 2) {
                    g0 += part[(k * 8 + uc) * 2 * IM + uf];
                    g1 += part[((k + 1) * 8 + uc) * 2 * IM + uf];
                }
                gs = g0 + g1;
            } else {
                gs = part[uc * 2 * IM + uf];
#pragma unroll
                for (int k = 1; k < NW; ++k) gs += part[(k * 8 + uc) * 2 * IM + uf];
            }
            hreg = fmaf(a.mu, gs, hreg);
            float* dst = reinterpret_cast<float*>(tapx + uc * S::TS + ut) + ((uf & 1) ? 2 : 0);
            dst[0] = hreg;
            dst[1] = hreg;
        }
        __syncthreads();
    }
    // final taps of the last segment, back from the rotating frame (the staged copy holds both components)
    if (seg == nseg - 1 && a.taps_out && tid < 2 * T) {
        const int tp = tid / T, tk = tid - tp * T, tr = tk & 1, ti = tk >> 1;
        const int tG = tr ? S::G1 : S::G0, tig = ti >= tG ? 1 : 0;
        const float4 hv = tapx[(tp * 4 + tr * 2 + tig) * S::TS + ti - tig * tG];
        float2 h = make_float2(hv.x, hv.z);
        if (inc) h = cmul(h, nco_conj(inc, tk));
        a.taps_out[q * 2 * T + tp * T + tk] = h;
    }
}

// the tiled kernel keeps one output phasor per block of a CTA (at most 256 blocks) and the sample
// offsets of its window copies as 32-bit integers
template <int LB>
inline bool lms_tile_fits(const LmsArgs& a) {
    return (a.L_seg + LB - 1) / LB + a.n_wu <= 256 && a.xstride < ((int64_t)1 << 30);
}

template <int NT, int T, int LB>
cudaError_t launch_lms_tile_t(const LmsArgs& a, cudaStream_t s) {
    using S = LmsTileShape<NT, T, LB>;
    const int64_t nseg = (a.n_sym + a.L_seg - 1) / a.L_seg;
    if (nseg <= 0) return cudaSuccess;
    const size_t smem = lms_launch_smem(sizeof(float4) * S::SMEM4, a.exclusive);
    static size_t attr = 0;
    if (smem > 48 * 1024 && smem > attr) {
        cudaFuncSetAttribute(k_lms_tile<NT, T, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    if (a.pdl) return launch_pdl(k_lms_tile<NT, T, LB>, dim3((unsigned)nseg, 2), dim3(NT), smem, s, a);
    k_lms_tile<NT, T, LB><<<dim3((unsigned)nseg, 2), NT, smem, s>>>(a);
    return cudaGetLastError();
}
