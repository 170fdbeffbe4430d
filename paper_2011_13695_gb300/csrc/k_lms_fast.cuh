// Block LMS (A2 CMA / DD acquisition, A4 segments) for a tap count T and block
// length LB known at compile time.
//
// Same recursion, schedule and CTA mapping as the generic kernel in k_mimo.cu
// (one CTA per output row q of one segment; Sec. IV-D's adaptive equaliser
// with block updates): per block, the outputs
//   y[n] = sum_p sum_k h_p[k] x_p[2n + c - k]
// then the error (CMA: y (R2 - |y|^2); DD: dec(y e^{-j psi}) e^{j psi} - y with
// psi = arg(-sum y^4) / 4) and the update h_p[k] += mu sum_n e[n] conj(x_p[2n + c - k]).
// What the compile-time shape buys is latency: every inner loop unrolls, so a
// thread issues all its shared-memory loads of a step back to back instead of
// one dependent pair per term. The per-block critical path is also shorter:
//   * outputs: P = NT / LB lanes per output, each with a fixed run of CS terms;
//   * the DD phase sum is reduced per warp while the outputs are still in
//     registers, and every thread then combines the NT/32 warp partials in the
//     same fixed order and takes the phase itself (no single-thread step and
//     no extra barrier);
//   * gradients: thread (g, t) sums tap t over symbols n = g (mod G), then the
//     2T tap threads add the G partials in a fixed order and update the taps;
//   * the next block's window is loaded into registers while the current one
//     is processed, and derotated with a per-kernel offset table as it is
//     written to shared memory; the whole range a CTA reads is requested into
//     L2 when it starts.
// The widely-linear form (WL; Sec. IV-D) adds conjugate taps g_p: the output
// gains sum_p sum_k g_p[k] conj(x_p[2n + c - k]) and g_p[k] += mu_c sum_n e[n]
// x_p[2n + c - k]. Every sample a lane loads then feeds both its direct and
// its conjugate product, and each gradient thread accumulates both sums of its
// tap (p, k) from the same loads. Taps per row: [h_0, h_1, g_0, g_1].
#pragma once

#include "rx_kernels.h"

template <int NT, int T, int LB, bool WL = false>
struct LmsFastShape {
    static constexpr int NV = WL ? 2 : 1;                  // tap sets: direct (and conjugate)
    static constexpr int C = (T - 1) / 2;
    static constexpr int XW = 2 * LB + T - 1;             // window samples per polarisation
    static constexpr int XS = 2 * LB + T + 1;             // natural staging stride per polarisation (even)
    static constexpr int XE = ((XW + 1) / 2 + 1) & ~1;     // split staging: even samples, odd ones at XE (even)
    static constexpr int Q = 2 * NT / LB;                  // lanes per output pair (pair path: 2 or 4)
    // the pair path for Q = 4 only: with Q = 2 (NT = LB) its registers cost segments CTAs per SM
    static constexpr bool PAIR = Q == 4 && (2 * NT) % LB == 0;
    static constexpr int RP = 2 * ((C + 2) / 2);           // split tap row: C + 1 even taps, padded to even
    static constexpr int P = NT / LB;                      // lanes per output
    static constexpr int PH = P >= 2 ? P / 2 : 1;          // lanes per polarisation (P >= 2)
    static constexpr int KC = 2 * ((T + 2 * PH - 1) / (2 * PH));   // taps per lane (even, P >= 2)
    static constexpr int G = NT / (2 * T);                 // gradient groups
    static constexpr int NG = (LB + G - 1) / G;            // symbols per group
    static constexpr int PF = (2 * XW + NT - 1) / NT;      // window registers per thread
    static constexpr int NWARP = NT / 32;
    static constexpr int NBT = 256;                        // derotation bases of the first NBT blocks
    static constexpr int SMEM =
        NV * (4 * RP + 2 * T) + 2 * (2 * XS + 4 * XE) + LB + G * NV * 2 * T + NWARP + XW + NBT;   // float2
    static_assert(NT % LB == 0 && (P & (P - 1)) == 0 && P <= 32, "NT must be a power-of-two multiple of LB");
    static_assert(G >= 1, "at least 2T threads");
    static_assert(T % 2 == 1, "odd tap count: window index parity follows the tap index");
};

template <int NT, int T, int LB, bool WL = false>
__global__ void __launch_bounds__(NT) k_lms_fast(LmsArgs a) {
    using S = LmsFastShape<NT, T, LB, WL>;
    constexpr int NV = S::NV;
    constexpr int NTAP = NV * 2 * T;                       // taps of one row
    extern __shared__ float4 smem4[];                      // 16-byte aligned
    float2* smem = reinterpret_cast<float2*>(smem4);
    if (a.run_if && *a.run_if == 0) return;
    float2* tps = smem;                                    // [v][p][parity][RP]: taps split by parity (16-B rows)
    float2* taps = tps + NV * 4 * S::RP;                   // [v][p][k]
    constexpr int WBUF = 2 * S::XS + 4 * S::XE;            // one window: natural [2][XS], split [2][2 XE]
    float2* xsb = taps + NTAP;                             // two windows
    float2* es = xsb + 2 * WBUF;                           // [LB]
    float2* part = es + LB;                                // [G][NTAP]
    float2* ypart = part + S::G * NTAP;                    // [NWARP]
    float2* tab = ypart + S::NWARP;                        // [XW]
    float2* btab = tab + S::XW;                            // [NBT]: derotation base of block b's window
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = blockIdx.y;
    const Qam qm = make_qam(a.m);
    const long long inc = a.derotate ? a.st->nco_inc : 0;
    auto tps_at = [&](int t) -> float2* {                  // split position of tap t = (v, p, k)
        const int v = t >= 2 * T ? 1 : 0, t2 = t - v * 2 * T;
        const int p = t2 >= T ? 1 : 0, k = t2 - p * T;
        return tps + v * 4 * S::RP + (2 * p + (k & 1)) * S::RP + (k >> 1);
    };
    for (int t = tid; t < NV * 4 * S::RP; t += NT) tps[t] = make_float2(0.0f, 0.0f);
    __syncthreads();
    for (int t = tid; t < NTAP; t += NT) {
        const float2 h = a.taps_in[q * NTAP + t];
        taps[t] = h;
        *tps_at(t) = h;
    }
    if (inc)
        for (int jj = tid; jj < S::XW; jj += NT) tab[jj] = nco_conj(inc, jj);

    const int64_t seg = blockIdx.x, nseg = gridDim.x;
    const int64_t start = seg * a.L_seg;
    const int64_t end = min(a.n_sym, start + a.L_seg);
    const int nwarm = seg > 0 ? a.n_wu : 0;
    const int nmain = (int)((end - start + LB - 1) / LB);
    const int nblk = nwarm + nmain;
    const int64_t nfirst = start - (int64_t)nwarm * LB;    // block b starts at symbol nfirst + b LB
    const float2* const xp0 = a.x;
    const float2* const xp1 = a.x + a.xstride;
    // the derotation of block b's window starts at input sample g0 + off + 2 (nfirst + b LB) - C; its
    // phasor is taken once per block here instead of by every thread at every commit
    const long long gfirst = a.g0 + a.off + 2 * nfirst - S::C;
    if (inc)
        for (int b = tid; b < nblk; b += NT) btab[b] = nco_conj(inc, gfirst + 2LL * LB * b);   // nblk <= NBT

    // every window the CTA will read, requested into L2 (128-byte lines)
    if (nblk > 0) {
        const int64_t lo = max(a.off + 2 * nfirst - (int64_t)S::C, (int64_t)0);
        const int64_t hi = min(a.off + 2 * (nfirst + (int64_t)nblk * LB) - (int64_t)S::C + T, a.xlen);
        const int64_t l0 = (lo * 8) >> 7, l1 = (hi * 8 + 127) >> 7;
        for (int64_t l = l0 + tid; l < l1; l += NT) {
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const char* adr = reinterpret_cast<const char*>(p ? xp1 : xp0) + (l << 7);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(adr));
            }
        }
    }

    float2 pf[S::PF];
    auto prefetch = [&](int64_t n0) {
        const int64_t i0 = a.off + 2 * n0 - S::C;
#pragma unroll
        for (int r = 0; r < S::PF; ++r) {
            const int t = tid + r * NT;
            float2 v = make_float2(0.0f, 0.0f);
            if (t < 2 * S::XW) {
                const int p = t >= S::XW ? 1 : 0, jj = t - p * S::XW;
                const int64_t i = i0 + jj;
                if (i >= 0 && i < a.xlen) v = __ldg((p ? xp1 : xp0) + i);
            }
            pf[r] = v;
        }
    };
    auto commit = [&](float2* xs, int blk) {
        const float2 base = inc ? btab[blk] : make_float2(1.0f, 0.0f);
#pragma unroll
        for (int r = 0; r < S::PF; ++r) {
            const int t = tid + r * NT;
            if (t < 2 * S::XW) {
                const int p = t >= S::XW ? 1 : 0, jj = t - p * S::XW;
                float2 v = pf[r];
                if (inc) v = cmul(v, cmul(base, tab[jj]));
                xs[p * S::XS + jj] = v;
                xs[2 * S::XS + p * 2 * S::XE + ((jj & 1) ? S::XE + (jj >> 1) : (jj >> 1))] = v;
            }
        }
    };

    __syncthreads();                                       // taps and table
    if (nblk > 0) {
        prefetch(nfirst);
        commit(xsb, 0);
    }
    __syncthreads();

    // Each window is staged twice: in natural order [p][jj] (the gradient's lanes run over taps, so
    // consecutive lanes read consecutive samples) and split by parity, sample jj at jj / 2 (even jj)
    // or XE + jj / 2 (odd jj) of the split plane of p (the outputs' lanes run over n, so the samples
    // x_p[2n + c - k] of consecutive outputs are consecutive); the parity of the window index
    // 2n + T - 1 - k is that of k.
    //
    // Output roles. Pair path (Q = 2 NT / LB lanes per pair of outputs 2m, 2m + 1, Q = 2 or 4): lane r
    // of the pair takes polarisation r / (Q / 2) and, for Q = 4, the taps of parity r % 2 (both
    // parities for Q = 2). With c = (T - 1) / 2, even taps k = 2i read E[2m + c - i] (output 2m) and
    // E[2m + 1 + c - i] (output 2m + 1), odd taps k = 2i + 1 read O[2m + c - 1 - i] and O[2m + c - i],
    // so the lane loads the runs E[2m .. 2m + c + 1] and O[2m .. 2m + c] with 16-byte loads and its
    // taps with 16-byte loads from the parity-split tap rows. Other shapes: P = NT / LB lanes per
    // output, the lane takes polarisation j / PH and taps k = h KC + i, h = j % PH (KC even).
    const int n_out = S::PAIR ? 2 * (tid / S::Q) : tid / S::P;
    const int j = S::PAIR ? tid % S::Q : tid % S::P;
    const int op = S::PAIR ? j / (S::Q / 2) : (S::P >= 2 ? j / S::PH : 0);
    const int opar = (S::PAIR && S::Q == 4) ? (j & 1) : 0;
    const int oh = S::P >= 2 ? j % S::PH : 0;
    const int olim = T - oh * S::KC;                      // taps i < olim exist for this lane (P path)
    // gradient role: tap t = (p, k), symbols n = g (mod G)
    const int gg = tid / (2 * T), gt = tid - gg * 2 * T;
    const bool grad_on = gg < S::G;
    const int gp = gt >= T ? 1 : 0, gk = gt - gp * T;
    const int goff = gp * S::XS + T - 1 - gk + 2 * gg;     // natural copy: x_p[2n + c - k], n = gg + G i

    for (int b = 0; b < nblk; ++b) {
        const int64_t n0 = nfirst + (int64_t)b * LB;
        const int L = b < nwarm ? LB : (int)min((int64_t)LB, end - n0);
        float2* xs = xsb + (b & 1) * WBUF;
        float2* xsplit = xs + 2 * S::XS;
        if (b + 1 < nblk) prefetch(n0 + LB);

        // outputs: y0 = y[n_out], y1 = y[n_out + 1] (pair path) or y0 = y[n_out]
        float2 y0 = make_float2(0.0f, 0.0f), y1 = make_float2(0.0f, 0.0f);
        if constexpr (S::PAIR) {
            constexpr int C = S::C;
            constexpr int NE = (C + 3) / 2;                 // float4 loads of the even run (C + 2 values)
            constexpr int NO = (C + 2) / 2;                 // float4 loads of the odd run (C + 1 values)
            const float4* E4 = reinterpret_cast<const float4*>(xsplit + op * 2 * S::XE + n_out);
            const float4* O4 = reinterpret_cast<const float4*>(xsplit + op * 2 * S::XE + S::XE + n_out);
            const float4* TE4 = reinterpret_cast<const float4*>(tps + (2 * op) * S::RP);
            const float4* TO4 = reinterpret_cast<const float4*>(tps + (2 * op + 1) * S::RP);
            float2 a0 = make_float2(0.0f, 0.0f), a1 = a0, b0 = a0, b1 = a0;
            if (S::Q == 2 || opar == 0) {
                float2 xv[2 * NE], hv[2 * NE];
#pragma unroll
                for (int u = 0; u < NE; ++u) {
                    const float4 v = E4[u];
                    xv[2 * u] = make_float2(v.x, v.y);
                    xv[2 * u + 1] = make_float2(v.z, v.w);
                }
#pragma unroll
                for (int u = 0; u < S::RP / 2; ++u) {
                    const float4 v = TE4[u];
                    hv[2 * u] = make_float2(v.x, v.y);
                    hv[2 * u + 1] = make_float2(v.z, v.w);
                }
#pragma unroll
                for (int i = 0; i <= C; ++i) {
                    if (i & 1) {
                        b0 = cmac(b0, hv[i], xv[C - i]);
                        b1 = cmac(b1, hv[i], xv[C + 1 - i]);
                    } else {
                        a0 = cmac(a0, hv[i], xv[C - i]);
                        a1 = cmac(a1, hv[i], xv[C + 1 - i]);
                    }
                }
                if constexpr (WL) {
                    const float4* GE4 = TE4 + 4 * S::RP / 2;    // conjugate taps: 4 RP float2 further
#pragma unroll
                    for (int u = 0; u < S::RP / 2; ++u) {
                        const float4 v = GE4[u];
                        hv[2 * u] = make_float2(v.x, v.y);
                        hv[2 * u + 1] = make_float2(v.z, v.w);
                    }
#pragma unroll
                    for (int i = 0; i <= C; ++i) {
                        if (i & 1) {
                            b0 = cmacc(b0, hv[i], xv[C - i]);
                            b1 = cmacc(b1, hv[i], xv[C + 1 - i]);
                        } else {
                            a0 = cmacc(a0, hv[i], xv[C - i]);
                            a1 = cmacc(a1, hv[i], xv[C + 1 - i]);
                        }
                    }
                }
            }
            if (S::Q == 2 || opar == 1) {
                float2 xv[2 * NO], hv[2 * NO];
#pragma unroll
                for (int u = 0; u < NO; ++u) {
                    const float4 v = O4[u];
                    xv[2 * u] = make_float2(v.x, v.y);
                    xv[2 * u + 1] = make_float2(v.z, v.w);
                }
#pragma unroll
                for (int u = 0; u < S::RP / 2; ++u) {
                    const float4 v = TO4[u];
                    hv[2 * u] = make_float2(v.x, v.y);
                    hv[2 * u + 1] = make_float2(v.z, v.w);
                }
#pragma unroll
                for (int i = 0; i < C; ++i) {
                    if (i & 1) {
                        b0 = cmac(b0, hv[i], xv[C - 1 - i]);
                        b1 = cmac(b1, hv[i], xv[C - i]);
                    } else {
                        a0 = cmac(a0, hv[i], xv[C - 1 - i]);
                        a1 = cmac(a1, hv[i], xv[C - i]);
                    }
                }
                if constexpr (WL) {
                    const float4* GO4 = TO4 + 4 * S::RP / 2;
#pragma unroll
                    for (int u = 0; u < S::RP / 2; ++u) {
                        const float4 v = GO4[u];
                        hv[2 * u] = make_float2(v.x, v.y);
                        hv[2 * u + 1] = make_float2(v.z, v.w);
                    }
#pragma unroll
                    for (int i = 0; i < C; ++i) {
                        if (i & 1) {
                            b0 = cmacc(b0, hv[i], xv[C - 1 - i]);
                            b1 = cmacc(b1, hv[i], xv[C - i]);
                        } else {
                            a0 = cmacc(a0, hv[i], xv[C - 1 - i]);
                            a1 = cmacc(a1, hv[i], xv[C - i]);
                        }
                    }
                }
            }
            y0 = cadd(a0, b0);
            y1 = cadd(a1, b1);
#pragma unroll
            for (int w = 1; w < S::Q; w <<= 1) {
                y0.x += __shfl_xor_sync(0xffffffffu, y0.x, w);
                y0.y += __shfl_xor_sync(0xffffffffu, y0.y, w);
                y1.x += __shfl_xor_sync(0xffffffffu, y1.x, w);
                y1.y += __shfl_xor_sync(0xffffffffu, y1.y, w);
            }
        } else {
            float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
            if constexpr (S::P == 1) {
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float2* be = xsplit + p * 2 * S::XE + n_out + S::C;   // even taps: be[-k/2]
                    const float2* bo = be + S::XE;                             // odd taps: bo[-(k+1)/2]
#pragma unroll
                    for (int k = 0; k < T; ++k) {
                        const float2 xv = (k & 1) ? bo[-((k + 1) >> 1)] : be[-(k >> 1)];
                        if (k & 1) acc1 = cmac(acc1, taps[p * T + k], xv);
                        else acc0 = cmac(acc0, taps[p * T + k], xv);
                        if constexpr (WL) {
                            if (k & 1) acc1 = cmacc(acc1, taps[2 * T + p * T + k], xv);
                            else acc0 = cmacc(acc0, taps[2 * T + p * T + k], xv);
                        }
                    }
                }
            } else {
                const float2* be = xsplit + op * 2 * S::XE + n_out + S::C - ((oh * S::KC) >> 1);
                const float2* bo = be + S::XE;
                const float2* hp = taps + op * T + oh * S::KC;
#pragma unroll
                for (int i = 0; i < S::KC; ++i) {
                    if (i < olim) {
                        const float2 xv = (i & 1) ? bo[-((i + 1) >> 1)] : be[-(i >> 1)];
                        if (i & 1) acc1 = cmac(acc1, hp[i], xv);
                        else acc0 = cmac(acc0, hp[i], xv);
                        if constexpr (WL) {
                            if (i & 1) acc1 = cmacc(acc1, hp[2 * T + i], xv);
                            else acc0 = cmacc(acc0, hp[2 * T + i], xv);
                        }
                    }
                }
            }
            y0 = cadd(acc0, acc1);
#pragma unroll
            for (int w = 1; w < S::P; w <<= 1) {
                y0.x += __shfl_xor_sync(0xffffffffu, y0.x, w);
                y0.y += __shfl_xor_sync(0xffffffffu, y0.y, w);
            }
        }
        constexpr int NOUT = S::PAIR ? 2 : 1;
        const bool lead = j == 0;
        const bool v0 = lead && n_out < L, v1 = lead && NOUT == 2 && n_out + 1 < L;
        // every lane of a pair holds both sums: lane 0 takes the first output, lane 1 the second
        const int jo = (NOUT == 2 && j < 2) ? j : 0;
        const bool vo = (NOUT == 2 ? j < 2 : lead) && n_out + jo < L;
        const float2 yo = jo ? y1 : y0;
        if (b >= nwarm && a.y != nullptr && vo) a.y[(int64_t)q * a.ystride + n0 + n_out + jo] = yo;
        if (a.cma) {
            if (vo) es[n_out + jo] = cscale(yo, a.R2 - cabs2(yo));
        } else {
            float2 c4 = make_float2(0.0f, 0.0f);
            if (v0) {
                const float2 y2 = cmul(y0, y0);
                c4 = cmul(y2, y2);
            }
            if (v1) {
                const float2 y2 = cmul(y1, y1);
                c4 = cadd(c4, cmul(y2, y2));
            }
            c4.x = warp_sum(c4.x);
            c4.y = warp_sum(c4.y);
            if (lane == 0) ypart[warp] = c4;
            __syncthreads();
            float2 sum = ypart[0];
#pragma unroll
            for (int w = 1; w < S::NWARP; ++w) sum = cadd(sum, ypart[w]);
            const float2 r = quarter_root_conj(make_float2(-sum.x, -sum.y));
            if (vo) {
                const float2 d = qam_decide(cmul(yo, r), qm);
                es[n_out + jo] = csub(cmulc(d, r), yo);
            }
        }
        __syncthreads();

        // gradient partials
        if (grad_on) {
            const float2* xg = xs + goff;
            float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
            float2 cc0 = make_float2(0.0f, 0.0f), cc1 = make_float2(0.0f, 0.0f);   // conjugate taps: e x
#pragma unroll
            for (int i = 0; i < S::NG; ++i) {
                if (gg + S::G * i < L) {
                    const float2 e = es[gg + S::G * i];
                    const float2 xv = xg[2 * S::G * i];
                    if (i & 1) acc1 = cmacc(acc1, e, xv);
                    else acc0 = cmacc(acc0, e, xv);
                    if constexpr (WL) {
                        if (i & 1) cc1 = cmac(cc1, e, xv);
                        else cc0 = cmac(cc0, e, xv);
                    }
                }
            }
            part[gg * NTAP + gt] = cadd(acc0, acc1);
            if constexpr (WL) part[gg * NTAP + 2 * T + gt] = cadd(cc0, cc1);
        }
        __syncthreads();
        if (tid < 2 * T) {
            float2 g = part[tid];
#pragma unroll
            for (int k = 1; k < S::G; ++k) g = cadd(g, part[k * NTAP + tid]);
            const float2 h = taps[tid];
            const float2 hn = make_float2(fmaf(a.mu, g.x, h.x), fmaf(a.mu, g.y, h.y));
            taps[tid] = hn;
            *tps_at(tid) = hn;
            if constexpr (WL) {
                float2 gc = part[2 * T + tid];
#pragma unroll
                for (int k = 1; k < S::G; ++k) gc = cadd(gc, part[k * NTAP + 2 * T + tid]);
                const float2 hc = taps[2 * T + tid];
                const float2 hcn = make_float2(fmaf(a.mu_c, gc.x, hc.x), fmaf(a.mu_c, gc.y, hc.y));
                taps[2 * T + tid] = hcn;
                *tps_at(2 * T + tid) = hcn;
            }
        }
        if (b + 1 < nblk) commit(xsb + ((b + 1) & 1) * WBUF, b + 1);
        __syncthreads();
    }
    if (seg == nseg - 1 && a.taps_out)
        for (int t = tid; t < NTAP; t += NT) a.taps_out[q * NTAP + t] = taps[t];
}

// the compile-time kernel keeps one derotation base per block of a CTA: at most NBT blocks
template <int LB>
inline bool lms_fast_fits(const LmsArgs& a) {
    return (a.L_seg + LB - 1) / LB + a.n_wu <= 256;
}

template <int NT, int T, int LB, bool WL = false>
cudaError_t launch_lms_fast_t(const LmsArgs& a, cudaStream_t s) {
    using S = LmsFastShape<NT, T, LB, WL>;
    const int64_t nseg = (a.n_sym + a.L_seg - 1) / a.L_seg;
    if (nseg <= 0) return cudaSuccess;
    const size_t smem = lms_launch_smem(sizeof(float2) * S::SMEM, a.exclusive);
    static size_t attr = 0;
    if (smem > 48 * 1024 && smem > attr) {
        cudaFuncSetAttribute(k_lms_fast<NT, T, LB, WL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    k_lms_fast<NT, T, LB, WL><<<dim3((unsigned)nseg, 2), NT, smem, s>>>(a);
    return cudaGetLastError();
}
