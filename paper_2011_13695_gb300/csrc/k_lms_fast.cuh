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
#pragma once

#include "rx_kernels.h"

template <int NT, int T, int LB>
struct LmsFastShape {
    static constexpr int C = (T - 1) / 2;
    static constexpr int XW = 2 * LB + T - 1;             // window samples per polarisation
    static constexpr int XS = 2 * LB + T;                 // staging stride per polarisation
    static constexpr int XE = (XW + 1) / 2;                // even-indexed samples first, odd ones at XE
    static constexpr int P = NT / LB;                      // lanes per output
    static constexpr int PH = P >= 2 ? P / 2 : 1;          // lanes per polarisation (P >= 2)
    static constexpr int KC = 2 * ((T + 2 * PH - 1) / (2 * PH));   // taps per lane (even, P >= 2)
    static constexpr int G = NT / (2 * T);                 // gradient groups
    static constexpr int NG = (LB + G - 1) / G;            // symbols per group
    static constexpr int PF = (2 * XW + NT - 1) / NT;      // window registers per thread
    static constexpr int NWARP = NT / 32;
    static constexpr int SMEM = 2 * T + 8 * XS + LB + G * 2 * T + NWARP + XW;   // float2 elements
    static_assert(NT % LB == 0 && (P & (P - 1)) == 0 && P <= 32, "NT must be a power-of-two multiple of LB");
    static_assert(G >= 1, "at least 2T threads");
    static_assert(T % 2 == 1, "odd tap count: window index parity follows the tap index");
};

template <int NT, int T, int LB>
__global__ void __launch_bounds__(NT) k_lms_fast(LmsArgs a) {
    using S = LmsFastShape<NT, T, LB>;
    extern __shared__ float2 smem[];
    if (a.run_if && *a.run_if == 0) return;
    float2* taps = smem;                                   // [p][k]
    float2* xsb = taps + 2 * T;                            // two windows of [2][XS] natural + [2][XS] split
    float2* es = xsb + 8 * S::XS;                          // [LB]
    float2* part = es + LB;                                // [G][2T]
    float2* ypart = part + S::G * 2 * T;                   // [NWARP]
    float2* tab = ypart + S::NWARP;                        // [XW]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = blockIdx.y;
    const Qam qm = make_qam(a.m);
    const long long inc = a.derotate ? a.st->nco_inc : 0;
    for (int t = tid; t < 2 * T; t += NT) taps[t] = a.taps_in[q * 2 * T + t];
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
    auto commit = [&](float2* xs, int64_t n0) {
        const long long g0 = a.g0 + a.off + 2 * n0 - S::C;
        const float2 base = inc ? nco_conj(inc, g0) : make_float2(1.0f, 0.0f);
#pragma unroll
        for (int r = 0; r < S::PF; ++r) {
            const int t = tid + r * NT;
            if (t < 2 * S::XW) {
                const int p = t >= S::XW ? 1 : 0, jj = t - p * S::XW;
                float2 v = pf[r];
                if (inc) v = cmul(v, cmul(base, tab[jj]));
                xs[p * S::XS + jj] = v;
                xs[(2 + p) * S::XS + ((jj & 1) ? S::XE + (jj >> 1) : (jj >> 1))] = v;
            }
        }
    };

    __syncthreads();                                       // taps and table
    if (nblk > 0) {
        prefetch(nfirst);
        commit(xsb, nfirst);
    }
    __syncthreads();

    // Each window is staged twice: in natural order [p][jj] (the gradient's lanes run over taps, so
    // consecutive lanes read consecutive samples) and split by parity, sample jj at jj / 2 (even jj)
    // or XE + jj / 2 (odd jj) of [2 + p] (the outputs' lanes run over n, so the samples x_p[2n + c - k]
    // of consecutive outputs are consecutive); the parity of the window index 2n + T - 1 - k is k's.
    // Output role: output n_out of the block, lane j of its P lanes; for P >= 2 the lane takes
    // polarisation j / PH and taps k = h KC + i, h = j % PH (KC even, so k and i share parity).
    const int n_out = tid / S::P, j = tid % S::P;
    const int op = S::P >= 2 ? j / S::PH : 0, oh = S::P >= 2 ? j % S::PH : 0;
    const int olim = T - oh * S::KC;                      // taps i < olim exist for this lane
    // gradient role: tap t = (p, k), symbols n = g (mod G)
    const int gg = tid / (2 * T), gt = tid - gg * 2 * T;
    const bool grad_on = gg < S::G;
    const int gp = gt >= T ? 1 : 0, gk = gt - gp * T;
    const int goff = gp * S::XS + T - 1 - gk + 2 * gg;     // natural copy: x_p[2n + c - k], n = gg + G i

    for (int b = 0; b < nblk; ++b) {
        const int64_t n0 = nfirst + (int64_t)b * LB;
        const int L = b < nwarm ? LB : (int)min((int64_t)LB, end - n0);
        float2* xs = xsb + (b & 1) * 4 * S::XS;
        if (b + 1 < nblk) prefetch(n0 + LB);

        // outputs
        const bool valid = n_out < L;
        float2 y;
        {
            float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
            if constexpr (S::P == 1) {
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float2* be = xs + (2 + p) * S::XS + n_out + S::C;      // even taps: be[-k/2]
                    const float2* bo = be + S::XE;                               // odd taps: bo[-(k+1)/2]
#pragma unroll
                    for (int k = 0; k < T; ++k) {
                        const float2 xv = (k & 1) ? bo[-((k + 1) >> 1)] : be[-(k >> 1)];
                        if (k & 1) acc1 = cmac(acc1, taps[p * T + k], xv);
                        else acc0 = cmac(acc0, taps[p * T + k], xv);
                    }
                }
            } else {
                const float2* be = xs + (2 + op) * S::XS + n_out + S::C - ((oh * S::KC) >> 1);
                const float2* bo = be + S::XE;
                const float2* hp = taps + op * T + oh * S::KC;
#pragma unroll
                for (int i = 0; i < S::KC; ++i) {
                    if (i < olim) {
                        const float2 xv = (i & 1) ? bo[-((i + 1) >> 1)] : be[-(i >> 1)];
                        if (i & 1) acc1 = cmac(acc1, hp[i], xv);
                        else acc0 = cmac(acc0, hp[i], xv);
                    }
                }
            }
            y = cadd(acc0, acc1);
#pragma unroll
            for (int w = 1; w < S::P; w <<= 1) {
                y.x += __shfl_xor_sync(0xffffffffu, y.x, w);
                y.y += __shfl_xor_sync(0xffffffffu, y.y, w);
            }
        }
        const bool owner = valid && j == 0;
        if (owner && b >= nwarm && a.y != nullptr) a.y[(int64_t)q * a.ystride + n0 + n_out] = y;
        if (a.cma) {
            if (owner) es[n_out] = cscale(y, a.R2 - cabs2(y));
        } else {
            float2 c4 = make_float2(0.0f, 0.0f);
            if (owner) {
                const float2 y2 = cmul(y, y);
                c4 = cmul(y2, y2);
            }
            c4.x = warp_sum(c4.x);
            c4.y = warp_sum(c4.y);
            if (lane == 0) ypart[warp] = c4;
            __syncthreads();
            float2 sum = ypart[0];
#pragma unroll
            for (int w = 1; w < S::NWARP; ++w) sum = cadd(sum, ypart[w]);
            const float2 r = quarter_root_conj(make_float2(-sum.x, -sum.y));
            if (owner) {
                const float2 d = qam_decide(cmul(y, r), qm);
                es[n_out] = csub(cmulc(d, r), y);
            }
        }
        __syncthreads();

        // gradient partials
        if (grad_on) {
            const float2* xg = xs + goff;
            float2 acc0 = make_float2(0.0f, 0.0f), acc1 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < S::NG; ++i) {
                if (gg + S::G * i < L) {
                    const float2 e = es[gg + S::G * i];
                    const float2 xv = xg[2 * S::G * i];
                    if (i & 1) acc1 = cmacc(acc1, e, xv);
                    else acc0 = cmacc(acc0, e, xv);
                }
            }
            part[gg * 2 * T + gt] = cadd(acc0, acc1);
        }
        __syncthreads();
        if (tid < 2 * T) {
            float2 g = part[tid];
#pragma unroll
            for (int k = 1; k < S::G; ++k) g = cadd(g, part[k * 2 * T + tid]);
            const float2 h = taps[tid];
            taps[tid] = make_float2(fmaf(a.mu, g.x, h.x), fmaf(a.mu, g.y, h.y));
        }
        if (b + 1 < nblk) commit(xsb + ((b + 1) & 1) * 4 * S::XS, n0 + LB);
        __syncthreads();
    }
    if (seg == nseg - 1 && a.taps_out)
        for (int t = tid; t < 2 * T; t += NT) a.taps_out[q * 2 * T + t] = taps[t];
}

template <int NT, int T, int LB>
cudaError_t launch_lms_fast_t(const LmsArgs& a, cudaStream_t s) {
    using S = LmsFastShape<NT, T, LB>;
    const int64_t nseg = (a.n_sym + a.L_seg - 1) / a.L_seg;
    if (nseg <= 0) return cudaSuccess;
    const size_t smem = sizeof(float2) * S::SMEM;
    static bool attr = false;
    if (smem > 48 * 1024 && !attr) {
        cudaFuncSetAttribute(k_lms_fast<NT, T, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    k_lms_fast<NT, T, LB><<<dim3((unsigned)nseg, 2), NT, smem, s>>>(a);
    return cudaGetLastError();
}
