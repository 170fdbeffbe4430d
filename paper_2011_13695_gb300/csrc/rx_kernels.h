// Host-side launchers of the librx kernels (one translation unit per stage group).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rx_dev.cuh"

// launch as a programmatic dependent of the stream's previous kernel (the kernel calls pdl_wait first)
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

struct CdcArgs {
    const void* in;        // [2][S] input samples
    int fmt;               // rx_input
    float in_scale;
    int64_t S;             // samples per polarisation in this frame
    int nfft;
    const float2* H;       // [nfft] FD filter, 1/nfft folded in
    const float2* tw;      // twiddle table
    const float2* tail;    // [2][nfft/2] carried scaled input (stream) or null (single frame)
    float2* out;           // buffer base; polarisation p writes out + p*ostride + obase
    int64_t ostride, obase;
    RxDevState* st;
    int64_t j0 = 0;        // first overlap-save block of this launch
    int64_t nblk = -1;     // blocks of this launch (-1: every block from j0 to the end of the frame)
};

struct LmsArgs {
    const float2* x;       // equaliser buffer base (polarisation stride xstride)
    int64_t xstride, xlen; // valid buffer indices [0, xlen)
    int64_t off;           // buffer index of symbol 0: off + 2n + c - k
    int T, Lb;
    int64_t n_sym;         // symbols the segments cover
    int64_t L_seg;         // symbols per segment
    int n_wu;              // warm-up blocks ahead of segments s >= 1
    int cma;               // 1 = CMA error, 0 = DD error
    float mu, R2;
    int m;
    int derotate;          // 1: multiply the input by the state's phase accumulator conjugate
    long long g0;          // input-sample index of buffer index 0
    const float2* taps_in; // [2][2][T]
    float2* taps_out;      // final taps of the last segment (may alias taps_in)
    float2* y;             // outputs [2][ystride] (nullable)
    int64_t ystride;
    const int* run_if;     // nullable: the kernel does nothing unless *run_if != 0
    RxDevState* st;
    int exclusive;         // 1: each CTA asks for a whole SM's shared memory, so that no other kernel's
                           // CTA shares its SM (the serial acquisition is latency-bound)
    float mu_c;            // widely-linear form only: step of the conjugate taps
    int npol = 2;          // input polarisations; 1 (generic kernel only): the second input plane reads as
                           // zero and only output row 0 runs, i.e. the single-polarisation equaliser
    int pdl = 0;           // tiled kernel only: launched as a programmatic dependent of the stream's previous
                           // kernel (its CTAs become resident early, issue their first window copies, and wait
                           // for that kernel's completion before reading anything else); x must not be
                           // written by that kernel
};

// shared memory a launch asks for: the kernel's need, or with `exclusive` the most a CTA may have
size_t lms_launch_smem(size_t need, int exclusive);

// A0 power of the first n_win samples; thread 0 of the first CTA also starts the frame's state (single:
// forget the unwrap carry and the alignment; always: forget the FO code and the CMA rerun)
cudaError_t launch_power(const void* in, int fmt, float in_scale, int64_t S, int64_t n_win, RxDevState* st,
                         int single, cudaStream_t s);
cudaError_t launch_cdc(const CdcArgs& a, cudaStream_t s);
cudaError_t launch_tail(const void* in, int fmt, float in_scale, int64_t S, int hop, float2* tail,
                        const RxDevState* st, cudaStream_t s);
cudaError_t launch_copy_hist(float2* buf, int64_t stride, int64_t S, int hist, cudaStream_t s);
cudaError_t launch_fill_twiddles(float2* tw, cudaStream_t s);
cudaError_t launch_fill_filter(float2* H, int nfft, double fs, double dl_lambda2_over_c, double rs, double rolloff,
                               cudaStream_t s);

cudaError_t launch_lms(const LmsArgs& a, int threads, cudaStream_t s);
int64_t lms_smem_bytes(int T, int Lb, int threads, bool wl = false);
// FFT size of a Kramers-Kronig front-end handle (k_kk.cu)
struct rx_kk;
int kk_fft_size(const rx_kk* k);
// widely-linear segmented DD-LMS: taps_in/taps_out are [2][4][T] (h_q0, h_q1, g_q0, g_q1 per row),
// mu_c the conjugate taps' step; threads 0 (choose), 128/256 for the compile-time shapes, else
// 256/512/1024 and >= 4T
cudaError_t launch_lms_wl(const LmsArgs& a, int threads, cudaStream_t s);
// the generic widely-linear kernel alone (any npol), threads 256/512/1024 and >= 4T
cudaError_t launch_lms_wl_generic(const LmsArgs& a, int threads, cudaStream_t s);

// A3 on the fixed CMA taps in one launch (a cluster of CTAs joined through distributed shared memory):
// the window outputs, the 4th-power periodogram of N = 2^kf points, its first maximum, the per-block
// phase slope, the code, the phase increment and the corrected taps
struct FoeArgs {
    const float2* x;       // equaliser input buffer (polarisation stride xstride), valid [0, xlen)
    int64_t xstride, xlen, off;
    int T;
    int64_t n0, nw;        // window: outputs n0 .. n0 + nw - 1 (2 nw <= 2^kf)
    const float2* taps;    // [2][2][T] fixed taps
    float2* yw;            // [2][nw] window outputs
    const float2* tw;      // FFT twiddle table
    int Lb;                // symbols per block of the fine stage
    double u_scale;        // Rs / (2 pi) / grid: rad/symbol to grid steps
    double f_scale;        // grid / fs: code to turns per sample
    RxDevState* st;
};
cudaError_t launch_foe(const FoeArgs& a, int kf, cudaStream_t s);
// the singularity check of the CMA outputs; pass 0 also rebuilds the second row into taps_init when the
// outputs correlate (the rerun's start)
cudaError_t launch_cma_check(const float2* yacq, int64_t ystride, int64_t nacq, int T, RxDevState* st,
                             int* flag_dev, int pass, cudaStream_t s);

cudaError_t launch_bps(const float2* y, int64_t ystride, int64_t N, int B, int W, int m, uint8_t* bstar,
                       int64_t bstride, cudaStream_t s);
// A5 unwrap and derotation in two passes; tile_sums holds 2 * ceil(N / 1024) + 4 ints (the per-tile
// jump sums, then a snapshot of the carried (b*, m) of each polarisation)
cudaError_t launch_unwrap(const float2* y, int64_t ystride, const uint8_t* bstar, int64_t bstride, int64_t N,
                          int B, int* tile_sums, int* m_out, int64_t mstride, float2* z, int64_t zstride,
                          RxDevState* st, cudaStream_t s, int* nlaunch);

// A6 alignment search; counts holds 16 * (2 * RX_MAX_DELAY + 1) + 1 ints, zero on entry and on return
// (the match counts, then the last-CTA arrival ticket)
cudaError_t launch_sync(const float2* z, int64_t zstride, const uint32_t* ref, int64_t refstride, int64_t n_ref,
                        int m, int64_t lo, int64_t hi, int max_delay, int64_t lat, int* counts, RxDevState* st,
                        cudaStream_t s, int* nlaunch);
cudaError_t launch_count(const float2* z, int64_t zstride, int64_t N, const uint32_t* ref, int64_t refstride,
                         int64_t n_ref, int m, int64_t lo, int64_t hi, int64_t lat, uint32_t* out,
                         int64_t outstride, RxDevState* st, cudaStream_t s);
