/*
 * rx.h - C ABI of librx, a dual-polarisation coherent receiver for sm_103a.
 *
 * One handle processes frames of 2 samples/symbol complex ADC samples of two
 * polarisations into decided bits, with BER/EVM counters:
 *
 *   A0  power normalisation of the ADC samples
 *   A1  overlap-save frequency-domain chromatic-dispersion compensation with
 *       the RRC matched filter (paper Sec. III-A: 1024-point FFT, "100 %"
 *       overlap-save, 512 valid samples per block, FD multiply with 128-bit
 *       accesses; Sec. IV-C: matched filtering in the FD static filter)
 *   A2  2x2 butterfly FIR MIMO: CMA acquisition, then block DD-LMS
 *   A3  frequency-offset estimate (4th-power periodogram peak + 4th-power
 *       phase slope) and derotation by a 64-bit fixed-point phase accumulator
 *   A4  segmented block DD-LMS with in-loop 4th-power block phase (the paper's
 *       serial TD DD-LMS with warp shuffles, Sec. IV-D, made parallel by a
 *       fixed segment schedule)
 *   A5  blind phase search with an exact integer unwrap (the paper's serial
 *       warp-level phase unwrap, Sec. III-B, becomes a parallel scan)
 *   A6  polarisation/rotation/delay alignment, Gray demapping, bit and symbol
 *       error counting (Sec. II-D Step 6; Q from BER, Sec. V-D)
 *
 * Conventions (all entry points):
 *  - Every pointer named d_* is DEVICE memory on the handle's device, owned by
 *    the caller; every pointer named h_* is HOST memory owned by the caller.
 *  - Sample layout: [2 polarisations][S] contiguous, S = 2 * n_sym samples per
 *    polarisation; complex samples are interleaved (I, Q) pairs of the input
 *    format (float32, float16 or int8).
 *  - Bit layout: [2][ceil(n_sym * m / 32)] uint32 words, bit i of a
 *    polarisation is bit (i % 32) of word i / 32; symbol n carries bits
 *    n*m .. n*m+m-1, the first m/2 are the Gray word of the in-phase level
 *    (MSB first), the last m/2 that of the quadrature level.
 *  - Work is enqueued on the caller's stream and is asynchronous; rx_process
 *    neither allocates nor synchronises. Handles are not thread-safe.
 *  - Errors are returned as rx_status and never thrown across the ABI.
 *    Faults seen on the device (non-finite input, a failed alignment) set
 *    bits of the error word reported by rx_stats.
 */
#ifndef RX_H
#define RX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* rx_stream_t; /* same object as cudaStream_t */
typedef struct rx_handle rx_handle;

typedef enum {
    RX_OK = 0,
    RX_EINVAL = -1,   /* bad argument or configuration */
    RX_ENOMEM = -2,   /* device allocation failed in rx_create */
    RX_ECUDA = -3,    /* a CUDA call failed; rx_stats reports the CUDA error text */
    RX_ETIMEOUT = -4, /* a bounded device wait gave up */
    RX_ESTATE = -5    /* call out of order (e.g. a state blob of another config) */
} rx_status;

typedef enum { RX_IN_C64 = 0, RX_IN_F16 = 1, RX_IN_I8 = 2 } rx_input;

/* Device error word bits (rx_stats.error_word). */
#define RX_ERR_NONFINITE 0x1u   /* a non-finite sample reached the equaliser */
#define RX_ERR_SYNC_LOST 0x2u   /* best alignment matched < 90 % of the sync window */
#define RX_ERR_SINGULAR 0x4u    /* CMA outputs still correlated after the rerun */
#define RX_ERR_TIMEOUT 0x8u     /* a bounded wait inside a pipelined kernel ran out; outputs invalid */

typedef struct rx_config {
    int32_t bits_per_sym;       /* m per polarisation: 2 (QPSK), 4 (16QAM), 6 (64QAM) */
    int32_t sps;                /* samples per symbol; must be 2 */
    double symbol_rate_hz;      /* Rs */
    double wavelength_m;        /* lambda, for the dispersion filter */
    double dispersion_s_per_m2; /* D (17e-6 = 17 ps/nm/km) */
    double length_m;            /* L; H_cdc = exp(+j pi D L lambda^2 f^2 / c) */
    double rrc_rolloff;         /* matched filter in the FD stage; 0 = none */
    int32_t fft_size;           /* FD block N = 2^K, 512..8192; keeps N/2 per block */
    int32_t n_taps;             /* T, odd, 3..63 */
    int32_t lms_block;          /* L_b symbols per block update, 16..256 */
    int32_t cma_blocks;         /* CMA acquisition blocks (first frame) */
    int32_t dd_acq_blocks;      /* DD-LMS acquisition blocks (first frame) */
    int32_t seg_blocks;         /* blocks per DD-LMS segment */
    int32_t warmup_blocks;      /* warm-up blocks ahead of every segment but the first */
    int32_t bps_phases;         /* B test phases, 2..64 */
    int32_t bps_window;         /* W symbols, a power of two, 2..64 */
    int32_t edge_skip;          /* E: symbols left out of the counts at each frame edge */
    int32_t sync_len;           /* symbols of the alignment window, 1..32768 */
    int32_t max_delay;          /* alignment searches delays in [-max_delay, max_delay] */
    float mu_cma;               /* CMA step */
    float mu_dd;                /* DD-LMS step */
    double fo_grid_hz;          /* frequency-offset quantum (code * grid = offset) */
    int32_t input_format;       /* rx_input */
    float input_scale;          /* multiplies every input value (e.g. the int8 step) */
    int32_t streaming;          /* 0: each call is one frame; 1: calls are frames of one stream */
    int64_t max_symbols;        /* largest n_sym per call (sizes the workspace) */
    int32_t lms_threads;        /* threads per CTA of the segmented DD-LMS: 128/256/512/1024; 0 = 256 */
} rx_config;

typedef struct rx_stats_t {
    uint64_t frames;            /* rx_process calls since create/reset */
    uint64_t symbols_processed; /* 2 * sum of n_sym */
    uint64_t bits_processed;    /* m * symbols_processed */
    uint64_t bits_counted;      /* bits inside the counted windows */
    uint64_t bit_errors;
    uint64_t symbols_counted;
    uint64_t symbol_errors;
    double evm_num, evm_den;    /* sum |z - s|^2 and sum |s|^2 over the counted symbols */
    double ber;                 /* bit_errors / bits_counted */
    double evm;                 /* sqrt(evm_num / evm_den) */
    double q_db;                /* 20 log10(sqrt(2) erfcinv(2 BER)); +inf when BER = 0 */
    int32_t fo_code;            /* frequency offset = fo_code * fo_grid_hz */
    double fo_hz;
    int32_t pol_map[2];         /* tx polarisation of each output */
    int32_t rotation[2];        /* quarter turns applied to each output */
    int32_t delay[2];           /* symbol delay of each output */
    int32_t sync_matches[2];    /* decisions matching in the sync window */
    int32_t sync_len;           /* length of the sync window used */
    int32_t cma_reran;          /* 1 if the singularity check restarted CMA */
    float cma_rho;              /* output correlation after the first CMA pass */
    int32_t latency_symbols;    /* output delay of a stream (0 for single frames) */
    uint32_t error_word;        /* RX_ERR_* bits */
} rx_stats_t;

/* Internal buffers that rx_get_buffer can export (for inspection and tests). */
typedef enum {
    RX_BUF_CDC = 0,      /* float2 [2][S]   A1 output of the last frame */
    RX_BUF_Y = 1,        /* float2 [2][N]   A4 equaliser output (P1) */
    RX_BUF_Z = 2,        /* float2 [2][N]   A5 carrier-recovered symbols (P2) */
    RX_BUF_BSTAR = 3,    /* uint8  [2][N]   A5 chosen test phase */
    RX_BUF_M = 4,        /* int32  [2][N]   A5 unwrap quarter-turn count */
    RX_BUF_TAPS_CMA = 5, /* float2 [2][2][T] taps after CMA (first frame) */
    RX_BUF_TAPS_INIT = 6,/* float2 [2][2][T] taps the segments start from */
    RX_BUF_TAPS_LAST = 7,/* float2 [2][2][T] final taps of the last segment */
    RX_BUF_Y_ACQ = 8,    /* float2 [2][N_acq] CMA outputs while adapting */
    RX_BUF_Y_FOE = 9,    /* float2 [2][N_acq/2] fixed-tap outputs the FO estimate uses */
    RX_BUF_SCALE = 10    /* float  [2]      A0 scale */
} rx_buffer;

/*
 * rx_create: validate *cfg, allocate every device buffer the handle will use
 * (sized by cfg->max_symbols) on the current device and precompute the FD
 * filter. No allocation happens after this call. Returns RX_EINVAL for an
 * invalid configuration, RX_ENOMEM when the device is out of memory.
 * The caller owns *out and frees it with rx_destroy.
 */
rx_status rx_create(const rx_config* cfg, rx_handle** out);

/*
 * rx_process: run the chain A0-A6 on one frame of n_sym symbols per
 * polarisation (d_in: [2][2*n_sym] samples of cfg->input_format).
 * d_ref_bits (nullable): the transmitted bits in the bit layout above; when
 * given, the frame is aligned (first frame of a stream, or every call in
 * single-frame mode) and errors are counted on [E, n_sym - E).
 * d_out_bits (nullable): receives the decided bits of each output
 * polarisation, quarter turn applied, in output order.
 * Asynchronous on `stream`; RX_EINVAL for n_sym < 1, n_sym > max_symbols or
 * (streaming) n_sym not a multiple of fft_size / 4.
 * Single-frame handles record the frame's launches as a CUDA graph on the
 * first call with a given (d_in, n_sym, d_ref_bits, d_out_bits) and replay it
 * on later calls with the same pointers and length (the data may change);
 * when the pointers change on three calls in a row, or a capture fails, the
 * handle launches directly from then on. Calls on a stream that the caller is
 * capturing always launch directly into that capture.
 */
rx_status rx_process(rx_handle* h, const void* d_in, int64_t n_sym, const uint32_t* d_ref_bits,
                     uint32_t* d_out_bits, rx_stream_t stream);

/*
 * rx_process_host: the same frame from HOST buffers. Copies h_in (and
 * h_ref_bits, nullable) to handle-owned device staging buffers on `stream`,
 * runs rx_process and copies the decided bits back to h_out_bits (nullable).
 * Asynchronous: the host buffers must stay valid until the stream reaches
 * this point (pinned memory makes the copies asynchronous).
 */
rx_status rx_process_host(rx_handle* h, const void* h_in, int64_t n_sym, const uint32_t* h_ref_bits,
                          uint32_t* h_out_bits, rx_stream_t stream);

/*
 * rx_decide: stage A6 alone (alignment, Gray demap, bit/symbol error and EVM
 * counting) on carrier-recovered symbols the caller supplies, e.g. the output
 * of the learned post-equaliser: d_z is DEVICE float [2][n_sym][2]. Counts
 * accumulate into the handle's statistics like rx_process's. Single-frame
 * handles only (RX_EINVAL for streaming handles).
 */
rx_status rx_decide(rx_handle* h, const float* d_z, int64_t n_sym, const uint32_t* d_ref_bits, uint32_t* d_out_bits,
                    rx_stream_t stream);

/* rx_stats: wait for the last stream used by the handle, then fill *out. */
rx_status rx_stats(rx_handle* h, rx_stats_t* out);

/*
 * rx_get_buffer: enqueue a device-to-device copy of an internal buffer
 * (rx_buffer) of the last frame into d_dst (bytes must equal the buffer
 * size, which rx_buffer_bytes returns). Not part of the timed path.
 */
rx_status rx_buffer_bytes(rx_handle* h, int32_t which, int64_t* bytes);
rx_status rx_get_buffer(rx_handle* h, int32_t which, void* d_dst, int64_t bytes, rx_stream_t stream);

/* rx_reset: forget the stream state and zero the counters (synchronous). */
rx_status rx_reset(rx_handle* h);

/*
 * Checkpoint/resume of a stream: rx_state_size gives the blob size; get
 * copies the carried state (dispersion tail, equaliser history, taps, FO
 * code, unwrap state, alignment, counters) to host memory; set restores it
 * into a handle created with the same configuration (RX_ESTATE otherwise).
 * Both synchronise the handle's last stream.
 */
rx_status rx_state_size(rx_handle* h, size_t* bytes);
rx_status rx_state_get(rx_handle* h, void* h_blob, size_t bytes);
rx_status rx_state_set(rx_handle* h, const void* h_blob, size_t bytes);

/*
 * Per-stage timing: with timing on, rx_process records CUDA events around
 * each stage on the caller's stream; rx_stage_times returns, per stage, the
 * total milliseconds and launch count since timing was switched on
 * (synchronises). Stage names come from rx_stage_name.
 */
rx_status rx_set_timing(rx_handle* h, int32_t enable);
int32_t rx_stage_count(void);
const char* rx_stage_name(int32_t stage);
rx_status rx_stage_times(rx_handle* h, double* ms, int64_t* launches, int32_t n);

/* Kernels launched by this handle since creation (all stages). */
uint64_t rx_launch_count(rx_handle* h);

/*
 * Batched channels. The paper keeps its GPU busy with one stream per buffer
 * and events between dependent kernels (Sec. II-C, Sec. III); a batch runs
 * many independent channels (single frames, each with its own format,
 * symbol rate, taps, dispersion and length) as ONE CUDA graph launch.
 *
 * rx_batch_create: n configurations (streaming must be 0). A channel with
 * fft_size == 0 gets the fastest N_fft in 512..8192 whose N/4 covers its
 * dispersion memory, and lms_threads == 0 the fastest DD-LMS CTA size, both
 * timed on the device at create time and cached per channel shape for the
 * process. Allocates every handle's workspace; RX_EINVAL on a bad config.
 * rx_batch_config returns channel i's configuration as tuned.
 */
typedef struct rx_batch rx_batch;
rx_status rx_batch_create(const rx_config* cfgs, int32_t n, rx_batch** out);
rx_status rx_batch_config(rx_batch* b, int32_t i, rx_config* out);
/* the handle of channel i (for rx_get_buffer); owned by the batch */
rx_handle* rx_batch_handle(rx_batch* b, int32_t i);
/*
 * rx_batch_process: d_in[i], n_sym[i], d_ref[i] (array or entries nullable),
 * d_out[i] (array or entries nullable) as for rx_process, per channel. The
 * first call with a given set of buffers and stream captures every channel's
 * chain (each on its own forked stream) into one graph; every call then
 * launches that graph once on `stream`. Asynchronous.
 */
rx_status rx_batch_process(rx_batch* b, const void* const* d_in, const int64_t* n_sym, const uint32_t* const* d_ref,
                           uint32_t* const* d_out, rx_stream_t stream);
/* rx_batch_stats: waits for the last batch launch, then rx_stats of channel i */
rx_status rx_batch_stats(rx_batch* b, int32_t i, rx_stats_t* out);
uint64_t rx_batch_launch_count(rx_batch* b);
void rx_batch_destroy(rx_batch* b);

/*
 * Learned post-equaliser (the paper has none): a 1-D CNN applied to the
 * carrier-recovered symbols z of both polarisations, out = z + f(z), with
 * f = conv(C->4) relu conv(C->C) relu conv(C->C) relu conv(4->C), kernel 9,
 * "same" zero padding, C = 64. Weights and activations BF16, products and
 * sums FP32, FP32 master weights updated by Adam (b1 0.9, b2 0.999, eps 1e-8)
 * on the mean squared error to the transmitted symbols.
 * Parameter order (h_params, d_grads): per layer W[out][in][9] then b[out],
 * layers 4->C, C->C, C->C, C->4; rx_pe_param_count gives the length.
 * Sequences: d_z, d_target, d_out are DEVICE float [2][T][2] (the layout of
 * rx_process's z), owned by the caller; T <= max_len given at create, which
 * allocates all working memory. Calls are asynchronous on `stream`.
 */
typedef struct rx_pe rx_pe;
int64_t rx_pe_param_count(int32_t channels, int32_t kernel);
rx_status rx_pe_create(int32_t channels, int32_t kernel, int64_t max_len, const float* h_params, rx_pe** out);
/* current FP32 master parameters into h_params (synchronises) */
rx_status rx_pe_params(rx_pe* p, float* h_params);
/* inference: d_out = d_z + f(d_z). Runs on the tcgen05 tensor cores with the hidden activations in
 * channel-chunk planes [C/8][T + 8][8]; training (rx_pe_gradients, rx_pe_train_step(s)) keeps its own
 * forward. */
rx_status rx_pe_forward(rx_pe* p, const float* d_z, int64_t T, float* d_out, rx_stream_t stream);
/* the post-equaliser's device error word (RX_ERR_TIMEOUT if a pipelined kernel gave up a wait;
 * synchronises) */
rx_status rx_pe_error_word(rx_pe* p, uint32_t* out);
/* loss (mean squared error) and its gradient w.r.t. every parameter, without updating them */
rx_status rx_pe_gradients(rx_pe* p, const float* d_z, const float* d_target, int64_t T, float* d_grads, float* d_loss,
                          rx_stream_t stream);
/* one Adam step on the sequence: forward, backward, update (d_loss nullable) */
rx_status rx_pe_train_step(rx_pe* p, const float* d_z, const float* d_target, int64_t T, float lr, float* d_loss,
                           rx_stream_t stream);
/* `steps` Adam steps in one call, step i on the window [offs[i], offs[i] + window) of the sequence pair
 * which[i]: d_z[k] and d_target[k] are device pointers to complex sequences [2][len[k]] (polarisation 1
 * at len[k] samples), read in place; host arrays which, offs, lrs (the step's learning rate) of `steps`
 * entries, d_losses (nullable) a device array of `steps` losses. The same steps as `steps` calls of
 * rx_pe_train_step on contiguous copies of the windows, bit for bit, without a host round trip or a
 * copy per step. RX_EINVAL for a window outside its sequence, a pair index outside [0, npairs) or
 * window > max_len. */
rx_status rx_pe_train_steps(rx_pe* p, const float* const* d_z, const float* const* d_target, const int64_t* len,
                            int32_t npairs, int64_t window, int32_t steps, const int32_t* which, const int64_t* offs,
                            const float* lrs, float* d_losses, rx_stream_t stream);
void rx_pe_destroy(rx_pe* p);

/*
 * rx_pe_targets: the post-equaliser's training labels on the device (no paper
 * counterpart: the paper has no learned equaliser). The label of output q at
 * index n is s_{p_q}[n + d_q] (-j)^{r_q}, the transmitted symbol that the
 * alignment of stage A6 (pol_map, rotation, delay as rx_stats reports them)
 * puts there, and 0 where n + d_q lies outside [0, n_ref). Each whole block of
 * `block` symbols is then turned by the quarter turn u in {1, j, -1, -j} that
 * minimises sum |z - label u|^2 over the block (the first minimum of FP32 sums
 * taken in a fixed order), so that labels follow a carrier slip of the chain
 * instead of teaching the network to undo it; a tail shorter than a block
 * keeps its labels. d_z: DEVICE float [2][n_sym][2] (I, Q) the chain's
 * carrier-recovered symbols; d_symbols: DEVICE float [2][n_ref][2] the
 * transmitted symbols; h_pol_map, h_rotation, h_delay: HOST int32 [2];
 * d_target: DEVICE float [2][n_sym][2] receives the labels (must not overlap
 * the inputs). Caller-owned; nothing is allocated; asynchronous on `stream`.
 * RX_EINVAL for NULL pointers, n_sym < 1, n_ref < 1, block < 1, a pol_map
 * entry outside {0, 1} or a rotation outside 0..3.
 */
rx_status rx_pe_targets(const float* d_z, int64_t n_sym, const float* d_symbols, int64_t n_ref,
                        const int32_t* h_pol_map, const int32_t* h_rotation, const int32_t* h_delay, int32_t block,
                        float* d_target, rx_stream_t stream);

/*
 * rx_fp32_fma_rate: measured FP32 FMA throughput of the current device (no
 * paper counterpart; the roofline of the chain's FP32-bound stages uses it).
 * One launch of every SM's worth of CTAs, each thread running eight
 * independent FMA chains of `iters` steps (packed != 0: fma.rn.f32x2, two
 * FMAs per instruction), timed with CUDA events after a warm-up launch.
 * *flops_per_s receives 2 flops per FMA over the timed launch; *ms
 * (nullable) its duration. Blocking (synchronises `stream`); allocates
 * nothing. RX_EINVAL for iters < 1 or a NULL flops_per_s.
 */
rx_status rx_fp32_fma_rate(int32_t packed, int32_t iters, double* flops_per_s, double* ms, rx_stream_t stream);

/*
 * rx_carrier_recovery_static: stage A5 alone (blind phase search, integer
 * unwrap, derotation) on one single frame of equalised symbols, for callers
 * that cannot allocate device memory when they process data (a real-time
 * ingest thread must not block in the CUDA allocator; some host frameworks
 * give the library a fixed memory budget at load time). The paper has no
 * counterpart: its kernels run inside a program that owns all its buffers.
 *
 * d_y: DEVICE float [2][n_sym][2] (I, Q) equalised symbols of the two
 * polarisations; d_z: DEVICE float [2][n_sym][2] receives the carrier-
 * recovered symbols; both owned by the caller. Same arithmetic and results
 * as the z of rx_process for the same y, with no carried unwrap state.
 * The working memory is one file-scope device array of RX_STATIC_MAX_SYMBOLS
 * symbols per polarisation (about 2.6 MB) that every device loading the
 * library keeps until the process exits; the function allocates nothing.
 * Its first call on a device looks up that array's device address, and with
 * lazy module loading (the CUDA default) it also loads the kernels it runs:
 * make one warm-up call on each device before any stream capture. Every call
 * shares the array (each call clears the carried unwrap state it uses):
 * calls that overlap on the GPU (other streams, other threads) race with
 * each other. `stream` must belong to the current device (RX_EINVAL
 * otherwise: the array's address is looked up per device).
 * RX_EINVAL for n_sym < 1, n_sym > RX_STATIC_MAX_SYMBOLS or invalid BPS
 * parameters (bps_phases 2..64, bps_window a power of two 2..64).
 * Asynchronous on `stream`.
 */
#define RX_STATIC_MAX_SYMBOLS 262144
rx_status rx_carrier_recovery_static(const float* d_y, int64_t n_sym, int32_t bits_per_sym, int32_t bps_phases,
                                     int32_t bps_window, float* d_z, rx_stream_t stream);

/*
 * rx_dd_lms_wl: the widely-linear form of stage A4 alone. Sec. IV-D's TD
 * equaliser is widely linear (it also undoes the transmitter's IQ
 * imbalance): every output adds conjugate taps to the 2x2 butterfly,
 *   y_q[n] = sum_p sum_k h_qp[k] x_p[2n + c - k] + g_qp[k] conj(x_p[2n + c - k]),
 * c = (T-1)/2, x zero outside [0, x_len), and per block of block_len symbols
 *   psi_q = arg(-sum_n y_q[n]^4) / 4,  d = dec(y e^{-j psi}),  e = d e^{j psi} - y,
 *   h_qp[k] += mu * sum_n e_q[n] conj(x_p[2n + c - k]),
 *   g_qp[k] += mu_conj * sum_n e_q[n] x_p[2n + c - k]
 * (the linear update on the augmented input [x, conj x]; the outputs of a
 * block use the taps it started with). Segment schedule as in rx_process:
 * segments of seg_blocks blocks all start from d_taps_in; every segment but
 * the first first runs warmup_blocks blocks on the symbols before it, whose
 * outputs are discarded. mu_conj = 0 with zero conjugate taps is the linear
 * DD-LMS.
 *
 * d_x: DEVICE float [2][x_len][2] (I, Q) input at 2 samples per symbol.
 * d_taps_in: DEVICE float [2 (q)][4][T][2]: per output row h_q0, h_q1, g_q0,
 * g_q1. d_y: DEVICE float [2][n_sym][2] outputs. d_taps_out: DEVICE, same
 * layout as d_taps_in, receives the last segment's final taps (NULL: not
 * written; must not overlap d_taps_in). All owned by the caller; nothing is
 * allocated. threads: CTA size. 0 lets the library choose (128 for the
 * compiled shapes, n_taps 15/21/31 with block_len 128, at most 256 blocks
 * per segment including warm-up; 256 otherwise); 128 or 256 run a compiled
 * shape; any other shape runs the generic kernel with 256, 512 or 1024
 * threads, at least 4 * n_taps. n_taps odd 3..63, block_len 16..256,
 * seg_blocks >= 1, warmup_blocks >= 0, bits_per_sym 2/4/6/8; RX_EINVAL
 * otherwise, for n_sym < 1, x_len < 1, a thread count the shape cannot use
 * or more than 2^31 - 1 segments. Asynchronous on `stream`.
 */
rx_status rx_dd_lms_wl(const float* d_x, int64_t x_len, int32_t n_taps, const float* d_taps_in, int64_t n_sym,
                       int32_t block_len, int32_t seg_blocks, int32_t warmup_blocks, int32_t bits_per_sym, float mu,
                       float mu_conj, float* d_y, float* d_taps_out, int32_t threads, rx_stream_t stream);

/*
 * Kramers-Kronig self-coherent front end (Sec. IV, Steps 1-8): one
 * polarisation at 4 samples/symbol, from the ADC's 12-bit unsigned codes to
 * the matched-filtered signal at 2 samples/symbol.
 *   Step 1: I[n] = max(code_scale * code[n] + dc_offset, min_intensity)
 *           (the static DC offset restores the term an AC-coupled digitiser
 *           drops); amplitude sqrt(I), log-amplitude ln sqrt(I).
 *   Steps 2-5: 100 % overlap-save blocks of N = fft_size samples (block j
 *           starts at j N/2 - N/4, zero outside the frame, keeps its centre
 *           N/2): FFT of the log-amplitude, times -j sgn(k) (0 at k = 0 and
 *           N/2), IFFT -> phase phi; field E[n] = sqrt(I[n]) exp(j phi[n])
 *           exp(-j 2 pi tone_over_fs n): the signal, which lies tone_over_fs
 *           above the carrier tone, moved to DC.
 *   Steps 6-8: second overlap-save pass on E: FFT, times 2 RRC(f_k)
 *           (matched filter of roll-off rrc_rolloff, symbol rate fs/4), the
 *           bins |f| < fs/4 into an N/2-point IFFT, i.e. 2 samples/symbol.
 * rx_kk_create: fft_size 1024..8192 (power of two; the paper uses 1024),
 * 0 < tone_over_fs < 0.5, 0 < rrc_rolloff <= 1, code_scale finite and
 * nonzero, dc_offset finite, min_intensity > 0; RX_EINVAL otherwise. It
 * allocates the twiddle table and the filter (RX_ENOMEM) and synchronises.
 * rx_kk_process: d_codes DEVICE uint16 [n_samples] (12-bit codes, 8-byte
 * aligned: read four at a time); first_sample: the stream index of
 * d_codes[0], which the downshift phase counts from (0 for a lone frame);
 * d_field
 * DEVICE float [n_samples][2] receives E (4 samples/symbol); d_out DEVICE
 * float [n_samples/2][2] the output (2 samples/symbol); all caller-owned.
 * n_samples even, 2..2^36; RX_EINVAL otherwise. No allocation;
 * asynchronous on `stream` (two kernel launches).
 */
typedef struct rx_kk rx_kk;
rx_status rx_kk_create(int32_t fft_size, double tone_over_fs, double rrc_rolloff, float code_scale, float dc_offset,
                       float min_intensity, rx_kk** out);
rx_status rx_kk_process(rx_kk* k, const uint16_t* d_codes, int64_t n_samples, int64_t first_sample, float* d_field,
                        float* d_out, rx_stream_t stream);
void rx_kk_destroy(rx_kk* k);
/*
 * rx_kk_equalise: Step 9 of the KK receiver (Sec. IV-D: a TD widely-linear
 * DD-LMS that also undoes the transmitter's IQ imbalance, then the decision
 * and demapping), on the front end's output at 2 samples/symbol:
 *   y[n] = sum_k h[k] x[2n + c - k] + g[k] conj(x[2n + c - k]),
 * c = (T-1)/2, x zero outside [0, x_len); per block of block_len symbols
 *   psi = arg(-sum_n y[n]^4) / 4,  d = dec(y e^{-j psi}),  e = d e^{j psi} - y,
 *   h[k] += mu sum_n e[n] conj(x[2n + c - k]),  g[k] += mu_conj sum_n e[n] x[2n + c - k];
 * the segment schedule of rx_dd_lms_wl (segments of seg_blocks blocks from
 * d_taps_in, warm-up blocks ahead of every segment but the first). The
 * decisions are the nearest square-QAM points of y (the front end keeps the
 * tone's phase, so no quarter-turn search), Gray-demapped.
 * d_x: DEVICE float [x_len][2] (I, Q), e.g. rx_kk_process's d_out;
 * d_taps_in: DEVICE float [2][T][2] (h, then g); d_y: DEVICE float
 * [n_sym][2] equalised symbols; d_bits: DEVICE uint32 [ceil(n_sym m / 32)]
 * decided bits in rx_process's layout for one polarisation (nullable);
 * d_taps_out: DEVICE, layout of d_taps_in, the last segment's final taps
 * (nullable). Caller-owned buffers; the taps pass through scratch the handle
 * allocated at rx_kk_create; nothing is allocated here. Runs the generic
 * widely-linear block-LMS kernel with one output row and one input
 * polarisation. n_taps odd 3..63, block_len 16..256, seg_blocks >= 1,
 * warmup_blocks >= 0, bits_per_sym 2/4/6/8; RX_EINVAL otherwise, for n_sym <
 * 1, x_len < 1 or a NULL handle, input, taps or output. Asynchronous on
 * `stream`; one handle's calls must not overlap (they share its scratch).
 */
rx_status rx_kk_equalise(rx_kk* k, const float* d_x, int64_t x_len, int32_t n_taps, const float* d_taps_in,
                         int64_t n_sym, int32_t block_len, int32_t seg_blocks, int32_t warmup_blocks,
                         int32_t bits_per_sym, float mu, float mu_conj, float* d_y, uint32_t* d_bits,
                         float* d_taps_out, rx_stream_t stream);

/*
 * rx_ingest_run: real-time ingest emulation (Sec. II-C, II-D). A digitiser
 * delivers n_buffers buffers of buffer_samples 12-bit codes at
 * sample_rate_hz (buffer i is ready buffer_samples * i / sample_rate_hz after
 * the start; its codes are h_source[(i * buffer_samples) mod
 * source_samples ...]). Each ready buffer takes a free one of n_streams GPU
 * slots (its own stream): copy in (the digitiser's DMA), the overlap step
 * (the last 2N codes of the previous buffer go in front, in buffer order,
 * through an event chain: each of the front end's two overlap-save passes
 * needs N/4 samples of context on either side of what a block keeps), the
 * KK front end of `kk` on the joined buffer, and the copy of its S/2 exact,
 * continuing outputs to host memory. A buffer that finds every slot busy is
 * dropped and the overlap chain restarts from zero codes: the first N/2
 * outputs of the stream from a (re)starting buffer's first sample on are a
 * start-up transient (the carry holds no data); every later output equals
 * that of the front end on the whole stream as one frame.
 * Output: buffer i's outputs are the 2-sample/symbol stream samples
 * [i S/2 - N/2, (i + 1) S/2 - N/2) (an N/2-sample delay), written
 * to h_out + i * S floats when h_out is not NULL (host, n_buffers * S/2
 * complex; dropped buffers leave theirs untouched). h_source (and h_out) are
 * page-locked (cudaHostRegister) at the start of every call and unlocked at
 * its end unless they already are page-locked: that costs host time before
 * pacing starts (it is not in the latency statistics), and a caller that
 * runs repeatedly passes memory it has already page-locked (cudaHostAlloc or
 * its own cudaHostRegister) to skip it. Blocking; it allocates
 * its slots before the first buffer and frees them at the end. RX_EINVAL for
 * buffer_samples not a multiple of N/2 or below 2N or above 2^30,
 * source_samples not a multiple of buffer_samples, sample_rate_hz <= 0,
 * n_streams outside 1..64 or n_buffers < 1.
 */
typedef struct rx_ingest_stats {
    uint64_t buffers;           /* buffers the digitiser delivered */
    uint64_t processed;         /* buffers that found a free slot */
    uint64_t dropped;           /* buffers lost: every slot busy */
    uint64_t pad0;
    double buffer_period_ms;    /* buffer_samples / sample_rate_hz */
    double mean_latency_ms;     /* ready -> outputs in host memory, processed buffers */
    double max_latency_ms;
    double wall_s;              /* the whole run */
} rx_ingest_stats;
rx_status rx_ingest_run(rx_kk* kk, const uint16_t* h_source, int64_t source_samples, int64_t buffer_samples,
                        double sample_rate_hz, int32_t n_streams, int64_t n_buffers, float* h_out,
                        rx_ingest_stats* stats);

/*
 * IM/DD PAM-M chain with frequency-domain clock recovery (Sec. III, Steps
 * 1-9), one real signal at 2 samples/symbol:
 *   Steps 1-2: v = code_scale * code + dc_offset; 100 % overlap-save blocks
 *     of N = fft_size (block j from j N/2 - N/4, zero outside the frame);
 *     FFT; the static FD equaliser as the RRC matched filter sqrt(2) RRC(f)
 *     (roll-off rrc_rolloff, symbol rate fs/2).
 *   Steps 3-4: clock product c_j = sum_{k < N/2} X_j[k] conj(X_j[k + N/2]);
 *     average over the 105 blocks |i - j| <= 52 inside the frame, phase
 *     phi_j = arg; winding numbers w_j from the unwrap steps (-1 when
 *     phi_j - phi_{j-1} > pi, +1 when < -pi).
 *   Steps 5-7: block spectrum times exp(-j phi_j f / Rs), IFFT; block j
 *     outputs the real parts of its samples N/4 + 2 i, i < N/4 + w_{j+1} -
 *     w_j (255, 256 or 257 symbols; the last block N/4, clipped to the
 *     frame), at offset j N/4 + w_j - w_0.
 *   Steps 8-9: u = (y - mean y) (M/2) / mean|y - mean y|; level index
 *     clip(rint((u + M - 1) / 2), 0, M - 1) (thresholds at the level
 *     midpoints; Gray word l ^ (l >> 1)).
 * rx_pam_create: fft_size 1024/2048/4096, levels 2/4/8, 0 < rrc_rolloff <=
 * 1, code_scale finite nonzero, dc_offset finite, max_samples 2..2^30;
 * allocates (RX_ENOMEM) and synchronises.
 * rx_pam_process: d_codes DEVICE uint16 [n_samples] (n_samples even, <=
 * max_samples); d_y DEVICE float (16-byte aligned) and d_levels DEVICE
 * uint8 (4-byte aligned), each with room for n_samples/2 +
 * n_samples/(fft_size/2) + 1 outputs; d_n_out DEVICE
 * int64 [1] receives the number of outputs. Asynchronous on `stream`, no
 * allocation. rx_pam_get copies one of the chain's internal arrays of the
 * last call (RX_PAM_*: float2 clock products, float phases, int32 winding
 * numbers, int64 offsets [blocks + 1], double [2] mean and mean absolute
 * deviation) into a DEVICE buffer; RX_EINVAL if bytes exceeds its size.
 */
typedef struct rx_pam rx_pam;
enum { RX_PAM_CLOCK = 0, RX_PAM_PHASE = 1, RX_PAM_WINDING = 2, RX_PAM_OFFSETS = 3, RX_PAM_STATS = 4 };
rx_status rx_pam_create(int32_t fft_size, int32_t levels, double rrc_rolloff, float code_scale, float dc_offset,
                        int64_t max_samples, rx_pam** out);
rx_status rx_pam_process(rx_pam* p, const uint16_t* d_codes, int64_t n_samples, float* d_y, uint8_t* d_levels,
                         int64_t* d_n_out, rx_stream_t stream);
rx_status rx_pam_get(rx_pam* p, int32_t which, void* d_dst, int64_t bytes, rx_stream_t stream);
void rx_pam_destroy(rx_pam* p);

void rx_destroy(rx_handle* h);
const char* rx_strerror(rx_status s);

#ifdef __cplusplus
}
#endif
#endif /* RX_H */
