/*
 * qrng.h -- C ABI of the GB300 QRNG post-processing library (libqrng_gb300.so).
 *
 * The library implements the data-parallel hot path of quantum-random-number post-processing:
 *   1. a min-entropy estimate of an ADC sample stream with the statistical-distance correction
 *      of Sec. II (histogram -> H_min -> Gaussian model -> d_U -> Delta H_m -> H_modify);
 *   2. Toeplitz-hashing randomness extraction k = T r (mod 2) over independent n-bit blocks of a
 *      raw bit stream (Sec. III.B standard matrix, Sec. III.D modified matrix (A, I_m),
 *      Sec. III.E block splitting).
 * Every step runs in CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Bits are packed LSB-first: bit t of a packed buffer is bit (t mod 8) of byte (t / 8).
 * 0-based indices: raw block r[0..n), seed a[0..L), output k[0..m).
 *   standard (Sec. III.B, T[i][j] = a_{n+i-j} 1-based):
 *       k_i = XOR_{j<n}    a[n-1+i-j]   AND r[j],                 L = n+m-1 seed bits
 *   modified (Sec. III.D, A[i][j] = a_{n-m+i-j} 1-based, then I_m):
 *       k_i = XOR_{j<n-m}  a[n-m-1+i-j] AND r[j]  XOR r[n-m+i],    L = n-1 seed bits
 * Block b of a stream occupies raw bits [b n, (b+1) n) and output bits [b m, (b+1) m).
 *
 * Pointers: every buffer argument is caller-owned. "device" pointers are CUDA device (or
 * managed) memory of the context's device; "host" pointers are host memory (pinned memory
 * gives the fastest copies). The context owns only its workspace, caches and statistics.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 * Extraction calls are asynchronous: they return after enqueueing the work on `stream`.
 * Calls that return host results (qrng_minentropy, qrng_postprocess, qrng_postprocess_host) synchronise
 * `stream` (qrng_postprocess only up to its estimate).
 *
 * Errors: every int-returning function returns a qrng_status; on failure the context keeps a
 * message (qrng_last_error). No function aborts or raises; a kernel never traps.
 *
 * Threads: a context may be used by one host thread at a time.
 */
#ifndef QRNG_H
#define QRNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define QRNG_API __attribute__((visibility("default")))
#else
#define QRNG_API
#endif

typedef enum {
  QRNG_OK = 0,
  QRNG_EINVAL = 1,      /* an argument is out of range, misaligned or NULL                  */
  QRNG_ENOMEM = 2,      /* device or pinned-host allocation failed                          */
  QRNG_ECUDA = 3,       /* a CUDA runtime call or a kernel launch failed                    */
  QRNG_ETIMEOUT = 4,    /* a bounded device-side wait gave up; the kernel returned cleanly  */
  QRNG_EPRECISION = 5,  /* a floating-point rounding guard tripped and could not be repaired */
  QRNG_ENOTSUP = 6      /* the requested algorithm does not support these arguments         */
} qrng_status;

typedef struct qrng_ctx qrng_ctx;
typedef void* qrng_stream_t; /* cudaStream_t */

/* Create a context bound to CUDA device `device` (makes it current on the calling thread).
 * *out receives the context, or NULL on failure. */
QRNG_API int qrng_create(qrng_ctx** out, int device);

/* Destroy a context: waits for its outstanding work and frees its workspace. NULL is ignored. */
QRNG_API void qrng_destroy(qrng_ctx* ctx);

/* Message describing the last failing call on `ctx` ("" if none). Valid until the next call. */
QRNG_API const char* qrng_last_error(const qrng_ctx* ctx);

/* Static name of a status code. */
QRNG_API const char* qrng_status_string(int status);

/* ----------------------------------------------------------------------------------------------
 * Min-entropy estimate (Sec. II)
 * --------------------------------------------------------------------------------------------*/

typedef struct {
  double h_modify;   /* corrected min-entropy max(0, h_model - delta_hm), bits per sample (Sec. II.C) */
  double h_emp;      /* -log2(max_count / count): min-entropy of the measured distribution P'      */
  double h_model;    /* -log2 max_v P_v of the ideal model P: the Gaussian with the measured mean and
                        population variance (Sec. II.B), rounded to codes, tails clipped into the
                        end codes 0 and 2^bits - 1; a point mass when the variance is 0             */
  double d_u;        /* statistical distance 1/2 sum_v |P'_v - P_v| over every code (Sec. II.C)    */
  double d_u_peak;   /* the same sum restricted to U = {argmax P'} (reported only)                */
  double delta_fs;   /* finite-size amplification 1/2 sqrt(2 (2^bits ln 2 + ln(1/eps)) / count)   */
  double delta_hm;   /* Delta H_m = log2((d_u + delta_fs) / 2^(-bits-1) + 1) (Sec. II.C)          */
  double mean;       /* sample mean                                                              */
  double var;        /* population variance                                                      */
  uint64_t count;    /* number of samples                                                        */
  uint64_t max_count;/* largest histogram bin                                                    */
  uint32_t argmax;   /* lowest code holding max_count                                            */
  uint32_t bits;     /* ADC resolution used                                                      */
} qrng_hmin_report;

/*
 * qrng_minentropy -- Sec. II.A (H_min = -log2 max P), Sec. II.B (Gaussian model fixed by the
 * measured variance), Sec. II.C (statistical distance, correction term Delta H_m, H_modify).
 *
 *   samples  device; `count` ADC codes, uint8 when bits <= 8, little-endian uint16 otherwise;
 *            any alignment.
 *   count    >= 1 samples.
 *   bits     ADC resolution, 1..16. A sample >= 2^bits makes the call fail with QRNG_EINVAL.
 *   eps      confidence parameter of the finite-size term, 0 < eps < 1.
 *   rep      host; receives the report.
 * Synchronises `stream`. Uses context workspace for the histogram.
 */
QRNG_API int qrng_minentropy(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, double eps,
                    qrng_hmin_report* rep, qrng_stream_t stream);

/*
 * qrng_minentropy_sampled -- the same estimate from a random subsample of the stream (Sec. II.C:
 * the corrected entropy may be computed from randomly selected samples). Sample i (0-based) is
 * used when output i+1 of the splitmix64 generator started at sel_seed, shifted right by 11 bits,
 * is below floor(fraction * 2^53); fraction = 1 uses every sample. The finite-size term follows
 * the number of samples kept (rep->count). 0 < fraction <= 1, otherwise as qrng_minentropy;
 * QRNG_EINVAL if no sample is kept.
 */
QRNG_API int qrng_minentropy_sampled(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, double eps,
                                     double fraction, uint64_t sel_seed, qrng_hmin_report* rep,
                                     qrng_stream_t stream);

/*
 * qrng_minentropy_quantum -- classical-noise subtraction (Sec. II.B): the laser-off stream holds
 * the classical noise alone, so the quantum noise variance is var_on - var_off and the ideal
 * model of the quantum part is the Gaussian of that variance around the laser-on mean, rounded
 * and clipped to codes. rep is the laser-on stream's report (counts, moments, empirical entropy,
 * its distance to its own Gaussian model, finite-size term, correction) except
 *   rep->h_model  = -log2 max of the quantum model,  rep->var = var_on - var_off,
 *   rep->h_modify = max(0, rep->h_model - rep->delta_hm).
 * *h_subtracted (may be NULL) receives the paper's H^{q+c} - H'^c: the model min-entropy of the
 * laser-on stream minus that of the laser-off stream. A laser-off stream without spread leaves
 * the plain estimate. QRNG_EINVAL when var_off >= var_on > 0. Synchronises `stream`.
 */
QRNG_API int qrng_minentropy_quantum(qrng_ctx* ctx, const void* samples_on, uint64_t count_on,
                                     const void* samples_off, uint64_t count_off, int bits, double eps,
                                     qrng_hmin_report* rep, double* h_subtracted, qrng_stream_t stream);

/*
 * qrng_minentropy_noalloc -- the same estimate and report as qrng_minentropy, for callers that
 * cannot allocate device memory. The paper has no counterpart; this is a deployment variant.
 *
 * Who it is for: acquisition loops that must not allocate once streaming has started (a device
 * allocation can block and synchronise the whole GPU, stalling the ADC data path), and programs
 * whose device memory belongs to another allocator or that keep no context object between calls.
 * It takes no context and allocates nothing: no cudaMalloc/cudaFree or other allocating call.
 * Its scratch is a fixed area compiled into the library (a histogram of up to 2^16 codes plus
 * the device-side report, about 513 KB), held on every GPU that loads the library until exit.
 *
 *   samples, count, eps, rep, stream   as for qrng_minentropy; samples on the current device.
 *   bits   1..16; a larger value (more codes than the fixed histogram holds) is QRNG_EINVAL.
 * Runs on the calling thread's current CUDA device and synchronises `stream`. Returns only a
 * status (there is no context to hold a message): QRNG_EINVAL for bad arguments or a sample
 * >= 2^bits, QRNG_ECUDA when a CUDA call fails.
 * Every call on a device shares the one scratch area (cleared at the start of each call): calls
 * whose GPU work overlaps, e.g. on two streams at once, race and return wrong reports. The first
 * call on a device looks up the scratch's device address; under CUDA's default lazy module
 * loading it is also the moment the driver loads the library's device code and places the
 * scratch, so make that first call during set-up, before streaming starts and before any stream
 * capture (CUDA_MODULE_LOADING=EAGER places it when the context is created instead). Later calls
 * allocate nothing.
 */
QRNG_API int qrng_minentropy_noalloc(const void* samples, uint64_t count, int bits, double eps,
                                     qrng_hmin_report* rep, qrng_stream_t stream);

/*
 * Output length of the extractor, Sec. III.B (leftover hash lemma):
 *   m = floor(n * h_per_sample / bits - 2 log2(1 / eps_lhl)), or 0 if that is not positive.
 * eps_lhl = 1 drops the security term (m = floor(n h / bits)). Pure host arithmetic.
 */
QRNG_API uint64_t qrng_output_length(uint64_t n, double h_per_sample, int bits, double eps_lhl);

/* ----------------------------------------------------------------------------------------------
 * Toeplitz extraction (Sec. III.B-E)
 * --------------------------------------------------------------------------------------------*/

enum { QRNG_FORM_STANDARD = 0, QRNG_FORM_MODIFIED = 1 };

enum {
  QRNG_ALGO_AUTO = 0,     /* the fastest algorithm for the shape: on the first call of a shape
                             class (n, form, the block count rounded up to a power of two, m with
                             its six leading bits kept: calls whose m differs by a few bits share
                             it) the candidates a cost model keeps are each run once and timed
                             (that call synchronises the stream), and the winner is cached on the
                             context; a later call of the class takes it where it applies to its
                             exact m, else the cost model's choice                                 */
  QRNG_ALGO_DIRECT = 1,   /* bit-packed AND/XOR + parity, each block on its own (Sec. III.B, O(mn)) */
  QRNG_ALGO_GEMM_TC = 2,  /* all blocks as one GF(2) matrix product T X on tcgen05 tensor cores   */
  QRNG_ALGO_FFT64 = 3,    /* circulant embedding + FP64 FFT convolution per block (Sec. III.B-D) */
  QRNG_ALGO_FFT32_SEG = 4,/* FP32 FFT over segments of S bits (S = 2048, 4096 or 8192; the
                             autotuner picks S with the route): every segment and seed window is
                             transformed once, T segment-window products are summed in the
                             frequency domain per inverse transform, T from a proven rounding bound
                             (qrng_fft32_terms_bound), each sum rounded to its exact integer and the
                             parities XOR-combined; if an observed rounding distance reaches 0.25,
                             or a sum reaches 2^20 (FP32 cannot show its rounding there), which only
                             happens with T forced past the bound, the exact direct kernel
                             recomputes the call on the GPU                                        */
  QRNG_ALGO_NTT = 5,      /* the circulant convolution of Sec. III.B with a number-theoretic
                             transform mod 2013265921 (exact integers, integer pipes); lengths up
                             to 2^27                                                                */
  QRNG_ALGO_GEMM_FP4 = 6, /* QRNG_ALGO_GEMM_TC with 4-bit operands (block-scaled E2M1, every scale
                             2^0): half the operand bytes and the FP4 tensor rate; same limits     */
  QRNG_ALGO_GEMM_FP4_PAIR = 7,/* QRNG_ALGO_GEMM_FP4 with each MMA spanning a pair of SMs (clusters
                             of two CTAs, M = 256): fewer shared-memory bytes per MAC; same limits */
  QRNG_ALGO_GEMM_KARATSUBA = 8 /* QRNG_ALGO_GEMM_FP4_PAIR on the 3^L sub-products of L rounds of
                             block Karatsuba over GF(2) (2x2 Toeplitz blocks need three products:
                             (3/4)^L of the multiply-adds, plus three memory-bound passes and
                             workspace of about 3^L (m + n) / 2^(L+3) bytes per block); same limits */
};

/* Seed length in bits: n+m-1 (standard) or n-1 (modified); 0 for an invalid shape. */
QRNG_API uint64_t qrng_seed_bits(uint64_t n, uint64_t m, int form);

/*
 * qrng_toeplitz_extract -- hash num_blocks independent n-bit blocks with one shared seed.
 *
 *   raw         device; num_blocks * n bits, block b at bit b*n (packed LSB-first).
 *   n, m        block length and output length per block; standard: 1 <= m <= n,
 *               modified: 1 <= m < n; n <= 2^26.
 *   seed        device; qrng_seed_bits(n, m, form) bits, shared by every block.
 *   form        QRNG_FORM_STANDARD or QRNG_FORM_MODIFIED.
 *   algo        QRNG_ALGO_*; an algorithm that cannot run these arguments returns QRNG_ENOTSUP.
 *   num_blocks  >= 1.
 *   out         device; ceil(num_blocks*m / 8) bytes; block b's output at bit b*m; the pad bits
 *               of the last byte are written as 0. Must not overlap raw or seed.
 * Asynchronous on `stream`. Any pointer alignment is accepted; 16-byte aligned raw and out with
 * n and m multiples of 128 take the copy-free path.
 */
QRNG_API int qrng_toeplitz_extract(qrng_ctx* ctx, const uint8_t* raw, uint64_t n, uint64_t m, const uint8_t* seed,
                          int form, int algo, uint64_t num_blocks, uint8_t* out, qrng_stream_t stream);

/* ----------------------------------------------------------------------------------------------
 * Uneven batches (Sec. III.E block processing, many independent requests)
 * --------------------------------------------------------------------------------------------*/

typedef struct {
  const uint8_t* raw;     /* device; the request's n raw bits start at bit raw_bit_off          */
  uint64_t raw_bit_off;
  uint64_t n, m;          /* one block: standard 1 <= m <= n, modified 1 <= m < n, n <= 2^26    */
  const uint8_t* seed;    /* device; qrng_seed_bits(n, m, form) bits from bit 0 (its own seed)  */
  int form;               /* QRNG_FORM_STANDARD or QRNG_FORM_MODIFIED                          */
  uint8_t* out;           /* device; the m output bits are written at bit out_bit_off; every
                             other bit of the buffer is left as it was (requests may share bytes) */
  uint64_t out_bit_off;
} qrng_request;

/*
 * qrng_extract_batch -- hash `count` independent requests, each one block with its own seed and
 * shape (Sec. III.B / III.D per request; Sec. III.E independence).
 * Requests on the direct route run in ONE persistent kernel launch: work items (request, output
 * tile, raw-word range) are numbered largest request first and taken from an atomic counter by
 * resident warps. The layout, hashing and output-merge kernels are captured once into a CUDA graph
 * cached on the context (keyed by the request table and its buffers); a repeated identical call
 * replays the graph. Requests on the transform route (exact number-theoretic transform of the
 * circulant convolution, three transforms each) run before the graph, batched by length.
 *   reqs   host; `count` >= 1 requests (device pointers inside; outputs must not overlap raw or
 *          seed data, and two requests' output bit ranges must not overlap).
 *   algo   QRNG_ALGO_AUTO (each request on the route its cost model prefers: the exact
 *          number-theoretic transform for long blocks), QRNG_ALGO_DIRECT (all direct),
 *          QRNG_ALGO_NTT or QRNG_ALGO_FFT64 (every request whose transform length fits 2^27 on that
 *          transform: the FP64 one packs seed and raw bits into one complex vector per request and
 *          two requests into one inverse); anything else (the shared-seed tensor-core product, the
 *          FP32 segmented route whose per-request seed windows would cost O(mn/S)) is
 *          QRNG_ENOTSUP.
 * Asynchronous on `stream`. Batch calls on one context must not overlap on the GPU.
 */
QRNG_API int qrng_extract_batch(qrng_ctx* ctx, const qrng_request* reqs, uint64_t count, int algo,
                                qrng_stream_t stream);

/* ----------------------------------------------------------------------------------------------
 * Whole pipeline
 * --------------------------------------------------------------------------------------------*/

/*
 * qrng_postprocess -- the post-processing of Sec. II + III on device buffers: estimate H_modify of
 * the ADC samples (as qrng_minentropy), size the output m = qrng_output_length(n, H_modify, bits,
 * eps_lhl) (m <= n - 1 for the modified form of Sec. III.D), treat the sample bytes as the raw bit
 * stream (sample s occupies raw bits [8s, 8s+8) for bits <= 8, [16s, 16s+16) otherwise) and hash
 * its floor(total_bits / n) whole n-bit blocks with `seed` (as qrng_toeplitz_extract with the
 * given form and algo) into `out`.
 *
 *   samples        device; count samples as for qrng_minentropy (also the raw stream).
 *   seed           device; at least seed_capacity_bits bits; must cover qrng_seed_bits(n, m, form).
 *   out            device; out_capacity_bytes bytes; must hold ceil(num_blocks*m/8) bytes, written
 *                  as by qrng_toeplitz_extract.
 *   m_out, num_blocks_out, rep   host; receive m, the number of blocks and the entropy report
 *                  (any of them may be NULL).
 * Returns QRNG_EINVAL when m comes out 0 or a capacity is too small (m_out / num_blocks_out are
 * still written). The call waits for the estimate (m is returned, and plans the hash) but not for
 * the hash, which is enqueued on `stream`. When the previous call on this context had the same n,
 * count, bits and form and its hash ran on the block-Karatsuba route, the derived raw operands of
 * that route (which do not depend on m in the standard form) are computed on a second stream of
 * the context while the estimate runs; a different m only costs computing them again. In the
 * standard form such a call (for n a multiple of 128, 16-byte aligned samples, a 4-byte aligned
 * `out` and a block count that is a multiple of 32) also enqueues the hash right behind the
 * estimate, before the host has read m: for up to m_cap rows, the previous m rounded up to the
 * route's row span (at most seed_capacity_bits - n + 1), with m itself computed on the device from
 * the report in the host's arithmetic. The hash's kernels do nothing unless m <= m_cap (and m >= 64)
 * and the call is valid; when m is outside, the call hashes again with m as an ordinary call
 * (qrng_stats counts both). Either way `out` receives exactly the ordinary call's bytes. The
 * buffers belong to the call until `stream` reaches its end, and calls on one context are made
 * on one stream (a call's work waits for the work earlier calls left on its stream).
 */
QRNG_API int qrng_postprocess(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, double eps,
                              double eps_lhl, uint64_t n, const uint8_t* seed, uint64_t seed_capacity_bits, int form,
                              int algo, uint8_t* out, uint64_t out_capacity_bytes, uint64_t* m_out,
                              uint64_t* num_blocks_out, qrng_hmin_report* rep, qrng_stream_t stream);

/*
 * qrng_postprocess_host -- the post-processing of Sec. II + III on host memory: copy the ADC
 * samples to the device, estimate H_modify (as qrng_minentropy), size the output
 * m = qrng_output_length(n, H_modify, bits, eps_lhl), treat the sample bytes as the raw bit
 * stream (sample s occupies raw bits [8s, 8s+8) for bits <= 8, [16s, 16s+16) otherwise), hash
 * its floor(total_bits / n) whole n-bit blocks, and copy the packed output back.
 *
 *   samples_host   host; count samples as for qrng_minentropy.
 *   seed_host      host; at least seed_capacity_bits bits; must cover qrng_seed_bits(n, m, form).
 *   out_host       host; out_capacity_bytes bytes; must hold ceil(num_blocks*m/8) bytes.
 *   m_out, num_blocks_out, rep   host; receive m, the number of blocks and the entropy report
 *                  (any of them may be NULL).
 * Returns QRNG_EINVAL when m comes out 0 or a capacity is too small (m_out / num_blocks_out
 * are still written). Synchronises `stream`. When n is a multiple of 128 and there are at least
 * 64 blocks, the blocks are hashed in two parts (the first about 7/8 of them) and the first part's
 * output is copied to the host (on a stream of the context) while the second is hashed; out_host
 * belongs to the call until it returns, like every other buffer.
 */
QRNG_API int qrng_postprocess_host(qrng_ctx* ctx, const void* samples_host, uint64_t count, int bits, double eps,
                          double eps_lhl, uint64_t n, const uint8_t* seed_host, uint64_t seed_capacity_bits,
                          int form, int algo, uint8_t* out_host, uint64_t out_capacity_bytes, uint64_t* m_out,
                          uint64_t* num_blocks_out, qrng_hmin_report* rep, qrng_stream_t stream);

/*
 * qrng_postprocess_host_async / qrng_postprocess_host_wait -- the host-buffer pipeline for a stream
 * of calls that overlap: each call uploads its samples and seed, estimates H_modify, sizes m and
 * hashes exactly as qrng_postprocess_host does (the whole seed_capacity_bits bits of seed_host are
 * uploaded), but returns as soon as its hash and the download of its output are enqueued. The
 * next call's upload then runs on a copy engine while this call hashes, and this call's download
 * while the next one hashes. Two calls' device buffers are kept (they alternate), so every call
 * returns once the call before it has finished hashing (its estimate waits for that on `stream`).
 * A call after one of the same shape enqueues its hash before reading m, under the conditions and
 * with the outcome qrng_postprocess states (the device buffers' alignment is the library's).
 * The caller keeps samples_host and out_host of a call untouched until a later
 * qrng_postprocess_host_wait has returned; pinned host memory is needed for the copies to
 * overlap. m_out, num_blocks_out and rep are written before the call returns.
 * qrng_postprocess_host_wait waits for every call submitted so far (and reports device-side
 * failures as qrng_synchronize does).
 */
QRNG_API int qrng_postprocess_host_async(qrng_ctx* ctx, const void* samples_host, uint64_t count, int bits,
                                         double eps, double eps_lhl, uint64_t n, const uint8_t* seed_host,
                                         uint64_t seed_capacity_bits, int form, int algo, uint8_t* out_host,
                                         uint64_t out_capacity_bytes, uint64_t* m_out, uint64_t* num_blocks_out,
                                         qrng_hmin_report* rep, qrng_stream_t stream);
QRNG_API int qrng_postprocess_host_wait(qrng_ctx* ctx, qrng_stream_t stream);

/* ----------------------------------------------------------------------------------------------
 * Statistics
 * --------------------------------------------------------------------------------------------*/

typedef struct {
  int last_algo;                 /* algorithm the last extraction ran (QRNG_ALGO_*)            */
  uint32_t last_kernels;         /* kernels the last extraction call launched                   */
  uint64_t kernels_launched;     /* kernels launched by this context since creation / reset    */
  double worst_fft_round_err;    /* max |s - round(s)| seen by the FFT paths since the reset    */
  uint64_t timed_launches;       /* main extraction kernels timed since the reset (see below)   */
  double timed_ms;               /* their summed device time, from CUDA events on their stream  */
  uint64_t hist_timed_launches;  /* histogram kernels of qrng_minentropy timed since the reset  */
  double hist_timed_ms;          /* their summed device time                                    */
  double batch_graph_ms;         /* qrng_extract_batch: device time of its graph replays        */
  uint64_t batch_requests[4];    /* requests of the last qrng_extract_batch call per route: the
                                    persistent direct kernel, the number-theoretic transform,
                                    the FP64 FFT and the FP32 segmented FFT                      */
  double batch_direct_bitmacs;   /* the last batch call: sum of m n_t over its direct requests  */
  double batch_transform_bytes;  /* the last batch call: (n + m) / 8 over its transform requests */
  double batch_direct_ms;        /* the last timed batch replay: its persistent direct kernel   */
  double batch_transform_ms;     /* the last timed batch replay: its transform groups           */
  double worst_fft32_round_err;  /* the FP32 segmented route's part of worst_fft_round_err      */
  uint64_t fft32_recomputed;     /* FP32 segmented calls whose rounding guard tripped and whose
                                    output the exact direct kernel recomputed                   */
  uint64_t last_fft32_segment;   /* segment length S of the last FP32 segmented call            */
  uint64_t kara_presplits;       /* qrng_postprocess / _host: derived operands of the block-
                                    Karatsuba route computed beside the estimate                 */
  uint64_t kara_presplits_used;  /* ... and taken by the hash (the rest were computed again)     */
  uint64_t autotune_runs;        /* QRNG_ALGO_AUTO calls that timed the candidates (one per shape
                                    class)                                                       */
  uint64_t speculative_hashes;   /* qrng_postprocess calls whose hash was enqueued before the
                                    host read m (see qrng_postprocess)                           */
  uint64_t speculative_misses;   /* ... of which m fell outside the enqueued rows and the hash
                                    ran again with m                                             */
} qrng_stats;

/* Statistics since creation or the last reset. When timing is on, this call waits for the
 * timed launches to finish (it synchronises their events). */
QRNG_API int qrng_get_stats(qrng_ctx* ctx, qrng_stats* out);

/* The precision evidence of the transform routes alone (Sec. III.B, the FFT route, computed in
 * floating point): the largest distance |s - round(s)| of a convolution sum from its
 * integer seen by the FP64 and FP32 segmented routes since creation or the last reset (0 when
 * neither ran; the number-theoretic transform is exact). Waits for the work that reports it. */
QRNG_API int qrng_extract_stats(qrng_ctx* ctx, double* worst_fft_round_err);
QRNG_API int qrng_reset_stats(qrng_ctx* ctx);

/* Waits for `stream` and reports device-side failures of the work enqueued so far: returns
 * QRNG_ETIMEOUT (and clears the condition) when a kernel's bounded wait gave up, in which case
 * the output of that call is incomplete, and QRNG_EPRECISION when an FFT path saw a convolution
 * sum 0.25 or more away from an integer since the last qrng_reset_stats (its rounding, hence its
 * parity, is then not trustworthy). Kernels never trap or hang on such a failure. */
QRNG_API int qrng_synchronize(qrng_ctx* ctx, qrng_stream_t stream);

/* Failure injection for testing the device-side failure path (no GPU fault involved): arms a
 * fault for the next tensor-core extraction on this context only.
 *   QRNG_FAULT_GEMM_NO_TMA  the kernel's loader publishes no raw tile; every wait that depends on
 *                           it gives up after its bound (about a second), the kernel frees its
 *                           tensor memory and returns, and qrng_synchronize reports QRNG_ETIMEOUT.
 * The context stays usable afterwards. */
enum { QRNG_FAULT_NONE = 0, QRNG_FAULT_GEMM_NO_TMA = 1 };
QRNG_API int qrng_inject_fault(qrng_ctx* ctx, int fault);

/* Autotuning of QRNG_ALGO_AUTO (on = 1, the default; off = 0 uses the cost model alone and never
 * synchronises). Changing it forgets the shapes tuned so far. */
QRNG_API int qrng_set_autotune(qrng_ctx* ctx, int on);

/* Block Karatsuba settings of QRNG_ALGO_GEMM_KARATSUBA (0 = chosen by the cost model, the default):
 *   levels          rounds of the 2x2 block split, 1..4 (3^levels sub-products);
 *   block_bits      h, the side of the square Toeplitz blocks: 256, 512, 1024, 2048, 4096 or 8192
 *                   (256 lets the two output tiles of a pair tile share T tiles across blocks: no
 *                   extra operand build per block);
 *   max_workspace   device bytes for the derived operands and sub-product parities of one pass
 *                   (the blocks are processed in passes that fit it; 0 = 1 GiB). A pass always
 *                   holds at least 224 blocks (one tile width of the product kernel), or every
 *                   block when there are fewer, so a budget below what 224 blocks need is
 *                   exceeded rather than refused.
 * Returns QRNG_EINVAL for values outside those sets. Forgets the shapes autotuned so far. */
QRNG_API int qrng_set_karatsuba(qrng_ctx* ctx, int levels, uint64_t block_bits, uint64_t max_workspace);

/* The block Karatsuba plan QRNG_ALGO_GEMM_KARATSUBA would run for this shape under the context's
 * settings (no GPU work): levels (0 when no plan fits), block side h in bits, the number of
 * sub-products (3^levels), each sub-product's rows and columns (multiples of h), blocks per pass
 * and the cost model's seconds for all blocks. Returns QRNG_EINVAL for an invalid shape. */
typedef struct {
  int levels;
  uint64_t block_bits;
  uint64_t products;
  uint64_t rows, cols;
  uint64_t blocks_per_pass;
  double model_seconds;
} qrng_karatsuba_plan_info;
QRNG_API int qrng_karatsuba_plan(qrng_ctx* ctx, uint64_t n, uint64_t m, int form, uint64_t num_blocks,
                                 qrng_karatsuba_plan_info* out);

/* FP32 segmented FFT settings of QRNG_ALGO_FFT32_SEG (Sec. III.B circulant route on segments):
 *   segment_bits   S: 2048, 4096 or 8192, or 0 (the default) to choose S per shape (the
 *                  autotuner times each S; without autotuning the cost model picks);
 *   terms          segment-window products summed per inverse transform, or 0 (the default) for
 *                  qrng_fft32_terms_bound(S). A larger value is allowed (a test of the rounding
 *                  guard): results stay exact, because a tripped guard makes the direct kernel
 *                  recompute the call, counted in qrng_stats.fft32_recomputed.
 * QRNG_EINVAL for other values. Forgets the shapes autotuned so far. */
QRNG_API int qrng_set_fft32(qrng_ctx* ctx, uint64_t segment_bits, int terms);

/* The largest number of product terms per inverse transform for which the FP32 rounding bound of
 * QRNG_ALGO_FFT32_SEG keeps every convolution sum within 0.45 of its integer: T with
 * T sqrt((2S-1) S) (eps_k + T u) <= 0.45, u = 2^-24, k = log2(2S), eps_k Percival's factor for
 * radix-2 transforms of length 2^k with twiddles rounded once (16, 8 and 3 for S = 2048, 4096,
 * 8192). 0 for another S. Pure host arithmetic. */
QRNG_API int qrng_fft32_terms_bound(uint64_t segment_bits);

/* Timing (on = 1, off = 0): CUDA event pairs on the caller's stream around the main extraction
 * kernel of each qrng_toeplitz_extract call (one pair per launch; the block-Karatsuba route
 * launches its product kernel once per pass), summed into timed_ms / timed_launches; around the
 * histogram kernel of qrng_minentropy (hist_timed_*); and around each qrng_extract_batch replay
 * (batch_graph_ms), whose graph also records the time of its transform groups and of its
 * persistent direct kernel (batch_transform_ms, batch_direct_ms: the last timed replay's). At most
 * 4096 pairs are kept between two qrng_get_stats calls; later ones are not timed. */
QRNG_API int qrng_set_timing(qrng_ctx* ctx, int on);

#ifdef __cplusplus
}
#endif

#endif /* QRNG_H */
