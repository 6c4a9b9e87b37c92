// C ABI of the library (declared in include/qrng.h): argument checks, workspace, dispatch of the
// min-entropy and extraction kernels, and the host-buffer pipeline.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cstdio>
#include <algorithm>
#include <new>
#include <vector>
#include <string>

#include "qrng_internal.h"

using namespace qrng;

namespace {

int fail(qrng_ctx* ctx, int status, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return status;
}

int cuda_fail(qrng_ctx* ctx, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(ctx, e == cudaErrorMemoryAllocation ? QRNG_ENOMEM : QRNG_ECUDA, msg);
}

#define QRNG_CUDA(ctx, call, where)                 \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

constexpr size_t kMaxTimed = 4096;
// Largest distance of an FFT convolution sum from its integer that still counts as exact.
constexpr double kFftRoundGuard = 0.25;

// CUDA-event timing of selected launches (qrng_set_timing): a begin/end pair on the launch's
// stream becomes one timed entry of a kind (summed per kind by qrng_get_stats). At most kMaxTimed
// entries are kept between two qrng_get_stats calls; later pairs are not timed.
enum TimeKind { kTimeExtract = 0, kTimeHist = 1, kTimeBatchGraph = 2 };

void timing_begin(qrng_ctx* ctx, int kind, cudaStream_t s) {
  ctx->ev_pending = (size_t)-1;
  if (!ctx->timing || ctx->ev_used >= kMaxTimed) return;
  if (ctx->ev_used == ctx->ev_start.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    ctx->ev_start.push_back(a);
    ctx->ev_end.push_back(b);
    ctx->ev_kind.push_back(0);
  }
  const size_t slot = ctx->ev_used;
  if (cudaEventRecord(ctx->ev_start[slot], s) != cudaSuccess) return;
  ctx->ev_kind[slot] = kind;
  ctx->ev_pending = slot;
}

void timing_end(qrng_ctx* ctx, cudaStream_t s) {
  const size_t slot = ctx->ev_pending;
  ctx->ev_pending = (size_t)-1;
  if (slot == (size_t)-1) return;
  if (cudaEventRecord(ctx->ev_end[slot], s) == cudaSuccess) ctx->ev_used = slot + 1;
}

// Times one launch: the pair brackets the object's lifetime up to done().
struct LaunchTimer {
  qrng_ctx* ctx;
  cudaStream_t s;
  bool open;
  LaunchTimer(qrng_ctx* c, cudaStream_t st, int kind = kTimeExtract) : ctx(c), s(st), open(true) {
    timing_begin(ctx, kind, s);
  }
  void done() {
    if (open) timing_end(ctx, s);
    open = false;
  }
};

// Hook for launchers that run their main kernel several times (one timed pair per launch).
TimingHook extract_hook(qrng_ctx* ctx) {
  TimingHook h;
  if (!ctx->timing) return h;
  h.user = ctx;
  h.begin = [](void* u, cudaStream_t st) { timing_begin(static_cast<qrng_ctx*>(u), kTimeExtract, st); };
  h.end = [](void* u, cudaStream_t st) { timing_end(static_cast<qrng_ctx*>(u), st); };
  return h;
}

bool shape_ok(uint64_t n, uint64_t m, int form) {
  if (n == 0 || m == 0 || n > kMaxBlockBits) return false;
  if (form == QRNG_FORM_STANDARD) return m <= n;
  if (form == QRNG_FORM_MODIFIED) return m < n;
  return false;
}

// Bit-packed extraction (direct kernel or tensor-core GEMM) of word-aligned or arbitrary layouts.
// FP32 segment length for a shape: the context's setting, else the cost model's best.
int fft32_pick_log_s(const qrng_ctx* ctx, uint64_t n_t, uint64_t m, uint64_t B) {
  if (ctx->fft32_log_s) return ctx->fft32_log_s;
  int best = 12;
  double best_t = 1e300;
  for (int ls = 11; ls <= 13; ++ls) {
    const int T = ctx->fft32_terms ? ctx->fft32_terms : fft32_terms_bound(ls);
    const double t = fft32_model_seconds(n_t, m, B, ls, T);
    if (t < best_t) {
      best_t = t;
      best = ls;
    }
  }
  return best;
}

int extract_bitwise(qrng_ctx* ctx, int algo, const uint8_t* raw, uint64_t n, uint64_t m, const uint8_t* seed,
                    int form, uint64_t num_blocks, uint8_t* out, cudaStream_t s, uint32_t* kernels,
                    int fft32_log_s = 0) {
  const uint64_t n_t = (form == QRNG_FORM_MODIFIED) ? n - m : n;
  const uint64_t L_t = n_t + m - 1;
  const bool fft = (algo == QRNG_ALGO_FFT64 || algo == QRNG_ALGO_FFT32_SEG || algo == QRNG_ALGO_NTT);

  // the bit-packed kernels read Toeplitz rows as windows of the reversed seed (the FP32 route keeps
  // one for its exact recomputation)
  if (!fft || algo == QRNG_ALGO_FFT32_SEG) {
    const uint64_t rev_words = kSeedFrontWords + ceil_div(L_t, 32) + kSeedBackWords;
    QRNG_CUDA(ctx, ctx->seed_rev.ensure(rev_words * 4), "seed workspace");
    QRNG_CUDA(ctx, launch_seed_reverse(seed, L_t, ctx->seed_rev.as<uint32_t>(), rev_words, s, kernels),
              "seed reverse");
  }

  DirectArgs a{};
  // The tensor-core kernel loads raw tiles with TMA: 16-byte aligned rows, a multiple of 4 words apart.
  const bool gemm = (algo == QRNG_ALGO_GEMM_TC || algo == QRNG_ALGO_GEMM_FP4 || algo == QRNG_ALGO_GEMM_FP4_PAIR ||
                     algo == QRNG_ALGO_GEMM_KARATSUBA);
  const bool raw_direct = gemm ? (n % 128 == 0) && ((reinterpret_cast<uintptr_t>(raw) & 15) == 0)
                               : (n % 32 == 0) && ((reinterpret_cast<uintptr_t>(raw) & 3) == 0);
  if (raw_direct) {
    a.raw = reinterpret_cast<const uint32_t*>(raw);
    a.raw_stride = n / 32;
  } else {
    const uint64_t stride = gemm ? ceil_div(n, 128) * 4 : ceil_div(n, 32);
    QRNG_CUDA(ctx, ctx->raw_stage.ensure(num_blocks * stride * 4), "raw staging workspace");
    QRNG_CUDA(ctx, launch_repack_blocks(raw, 0, n, num_blocks, ctx->raw_stage.as<uint32_t>(), stride, s, kernels),
              "raw repack");
    a.raw = ctx->raw_stage.as<uint32_t>();
    a.raw_stride = stride;
  }
  const uint64_t mw = ceil_div(m, 32);
  const bool out_direct = (m % 32 == 0) && ((reinterpret_cast<uintptr_t>(out) & 3) == 0);
  uint32_t* out_w;
  if (out_direct) {
    out_w = reinterpret_cast<uint32_t*>(out);
  } else {
    QRNG_CUDA(ctx, ctx->out_stage.ensure(num_blocks * mw * 4), "output staging workspace");
    out_w = ctx->out_stage.as<uint32_t>();
  }

  a.n_t = n_t;
  a.nw_t = (uint32_t)ceil_div(n_t, 32);
  a.tail_mask = (n_t % 32) ? ((1u << (n_t % 32)) - 1u) : 0xffffffffu;
  a.m = (uint32_t)m;
  a.mw = (uint32_t)mw;
  a.seed_rev = ctx->seed_rev.as<uint32_t>();
  a.modified = (form == QRNG_FORM_MODIFIED);
  a.id_off = (uint32_t)(n - m);
  a.out = out_w;
  a.out_stride = mw;
  a.num_blocks = num_blocks;
  if (algo == QRNG_ALGO_FFT32_SEG) {
    const int log_s = fft32_log_s ? fft32_log_s : fft32_pick_log_s(ctx, n_t, m, num_blocks);
    const int T = ctx->fft32_terms ? ctx->fft32_terms : fft32_terms_bound(log_s);
    ctx->fft.worst = ctx->fft_worst.as<unsigned long long>() + 1;  // its own word: a trip is repaired
    int* flag = ctx->fft32_guard.as<int>();
    QRNG_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), s), "guard clear");
    LaunchTimer timer(ctx, s);
    const cudaError_t e = launch_fft32_seg(a, seed, L_t, log_s, T, ctx->fft, flag, s, kernels);
    timer.done();
    QRNG_CUDA(ctx, e, "FP32 segmented FFT extraction");
    // exact recomputation by the direct kernel, which returns at once unless the guard tripped
    DirectArgs r = a;
    r.tiles = (uint32_t)ceil_div(m, (uint64_t)direct_outputs_per_warp());
    r.splits = 1;
    r.words_per_split = a.nw_t;
    r.guard = flag;
    r.repairs = reinterpret_cast<unsigned long long*>(ctx->fft32_guard.as<char>() + 8);
    QRNG_CUDA(ctx, launch_direct(r, s, kernels), "FP32 route recomputation");
    ctx->last_fft32_log_s = log_s;
    if (!out_direct)
      QRNG_CUDA(ctx, launch_pack_blocks(out_w, mw, m, num_blocks, out, s, kernels), "output pack");
    return QRNG_OK;
  }
  if (fft) {
    ctx->fft.worst = ctx->fft_worst.as<unsigned long long>();
    LaunchTimer timer(ctx, s);
    const cudaError_t e = algo == QRNG_ALGO_FFT64 ? launch_fft64(a, seed, L_t, ctx->fft, s, kernels)
                                                  : launch_ntt(a, seed, L_t, ctx->fft, s, kernels);
    timer.done();
    QRNG_CUDA(ctx, e, algo == QRNG_ALGO_FFT64 ? "FP64 FFT extraction" : "number-theoretic transform extraction");
    if (!out_direct)
      QRNG_CUDA(ctx, launch_pack_blocks(out_w, mw, m, num_blocks, out, s, kernels), "output pack");
    return QRNG_OK;
  }
  if (gemm) {
    QRNG_CUDA(ctx, ctx->dev_err.ensure(sizeof(int)), "error word");
    const int fault = ctx->fault;
    ctx->fault = 0;  // one-shot
    if (algo == QRNG_ALGO_GEMM_KARATSUBA) {
      const KaraPlan plan = karatsuba_plan(n_t, m, num_blocks, ctx->num_sms, ctx->kara_levels, ctx->kara_h,
                                           ctx->kara_workspace);
      if (plan.levels == 0) return fail(ctx, QRNG_ENOTSUP, "qrng_toeplitz_extract: no block Karatsuba plan fits");
      // the combination writes the packed stream itself when its layout allows (no pack pass)
      const uint64_t out_bytes = ceil_div(num_blocks * m, 8);
      const bool fused = !out_direct && (reinterpret_cast<uintptr_t>(out) & 3) == 0 && out_bytes % 4 == 0 &&
                         m >= 64 && m <= kKaraPackMaxBits;
      // one timed pair around each pass's product kernel
      QRNG_CUDA(ctx,
                launch_gemm_karatsuba(a, plan, ctx->kara, ctx->dev_err.as<int>(), fault, ctx->num_sms, s, kernels,
                                      extract_hook(ctx), fused ? out : nullptr),
                "block Karatsuba extraction");
      if (fused) return QRNG_OK;
    } else {
      LaunchTimer timer(ctx, s);
      QRNG_CUDA(ctx,
                algo == QRNG_ALGO_GEMM_FP4_PAIR
                    ? launch_gemm_pair(a, ctx->dev_err.as<int>(), fault, ctx->num_sms, s, kernels)
                    : launch_gemm_tc(a, algo == QRNG_ALGO_GEMM_FP4, ctx->dev_err.as<int>(), fault, ctx->num_sms, s,
                                     kernels),
                "tensor-core extraction kernel");
      timer.done();
    }
    if (!out_direct)
      QRNG_CUDA(ctx, launch_pack_blocks(out_w, mw, m, num_blocks, out, s, kernels), "output pack");
    return QRNG_OK;
  }
  const uint64_t per_warp = (uint64_t)direct_outputs_per_warp();
  const uint64_t R = per_warp / 32;
  a.tiles = (uint32_t)ceil_div(m, per_warp);
  const uint64_t base_warps = num_blocks * a.tiles;
  const uint64_t target_warps = (uint64_t)ctx->num_sms * 32;
  uint64_t splits = 1;
  if (base_warps < target_warps) {
    splits = ceil_div(target_warps, base_warps);
    const uint64_t max_splits = ceil_div(a.nw_t, R);
    if (splits > max_splits) splits = max_splits;
  }
  uint64_t wps = ceil_div(ceil_div(a.nw_t, splits), R) * R;
  splits = ceil_div(a.nw_t, wps);
  a.splits = (uint32_t)splits;
  a.words_per_split = (uint32_t)wps;
  if (splits > 1) QRNG_CUDA(ctx, cudaMemsetAsync(out_w, 0, num_blocks * mw * 4, s), "output clear");
  LaunchTimer timer(ctx, s);
  QRNG_CUDA(ctx, launch_direct(a, s, kernels), "direct extraction kernel");
  timer.done();
  if (!out_direct)
    QRNG_CUDA(ctx, launch_pack_blocks(out_w, mw, m, num_blocks, out, s, kernels), "output pack");
  return QRNG_OK;
}

// Histogram (all samples, or the random subsample when thr < 2^53) and FP64 finaliser enqueued on
// `s`; the report stays on the device (ctx->result).
int minentropy_enqueue(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, double eps, cudaStream_t s,
                       uint64_t thr = 1ull << 53, uint64_t sel_seed = 0, double var_sub = 0.0, double h_ref = 0.0) {
  const uint64_t K = 1ull << bits;
  uint32_t kernels = 0;
  QRNG_CUDA(ctx, ctx->hist.ensure((K + 1) * sizeof(unsigned long long)), "histogram workspace");
  const bool fresh_result = ctx->result.cap < sizeof(DevHminResult);
  QRNG_CUDA(ctx, ctx->result.ensure(sizeof(DevHminResult)), "result workspace");
  // the finaliser's accumulators start at zero once; every finaliser run leaves them so
  if (fresh_result) QRNG_CUDA(ctx, cudaMemsetAsync(ctx->result.p, 0, sizeof(DevHminResult), s), "result clear");
  if (thr >= (1ull << 53)) {
    LaunchTimer timer(ctx, s, kTimeHist);
    QRNG_CUDA(ctx, launch_histogram(samples, count, bits, ctx->hist.as<unsigned long long>(), ctx->num_sms, s, &kernels),
              "histogram kernel");
    timer.done();
  } else {
    QRNG_CUDA(ctx, launch_histogram_sampled(samples, count, bits, thr, sel_seed, ctx->hist.as<unsigned long long>(),
                                            ctx->num_sms, s, &kernels),
              "sampled histogram kernel");
  }
  QRNG_CUDA(ctx, launch_hmin_finalize(ctx->hist.as<unsigned long long>(), bits, eps, ctx->result.as<DevHminResult>(),
                                      s, &kernels, var_sub, h_ref),
            "min-entropy finaliser kernel");
  ctx->stats.kernels_launched += kernels;
  return QRNG_OK;
}

// The report in ctx->result_host (its copy complete), the finaliser's failures as statuses.
int minentropy_read(qrng_ctx* ctx, qrng_hmin_report* rep, double var_sub = 0.0, double* h_subtracted = nullptr) {
  const DevHminResult& r = *ctx->result_host;
  if (r.out_of_range)
    return fail(ctx, QRNG_EINVAL, "qrng_minentropy: " + std::to_string(r.out_of_range) + " samples are >= 2^bits");
  if (r.status != QRNG_OK)
    return fail(ctx, r.status,
                var_sub > 0.0 ? "qrng_minentropy_quantum: the laser-off variance is not below the laser-on variance"
                              : "qrng_minentropy: finaliser reported an error (no sample selected?)");
  *rep = r.rep;
  if (h_subtracted) *h_subtracted = r.h_subtracted;
  return QRNG_OK;
}

// Histogram (all samples, or the random subsample when thr < 2^53) + FP64 finaliser, report read back.
int minentropy_dev(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, double eps, qrng_hmin_report* rep,
                   cudaStream_t s, uint64_t thr = 1ull << 53, uint64_t sel_seed = 0, double var_sub = 0.0,
                   double h_ref = 0.0, double* h_subtracted = nullptr) {
  const int st = minentropy_enqueue(ctx, samples, count, bits, eps, s, thr, sel_seed, var_sub, h_ref);
  if (st) return st;
  QRNG_CUDA(ctx, cudaMemcpyAsync(ctx->result_host, ctx->result.p, sizeof(DevHminResult), cudaMemcpyDeviceToHost, s),
            "report copy");
  QRNG_CUDA(ctx, cudaStreamSynchronize(s), "min-entropy synchronise");
  return minentropy_read(ctx, rep, var_sub, h_subtracted);
}

int check_minentropy_args(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, double eps,
                          const qrng_hmin_report* rep) {
  if (!samples || !rep) return fail(ctx, QRNG_EINVAL, "qrng_minentropy: NULL pointer");
  if (count == 0) return fail(ctx, QRNG_EINVAL, "qrng_minentropy: count must be >= 1");
  if (bits < 1 || bits > 16) return fail(ctx, QRNG_EINVAL, "qrng_minentropy: bits must be in [1, 16]");
  if (!(eps > 0.0 && eps < 1.0)) return fail(ctx, QRNG_EINVAL, "qrng_minentropy: eps must be in (0, 1)");
  return QRNG_OK;
}

int check_extract_args(qrng_ctx* ctx, const uint8_t* raw, uint64_t n, uint64_t m, const uint8_t* seed, int form,
                       int algo, uint64_t num_blocks, const uint8_t* out) {
  if (!raw || !seed || !out) return fail(ctx, QRNG_EINVAL, "qrng_toeplitz_extract: NULL pointer");
  if (form != QRNG_FORM_STANDARD && form != QRNG_FORM_MODIFIED)
    return fail(ctx, QRNG_EINVAL, "qrng_toeplitz_extract: unknown form");
  if (!shape_ok(n, m, form))
    return fail(ctx, QRNG_EINVAL,
                "qrng_toeplitz_extract: need 1 <= m <= n (standard) or 1 <= m < n (modified), n <= 2^26");
  if (num_blocks == 0) return fail(ctx, QRNG_EINVAL, "qrng_toeplitz_extract: num_blocks must be >= 1");
  if (num_blocks > (1ull << 62) / n) return fail(ctx, QRNG_EINVAL, "qrng_toeplitz_extract: stream too long");
  if (algo < QRNG_ALGO_AUTO || algo > QRNG_ALGO_GEMM_KARATSUBA)
    return fail(ctx, QRNG_EINVAL, "qrng_toeplitz_extract: unknown algorithm");
  return QRNG_OK;
}

// Rough time model (seconds) of each algorithm, used to prune the autotuner's candidates and as
// the choice when autotuning is off. Rates are the ones measured on GB300 for these kernels.
double model_seconds(const qrng_ctx* ctx, int algo, uint64_t n_t, uint64_t m, uint64_t B) {
  const double bm = (double)m * (double)n_t * (double)B;
  switch (algo) {
    case QRNG_ALGO_DIRECT:
      return bm / 5.6e14 + 5e-6;
    case QRNG_ALGO_GEMM_TC: {
      const double mp = (double)ceil_div(m, 256) * 256, bp = (double)ceil_div(B, 256) * 256;
      return mp * (double)n_t * bp / 1.75e15 + 1e-5;
    }
    case QRNG_ALGO_GEMM_FP4: {
      const double mp = (double)ceil_div(m, 256) * 256, bp = (double)ceil_div(B, 224) * 224;
      return mp * (double)n_t * bp / 3.0e15 + 1e-5;
    }
    case QRNG_ALGO_GEMM_FP4_PAIR: {
      const double mp = (double)ceil_div(m, 256) * 256, bp = (double)ceil_div(B, 256) * 256;
      return mp * (double)n_t * bp / 4.5e15 + 1e-5;
    }
    case QRNG_ALGO_GEMM_KARATSUBA: {
      const KaraPlan p = karatsuba_plan(n_t, m, B, ctx->num_sms, ctx->kara_levels, ctx->kara_h, ctx->kara_workspace);
      return p.levels ? p.model_s : 1e30;
    }
    case QRNG_ALGO_FFT64: {
      const double P = (double)fft64_length(n_t, m), lg = log2(P), pairs = (double)ceil_div(B, 2);
      return pairs * (10.0 * P * lg / 6e11 + 64.0 * P * lg / 6e12) + 2.0 * lg * 4e-6;
    }
    case QRNG_ALGO_NTT: {  // measured: about 0.9 ps per element and log2 P per block (two transforms)
      const double P = (double)fft64_length(n_t, m), lg = log2(P);
      return (double)B * P * lg * 0.9e-12 + 6e-5;
    }
    case QRNG_ALGO_FFT32_SEG: {
      const int ls = fft32_pick_log_s(ctx, n_t, m, B);
      return fft32_model_seconds(n_t, m, B, ls, ctx->fft32_terms ? ctx->fft32_terms : fft32_terms_bound(ls));
    }
  }
  return 1e30;
}

bool algo_applicable(int algo, uint64_t n_t, uint64_t m, uint64_t B) {
  switch (algo) {
    case QRNG_ALGO_DIRECT:
      return true;
    case QRNG_ALGO_GEMM_TC:
    case QRNG_ALGO_GEMM_FP4:
    case QRNG_ALGO_GEMM_FP4_PAIR:
    case QRNG_ALGO_GEMM_KARATSUBA:
      return n_t <= kGemmMaxColumns;
    case QRNG_ALGO_FFT64:
    case QRNG_ALGO_NTT:
      return fft64_length(n_t, m) <= (1ull << 27);
    case QRNG_ALGO_FFT32_SEG:
      return true;
  }
  return false;
}

int extract_one(qrng_ctx* ctx, int algo, const uint8_t* raw, uint64_t n, uint64_t m, const uint8_t* seed, int form,
                uint64_t num_blocks, uint8_t* out, cudaStream_t s, uint32_t* kernels, int fft32_log_s = 0) {
  return extract_bitwise(ctx, algo, raw, n, m, seed, form, num_blocks, out, s, kernels, fft32_log_s);
}

// The autotuner's class of an output length: m with its six leading bits kept (the class is 1/64
// to 1/32 of m wide). The corrected min-entropy of a live stream moves m by a few bits from call
// to call; the routes' costs do not change over such a step, so those calls share one tuning.
uint64_t tune_m_class(uint64_t m) {
  uint32_t lg = 0;
  while (lg < 63 && (2ull << lg) <= m) ++lg;  // floor(log2 m) for m >= 1
  const uint32_t sh = lg > 5 ? lg - 5 : 0;
  return (m >> sh) << sh;
}

qrng_ctx::TuneKey tune_key(uint64_t n, uint64_t m, uint64_t num_blocks, int form) {
  uint32_t lb = 0;
  while ((1ull << lb) < num_blocks) ++lb;
  return qrng_ctx::TuneKey{n, tune_m_class(m), lb, form};
}

// QRNG_ALGO_AUTO: the candidates within 4x of the best modelled time are each run once on the
// call's own data (they give identical bits), timed with CUDA events, and the fastest is kept for
// this shape class; later calls of the class use it directly (or the cost model's choice when the
// kept route does not apply to their exact m). The FP32 route is a candidate once per
// segment length (unless the context fixes it), so the segment length is tuned with it.
int choose_auto(qrng_ctx* ctx, const uint8_t* raw, uint64_t n, uint64_t m, const uint8_t* seed, int form,
                uint64_t num_blocks, uint8_t* out, cudaStream_t s, uint32_t* kernels, int* chosen, int* chosen_log_s,
                bool* done) {
  const uint64_t n_t = (form == QRNG_FORM_MODIFIED) ? n - m : n;
  struct Cand {
    int algo, log_s;
    double model;
  };
  std::vector<Cand> cands;
  const int algos[7] = {QRNG_ALGO_DIRECT, QRNG_ALGO_GEMM_TC, QRNG_ALGO_GEMM_FP4, QRNG_ALGO_GEMM_FP4_PAIR,
                        QRNG_ALGO_GEMM_KARATSUBA, QRNG_ALGO_NTT, QRNG_ALGO_FFT64};
  for (int a : algos)
    if (algo_applicable(a, n_t, m, num_blocks)) cands.push_back({a, 0, model_seconds(ctx, a, n_t, m, num_blocks)});
  for (int ls = 11; ls <= 13; ++ls) {
    if (ctx->fft32_log_s && ctx->fft32_log_s != ls) continue;
    const int T = ctx->fft32_terms ? ctx->fft32_terms : fft32_terms_bound(ls);
    cands.push_back({QRNG_ALGO_FFT32_SEG, ls, fft32_model_seconds(n_t, m, num_blocks, ls, T)});
  }
  double best_model = 1e300;
  Cand best_c{QRNG_ALGO_DIRECT, 0, 0.0};
  for (const Cand& c : cands)
    if (c.model < best_model) {
      best_model = c.model;
      best_c = c;
    }
  *done = false;
  *chosen_log_s = 0;
  if (!ctx->autotune) {
    *chosen = best_c.algo;
    *chosen_log_s = best_c.log_s;
    return QRNG_OK;
  }
  const qrng_ctx::TuneKey key = tune_key(n, m, num_blocks, form);
  for (const auto& e : ctx->tuned)
    if (e.first == key) {
      const bool fits = algo_applicable(e.second.algo, n_t, m, num_blocks);
      *chosen = fits ? e.second.algo : best_c.algo;
      *chosen_log_s = fits ? e.second.fft32_log_s : best_c.log_s;
      return QRNG_OK;
    }
  ++ctx->stats.autotune_runs;
  int best = -1, best_ls = 0;
  float best_ms = 0.f;
  bool last_ok = true;
  for (const Cand& c : cands) {
    if (c.model > 4.0 * best_model) continue;
    cudaEvent_t e0, e1;
    QRNG_CUDA(ctx, cudaEventCreate(&e0), "autotune event");
    QRNG_CUDA(ctx, cudaEventCreate(&e1), "autotune event");
    QRNG_CUDA(ctx, cudaEventRecord(e0, s), "autotune event");
    const int st = extract_one(ctx, c.algo, raw, n, m, seed, form, num_blocks, out, s, kernels, c.log_s);
    QRNG_CUDA(ctx, cudaEventRecord(e1, s), "autotune event");
    QRNG_CUDA(ctx, cudaEventSynchronize(e1), "autotune wait");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    last_ok = (st == QRNG_OK);
    if (st == QRNG_OK && (best < 0 || ms < best_ms)) {
      best = c.algo;
      best_ls = c.log_s;
      best_ms = ms;
    }
  }
  if (best < 0) best = QRNG_ALGO_DIRECT;
  if (best != QRNG_ALGO_FFT32_SEG) best_ls = 0;
  // every candidate that succeeds writes the same bits; a failed last candidate may have left a
  // partial output, so the winner runs once more then
  if (!last_ok) {
    const int st = extract_one(ctx, best, raw, n, m, seed, form, num_blocks, out, s, kernels, best_ls);
    if (st != QRNG_OK) return st;
  }
  ctx->tuned.push_back({key, {best, best_ls}});
  *chosen = best;
  *chosen_log_s = best_ls;
  *done = true;  // the output already holds the result (every candidate writes the same bits)
  return QRNG_OK;
}

int extract_dispatch(qrng_ctx* ctx, const uint8_t* raw, uint64_t n, uint64_t m, const uint8_t* seed, int form,
                     int algo, uint64_t num_blocks, uint8_t* out, cudaStream_t s) {
  uint32_t kernels = 0;
  int st;
  const uint64_t n_t = (form == QRNG_FORM_MODIFIED) ? n - m : n;
  int used = algo, used_log_s = 0;
  if (used == QRNG_ALGO_AUTO) {
    bool done = false;
    st = choose_auto(ctx, raw, n, m, seed, form, num_blocks, out, s, &kernels, &used, &used_log_s, &done);
    if (st != QRNG_OK) return st;
    if (done) {
      ctx->stats.kernels_launched += kernels;
      ctx->stats.last_algo = used;
      ctx->stats.last_kernels = kernels;
      return QRNG_OK;
    }
  }
  switch (used) {
    case QRNG_ALGO_DIRECT:
      st = extract_bitwise(ctx, used, raw, n, m, seed, form, num_blocks, out, s, &kernels);
      break;
    case QRNG_ALGO_FFT64:
    case QRNG_ALGO_FFT32_SEG:
      st = extract_bitwise(ctx, used, raw, n, m, seed, form, num_blocks, out, s, &kernels, used_log_s);
      break;
    case QRNG_ALGO_NTT:
      if (fft64_length(n_t, m) > (1ull << 27))
        return fail(ctx, QRNG_ENOTSUP, "qrng_toeplitz_extract: the transform length exceeds 2^27");
      st = extract_bitwise(ctx, used, raw, n, m, seed, form, num_blocks, out, s, &kernels);
      break;
    case QRNG_ALGO_GEMM_TC:
    case QRNG_ALGO_GEMM_FP4:
    case QRNG_ALGO_GEMM_FP4_PAIR:
    case QRNG_ALGO_GEMM_KARATSUBA:
      if (n_t > kGemmMaxColumns)
        return fail(ctx, QRNG_ENOTSUP, "qrng_toeplitz_extract: the tensor-core path needs n (n-m modified) <= 2^22");
      st = extract_bitwise(ctx, used, raw, n, m, seed, form, num_blocks, out, s, &kernels);
      break;
    default:
      return fail(ctx, QRNG_ENOTSUP, "qrng_toeplitz_extract: algorithm not available for these arguments");
  }
  ctx->stats.kernels_launched += kernels;
  if (st == QRNG_OK) {
    ctx->stats.last_algo = used;
    ctx->stats.last_kernels = kernels;
  }
  return st;
}

uint64_t fnv1a(const void* data, size_t bytes, uint64_t h = 1469598103934665603ull) {
  const uint8_t* p = static_cast<const uint8_t*>(data);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

void drop_graph(qrng_ctx::BatchGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  if (g.meta_host) cudaFreeHost(g.meta_host);
  for (cudaEvent_t& e : g.ev)
    if (e) cudaEventDestroy(e);
  g = qrng_ctx::BatchGraph{};
}

void drop_all_graphs(qrng_ctx* ctx) {
  for (auto& g : ctx->graphs) drop_graph(g);
  ctx->graphs.clear();
}

// Grows a buffer a batch graph uses; any move invalidates the graphs that captured the old address.
cudaError_t ensure_batch(qrng_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes <= b.cap) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(ctx->capture_stream);
  if (e != cudaSuccess) return e;
  e = cudaDeviceSynchronize();  // a replay may still read the old buffer
  if (e != cudaSuccess) return e;
  drop_all_graphs(ctx);
  ++ctx->batch_generation;
  return b.ensure(bytes);
}

constexpr size_t kMaxGraphs = 4;
constexpr uint64_t kFft32BatchBudget = 1ull << 30;  // bytes of FP32 spectra per group

// ---- uneven batches ----
//
// A call is planned on the host: every request gets a route (the persistent direct kernel, or one
// of the batched circulant routes: number-theoretic transform, FP64 FFT, FP32 segmented FFT);
// direct requests come first in the device table (largest work first), then the transform
// requests in groups (one transform length, or one FP32 segment length, per group, within a
// workspace budget). One launch sequence runs the plan: table upload, staging of the direct
// requests, every transform group, the persistent kernel, and the merge of all outputs into the
// callers' bit offsets. The sequence is captured once into a CUDA graph cached on the context, so
// every call is one graph replay; the transform workspace belongs to the batch path alone and is
// sized before capture, and each group recomputes its twiddle tables inside the graph.

struct BatchGroup {
  uint64_t begin, end;  // device-table range
  int route;
  uint64_t P;           // transform length (NTT, FP64)
  int log_s;            // FP32 segment length
  uint64_t max_mw, spec_items, mac_ctas, spec_rows;
};

struct BatchPlan {
  std::vector<BatchReq> reqs;  // device order
  std::vector<BatchGroup> groups;
  uint64_t raw_total = 0, rev_total = 0, out_total = 0, items = 0, dst_total = 0, direct_out = 0;
  size_t buf0 = 0, buf1 = 0, spec = 0, ntt_tw = 0, tw = 0, tw32 = 0;  // transform workspace needs
  uint64_t routes[4] = {0, 0, 0, 0};
};

uint64_t ilog2_ceil(uint64_t x) {
  uint64_t l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

// Modelled seconds of one request on a route (prunes the autotuner's candidates; the choice when
// autotuning is off). Rates measured on GB300 for the batched kernels.
double route_model(int route, uint64_t n_t, uint64_t m, int log_s) {
  const uint64_t P = fft64_length(n_t, m);
  const double lg = log2((double)P);
  switch (route) {
    case kRouteDirect:
      return (double)m * (double)n_t / 5.6e14 + 2e-8;
    case kRouteNtt:
      return P > (1ull << 27) ? 1e30 : (double)P * lg * 1.3e-12;
    case kRouteFft64:
      return P > (1ull << 27) ? 1e30 : (double)P * lg * 1.6e-11;
    case kRouteFft32:
      return fft32_model_seconds(n_t, m, 1, log_s, fft32_terms_bound(log_s)) - 2e-5;
  }
  return 1e30;
}

BatchReq base_request(const qrng_request& r) {
  BatchReq q{};
  q.raw = r.raw;
  q.raw_bit_off = r.raw_bit_off;
  q.n = r.n;
  q.m = r.m;
  q.seed = r.seed;
  q.form = r.form;
  q.out = r.out;
  q.out_bit_off = r.out_bit_off;
  q.n_t = r.form == QRNG_FORM_MODIFIED ? r.n - r.m : r.n;
  q.L_t = q.n_t + r.m - 1;
  q.nw_t = (uint32_t)ceil_div(q.n_t, 32);
  q.tail_mask = (q.n_t % 32) ? ((1u << (q.n_t % 32)) - 1u) : 0xffffffffu;
  q.mw = (uint32_t)ceil_div(r.m, 32);
  q.id_off = (uint32_t)(r.n - r.m);
  const uint64_t first = (reinterpret_cast<uintptr_t>(r.out) * 8 + r.out_bit_off);
  q.dst_word0 = first / 32;
  q.dst_words = (first + r.m - 1) / 32 - q.dst_word0 + 1;
  return q;
}

// Plan of the requests idx[...] (indices into reqs) with routes route[i] and FP32 segment lengths log_s[i].
BatchPlan make_plan(const qrng_request* reqs, const std::vector<uint64_t>& idx, const std::vector<int>& route,
                    const std::vector<int>& log_s) {
  BatchPlan p;
  std::vector<BatchReq> t;
  std::vector<uint64_t> key;  // group key of transform requests
  t.reserve(idx.size());
  for (uint64_t i : idx) {
    BatchReq q = base_request(reqs[i]);
    q.route = route[i];
    if (q.route == kRouteDirect) {
      q.tiles = (uint32_t)ceil_div(q.m, (uint64_t)direct_outputs_per_warp());
      q.splits = (uint32_t)ceil_div(q.nw_t, kBatchWordsPerSplit);
      q.raw_words = ceil_div(q.n, 32);
      q.rev_words = kSeedFrontWords + ceil_div(q.L_t, 32) + kSeedBackWords;
    } else if (q.route == kRouteFft32) {
      const uint64_t S = 1ull << log_s[i];
      q.seg_ns = (uint32_t)ceil_div(q.n_t, S);
      q.seg_nq = (uint32_t)ceil_div(q.m, S);
    }
    t.push_back(q);
    key.push_back(q.route == kRouteFft32 ? (uint64_t)log_s[i] : fft64_length(q.n_t, q.m));
  }
  std::vector<uint64_t> order(t.size());
  for (uint64_t k = 0; k < order.size(); ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](uint64_t x, uint64_t y) {
    const bool dx = t[x].route == kRouteDirect, dy = t[y].route == kRouteDirect;
    if (dx != dy) return dx;                                         // direct requests first
    if (!dx && t[x].route != t[y].route) return t[x].route < t[y].route;
    if (!dx && key[x] != key[y]) return key[x] > key[y];              // transforms grouped
    return t[x].m * t[x].n_t > t[y].m * t[y].n_t;                     // largest work first
  });
  p.reqs.resize(t.size());
  for (uint64_t k = 0; k < order.size(); ++k) {
    BatchReq q = t[order[k]];
    ++p.routes[q.route];
    q.raw_stage_off = p.raw_total;
    p.raw_total += q.raw_words;
    q.rev_off = p.rev_total;
    p.rev_total += q.rev_words;
    q.out_stage_off = p.out_total;
    p.out_total += q.mw;
    q.item_begin = p.items;
    p.items += (uint64_t)q.tiles * q.splits;
    q.dst_begin = p.dst_total;
    p.dst_total += q.dst_words;
    if (q.route == kRouteDirect) p.direct_out = p.out_total;
    p.reqs[k] = q;
  }
  // transform groups within the workspace budget
  for (uint64_t k = 0; k < p.reqs.size();) {
    BatchReq& q0 = p.reqs[k];
    if (q0.route == kRouteDirect) {
      ++k;
      continue;
    }
    BatchGroup g{};
    g.begin = k;
    g.route = q0.route;
    const uint64_t gk = key[order[k]];
    if (g.route == kRouteFft32) g.log_s = (int)gk;
    else g.P = gk;
    const uint64_t S = g.route == kRouteFft32 ? (1ull << g.log_s) : 0;
    const int qt = g.route == kRouteFft32 ? fft32_batch_tiles(g.log_s) : 1;
    uint64_t e = k, bytes = 0;
    while (e < p.reqs.size() && p.reqs[e].route == g.route && key[order[e]] == gk) {
      BatchReq& q = p.reqs[e];
      uint64_t need;
      if (g.route == kRouteFft32) need = ((uint64_t)q.seg_nq + 2ull * q.seg_ns - 1) * S * 8;
      else if (g.route == kRouteNtt) need = 2 * g.P * 4;
      else need = 2 * g.P * 16;
      const uint64_t budget = g.route == kRouteFft32 ? kFft32BatchBudget : kFftWorkspaceBytes;
      if (e > k && bytes + need > budget) break;
      if (g.route == kRouteFft32) {
        q.spec_row = g.spec_rows;
        q.spec_item_begin = g.spec_items;
        q.mac_cta_begin = g.mac_ctas;
        const uint64_t rows = (uint64_t)q.seg_nq + 2ull * q.seg_ns - 1;
        g.spec_rows += rows;
        g.spec_items += rows;
        g.mac_ctas += ceil_div(q.seg_nq, (uint64_t)qt);
      }
      if (q.mw > g.max_mw) g.max_mw = q.mw;
      bytes += need;
      ++e;
    }
    g.end = e;
    const uint64_t nr = e - k;
    if (g.route == kRouteNtt) {
      p.buf0 = std::max<size_t>(p.buf0, 2 * nr * g.P * 4);
      p.buf1 = std::max<size_t>(p.buf1, nr * (g.P / 8));
      p.ntt_tw = std::max<size_t>(p.ntt_tw, (g.P / 2) * 4);
    } else if (g.route == kRouteFft64) {
      p.buf0 = std::max<size_t>(p.buf0, nr * g.P * 16);
      p.buf1 = std::max<size_t>(p.buf1, nr * g.P * 16);
      p.tw = std::max<size_t>(p.tw, (g.P / 2) * 16);
    } else {
      p.spec = std::max<size_t>(p.spec, g.spec_rows * S * 8);
      p.tw32 = std::max<size_t>(p.tw32, S * 8);
    }
    p.groups.push_back(g);
    k = e;
  }
  return p;
}

// Buffers of a plan (grown before any capture; a move drops the cached graphs).
int ensure_plan(qrng_ctx* ctx, const BatchPlan& p) {
  FftWorkspace& w = ctx->batch_fft;
  QRNG_CUDA(ctx, ensure_batch(ctx, ctx->batch_meta, p.reqs.size() * sizeof(BatchReq)), "batch table workspace");
  QRNG_CUDA(ctx, ensure_batch(ctx, ctx->batch_raw, (p.raw_total ? p.raw_total : 1) * 4), "batch raw workspace");
  QRNG_CUDA(ctx, ensure_batch(ctx, ctx->batch_rev, (p.rev_total ? p.rev_total : 1) * 4), "batch seed workspace");
  QRNG_CUDA(ctx, ensure_batch(ctx, ctx->batch_out, (p.out_total ? p.out_total : 1) * 4), "batch output workspace");
  QRNG_CUDA(ctx, ensure_batch(ctx, ctx->batch_counter, sizeof(unsigned long long)), "batch counter");
  QRNG_CUDA(ctx, ensure_batch(ctx, w.buf0, p.buf0 ? p.buf0 : 1), "batch transform workspace");
  QRNG_CUDA(ctx, ensure_batch(ctx, w.buf1, p.buf1 ? p.buf1 : 1), "batch transform workspace");
  QRNG_CUDA(ctx, ensure_batch(ctx, w.spec, p.spec ? p.spec : 1), "batch spectra workspace");
  QRNG_CUDA(ctx, ensure_batch(ctx, w.ntt_tw, p.ntt_tw ? p.ntt_tw : 1), "batch twiddle workspace");
  QRNG_CUDA(ctx, ensure_batch(ctx, w.tw, p.tw ? p.tw : 1), "batch twiddle workspace");
  QRNG_CUDA(ctx, ensure_batch(ctx, w.tw32, p.tw32 ? p.tw32 : 1), "batch twiddle workspace");
  for (const BatchGroup& g : p.groups)
    if (g.route == kRouteNtt && !w.ntt_stage.p) {
      // the NTT's constant stage table, once, outside any capture (its buffer never moves)
      uint32_t k = 0;
      QRNG_CUDA(ctx, ntt_prepare(w, g.P, ctx->capture_stream, &k), "batch NTT tables");
      QRNG_CUDA(ctx, cudaStreamSynchronize(ctx->capture_stream), "batch NTT tables");
    }
  return QRNG_OK;
}

// The launch sequence of a plan on stream cs; its request table is uploaded from pinned `meta_host`.
// ev (may be null): events recorded before and after the transform groups and the direct kernel.
cudaError_t run_plan(qrng_ctx* ctx, const BatchPlan& p, const void* meta_host, bool merge, cudaStream_t cs,
                     uint32_t* kernels, const cudaEvent_t* ev = nullptr) {
  const uint32_t count = (uint32_t)p.reqs.size();
  BatchReq* meta = ctx->batch_meta.as<BatchReq>();
  cudaError_t e = cudaMemcpyAsync(meta, meta_host, count * sizeof(BatchReq), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->batch_counter.p, 0, sizeof(unsigned long long), cs);
  if (e == cudaSuccess && p.direct_out) e = cudaMemsetAsync(ctx->batch_out.p, 0, p.direct_out * 4, cs);
  if (e == cudaSuccess && p.raw_total)
    e = launch_batch_layout(meta, count, p.raw_total, p.rev_total, ctx->batch_raw.as<uint32_t>(),
                            ctx->batch_rev.as<uint32_t>(), cs, kernels);
  FftWorkspace& w = ctx->batch_fft;
  w.worst = ctx->fft_worst.as<unsigned long long>();  // a batch trip is reported by qrng_synchronize
  // graph nodes that record the events on every replay (external records of a capture)
  if (e == cudaSuccess && ev && !p.groups.empty()) e = cudaEventRecordWithFlags(ev[0], cs, cudaEventRecordExternal);
  for (const BatchGroup& g : p.groups) {
    if (e != cudaSuccess) break;
    const uint64_t nr = g.end - g.begin;
    if (g.route == kRouteNtt) {
      w.ntt_P = 0;  // the group's twiddles are computed inside the sequence
      e = launch_ntt_batch(meta + g.begin, nr, g.P, g.max_mw, w, ctx->batch_out.as<uint32_t>(), cs, kernels);
    } else if (g.route == kRouteFft64) {
      w.tw_P = 0;
      e = launch_fft64_batch(meta + g.begin, nr, g.P, g.max_mw, w, ctx->batch_out.as<uint32_t>(), cs, kernels);
    } else {
      w.tw32_S = 0;
      e = launch_fft32_batch(meta + g.begin, nr, g.spec_items, g.mac_ctas, g.log_s, fft32_terms_bound(g.log_s), w,
                             ctx->batch_out.as<uint32_t>(), cs, kernels);
    }
  }
  if (e == cudaSuccess && ev && !p.groups.empty()) e = cudaEventRecordWithFlags(ev[1], cs, cudaEventRecordExternal);
  if (e == cudaSuccess && ev && p.items) e = cudaEventRecordWithFlags(ev[2], cs, cudaEventRecordExternal);
  if (e == cudaSuccess && p.items)
    e = launch_batch_direct(meta, count, p.items, ctx->batch_raw.as<uint32_t>(), ctx->batch_rev.as<uint32_t>(),
                            ctx->batch_out.as<uint32_t>(), ctx->batch_counter.as<unsigned long long>(), ctx->num_sms,
                            cs, kernels);
  if (e == cudaSuccess && ev && p.items) e = cudaEventRecordWithFlags(ev[3], cs, cudaEventRecordExternal);
  if (e == cudaSuccess && merge)
    e = launch_batch_pack(meta, count, p.dst_total, ctx->batch_out.as<uint32_t>(), cs, kernels);
  return e;
}

// Pinned host staging of at least `bytes` for a tuner's table.
int tune_staging(qrng_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->tune_host_cap) return QRNG_OK;
  if (ctx->tune_host) cudaFreeHost(ctx->tune_host);
  ctx->tune_host = nullptr;
  ctx->tune_host_cap = 0;
  QRNG_CUDA(ctx, cudaMallocHost(&ctx->tune_host, bytes), "pinned tuner table");
  ctx->tune_host_cap = bytes;
  return QRNG_OK;
}

// QRNG_ALGO_AUTO: the route of each shape class (transform length P). A class seen for the first
// time has the routes the cost model keeps (within 4x of its best) each run once on the class's
// requests of this call, timed with CUDA events; the fastest is kept on the context.
int tune_classes(qrng_ctx* ctx, const qrng_request* reqs, uint64_t count, std::vector<int>& route,
                 std::vector<int>& log_s) {
  std::vector<uint64_t> cls(count);
  for (uint64_t i = 0; i < count; ++i) {
    const BatchReq q = base_request(reqs[i]);
    cls[i] = fft64_length(q.n_t, q.m);
  }
  std::vector<uint64_t> todo;
  for (uint64_t i = 0; i < count; ++i) {
    bool known = false;
    for (const auto& bt : ctx->batch_tuned) known = known || bt.P == cls[i];
    for (uint64_t c : todo) known = known || c == cls[i];
    if (!known) todo.push_back(cls[i]);
  }
  cudaStream_t cs = ctx->capture_stream;
  for (uint64_t P : todo) {
    std::vector<uint64_t> members;
    for (uint64_t i = 0; i < count; ++i)
      if (cls[i] == P) members.push_back(i);
    struct Cand {
      int route, log_s;
      double model;
    };
    std::vector<Cand> cands;
    for (int r = kRouteDirect; r <= kRouteFft32; ++r) {
      for (int ls = 11; ls <= (r == kRouteFft32 ? 13 : 11); ++ls) {
        double t = 0;
        for (uint64_t i : members) {
          const BatchReq q = base_request(reqs[i]);
          t += route_model(r, q.n_t, q.m, ls);
        }
        cands.push_back({r, r == kRouteFft32 ? ls : 0, t});
      }
    }
    double best_model = 1e300;
    for (const Cand& c : cands) best_model = std::min(best_model, c.model);
    int best_r = kRouteDirect, best_ls = 0;
    float best_ms = -1.f;
    for (const Cand& c : cands) {
      if (c.model > 4.0 * best_model || c.model >= 1e29) continue;
      std::vector<int> r2(count, c.route), l2(count, c.log_s);
      const BatchPlan sub = make_plan(reqs, members, r2, l2);
      int st = ensure_plan(ctx, sub);
      if (st) return st;
      st = tune_staging(ctx, sub.reqs.size() * sizeof(BatchReq));
      if (st) return st;
      QRNG_CUDA(ctx, cudaStreamSynchronize(cs), "batch tuner");
      memcpy(ctx->tune_host, sub.reqs.data(), sub.reqs.size() * sizeof(BatchReq));
      cudaEvent_t e0, e1;
      QRNG_CUDA(ctx, cudaEventCreate(&e0), "batch tuner event");
      QRNG_CUDA(ctx, cudaEventCreate(&e1), "batch tuner event");
      uint32_t k = 0;
      QRNG_CUDA(ctx, cudaEventRecord(e0, cs), "batch tuner event");
      const cudaError_t e = run_plan(ctx, sub, ctx->tune_host, false, cs, &k);
      QRNG_CUDA(ctx, cudaEventRecord(e1, cs), "batch tuner event");
      QRNG_CUDA(ctx, cudaEventSynchronize(e1), "batch tuner wait");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      ctx->stats.kernels_launched += k;
      if (e == cudaSuccess && (best_ms < 0 || ms < best_ms)) {
        best_ms = ms;
        best_r = c.route;
        best_ls = c.log_s;
      }
    }
    ctx->batch_tuned.push_back({P, best_r, best_ls});
  }
  for (uint64_t i = 0; i < count; ++i)
    for (const auto& bt : ctx->batch_tuned)
      if (bt.P == cls[i]) {
        route[i] = bt.route;
        log_s[i] = bt.log_s;
      }
  return QRNG_OK;
}

int extract_batch(qrng_ctx* ctx, const qrng_request* reqs, uint64_t count, int algo, cudaStream_t s) {
  std::vector<int> route(count, kRouteDirect), log_s(count, 0);
  for (uint64_t i = 0; i < count; ++i) {
    const BatchReq q = base_request(reqs[i]);
    const bool fits = fft64_length(q.n_t, q.m) <= (1ull << 27);
    if (algo == QRNG_ALGO_NTT && fits) route[i] = kRouteNtt;
    else if (algo == QRNG_ALGO_FFT64 && fits) route[i] = kRouteFft64;
    else if (algo == QRNG_ALGO_FFT32_SEG) {
      route[i] = kRouteFft32;
      int best = 12;
      double bt = 1e300;
      for (int ls = 11; ls <= 13; ++ls) {
        if (ctx->fft32_log_s && ctx->fft32_log_s != ls) continue;
        const double t = route_model(kRouteFft32, q.n_t, q.m, ls);
        if (t < bt) {
          bt = t;
          best = ls;
        }
      }
      log_s[i] = best;
    }
  }
  if (algo == QRNG_ALGO_AUTO) {
    if (ctx->autotune) {
      const int st = tune_classes(ctx, reqs, count, route, log_s);
      if (st) return st;
    } else {
      for (uint64_t i = 0; i < count; ++i) {  // the cost model alone
        const BatchReq q = base_request(reqs[i]);
        double bt = 1e300;
        for (int r = kRouteDirect; r <= kRouteFft32; ++r)
          for (int ls = 11; ls <= (r == kRouteFft32 ? 13 : 11); ++ls) {
            const double t = route_model(r, q.n_t, q.m, ls);
            if (t < bt) {
              bt = t;
              route[i] = r;
              log_s[i] = r == kRouteFft32 ? ls : 0;
            }
          }
      }
    }
  }
  std::vector<uint64_t> all(count);
  for (uint64_t i = 0; i < count; ++i) all[i] = i;
  const BatchPlan plan = make_plan(reqs, all, route, log_s);
  const uint64_t key = fnv1a(plan.reqs.data(), plan.reqs.size() * sizeof(BatchReq), fnv1a(&count, sizeof(count)));
  int st = ensure_plan(ctx, plan);
  if (st) return st;

  qrng_ctx::BatchGraph* hit = nullptr;
  for (auto& g : ctx->graphs)
    if (g.key == key && g.generation == ctx->batch_generation) hit = &g;
  if (!hit) {
    if (ctx->graphs.size() >= kMaxGraphs) {  // evict the least recently used graph
      size_t victim = 0;
      for (size_t i = 1; i < ctx->graphs.size(); ++i)
        if (ctx->graphs[i].stamp < ctx->graphs[victim].stamp) victim = i;
      QRNG_CUDA(ctx, cudaStreamSynchronize(s), "graph eviction");
      drop_graph(ctx->graphs[victim]);
      ctx->graphs.erase(ctx->graphs.begin() + victim);
    }
    qrng_ctx::BatchGraph g;
    g.key = key;
    g.generation = ctx->batch_generation;
    for (int r = 0; r < 4; ++r) g.routes[r] = plan.routes[r];
    for (const BatchReq& q : plan.reqs) {
      if (q.route == kRouteDirect) g.direct_bitmacs += (double)q.m * (double)q.n_t;
      else g.transform_bytes += (double)(q.n + q.m) / 8.0;
    }
    g.has_transform = !plan.groups.empty();
    g.has_direct = plan.items != 0;
    for (cudaEvent_t& ev : g.ev) {
      const cudaError_t ee = cudaEventCreate(&ev);
      if (ee != cudaSuccess) {
        drop_graph(g);
        return cuda_fail(ctx, ee, "batch graph events");
      }
    }
    QRNG_CUDA(ctx, cudaMallocHost(&g.meta_host, count * sizeof(BatchReq)), "pinned request table");
    memcpy(g.meta_host, plan.reqs.data(), count * sizeof(BatchReq));
    cudaStream_t cs = ctx->capture_stream;
    QRNG_CUDA(ctx, cudaStreamSynchronize(cs), "batch capture");
    // relaxed: the launchers set kernel attributes while the sequence is captured
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) e = run_plan(ctx, plan, g.meta_host, true, cs, &g.kernels, g.ev);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    g.graph = graph;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (e != cudaSuccess) {
      drop_graph(g);
      return cuda_fail(ctx, e, "batch graph capture");
    }
    ctx->graphs.push_back(g);
    hit = &ctx->graphs.back();
  }
  hit->stamp = ++ctx->graph_clock;
  LaunchTimer gtimer(ctx, s, kTimeBatchGraph);
  QRNG_CUDA(ctx, cudaGraphLaunch(hit->exec, s), "batch graph launch");
  gtimer.done();
  ctx->stats.kernels_launched += hit->kernels;
  ctx->stats.last_kernels = hit->kernels;
  for (int r = 0; r < 4; ++r) ctx->stats.batch_requests[r] = hit->routes[r];
  ctx->stats.batch_direct_bitmacs = hit->direct_bitmacs;
  ctx->stats.batch_transform_bytes = hit->transform_bytes;
  if (ctx->timing) {
    ctx->timed_graph_pending = true;
    ctx->timed_graph_key = hit->key;
    ctx->timed_graph_generation = hit->generation;
  }
  static const int kAlgoOfRoute[4] = {QRNG_ALGO_DIRECT, QRNG_ALGO_NTT, QRNG_ALGO_FFT64, QRNG_ALGO_FFT32_SEG};
  int used = -1;
  for (int r = 0; r < 4; ++r)
    if (hit->routes[r]) used = (used == -1) ? kAlgoOfRoute[r] : QRNG_ALGO_AUTO;
  ctx->stats.last_algo = used < 0 ? QRNG_ALGO_DIRECT : used;
  return QRNG_OK;
}

// The QRNG_ALGO_AUTO choice already tuned for this shape, or -1.
int tuned_choice(const qrng_ctx* ctx, uint64_t n, uint64_t m, uint64_t num_blocks, int form) {
  if (!ctx->autotune) return -1;
  const qrng_ctx::TuneKey key = tune_key(n, m, num_blocks, form);
  for (const auto& e : ctx->tuned)
    if (e.first == key) return e.second.algo;
  return -1;
}

// The block-Karatsuba route's derived operands depend on the raw blocks, n_t and the plan, not on
// the seed: when the previous pipeline call of this stream shape settled on that route, they are
// computed on the context's second stream while the min-entropy estimate and its read-back run,
// for the m that call found (a different m this time only costs the split again). The pipeline
// makes its stream wait for the second stream before hashing.
bool pipeline_presplit(qrng_ctx* ctx, const uint8_t* raw, uint64_t n, int form, int algo, uint64_t num_blocks,
                       uint64_t count, int bits, cudaStream_t s) {
  ctx->kara.xk_ready = false;
  const qrng_ctx::PipelineShape shape{n, count, bits, form, num_blocks};
  if (!ctx->pipeline_seen || !(ctx->pipeline_shape == shape) || num_blocks == 0) return false;
  const uint64_t m = ctx->pipeline_m;
  if (m == 0 || m > n || (form == QRNG_FORM_MODIFIED && m >= n)) return false;
  const int a = algo == QRNG_ALGO_AUTO ? tuned_choice(ctx, n, m, num_blocks, form) : algo;
  if (a != QRNG_ALGO_GEMM_KARATSUBA) return false;
  const uint64_t n_t = form == QRNG_FORM_MODIFIED ? n - m : n;
  if (!algo_applicable(QRNG_ALGO_GEMM_KARATSUBA, n_t, m, num_blocks)) return false;
  // only when the extraction reads the raw blocks in place (otherwise it repacks them first)
  if (n % 128 != 0 || (reinterpret_cast<uintptr_t>(raw) & 15) != 0) return false;
  const KaraPlan plan = karatsuba_plan(n_t, m, num_blocks, ctx->num_sms, ctx->kara_levels, ctx->kara_h,
                                       ctx->kara_workspace);
  if (plan.levels == 0) return false;
  DirectArgs a_args{};
  a_args.n_t = n_t;
  a_args.raw = reinterpret_cast<const uint32_t*>(raw);
  a_args.raw_stride = n / 32;
  a_args.nw_t = (uint32_t)ceil_div(n_t, 32);
  a_args.tail_mask = (n_t % 32) ? ((1u << (n_t % 32)) - 1u) : 0xffffffffu;
  a_args.num_blocks = num_blocks;
  if (cudaEventRecord(ctx->pre_ready, s) != cudaSuccess) return false;
  if (cudaStreamWaitEvent(ctx->copy_stream, ctx->pre_ready, 0) != cudaSuccess) return false;
  uint32_t kernels = 0;
  if (launch_kara_presplit(a_args, plan, ctx->kara, ctx->num_sms, ctx->copy_stream, &kernels) != cudaSuccess) {
    ctx->kara.xk_ready = false;
    cudaGetLastError();
    return false;
  }
  ctx->stats.kernels_launched += kernels;
  ++ctx->stats.kara_presplits;
  if (cudaEventRecord(ctx->pre_done, ctx->copy_stream) != cudaSuccess) {
    cudaStreamSynchronize(ctx->copy_stream);
    ctx->kara.xk_ready = false;
  }
  return true;
}

// The pipeline's first half on device samples: the pre-split above, the min-entropy estimate
// (which synchronises `s`) and the output length; `first_blocks` is the block count of the first
// extraction call that follows. On return `s` is ordered after the pre-split.
int pipeline_size(qrng_ctx* ctx, const char* who, const void* samples, uint64_t count, int bits, double eps,
                  double eps_lhl, uint64_t n, uint64_t seed_capacity_bits, int form, int algo,
                  uint64_t first_blocks, cudaStream_t s, uint64_t* m_out, qrng_hmin_report* rep) {
  *m_out = 0;
  const std::string w(who);
  if (form != QRNG_FORM_STANDARD && form != QRNG_FORM_MODIFIED) return fail(ctx, QRNG_EINVAL, w + ": unknown form");
  if (n < 2 || n > kMaxBlockBits) return fail(ctx, QRNG_EINVAL, w + ": n must be in [2, 2^26]");
  if (!(eps_lhl > 0.0 && eps_lhl <= 1.0)) return fail(ctx, QRNG_EINVAL, w + ": eps_lhl in (0, 1]");
  qrng_hmin_report local{};
  int st = check_minentropy_args(ctx, samples, count, bits, eps, &local);
  if (st) return st;
  const uint64_t bytes = count * (bits <= 8 ? 1 : 2);
  const uint64_t num_blocks = bytes * 8 / n;
  const bool pre = pipeline_presplit(ctx, static_cast<const uint8_t*>(samples), n, form, algo, first_blocks, count,
                                     bits, s);
  st = minentropy_dev(ctx, samples, count, bits, eps, &local, s);
  if (pre) {
    const cudaError_t e = cudaStreamWaitEvent(s, ctx->pre_done, 0);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(ctx->copy_stream);
      ctx->kara.xk_ready = false;
    }
  }
  if (st) {
    ctx->kara.xk_ready = false;
    return st;
  }
  if (rep) *rep = local;
  uint64_t m = qrng_output_length(n, local.h_modify, bits, eps_lhl);
  if (form == QRNG_FORM_MODIFIED && m >= n) m = n - 1;
  if (m > n) m = n;
  *m_out = m;
  ctx->pipeline_seen = true;
  ctx->pipeline_shape = qrng_ctx::PipelineShape{n, count, bits, form, first_blocks};
  ctx->pipeline_m = m;
  const char* bad = m == 0 ? ": the corrected min-entropy gives m = 0"
                    : num_blocks == 0 ? ": fewer than n raw bits"
                    : seed_capacity_bits < qrng_seed_bits(n, m, form) ? ": seed shorter than the hash needs"
                    : nullptr;
  if (bad) {
    ctx->kara.xk_ready = false;
    return fail(ctx, QRNG_EINVAL, w + bad);
  }
  return QRNG_OK;
}

// ---- speculative hash of the pipeline ----
//
// After a qrng_postprocess call of a stream shape that hashed on the block-Karatsuba route in the
// standard form, the next call of that shape does not wait for its estimate before hashing: it
// enqueues the estimate, the output length computed from it on the device, and the hash for up to
// m_cap rows (the previous m rounded up to the plan's row span, so the product issues the tiles the
// previous call did), with the derived operands and seeds on the second stream beside the
// estimate. The product kernel returns at once and the combination writes nothing unless the
// device's m is at most m_cap (and at least kSpecMinBits) and the call is valid; the host reads
// the report while the product runs, finds the same m, and hashes again on the ordinary path when
// the hash did not stand.
struct SpecPlan {
  uint64_t m_cap = 0;
  KaraPlan plan;
};

bool spec_plan(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, uint64_t n, int form, int algo,
               uint64_t nb, uint64_t seed_capacity_bits, const uint8_t* out, SpecPlan* sp) {
  const qrng_ctx::PipelineShape shape{n, count, bits, form, nb};
  if (!ctx->pipeline_seen || !(ctx->pipeline_shape == shape) || form != QRNG_FORM_STANDARD || nb == 0) return false;
  const uint64_t m_prev = ctx->pipeline_m;
  if (m_prev < kSpecMinBits || m_prev > n || seed_capacity_bits < n + m_prev - 1) return false;
  const int a = algo == QRNG_ALGO_AUTO ? tuned_choice(ctx, n, m_prev, nb, form) : algo;
  if (a != QRNG_ALGO_GEMM_KARATSUBA || !algo_applicable(a, n, m_prev, nb)) return false;
  // raw blocks read in place; the packed output a whole number of aligned words for every m
  if (n % 128 != 0 || (reinterpret_cast<uintptr_t>(samples) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(out) & 3) != 0 || nb % 32 != 0)
    return false;
  const KaraPlan p0 = karatsuba_plan(n, m_prev, nb, ctx->num_sms, ctx->kara_levels, ctx->kara_h, ctx->kara_workspace);
  if (p0.levels == 0) return false;
  uint64_t m_cap = ceil_div(m_prev, p0.span) * p0.span;
  if (m_cap > n) m_cap = n;
  if (m_cap > seed_capacity_bits - n + 1) m_cap = seed_capacity_bits - n + 1;  // >= m_prev
  const KaraPlan p = karatsuba_plan(n, m_cap, nb, ctx->num_sms, ctx->kara_levels, ctx->kara_h, ctx->kara_workspace);
  if (!kara_speculation_fits(p, m_cap, nb)) return false;
  sp->m_cap = m_cap;
  sp->plan = p;
  return true;
}

// Enqueues the speculative call and reads its report. *done: the output is written (or the call
// refused, st != 0); otherwise the caller hashes with *m_out on the ordinary path.
// ws, seed_rev and spec_buf hold the hash's derived operands, seeds, reversed seed and device-side
// m; the second stream's part waits for `inputs_ready` when given (the samples and seed are the
// library's own upload and nothing on `s` touches those buffers before it), else for the work
// already on `s`. With combine_stream the combination runs there, after the product.
int postprocess_speculative(qrng_ctx* ctx, const SpecPlan& sp, const void* samples, uint64_t count, int bits,
                            double eps, double eps_lhl, uint64_t n, const uint8_t* seed, uint64_t seed_capacity_bits,
                            uint8_t* out, uint64_t out_capacity_bytes, uint64_t nb, cudaStream_t s, uint64_t* m_out,
                            qrng_hmin_report* rep, bool* done, KaraWorkspace& ws, DevBuf& seed_rev,
                            DevBuf& spec_buf, cudaEvent_t inputs_ready = nullptr,
                            cudaStream_t combine_stream = nullptr) {
  *done = false;
  *m_out = 0;
  const std::string w("qrng_postprocess");
  qrng_hmin_report local{};
  int st = check_minentropy_args(ctx, samples, count, bits, eps, &local);
  if (st) return st;
  // the derived operands enqueued below belong to this call's hash alone: whatever way the call
  // returns, no later launch may take them for its own
  struct NotReady {
    KaraWorkspace& w;
    ~NotReady() { w.xk_ready = false; }
  } not_ready{ws};
  ws.xk_ready = false;
  QRNG_CUDA(ctx, spec_buf.ensure(sizeof(DevSpec)), "pipeline size word");
  if (!ctx->report_stream) {
    QRNG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->report_stream, cudaStreamNonBlocking), "report stream");
    QRNG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->spec_sized, cudaEventDisableTiming), "event");
    QRNG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->spec_est, cudaEventDisableTiming), "event");
    QRNG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->spec_product, cudaEventDisableTiming), "event");
    QRNG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->spec_hashed, cudaEventDisableTiming), "event");
  }
  const uint64_t m_cap = sp.m_cap;
  const uint64_t rev_words = kSeedFrontWords + ceil_div(n + m_cap - 1, 32) + kSeedBackWords;
  QRNG_CUDA(ctx, seed_rev.ensure(rev_words * 4), "seed workspace");
  DirectArgs a{};
  a.raw = static_cast<const uint32_t*>(samples);
  a.raw_stride = n / 32;
  a.n_t = n;
  a.nw_t = (uint32_t)ceil_div(n, 32);
  a.tail_mask = 0xffffffffu;  // n is a multiple of 128
  a.m = (uint32_t)m_cap;
  a.mw = (uint32_t)ceil_div(m_cap, 32);
  a.seed_rev = seed_rev.as<uint32_t>();
  a.modified = 0;
  a.id_off = (uint32_t)(n - m_cap);
  a.out = nullptr;  // the combination writes the packed stream
  a.out_stride = a.mw;
  a.num_blocks = nb;

  // second stream: derived operands, reversed seed, derived seeds
  uint32_t kernels = 0;
  if (!inputs_ready) {
    QRNG_CUDA(ctx, cudaEventRecord(ctx->pre_ready, s), "pipeline event");
    inputs_ready = ctx->pre_ready;
  }
  QRNG_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, inputs_ready, 0), "pipeline event");
  QRNG_CUDA(ctx, launch_kara_presplit(a, sp.plan, ws, ctx->num_sms, ctx->copy_stream, &kernels),
            "derived operands");
  ++ctx->stats.kara_presplits;
  QRNG_CUDA(ctx, launch_seed_reverse(seed, n + m_cap - 1, seed_rev.as<uint32_t>(), rev_words, ctx->copy_stream,
                                     &kernels),
            "seed reverse");
  QRNG_CUDA(ctx, launch_kara_seeds(a, sp.plan, ws, ctx->copy_stream, &kernels), "derived seeds");
  QRNG_CUDA(ctx, cudaEventRecord(ctx->pre_done, ctx->copy_stream), "pipeline event");
  ctx->stats.kernels_launched += kernels;
  kernels = 0;

  // `s`: estimate, device-side m, the report's copy, then the hash
  st = minentropy_enqueue(ctx, samples, count, bits, eps, s);
  if (st) {
    cudaStreamSynchronize(ctx->copy_stream);
    ws.xk_ready = false;
    return st;
  }
  DevSpec* dspec = spec_buf.as<DevSpec>();
  const double lhl_term = 2.0 * log2(1.0 / eps_lhl);  // as qrng_output_length forms it
  QRNG_CUDA(ctx,
            launch_pipeline_size(ctx->result.as<DevHminResult>(), n, bits, lhl_term, m_cap, seed_capacity_bits,
                                 out_capacity_bytes, nb, dspec, s, &kernels),
            "pipeline size kernel");
  // the report and m go to the host on a stream of their own, so the hash does not wait for them
  // (this call waits for the copies before it returns: no later call rewrites them first)
  QRNG_CUDA(ctx, cudaEventRecord(ctx->spec_sized, s), "pipeline event");
  QRNG_CUDA(ctx, cudaStreamWaitEvent(ctx->report_stream, ctx->spec_sized, 0), "pipeline event");
  QRNG_CUDA(ctx,
            cudaMemcpyAsync(ctx->result_host, ctx->result.p, sizeof(DevHminResult), cudaMemcpyDeviceToHost,
                            ctx->report_stream),
            "report copy");
  QRNG_CUDA(ctx, cudaMemcpyAsync(ctx->spec_host, dspec, sizeof(DevSpec), cudaMemcpyDeviceToHost, ctx->report_stream),
            "size copy");
  QRNG_CUDA(ctx, cudaEventRecord(ctx->spec_est, ctx->report_stream), "pipeline event");
  QRNG_CUDA(ctx, cudaStreamWaitEvent(s, ctx->pre_done, 0), "pipeline event");
  QRNG_CUDA(ctx,
            launch_gemm_karatsuba(a, sp.plan, ws, ctx->dev_err.as<int>(), 0, ctx->num_sms, s, &kernels,
                                  extract_hook(ctx), out, dspec, true, combine_stream,
                                  combine_stream ? ctx->spec_product : nullptr),
            "speculative block Karatsuba extraction");
  ws.xk_ready = false;
  ctx->stats.kernels_launched += kernels;
  ++ctx->stats.speculative_hashes;

  // the host side of the call while the product runs
  QRNG_CUDA(ctx, cudaEventSynchronize(ctx->spec_est), "min-entropy synchronise");
  st = minentropy_read(ctx, &local);
  if (st) return st;  // the device refused the hash too (status 2)
  if (rep) *rep = local;
  uint64_t m = qrng_output_length(n, local.h_modify, bits, eps_lhl);
  if (m > n) m = n;
  *m_out = m;
  ctx->pipeline_m = m;
  const char* bad = m == 0 ? ": the corrected min-entropy gives m = 0"
                    : seed_capacity_bits < qrng_seed_bits(n, m, QRNG_FORM_STANDARD) ? ": seed shorter than the hash needs"
                    : out_capacity_bytes < ceil_div(nb * m, 8) ? ": output buffer too small"
                    : nullptr;
  if (bad) return fail(ctx, QRNG_EINVAL, w + bad);
  const DevSpec& d = *ctx->spec_host;
  if (d.status == 0 && d.m == m) {
    ctx->stats.last_algo = QRNG_ALGO_GEMM_KARATSUBA;
    ctx->stats.last_kernels = kernels;
    *done = true;
    return QRNG_OK;
  }
  ++ctx->stats.speculative_misses;  // m outside the enqueued rows: the ordinary path hashes with m
  return QRNG_OK;
}

}  // namespace

extern "C" {

int qrng_create(qrng_ctx** out, int device) {
  if (!out) return QRNG_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return QRNG_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return QRNG_ECUDA;
  qrng_ctx* ctx = new (std::nothrow) qrng_ctx();
  if (!ctx) return QRNG_ENOMEM;
  ctx->device = device;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete ctx;
    return QRNG_ECUDA;
  }
  // the report and the pipeline's device-side size word, read back side by side
  if (cudaMallocHost(reinterpret_cast<void**>(&ctx->result_host), sizeof(DevHminResult) + sizeof(DevSpec)) !=
      cudaSuccess) {
    delete ctx;
    return QRNG_ENOMEM;
  }
  ctx->spec_host = reinterpret_cast<DevSpec*>(ctx->result_host + 1);
  if (ctx->dev_err.ensure(sizeof(int)) != cudaSuccess || cudaMemset(ctx->dev_err.p, 0, sizeof(int)) != cudaSuccess ||
      ctx->fft_worst.ensure(2 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(ctx->fft_worst.p, 0, 2 * sizeof(unsigned long long)) != cudaSuccess ||
      ctx->fft32_guard.ensure(16) != cudaSuccess || cudaMemset(ctx->fft32_guard.p, 0, 16) != cudaSuccess) {
    cudaFreeHost(ctx->result_host);
    ctx->dev_err.release();
    ctx->fft_worst.release();
    ctx->fft32_guard.release();
    delete ctx;
    return QRNG_ENOMEM;
  }
  if (cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->copy_ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->copy_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->pre_ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->pre_done, cudaEventDisableTiming) != cudaSuccess) {
    if (ctx->pre_done) cudaEventDestroy(ctx->pre_done);
    if (ctx->pre_ready) cudaEventDestroy(ctx->pre_ready);
    if (ctx->copy_done) cudaEventDestroy(ctx->copy_done);
    if (ctx->copy_ready) cudaEventDestroy(ctx->copy_ready);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    cudaFreeHost(ctx->result_host);
    ctx->dev_err.release();
    ctx->fft_worst.release();
    ctx->fft32_guard.release();
    delete ctx;
    return QRNG_ECUDA;
  }
  *out = ctx;
  return QRNG_OK;
}

void qrng_destroy(qrng_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  ctx->hist.release();
  ctx->result.release();
  ctx->seed_rev.release();
  ctx->raw_stage.release();
  ctx->out_stage.release();
  ctx->samples_dev.release();
  ctx->out_dev.release();
  ctx->seed_dev.release();
  ctx->dev_err.release();
  ctx->fft_worst.release();
  ctx->fft32_guard.release();
  ctx->fft.release();
  ctx->kara.release();
  ctx->spec.release();
  if (ctx->spec_sized) cudaEventDestroy(ctx->spec_sized);
  if (ctx->spec_product) cudaEventDestroy(ctx->spec_product);
  if (ctx->spec_hashed) cudaEventDestroy(ctx->spec_hashed);
  if (ctx->spec_est) cudaEventDestroy(ctx->spec_est);
  if (ctx->report_stream) cudaStreamDestroy(ctx->report_stream);
  drop_all_graphs(ctx);
  ctx->batch_meta.release();
  ctx->batch_raw.release();
  ctx->batch_rev.release();
  ctx->batch_out.release();
  ctx->batch_counter.release();
  ctx->batch_fft.release();
  if (ctx->tune_host) cudaFreeHost(ctx->tune_host);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->copy_ready) cudaEventDestroy(ctx->copy_ready);
  if (ctx->copy_done) cudaEventDestroy(ctx->copy_done);
  if (ctx->pre_ready) cudaEventDestroy(ctx->pre_ready);
  if (ctx->pre_done) cudaEventDestroy(ctx->pre_done);
  for (auto& sl : ctx->async_slot) {
    sl.samples.release();
    sl.seed.release();
    sl.out.release();
    sl.kara.release();
    sl.seed_rev.release();
    sl.spec.release();
    if (sl.uploaded) cudaEventDestroy(sl.uploaded);
    if (sl.computed) cudaEventDestroy(sl.computed);
    if (sl.downloaded) cudaEventDestroy(sl.downloaded);
  }
  if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
  if (ctx->down_stream) cudaStreamDestroy(ctx->down_stream);
  if (ctx->result_host) cudaFreeHost(ctx->result_host);
  for (cudaEvent_t e : ctx->ev_start) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->ev_end) cudaEventDestroy(e);
  delete ctx;
}

const char* qrng_last_error(const qrng_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

const char* qrng_status_string(int status) {
  switch (status) {
    case QRNG_OK: return "QRNG_OK";
    case QRNG_EINVAL: return "QRNG_EINVAL";
    case QRNG_ENOMEM: return "QRNG_ENOMEM";
    case QRNG_ECUDA: return "QRNG_ECUDA";
    case QRNG_ETIMEOUT: return "QRNG_ETIMEOUT";
    case QRNG_EPRECISION: return "QRNG_EPRECISION";
    case QRNG_ENOTSUP: return "QRNG_ENOTSUP";
    default: return "unknown status";
  }
}

int qrng_minentropy(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, double eps, qrng_hmin_report* rep,
                    qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  int st = check_minentropy_args(ctx, samples, count, bits, eps, rep);
  if (st) return st;
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  return minentropy_dev(ctx, samples, count, bits, eps, rep, static_cast<cudaStream_t>(stream));
}

int qrng_minentropy_sampled(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, double eps, double fraction,
                            uint64_t sel_seed, qrng_hmin_report* rep, qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  int st = check_minentropy_args(ctx, samples, count, bits, eps, rep);
  if (st) return st;
  if (!(fraction > 0.0 && fraction <= 1.0))
    return fail(ctx, QRNG_EINVAL, "qrng_minentropy_sampled: fraction must be in (0, 1]");
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  const uint64_t thr = (uint64_t)floor(fraction * 9007199254740992.0);  // fraction * 2^53
  return minentropy_dev(ctx, samples, count, bits, eps, rep, static_cast<cudaStream_t>(stream), thr, sel_seed);
}

int qrng_minentropy_quantum(qrng_ctx* ctx, const void* samples_on, uint64_t count_on, const void* samples_off,
                            uint64_t count_off, int bits, double eps, qrng_hmin_report* rep, double* h_subtracted,
                            qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  int st = check_minentropy_args(ctx, samples_on, count_on, bits, eps, rep);
  if (st) return st;
  qrng_hmin_report off{};
  st = check_minentropy_args(ctx, samples_off, count_off, bits, eps, &off);
  if (st) return st;
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = minentropy_dev(ctx, samples_off, count_off, bits, eps, &off, s);
  if (st) return st;
  // var_sub > 0 selects the quantum model; a noiseless laser-off stream leaves the plain estimate
  const double var_sub = off.var > 0.0 ? off.var : 0.0;
  double hs = 0.0;
  st = minentropy_dev(ctx, samples_on, count_on, bits, eps, rep, s, 1ull << 53, 0, var_sub, off.h_model, &hs);
  if (st) return st;
  if (h_subtracted) *h_subtracted = hs;
  return QRNG_OK;
}

uint64_t qrng_output_length(uint64_t n, double h_per_sample, int bits, double eps_lhl) {
  if (bits < 1 || !(h_per_sample >= 0.0) || !(eps_lhl > 0.0 && eps_lhl <= 1.0)) return 0;
  const double m = (double)n * h_per_sample / (double)bits - 2.0 * log2(1.0 / eps_lhl);
  if (!(m > 0.0)) return 0;
  return (uint64_t)floor(m);
}

uint64_t qrng_seed_bits(uint64_t n, uint64_t m, int form) {
  if (!shape_ok(n, m, form)) return 0;
  return form == QRNG_FORM_STANDARD ? n + m - 1 : n - 1;
}

int qrng_toeplitz_extract(qrng_ctx* ctx, const uint8_t* raw, uint64_t n, uint64_t m, const uint8_t* seed, int form,
                          int algo, uint64_t num_blocks, uint8_t* out, qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  int st = check_extract_args(ctx, raw, n, m, seed, form, algo, num_blocks, out);
  if (st) return st;
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  return extract_dispatch(ctx, raw, n, m, seed, form, algo, num_blocks, out, static_cast<cudaStream_t>(stream));
}

int qrng_extract_batch(qrng_ctx* ctx, const qrng_request* reqs, uint64_t count, int algo, qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  if (!reqs || count == 0 || count > (1ull << 31)) return fail(ctx, QRNG_EINVAL, "qrng_extract_batch: bad request table");
  if (algo != QRNG_ALGO_AUTO && algo != QRNG_ALGO_DIRECT && algo != QRNG_ALGO_NTT && algo != QRNG_ALGO_FFT64 &&
      algo != QRNG_ALGO_FFT32_SEG)
    return fail(ctx, QRNG_ENOTSUP, "qrng_extract_batch: batches run AUTO, DIRECT, NTT, FFT64 or FFT32_SEG");
  for (uint64_t i = 0; i < count; ++i) {
    const qrng_request& r = reqs[i];
    if (!r.raw || !r.seed || !r.out)
      return fail(ctx, QRNG_EINVAL, "qrng_extract_batch: request " + std::to_string(i) + " has a NULL pointer");
    if ((r.form != QRNG_FORM_STANDARD && r.form != QRNG_FORM_MODIFIED) || !shape_ok(r.n, r.m, r.form))
      return fail(ctx, QRNG_EINVAL, "qrng_extract_batch: request " + std::to_string(i) + " has a bad shape or form");
  }
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  return extract_batch(ctx, reqs, count, algo, static_cast<cudaStream_t>(stream));
}

int qrng_postprocess(qrng_ctx* ctx, const void* samples, uint64_t count, int bits, double eps, double eps_lhl,
                     uint64_t n, const uint8_t* seed, uint64_t seed_capacity_bits, int form, int algo, uint8_t* out,
                     uint64_t out_capacity_bytes, uint64_t* m_out, uint64_t* num_blocks_out, qrng_hmin_report* rep,
                     qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  if (!samples || !seed || !out) return fail(ctx, QRNG_EINVAL, "qrng_postprocess: NULL pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  const uint64_t bytes = count * (bits <= 8 ? 1 : 2);
  const uint64_t nb = n >= 2 ? bytes * 8 / n : 0;
  uint64_t m = 0;
  if (num_blocks_out) *num_blocks_out = nb;
  SpecPlan sp;
  if (eps_lhl > 0.0 && eps_lhl <= 1.0 && n <= kMaxBlockBits &&
      spec_plan(ctx, samples, count, bits, n, form, algo, nb, seed_capacity_bits, out, &sp)) {
    bool done = false;
    int st = postprocess_speculative(ctx, sp, samples, count, bits, eps, eps_lhl, n, seed, seed_capacity_bits, out,
                                     out_capacity_bytes, nb, s, &m, rep, &done, ctx->kara, ctx->seed_rev, ctx->spec);
    if (m_out) *m_out = m;
    if (st || done) return st;
    // the enqueued hash did not stand (m outside its rows): hash with m, as below
    st = extract_dispatch(ctx, static_cast<const uint8_t*>(samples), n, m, seed, form, algo, nb, out, s);
    ctx->kara.xk_ready = false;
    return st;
  }
  int st = pipeline_size(ctx, "qrng_postprocess", samples, count, bits, eps, eps_lhl, n, seed_capacity_bits, form,
                         algo, nb, s, &m, rep);
  if (m_out) *m_out = m;
  if (st) return st;
  if (out_capacity_bytes < ceil_div(nb * m, 8)) {
    ctx->kara.xk_ready = false;
    return fail(ctx, QRNG_EINVAL, "qrng_postprocess: output buffer too small");
  }
  st = extract_dispatch(ctx, static_cast<const uint8_t*>(samples), n, m, seed, form, algo, nb, out, s);
  ctx->kara.xk_ready = false;
  return st;
}

int qrng_postprocess_host(qrng_ctx* ctx, const void* samples_host, uint64_t count, int bits, double eps,
                          double eps_lhl, uint64_t n, const uint8_t* seed_host, uint64_t seed_capacity_bits,
                          int form, int algo, uint8_t* out_host, uint64_t out_capacity_bytes, uint64_t* m_out,
                          uint64_t* num_blocks_out, qrng_hmin_report* rep, qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  if (!samples_host || !seed_host || !out_host) return fail(ctx, QRNG_EINVAL, "qrng_postprocess_host: NULL pointer");
  qrng_hmin_report local{};
  int st = check_minentropy_args(ctx, samples_host, count, bits, eps, &local);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");

  const uint64_t bytes = count * (bits <= 8 ? 1 : 2);
  QRNG_CUDA(ctx, ctx->samples_dev.ensure(bytes), "sample workspace");
  QRNG_CUDA(ctx, cudaMemcpyAsync(ctx->samples_dev.p, samples_host, bytes, cudaMemcpyHostToDevice, s), "sample upload");
  const uint64_t num_blocks = n >= 2 ? bytes * 8 / n : 0;
  // Two parts when the split keeps both raw and output chunks aligned (n a multiple of 128 bits, the
  // first part a multiple of 32 blocks): the first 7/8 of the blocks' output travels to the host on the
  // copy stream while the last 1/8 is hashed, so only 1/8 of the download is left after the last kernel.
  const uint64_t first = ((num_blocks * 7) / 8) & ~31ull;
  const bool split = (n % 128 == 0) && num_blocks >= 64 && first >= 32 && first < num_blocks;
  const uint64_t b0 = split ? first : num_blocks;
  uint64_t m = 0;
  st = pipeline_size(ctx, "qrng_postprocess_host", ctx->samples_dev.p, count, bits, eps, eps_lhl, n,
                     seed_capacity_bits, form, algo, b0, s, &m, rep);
  if (m_out) *m_out = m;
  if (num_blocks_out) *num_blocks_out = num_blocks;
  if (st) return st;
  const uint64_t out_bytes = ceil_div(num_blocks * m, 8);
  if (out_capacity_bytes < out_bytes) {
    ctx->kara.xk_ready = false;
    return fail(ctx, QRNG_EINVAL, "qrng_postprocess_host: output buffer too small");
  }
  const uint64_t L = qrng_seed_bits(n, m, form);
  QRNG_CUDA(ctx, ctx->seed_dev.ensure(ceil_div(L, 8)), "seed workspace");
  QRNG_CUDA(ctx, cudaMemcpyAsync(ctx->seed_dev.p, seed_host, ceil_div(L, 8), cudaMemcpyHostToDevice, s), "seed upload");
  QRNG_CUDA(ctx, ctx->out_dev.ensure(out_bytes), "output workspace");
  uint8_t* out_d = ctx->out_dev.as<uint8_t>();
  st = extract_dispatch(ctx, ctx->samples_dev.as<uint8_t>(), n, m, ctx->seed_dev.as<uint8_t>(), form, algo, b0, out_d,
                        s);
  ctx->kara.xk_ready = false;
  if (st) return st;
  if (split) {
    const uint64_t bytes0 = b0 * m / 8;  // b0 m is a multiple of 32 bits
    QRNG_CUDA(ctx, cudaEventRecord(ctx->copy_ready, s), "copy event");
    QRNG_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_ready, 0), "copy stream wait");
    QRNG_CUDA(ctx, cudaMemcpyAsync(out_host, out_d, bytes0, cudaMemcpyDeviceToHost, ctx->copy_stream),
              "output download");
    QRNG_CUDA(ctx, cudaEventRecord(ctx->copy_done, ctx->copy_stream), "copy event");
    st = extract_dispatch(ctx, ctx->samples_dev.as<uint8_t>() + b0 * n / 8, n, m, ctx->seed_dev.as<uint8_t>(), form,
                          algo, num_blocks - b0, out_d + bytes0, s);
    if (st) {
      cudaStreamSynchronize(ctx->copy_stream);
      return st;
    }
    QRNG_CUDA(ctx, cudaMemcpyAsync(out_host + bytes0, out_d + bytes0, out_bytes - bytes0, cudaMemcpyDeviceToHost, s),
              "output download");
    QRNG_CUDA(ctx, cudaStreamWaitEvent(s, ctx->copy_done, 0), "copy join");
  } else {
    QRNG_CUDA(ctx, cudaMemcpyAsync(out_host, out_d, out_bytes, cudaMemcpyDeviceToHost, s), "output download");
  }
  return qrng_synchronize(ctx, stream);
}

int qrng_postprocess_host_async(qrng_ctx* ctx, const void* samples_host, uint64_t count, int bits, double eps,
                                double eps_lhl, uint64_t n, const uint8_t* seed_host, uint64_t seed_capacity_bits,
                                int form, int algo, uint8_t* out_host, uint64_t out_capacity_bytes, uint64_t* m_out,
                                uint64_t* num_blocks_out, qrng_hmin_report* rep, qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  if (!samples_host || !seed_host || !out_host)
    return fail(ctx, QRNG_EINVAL, "qrng_postprocess_host_async: NULL pointer");
  qrng_hmin_report local{};
  int st = check_minentropy_args(ctx, samples_host, count, bits, eps, &local);
  if (st) return st;
  if (seed_capacity_bits == 0) return fail(ctx, QRNG_EINVAL, "qrng_postprocess_host_async: empty seed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (!ctx->up_stream) {
    QRNG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking), "upload stream");
    QRNG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->down_stream, cudaStreamNonBlocking), "download stream");
    for (auto& sl : ctx->async_slot) {
      QRNG_CUDA(ctx, cudaEventCreateWithFlags(&sl.uploaded, cudaEventDisableTiming), "pipeline event");
      QRNG_CUDA(ctx, cudaEventCreateWithFlags(&sl.computed, cudaEventDisableTiming), "pipeline event");
      QRNG_CUDA(ctx, cudaEventCreateWithFlags(&sl.downloaded, cudaEventDisableTiming), "pipeline event");
    }
  }
  qrng_ctx::AsyncSlot& sl = ctx->async_slot[ctx->async_calls & 1];
  const uint64_t bytes = count * (bits <= 8 ? 1 : 2);
  const uint64_t seed_bytes = ceil_div(seed_capacity_bits, 8);
  // the slot's earlier call must have finished hashing before its samples and seed are replaced
  if (sl.used) QRNG_CUDA(ctx, cudaStreamWaitEvent(ctx->up_stream, sl.computed, 0), "pipeline wait");
  if (sl.used && (sl.samples.cap < bytes || sl.seed.cap < seed_bytes))  // growing frees the old buffer
    QRNG_CUDA(ctx, cudaEventSynchronize(sl.computed), "pipeline wait");
  QRNG_CUDA(ctx, sl.samples.ensure(bytes), "pipeline sample workspace");
  QRNG_CUDA(ctx, sl.seed.ensure(seed_bytes), "pipeline seed workspace");
  QRNG_CUDA(ctx, cudaMemcpyAsync(sl.samples.p, samples_host, bytes, cudaMemcpyHostToDevice, ctx->up_stream),
            "sample upload");
  QRNG_CUDA(ctx, cudaMemcpyAsync(sl.seed.p, seed_host, seed_bytes, cudaMemcpyHostToDevice, ctx->up_stream),
            "seed upload");
  QRNG_CUDA(ctx, cudaEventRecord(sl.uploaded, ctx->up_stream), "pipeline event");
  QRNG_CUDA(ctx, cudaStreamWaitEvent(s, sl.uploaded, 0), "pipeline wait");
  const uint64_t num_blocks = n >= 2 ? bytes * 8 / n : 0;
  uint64_t m = 0;
  if (num_blocks_out) *num_blocks_out = num_blocks;
  SpecPlan sp;
  if (eps_lhl > 0.0 && eps_lhl <= 1.0 && n <= kMaxBlockBits &&
      spec_plan(ctx, sl.samples.p, count, bits, n, form, algo, num_blocks, seed_capacity_bits, sl.out.as<uint8_t>(),
                &sp)) {
    // the hash is enqueued before m is known (as qrng_postprocess does): the slot's output holds
    // the enqueued rows, and its earlier download is over before the hash writes it
    const uint64_t cap_bytes = ceil_div(num_blocks * sp.m_cap, 8);
    if (sl.used && sl.out.cap < cap_bytes) QRNG_CUDA(ctx, cudaEventSynchronize(sl.downloaded), "pipeline wait");
    QRNG_CUDA(ctx, sl.out.ensure(cap_bytes), "pipeline output workspace");
    if (sl.used) QRNG_CUDA(ctx, cudaStreamWaitEvent(s, sl.downloaded, 0), "pipeline wait");
    // the combination runs on the download stream, right before this call's download (the slot's
    // parities, size word and output are its own), so the caller's stream takes the next call's
    // estimate as soon as the product has run
    bool done = false;
    st = postprocess_speculative(ctx, sp, sl.samples.p, count, bits, eps, eps_lhl, n, sl.seed.as<uint8_t>(),
                                 seed_capacity_bits, sl.out.as<uint8_t>(), out_capacity_bytes, num_blocks, s, &m, rep,
                                 &done, sl.kara, sl.seed_rev, sl.spec, sl.uploaded, ctx->down_stream);
    if (m_out) *m_out = m;
    if (st == QRNG_OK && !done) {  // m outside the enqueued rows: hash again with m
      const uint64_t out_bytes = ceil_div(num_blocks * m, 8);
      if (sl.out.cap < out_bytes)  // growing frees the old buffer: the enqueued combination must be over
        QRNG_CUDA(ctx, cudaStreamSynchronize(ctx->down_stream), "pipeline wait");
      QRNG_CUDA(ctx, sl.out.ensure(out_bytes), "pipeline output workspace");
      st = extract_dispatch(ctx, sl.samples.as<uint8_t>(), n, m, sl.seed.as<uint8_t>(), form, algo, num_blocks,
                            sl.out.as<uint8_t>(), s);
    }
    ctx->kara.xk_ready = false;
    // the slot's call is over once the caller's stream (the estimate, the product, a repeated hash)
    // and the download stream (the combination) have passed it
    if (ctx->spec_hashed) {
      QRNG_CUDA(ctx, cudaEventRecord(ctx->spec_hashed, s), "pipeline event");
      QRNG_CUDA(ctx, cudaStreamWaitEvent(ctx->down_stream, ctx->spec_hashed, 0), "pipeline wait");
      QRNG_CUDA(ctx, cudaEventRecord(sl.computed, ctx->down_stream), "pipeline event");
    } else {
      QRNG_CUDA(ctx, cudaEventRecord(sl.computed, s), "pipeline event");
    }
    sl.used = true;
    ++ctx->async_calls;
    if (st) return st;
    QRNG_CUDA(ctx, cudaStreamWaitEvent(ctx->down_stream, sl.computed, 0), "pipeline wait");
    QRNG_CUDA(ctx,
              cudaMemcpyAsync(out_host, sl.out.p, ceil_div(num_blocks * m, 8), cudaMemcpyDeviceToHost,
                              ctx->down_stream),
              "output download");
    QRNG_CUDA(ctx, cudaEventRecord(sl.downloaded, ctx->down_stream), "pipeline event");
    return QRNG_OK;
  }
  st = pipeline_size(ctx, "qrng_postprocess_host_async", sl.samples.p, count, bits, eps, eps_lhl, n,
                     seed_capacity_bits, form, algo, num_blocks, s, &m, rep);
  if (m_out) *m_out = m;
  if (st) {
    sl.used = true;  // its upload is in flight: the next use of the slot orders after the compute stream
    QRNG_CUDA(ctx, cudaEventRecord(sl.computed, s), "pipeline event");
    ++ctx->async_calls;
    return st;
  }
  const uint64_t out_bytes = ceil_div(num_blocks * m, 8);
  if (out_capacity_bytes < out_bytes) {
    ctx->kara.xk_ready = false;
    sl.used = true;
    QRNG_CUDA(ctx, cudaEventRecord(sl.computed, s), "pipeline event");
    ++ctx->async_calls;
    return fail(ctx, QRNG_EINVAL, "qrng_postprocess_host_async: output buffer too small");
  }
  if (sl.used && sl.out.cap < out_bytes) {
    // growing the buffer frees the old one: its download must be over first
    QRNG_CUDA(ctx, cudaEventSynchronize(sl.downloaded), "pipeline wait");
  }
  QRNG_CUDA(ctx, sl.out.ensure(out_bytes), "pipeline output workspace");
  // the slot's earlier call must have finished downloading before its output is overwritten
  if (sl.used) QRNG_CUDA(ctx, cudaStreamWaitEvent(s, sl.downloaded, 0), "pipeline wait");
  st = extract_dispatch(ctx, sl.samples.as<uint8_t>(), n, m, sl.seed.as<uint8_t>(), form, algo, num_blocks,
                        sl.out.as<uint8_t>(), s);
  ctx->kara.xk_ready = false;
  QRNG_CUDA(ctx, cudaEventRecord(sl.computed, s), "pipeline event");
  sl.used = true;
  ++ctx->async_calls;
  if (st) return st;
  QRNG_CUDA(ctx, cudaStreamWaitEvent(ctx->down_stream, sl.computed, 0), "pipeline wait");
  QRNG_CUDA(ctx, cudaMemcpyAsync(out_host, sl.out.p, out_bytes, cudaMemcpyDeviceToHost, ctx->down_stream),
            "output download");
  QRNG_CUDA(ctx, cudaEventRecord(sl.downloaded, ctx->down_stream), "pipeline event");
  return QRNG_OK;
}

int qrng_postprocess_host_wait(qrng_ctx* ctx, qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (ctx->up_stream) {
    QRNG_CUDA(ctx, cudaStreamSynchronize(ctx->up_stream), "pipeline wait");
    QRNG_CUDA(ctx, cudaStreamSynchronize(ctx->down_stream), "pipeline wait");
  }
  return qrng_synchronize(ctx, stream);
}

int qrng_get_stats(qrng_ctx* ctx, qrng_stats* out) {
  if (!ctx || !out) return QRNG_EINVAL;
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    float ms = 0.f;
    QRNG_CUDA(ctx, cudaEventSynchronize(ctx->ev_end[i]), "timing event wait");
    QRNG_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_start[i], ctx->ev_end[i]), "timing event read");
    switch (ctx->ev_kind[i]) {
      case kTimeHist:
        ctx->stats.hist_timed_ms += ms;
        ctx->stats.hist_timed_launches += 1;
        break;
      case kTimeBatchGraph:
        ctx->stats.batch_graph_ms += ms;
        break;
      default:
        ctx->stats.timed_ms += ms;
        ctx->stats.timed_launches += 1;
    }
  }
  ctx->ev_used = 0;
  if (ctx->timed_graph_pending) {  // the parts of the last timed batch replay
    ctx->timed_graph_pending = false;
    for (const auto& g : ctx->graphs) {
      if (g.key != ctx->timed_graph_key || g.generation != ctx->timed_graph_generation) continue;
      float ms = 0.f;
      if (g.has_transform) {
        QRNG_CUDA(ctx, cudaEventSynchronize(g.ev[1]), "batch timing wait");
        QRNG_CUDA(ctx, cudaEventElapsedTime(&ms, g.ev[0], g.ev[1]), "batch timing read");
        ctx->stats.batch_transform_ms = ms;
      }
      if (g.has_direct) {
        QRNG_CUDA(ctx, cudaEventSynchronize(g.ev[3]), "batch timing wait");
        QRNG_CUDA(ctx, cudaEventElapsedTime(&ms, g.ev[2], g.ev[3]), "batch timing read");
        ctx->stats.batch_direct_ms = ms;
      }
    }
  }
  unsigned long long worst[2] = {0, 0}, repairs = 0;
  QRNG_CUDA(ctx, cudaMemcpy(worst, ctx->fft_worst.p, sizeof(worst), cudaMemcpyDeviceToHost), "FFT error read");
  QRNG_CUDA(ctx, cudaMemcpy(&repairs, ctx->fft32_guard.as<char>() + 8, sizeof(repairs), cudaMemcpyDeviceToHost),
            "repair count read");
  double w64, w32;
  memcpy(&w64, &worst[0], sizeof(w64));
  memcpy(&w32, &worst[1], sizeof(w32));
  ctx->stats.worst_fft_round_err = w64 > w32 ? w64 : w32;
  ctx->stats.worst_fft32_round_err = w32;
  ctx->stats.fft32_recomputed = repairs;
  ctx->stats.last_fft32_segment = ctx->last_fft32_log_s ? (1ull << ctx->last_fft32_log_s) : 0;
  ctx->stats.kara_presplits_used =
      ctx->kara.presplits_used + ctx->async_slot[0].kara.presplits_used + ctx->async_slot[1].kara.presplits_used;
  *out = ctx->stats;
  return QRNG_OK;
}

int qrng_extract_stats(qrng_ctx* ctx, double* worst_fft_round_err) {
  if (!ctx) return QRNG_EINVAL;
  if (!worst_fft_round_err) return fail(ctx, QRNG_EINVAL, "qrng_extract_stats: NULL pointer");
  qrng_stats st{};
  const int r = qrng_get_stats(ctx, &st);
  if (r) return r;
  *worst_fft_round_err = st.worst_fft_round_err;
  return QRNG_OK;
}

int qrng_reset_stats(qrng_ctx* ctx) {
  if (!ctx) return QRNG_EINVAL;
  for (size_t i = 0; i < ctx->ev_used; ++i) cudaEventSynchronize(ctx->ev_end[i]);
  ctx->ev_used = 0;
  ctx->stats = qrng_stats{};
  ctx->kara.presplits_used = 0;
  for (auto& sl : ctx->async_slot) sl.kara.presplits_used = 0;
  QRNG_CUDA(ctx, cudaMemset(ctx->fft_worst.p, 0, 2 * sizeof(unsigned long long)), "FFT error reset");
  QRNG_CUDA(ctx, cudaMemset(ctx->fft32_guard.p, 0, 16), "repair count reset");
  return QRNG_OK;
}

int qrng_synchronize(qrng_ctx* ctx, qrng_stream_t stream) {
  if (!ctx) return QRNG_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  QRNG_CUDA(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  QRNG_CUDA(ctx, cudaStreamSynchronize(s), "stream synchronise");
  int code = 0;
  QRNG_CUDA(ctx, cudaMemcpy(&code, ctx->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost), "error word read");
  if (code != 0) {
    QRNG_CUDA(ctx, cudaMemset(ctx->dev_err.p, 0, sizeof(int)), "error word clear");
    return fail(ctx, QRNG_ETIMEOUT,
                "a bounded device wait gave up (site " + std::to_string(code) + "); the affected output is incomplete");
  }
  unsigned long long worst = 0;
  QRNG_CUDA(ctx, cudaMemcpy(&worst, ctx->fft_worst.p, sizeof(worst), cudaMemcpyDeviceToHost), "FFT error read");
  double w;
  memcpy(&w, &worst, sizeof(w));
  if (w >= kFftRoundGuard)
    return fail(ctx, QRNG_EPRECISION,
                "an FFT convolution sum was " + std::to_string(w) + " away from an integer; its parity is unreliable");
  return QRNG_OK;
}

int qrng_inject_fault(qrng_ctx* ctx, int fault) {
  if (!ctx || (fault != QRNG_FAULT_NONE && fault != QRNG_FAULT_GEMM_NO_TMA)) return QRNG_EINVAL;
  ctx->fault = fault;
  return QRNG_OK;
}

int qrng_set_autotune(qrng_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return QRNG_EINVAL;
  ctx->autotune = (on == 1);
  ctx->tuned.clear();
  ctx->batch_tuned.clear();
  return QRNG_OK;
}

int qrng_set_karatsuba(qrng_ctx* ctx, int levels, uint64_t block_bits, uint64_t max_workspace) {
  if (!ctx) return QRNG_EINVAL;
  if (levels < 0 || levels > (int)kMaxLevels) return fail(ctx, QRNG_EINVAL, "qrng_set_karatsuba: levels must be 0..4");
  if (block_bits != 0 && (block_bits < 256 || block_bits > 8192 || (block_bits & (block_bits - 1)) != 0))
    return fail(ctx, QRNG_EINVAL, "qrng_set_karatsuba: block_bits must be 0 or a power of two in [256, 8192]");
  ctx->kara_levels = levels;
  ctx->kara_h = block_bits;
  ctx->kara_workspace = max_workspace;
  ctx->tuned.clear();
  return QRNG_OK;
}

int qrng_karatsuba_plan(qrng_ctx* ctx, uint64_t n, uint64_t m, int form, uint64_t num_blocks,
                        qrng_karatsuba_plan_info* out) {
  if (!ctx || !out) return QRNG_EINVAL;
  if (!shape_ok(n, m, form) || num_blocks == 0) return fail(ctx, QRNG_EINVAL, "qrng_karatsuba_plan: invalid shape");
  const uint64_t n_t = (form == QRNG_FORM_MODIFIED) ? n - m : n;
  const KaraPlan p = karatsuba_plan(n_t, m, num_blocks, ctx->num_sms, ctx->kara_levels, ctx->kara_h,
                                    ctx->kara_workspace);
  *out = qrng_karatsuba_plan_info{};
  out->levels = (int)p.levels;
  out->block_bits = p.h;
  out->products = p.groups;
  out->rows = p.mq;
  out->cols = p.kq;
  out->blocks_per_pass = p.chunk_blocks;
  out->model_seconds = p.model_s;
  return QRNG_OK;
}

int qrng_set_fft32(qrng_ctx* ctx, uint64_t segment_bits, int terms) {
  if (!ctx) return QRNG_EINVAL;
  int ls = 0;
  if (segment_bits != 0) {
    while ((1ull << ls) < segment_bits) ++ls;
    if ((1ull << ls) != segment_bits || !fft32_log_s_ok(ls))
      return fail(ctx, QRNG_EINVAL, "qrng_set_fft32: segment_bits must be 0, 2048, 4096 or 8192");
  }
  if (terms < 0 || terms > 1 << 20) return fail(ctx, QRNG_EINVAL, "qrng_set_fft32: terms must be in [0, 2^20]");
  ctx->fft32_log_s = ls;
  ctx->fft32_terms = terms;
  ctx->tuned.clear();
  return QRNG_OK;
}

int qrng_fft32_terms_bound(uint64_t segment_bits) {
  for (int ls = 11; ls <= 13; ++ls)
    if (segment_bits == (1ull << ls)) return fft32_terms_bound(ls);
  return 0;
}

int qrng_set_timing(qrng_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return QRNG_EINVAL;
  ctx->timing = (on == 1);
  return QRNG_OK;
}

}  // extern "C"
