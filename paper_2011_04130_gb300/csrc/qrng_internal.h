// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qrng.h"

namespace qrng {

// Front padding (in 32-bit words) of the bit-reversed seed buffer, so that every window the
// extraction kernels read sits at a non-negative word index.
constexpr int kSeedFrontWords = 64;
// Back padding beyond the last seed word.
constexpr int kSeedBackWords = 72;

constexpr uint64_t kMaxBlockBits = 1ull << 26;

inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// Grow-only device buffer owned by a context.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) {
      cudaError_t e = cudaFree(p);
      p = nullptr;
      cap = 0;
      if (e != cudaSuccess) return e;
    }
    size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

// Device-side min-entropy result: the public report plus the count of out-of-range samples.
struct DevHminResult {
  qrng_hmin_report rep;
  unsigned long long out_of_range;
  int status;
  double h_subtracted;  // classical-noise route: model entropy of this stream minus h_ref
  // handed from the moments kernel to the cells kernels
  unsigned long long n;
  double mu, sigma, sigma_q;
  int point, bad_sub;
  // accumulated by the cells kernels: bits of the largest cells (non-negative doubles), the
  // distance sum in units of 2^-62, the cell of the argmax code, the count of finished CTAs
  unsigned long long pmax_bits, pmax_full_bits, dsum_fixed;
  double p_argmax;
  unsigned int done;
};

// Output length of a pipeline call found on the device from the finaliser's report, for a hash
// enqueued before the host has read that report. status 0: the hash enqueued for at most m_cap
// rows stands; 1: m is above m_cap or below kSpecMinBits (the host hashes again with m); 2: the
// call is refused (the estimate failed, m = 0, or the seed or the output buffer is too short).
struct DevSpec {
  unsigned long long m;
  uint32_t mw;  // ceil(m / 32)
  int status;
};
constexpr uint64_t kSpecMinBits = 64;

// ---- histogram + finaliser (k_hist.cu) ----
// hist: (2^bits + 1) uint64 counters, the last one counts samples >= 2^bits. Zeroed by the launcher.
cudaError_t launch_histogram(const void* samples, uint64_t count, int bits, unsigned long long* hist, int num_sms,
                             cudaStream_t s, uint32_t* kernels);
// var_sub > 0: the model entropy is that of the Gaussian with the measured variance minus var_sub
// (classical-noise subtraction), the distance stays the one to the measured-variance model, and
// h_subtracted = (model entropy at the measured variance) - h_ref.
cudaError_t launch_hmin_finalize(const unsigned long long* hist, int bits, double eps, DevHminResult* out,
                                 cudaStream_t s, uint32_t* kernels, double var_sub = 0.0, double h_ref = 0.0);
// One thread: m = floor(n h_modify / bits - lhl_term) (clipped to n) from the report, in the
// operation order and rounding of the host's qrng_output_length (lhl_term = 2 log2(1 / eps_lhl)
// computed by the host), then the checks of DevSpec.status against m_cap and the capacities.
cudaError_t launch_pipeline_size(const DevHminResult* res, uint64_t n, int bits, double lhl_term, uint64_t m_cap,
                                 uint64_t seed_capacity_bits, uint64_t out_capacity_bytes, uint64_t num_blocks,
                                 DevSpec* spec, cudaStream_t s, uint32_t* kernels);
// Histogram of the samples kept by the random selection: sample i is kept when output i+1 of
// splitmix64 started at sel_seed, shifted right by 11, is below thr (thr = 2^53 keeps all).
cudaError_t launch_histogram_sampled(const void* samples, uint64_t count, int bits, uint64_t thr, uint64_t sel_seed,
                                     unsigned long long* hist, int num_sms, cudaStream_t s, uint32_t* kernels);

// ---- bit layout helpers (k_bits.cu) ----
// Bit-reversed, padded copy of seed bits [0, L): word kSeedFrontWords+w, bit t holds a[L-1-(32w+t)]
// (zero outside [0, L)). rev_words = kSeedFrontWords + ceil(L/32) + kSeedBackWords.
cudaError_t launch_seed_reverse(const uint8_t* seed, uint64_t L, uint32_t* rev, uint64_t rev_words, cudaStream_t s,
                                uint32_t* kernels);
// Copy num_blocks blocks of n bits (block b at bit raw_bit_off + b*n of src) into word-aligned
// blocks of `stride_w` words each, bits beyond n zero.
cudaError_t launch_repack_blocks(const uint8_t* src, uint64_t raw_bit_off, uint64_t n, uint64_t num_blocks,
                                 uint32_t* dst, uint64_t stride_w, cudaStream_t s, uint32_t* kernels);
// Pack per-block word-aligned outputs (stride_w words per block, m valid bits each) into a
// bit-contiguous stream at bit out_bit_off of dst (bits outside the range untouched except
// the pad bits of the final byte when out_bit_off == 0, which are zeroed).
cudaError_t launch_pack_blocks(const uint32_t* src, uint64_t stride_w, uint64_t m, uint64_t num_blocks, uint8_t* dst,
                               cudaStream_t s, uint32_t* kernels);

// ---- direct bit-packed extraction (k_direct.cu) ----
struct DirectArgs {
  uint64_t n_t;          // Toeplitz columns: n (standard) or n-m (modified)
  const uint32_t* raw;   // word-aligned blocks
  uint64_t raw_stride;   // words per block
  uint32_t nw_t;         // words of the Toeplitz part: ceil(n_t/32), n_t = n (standard) or n-m (modified)
  uint32_t tail_mask;    // valid bits of word nw_t-1
  uint32_t m;
  uint32_t mw;           // ceil(m/32)
  const uint32_t* seed_rev;  // from launch_seed_reverse with L = n_t + m - 1
  int modified;
  uint32_t id_off;       // n - m (modified only)
  uint32_t* out;         // word-aligned outputs
  uint64_t out_stride;   // words per block
  uint64_t num_blocks;
  uint32_t tiles;        // output tiles per block
  uint32_t splits;       // split of the raw words across warps (XOR-combined)
  uint32_t words_per_split;
  // optional: the kernel does nothing unless *guard != 0 (an exact recomputation after an FP32
  // rounding guard tripped; splits must be 1); then block 0 counts it in *repairs
  const int* guard;
  unsigned long long* repairs;
};
int direct_outputs_per_warp();
cudaError_t launch_direct(const DirectArgs& a, cudaStream_t s, uint32_t* kernels);

// ---- uneven batched requests (k_direct.cu persistent kernel, k_bits.cu layout kernels) ----
constexpr uint32_t kBatchWordsPerSplit = 2048;  // raw words per work item (a multiple of the tile depth)
struct BatchReq {
  // caller's request
  const uint8_t* raw;
  uint64_t raw_bit_off;
  uint64_t n, m;
  const uint8_t* seed;
  int form;
  uint8_t* out;
  uint64_t out_bit_off;
  // derived layout
  uint64_t n_t, L_t;
  uint32_t nw_t, tail_mask, mw, tiles, splits, id_off;
  uint64_t raw_words;      // words of the request's staged raw block
  uint64_t raw_stage_off;  // first word in the raw staging buffer
  uint64_t rev_off;        // first word of its reversed, padded seed
  uint64_t rev_words;
  uint64_t out_stage_off;  // first word in the output staging buffer
  uint64_t item_begin;     // first work item of the persistent kernel
  uint64_t dst_word0;      // absolute index of the first 32-bit destination word ((addr*8 + off) / 32)
  uint64_t dst_begin;      // first destination word in the pack kernel's numbering
  uint64_t dst_words;
  // route (kRoute*) and, for the FP32 segmented route, the request's place in its group
  int route;
  uint32_t seg_ns, seg_nq;     // segments and output tiles of S bits
  uint64_t spec_row;           // first spectrum row (windows d = -(NS-1).., then segments) in the group buffer
  uint64_t spec_item_begin;    // first spectra item of the request within its group
  uint64_t mac_cta_begin;      // first multiply-and-inverse CTA of the request within its group
};
enum { kRouteDirect = 0, kRouteNtt = 1, kRouteFft64 = 2, kRouteFft32 = 3 };
cudaError_t launch_batch_direct(const BatchReq* reqs, uint32_t nreq, uint64_t total_items, const uint32_t* raw_stage,
                                const uint32_t* rev, uint32_t* out_stage, unsigned long long* counter, int num_sms,
                                cudaStream_t s, uint32_t* kernels);
cudaError_t launch_batch_layout(const BatchReq* reqs, uint32_t nreq, uint64_t raw_words_total, uint64_t rev_words_total,
                                uint32_t* raw_stage, uint32_t* rev, cudaStream_t s, uint32_t* kernels);
cudaError_t launch_batch_pack(const BatchReq* reqs, uint32_t nreq, uint64_t dst_words_total, const uint32_t* out_stage,
                              cudaStream_t s, uint32_t* kernels);

// ---- FFT routes (k_fft.cu) ----
constexpr uint64_t kFftWorkspaceBytes = 1ull << 31;  // budget for the FP64 ping-pong buffers
struct FftWorkspace {
  DevBuf buf0, buf1, spec, tw, tw32, ntt_tw, ntt_stage;
  uint64_t tw_P = 0;                    // length the FP64 twiddle table holds
  uint64_t tw32_S = 0;                  // segment length the FP32 twiddle table holds
  uint64_t ntt_P = 0;                   // length the number-theoretic twiddle table holds
  unsigned long long* worst = nullptr;  // device: bits of the largest |s - round(s)| (a double)
  void release() {
    buf0.release();
    buf1.release();
    spec.release();
    tw.release();
    tw32.release();
    ntt_tw.release();
    ntt_stage.release();
    tw_P = 0;
    tw32_S = 0;
    ntt_P = 0;
  }
};
uint64_t fft64_length(uint64_t n_t, uint64_t m);
cudaError_t launch_fft64(const DirectArgs& a, const uint8_t* seed, uint64_t L_t, FftWorkspace& ws, cudaStream_t s,
                         uint32_t* kernels);
cudaError_t launch_ntt(const DirectArgs& a, const uint8_t* seed, uint64_t L_t, FftWorkspace& ws, cudaStream_t s,
                       uint32_t* kernels);
// The NTT's constant stage table and the twiddles of length P (a no-op when both are current).
cudaError_t ntt_prepare(FftWorkspace& ws, uint64_t P, cudaStream_t s, uint32_t* kernels);
// Requests reqs_dev[0..nr) (own seeds, all with transform length P) by NTT into their word-aligned
// output staging.
cudaError_t launch_ntt_batch(const BatchReq* reqs_dev, uint64_t nr, uint64_t P,
                             uint64_t max_mw, FftWorkspace& ws, uint32_t* out_stage, cudaStream_t s,
                             uint32_t* kernels);
cudaError_t launch_fft64_batch(const BatchReq* reqs_dev, uint64_t nr, uint64_t P, uint64_t max_mw, FftWorkspace& ws,
                               uint32_t* out_stage, cudaStream_t s, uint32_t* kernels);
// ---- FP32 segmented FFT (k_fft32.cu) ----
// Segments of S = 2^log_s bits, log_s in 11..13; T product terms summed per inverse transform.
bool fft32_log_s_ok(int log_s);
// The largest T for which the FP32 rounding bound keeps every sum within 0.45 of its integer.
int fft32_terms_bound(int log_s);
double fft32_model_seconds(uint64_t n_t, uint64_t m, uint64_t num_blocks, int log_s, int T);
// Writes a.out for every block; worst rounding distance into ws.worst; *guard_flag = 1 if it
// reached the guard (the caller then recomputes exactly).
cudaError_t launch_fft32_seg(const DirectArgs& a, const uint8_t* seed, uint64_t L_t, int log_s, int T,
                             FftWorkspace& ws, int* guard_flag, cudaStream_t s, uint32_t* kernels);
// Tiles one multiply-and-inverse CTA of the FP32 route covers (its accumulators).
int fft32_batch_tiles(int log_s);
// Requests reqs_dev[0..nr) of one FP32 group (segment length 2^log_s, spec_row / spec_item_begin /
// mac_cta_begin laid out by the caller; ws.spec must hold `rows` rows of 2^log_s bins) into their
// word-aligned output staging. The worst rounding distance goes to ws.worst.
cudaError_t launch_fft32_batch(const BatchReq* reqs_dev, uint64_t nr, uint64_t spec_items, uint64_t mac_ctas,
                               int log_s, int T, FftWorkspace& ws, uint32_t* out_stage, cudaStream_t s,
                               uint32_t* kernels);

// ---- tensor-core block-batched extraction (k_gemm_tc.cu) ----
// Same layout arguments as the direct kernel (splits unused). Exact for n_t <= kGemmMaxColumns.
constexpr uint64_t kGemmMaxColumns = 1ull << 22;
// fp4 selects the block-scaled E2M1 operand encoding (kind::mxf4) over E4M3 (kind::f8f6f4).
cudaError_t launch_gemm_tc(const DirectArgs& a, bool fp4, int* err, int fault, int num_sms, cudaStream_t s,
                           uint32_t* kernels);
// The FP4 product on SM pairs (k_gemm_pair.cu): clusters of two CTAs, cta_group::2 MMAs.
cudaError_t launch_gemm_pair(const DirectArgs& a, int* err, int fault, int num_sms, cudaStream_t s, uint32_t* kernels);

// Optional callbacks a launcher calls around each launch of its main kernel (event timing).
struct TimingHook {
  void* user = nullptr;
  void (*begin)(void* user, cudaStream_t s) = nullptr;
  void (*end)(void* user, cudaStream_t s) = nullptr;
  void on_begin(cudaStream_t s) const {
    if (begin) begin(user, s);
  }
  void on_end(cudaStream_t s) const {
    if (end) end(user, s);
  }
};

// ---- block Karatsuba over GF(2) on the SM-pair product (k_karatsuba.cu, k_gemm_pair.cu) ----
// The zero-padded Toeplitz matrix, cut into h x h blocks, is block Toeplitz; `levels` rounds of the
// 2x2 split [[T_d, T_d+1], [T_d-1, T_d]] (three products: T_d (x0^x1), (T_d+1 ^ T_d) x1,
// (T_d-1 ^ T_d) x0) leave 3^levels sub-products of mq x kq, each a Toeplitz matrix of a derived
// seed restricted to every span-th h-block (span = h << levels); output block r = (R << levels) + q
// is the XOR of the 2^levels sub-products that level l's bit of q selects (A and, by that bit, B or C).
constexpr uint32_t kMaxLevels = 4;  // rounds of the 2 x 2 block split (3^4 = 81 sub-products at most)
struct KaraPlan {
  uint32_t levels = 0;   // 0: no plan (the plain product)
  uint64_t h = 0, span = 0;
  uint32_t groups = 0;   // 3^levels
  uint64_t mq = 0, kq = 0;          // rows and columns of every sub-product (multiples of h)
  uint32_t seed_front = 0;          // front padding (words) of every derived seed
  uint64_t seed_stride = 0;         // words per derived seed
  uint64_t chunk_blocks = 0;        // blocks per pass (bounds the workspace)
  double model_s = 0;               // modelled seconds for all blocks
};
// forced_levels / forced_h = 0 choose by the cost model; max_workspace = 0 takes 1 GiB for the
// derived operands and sub-product parities of one pass. The plan is empty when nothing fits.
KaraPlan karatsuba_plan(uint64_t n_t, uint64_t m, uint64_t num_blocks, int num_sms, int forced_levels,
                        uint64_t forced_h, uint64_t max_workspace);
// The arguments of the first pass's derived-operand kernel: a launch whose first pass matches the
// key of a split already enqueued (launch_kara_presplit) skips that split.
struct KaraSplitKey {
  const uint32_t* raw = nullptr;
  uint64_t raw_stride = 0, blocks = 0, xk_words = 0;
  uint32_t nw_t = 0, tail_mask = 0, hw = 0, kblocks = 0, levels = 0;
  bool operator==(const KaraSplitKey& o) const {
    return raw == o.raw && raw_stride == o.raw_stride && blocks == o.blocks && xk_words == o.xk_words &&
           nw_t == o.nw_t && tail_mask == o.tail_mask && hw == o.hw && kblocks == o.kblocks && levels == o.levels;
  }
};
struct KaraWorkspace {
  DevBuf seeds, xk, qpar;
  bool xk_ready = false;  // xk holds the derived operands of xk_key (consumed by the next launch)
  KaraSplitKey xk_key;
  uint64_t presplits_used = 0;
  void release() {
    seeds.release();
    xk.release();
    qpar.release();
    xk_ready = false;
  }
};
// The pair kernel on the sub-products: derived seeds (seed_stride words each, front padding
// seed_front), derived raw operands xk (row z * num_blocks + b, kq / 32 words), sub-product
// parities into qpar (row b * groups + z, mq / 32 words: a block's parities are contiguous, so
// the combining pass reads each block's share in one stream).
struct PairKara {
  const uint32_t* seeds;
  uint64_t seed_stride;
  uint32_t seed_front;
  const uint32_t* xk;
  uint64_t xk_words;
  uint32_t* qpar;
  uint64_t h, span, mq, kq;
  uint64_t mq_live;  // sub-product rows that feed an output row below m: ceil(m / span) h
  uint32_t groups;
  const int* skip;   // non-null: the kernel returns at once unless *skip == 0 (a speculative hash)
};
cudaError_t launch_gemm_pair_kara(const DirectArgs& a, const PairKara& k, int* err, int fault, int num_sms,
                                  cudaStream_t s, uint32_t* kernels);
// The whole Karatsuba extraction of a.num_blocks blocks (chunked by plan.chunk_blocks); `hook` is
// called around every launch of the product kernel (one per pass). With packed_out the output goes
// straight into that bit-contiguous stream (block b at bit b m; 4-byte aligned, a whole number of
// 4-byte words long, m >= 64, m <= kKaraPackMaxBits) instead of the word-aligned a.out.
constexpr uint64_t kKaraPackMaxBits = 1ull << 18;  // 32 KB of output words per CTA
//
// A speculative hash (spec non-null) is enqueued before m is known: a.m is the row capacity m_cap,
// the product kernel returns at once unless spec->status is 0, and the combination writes
// spec->m bits per block. It needs packed_out, one pass and the double-buffered combination
// (kara_speculation_fits); seeds_done says the derived seeds are already enqueued
// (launch_kara_seeds with the same a and plan).
// With combine_stream (and an event product_done) the combination runs on that stream after the
// product (recorded on `s`), so `s` is free for other work once the product has run.
cudaError_t launch_gemm_karatsuba(const DirectArgs& a, const KaraPlan& plan, KaraWorkspace& ws, int* err, int fault,
                                  int num_sms, cudaStream_t s, uint32_t* kernels, const TimingHook& hook = TimingHook(),
                                  uint8_t* packed_out = nullptr, const DevSpec* spec = nullptr,
                                  bool seeds_done = false, cudaStream_t combine_stream = nullptr,
                                  cudaEvent_t product_done = nullptr);
// The derived seeds of a plan (3^levels windows of a.seed_rev), as launch_gemm_karatsuba enqueues
// them first.
cudaError_t launch_kara_seeds(const DirectArgs& a, const KaraPlan& plan, KaraWorkspace& ws, cudaStream_t s,
                              uint32_t* kernels);
// Whether a speculative hash of num_blocks blocks with row capacity m_cap runs on this plan.
bool kara_speculation_fits(const KaraPlan& plan, uint64_t m_cap, uint64_t num_blocks);
// Enqueues on `s` the derived operands of the first pass of launch_gemm_karatsuba(a, plan, ...)
// (a needs n_t, raw, raw_stride, nw_t, tail_mask and num_blocks only) and marks them ready: the
// next launch whose first pass has the same split arguments skips its split. The caller orders `s`
// before that launch and clears ws.xk_ready when the operands may go stale.
cudaError_t launch_kara_presplit(const DirectArgs& a, const KaraPlan& plan, KaraWorkspace& ws, int num_sms,
                                 cudaStream_t s, uint32_t* kernels);

}  // namespace qrng

struct qrng_ctx {
  int device = 0;
  int num_sms = 0;
  std::string err;
  qrng::DevBuf hist, result, seed_rev, raw_stage, out_stage, samples_dev, out_dev, seed_dev;
  qrng::DevBuf dev_err;  // int error word written by kernels with bounded waits (0 = no error)
  qrng::DevBuf fft_worst;  // double bits of the worst FFT rounding distance since the last reset
  qrng::FftWorkspace fft;
  qrng::KaraWorkspace kara;
  int kara_levels = 0;       // 0 = chosen by the cost model
  uint64_t kara_h = 0;
  uint64_t kara_workspace = 0;  // 0 = the default budget
  // uneven-batch workspace and its captured graphs (see api.cu)
  qrng::DevBuf batch_meta, batch_raw, batch_rev, batch_out, batch_counter;
  uint64_t batch_generation = 0;  // bumped whenever a batch buffer moves (invalidates cached graphs)
  cudaStream_t capture_stream = nullptr;
  cudaStream_t copy_stream = nullptr;      // host pipeline: output download beside the extraction;
                                           // pipelines: derived operands beside the estimate
  cudaEvent_t copy_ready = nullptr, copy_done = nullptr;
  cudaEvent_t pre_ready = nullptr, pre_done = nullptr;
  // speculative hash: the device-side output length, its pinned copy (beside result_host) and
  // the event after the report's copy
  qrng::DevBuf spec;
  qrng::DevSpec* spec_host = nullptr;
  cudaEvent_t spec_sized = nullptr, spec_est = nullptr, spec_product = nullptr, spec_hashed = nullptr;
  cudaStream_t report_stream = nullptr;  // the report's read-back, beside the hash
  // the last pipeline call's stream shape and output length (predicts the next call's m)
  struct PipelineShape {
    uint64_t n, count;
    int bits, form;
    uint64_t blocks;
    bool operator==(const PipelineShape& o) const {
      return n == o.n && count == o.count && bits == o.bits && form == o.form && blocks == o.blocks;
    }
  };
  bool pipeline_seen = false;
  PipelineShape pipeline_shape{};
  uint64_t pipeline_m = 0;
  // overlapped host pipeline (qrng_postprocess_host_async): two slots of device buffers, used by
  // calls in turn; a slot's buffers are reused once its earlier call's hash (samples, seed) and
  // download (output) are done
  struct AsyncSlot {
    qrng::DevBuf samples, seed, out;
    // the speculative hash's workspace of this slot's calls: the next call's derived operands and
    // seeds are computed right after its upload, while the other slot's call still hashes
    qrng::KaraWorkspace kara;
    qrng::DevBuf seed_rev;
    qrng::DevBuf spec;  // the device-side m of the slot's call (its combination runs on the download stream)
    cudaEvent_t uploaded = nullptr, computed = nullptr, downloaded = nullptr;
    bool used = false;
  };
  AsyncSlot async_slot[2];
  uint64_t async_calls = 0;
  cudaStream_t up_stream = nullptr, down_stream = nullptr;
  struct BatchGraph {
    uint64_t key = 0, generation = 0, stamp = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* meta_host = nullptr;  // pinned copy of the request table the graph uploads
    uint32_t kernels = 0;       // kernels one replay runs
    uint64_t routes[4] = {0, 0, 0, 0};  // requests per route (kRoute*)
    double direct_bitmacs = 0, transform_bytes = 0;
    // recorded by the graph: transform groups [0, 1), persistent direct kernel [2, 3)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool has_transform = false, has_direct = false;
  };
  uint64_t timed_graph_key = 0, timed_graph_generation = 0;  // the last replay made while timing
  bool timed_graph_pending = false;
  qrng::FftWorkspace batch_fft;  // transform workspace of batch graphs only (addresses stay put)
  // per-class routes of QRNG_ALGO_AUTO batches, keyed by transform length: route and FP32 segment
  struct BatchTune {
    uint64_t P;
    int route, log_s;
  };
  std::vector<BatchTune> batch_tuned;
  void* tune_host = nullptr;   // pinned staging of the tuner's request tables
  size_t tune_host_cap = 0;
  std::vector<BatchGraph> graphs;
  uint64_t graph_clock = 0;
  // autotuner: fastest measured algorithm per shape class (n, m to its six leading bits, log2 of
  // the block count rounded up, form)
  struct TuneKey {
    uint64_t n, m;  // m: the class's lower end
    uint32_t log2_blocks;
    int form;
    bool operator==(const TuneKey& o) const {
      return n == o.n && m == o.m && log2_blocks == o.log2_blocks && form == o.form;
    }
  };
  bool autotune = true;
  int fault = 0;  // QRNG_FAULT_* armed for the next tensor-core extraction only
  struct TuneChoice {
    int algo;
    int fft32_log_s;  // segment length of the FP32 route when it won (0 otherwise)
  };
  std::vector<std::pair<TuneKey, TuneChoice>> tuned;
  // FP32 segmented FFT settings (0 = chosen per shape) and its guard word and repair counter
  int fft32_log_s = 0;
  int fft32_terms = 0;
  int last_fft32_log_s = 0;
  qrng::DevBuf fft32_guard;  // int per-call flag + unsigned long long repair count
  qrng::DevHminResult* result_host = nullptr;  // pinned
  qrng_stats stats{};
  // optional CUDA-event timing of the main extraction kernel
  bool timing = false;
  std::vector<cudaEvent_t> ev_start, ev_end;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  size_t ev_pending = (size_t)-1;
};
