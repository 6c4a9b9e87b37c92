// Direct bit-packed Toeplitz hashing, k = T r (mod 2) (Sec. III.B; the O(mn) product the paper
// starts from), each block on its own.
//
// Formulation. With the seed reversed (rev[u] = a[L-1-u]) the bits of row i of T that meet raw
// word w (raw bits 32w..32w+31) are the 32 consecutive reversed-seed bits starting at
//     p(i, w) = m - 1 - i + 32 w,
// so   k_i = parity( XOR_w  window(p(i, w)) AND r_w ).
// Each window is one funnel shift of two reversed-seed words, and the XOR accumulation needs one
// LOP3 per 32 bit-products; the parity (POPC) is taken once per output at the end.
//
// Register blocking. Lane l of a warp owns outputs i = i0 + l + 32k, k = 0..R-1. Because
// p(i + 32k, w) = p(i, w - k), output i+32k at word w uses the window output i used at word w-k:
// each lane computes ONE new window per raw word and keeps the last R windows in registers, so a
// raw word costs R LOP3 + 1 funnel shift + 2 loads per lane. The warp's 32R parities become R
// output words through __ballot_sync. Long blocks may split the raw words over several warps;
// their partial parities are XOR-combined in global memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qrng_internal.h"

namespace qrng {
namespace {

constexpr int kR = 32;           // output words per warp (= outputs per lane)
constexpr int kWarpsPerCta = 4;

// Parities of the 32R outputs i0 .. i0+32R-1 (i0 = 32 R tile) over raw words [w_begin, w_end) of
// one block; lane k < R returns output word (R tile + k), unmasked. Warp-uniform arguments.
template <int R>
__device__ __forceinline__ uint32_t direct_tile(const uint32_t* __restrict__ raw, uint32_t nw_t, uint32_t tail_mask,
                                                const uint32_t* __restrict__ seed, uint32_t m, uint32_t tile,
                                                uint32_t w_begin, uint32_t w_end, uint32_t lane) {
  // Padded reversed-seed bit of window (lane, t):  P(t) = c + 32 t, c = m-1-i0-lane + 32*front.
  const int64_t i0 = (int64_t)tile * 32 * R;
  const int64_t c = (int64_t)m - 1 - i0 - (int64_t)lane + 32 * (int64_t)kSeedFrontWords;
  const uint32_t sh = (uint32_t)(c & 31);
  // word index of window t is (c >> 5) + t
  const int64_t qbase = c >> 5;

  uint32_t acc[R];
  uint32_t win[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = 0;

  // Prologue: win[j] = window(w_begin - R + j) for j = 1..R-1 (win[0] is never read before it is set).
  int64_t q = qbase + (int64_t)w_begin - R;  // word of window (w_begin - R)
  uint32_t lo = __ldg(seed + q + 1);
#pragma unroll
  for (int j = 1; j < R; ++j) {
    uint32_t hi = __ldg(seed + q + j + 1);
    win[j] = __funnelshift_r(lo, hi, sh);
    lo = hi;
  }
  win[0] = 0;
  q += R;  // now: word of window w_begin; lo holds seed[q]

  const uint32_t nfull = (tail_mask == 0xffffffffu) ? nw_t : nw_t - 1;  // words needing no mask
  for (uint32_t base = w_begin; base < w_end; base += R) {
    uint32_t r[R];
    if (base + R <= w_end && base + R <= nfull) {
#pragma unroll
      for (int u = 0; u < R; ++u) r[u] = __ldg(raw + base + u);
    } else {
#pragma unroll
      for (int u = 0; u < R; ++u) {
        uint32_t w = base + u;
        uint32_t x = (w < w_end) ? __ldg(raw + w) : 0u;
        if (w == nw_t - 1) x &= tail_mask;
        r[u] = x;
      }
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
      uint32_t hi = __ldg(seed + q + u + 1);
      win[u] = __funnelshift_r(lo, hi, sh);
      lo = hi;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        // acc[k] ^= window(base + u - k) & r[u]
        acc[k] ^= win[(u - k + R) % R] & r[u];
      }
    }
    q += R;
  }

  // parities -> output words (lane k keeps word k of this tile)
  uint32_t myword = 0;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    uint32_t wrd = __ballot_sync(0xffffffffu, __popc(acc[k]) & 1u);
    if (lane == (uint32_t)k) myword = wrd;
  }
  return myword;
}

// Masks output word ow (32 outputs) to m and, for the modified form, XORs in raw bits
// [id_off + 32 ow, +32) of the block (the identity block I_m).
__device__ __forceinline__ uint32_t finish_word(uint32_t word, uint32_t ow, uint32_t m, int modified,
                                                uint32_t id_off, const uint32_t* __restrict__ raw,
                                                uint64_t raw_words) {
  const uint32_t rem = m - 32 * ow;
  const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
  word &= omask;
  if (modified) {
    const uint64_t bit = (uint64_t)id_off + 32ull * ow;
    const uint64_t rq = bit >> 5;
    const uint32_t rs = (uint32_t)(bit & 31);
    const uint32_t rlo = __ldg(raw + rq);
    const uint32_t rhi = (rs && rq + 1 < raw_words) ? __ldg(raw + rq + 1) : 0u;
    word ^= __funnelshift_r(rlo, rhi, rs) & omask;
  }
  return word;
}

template <int R>
__global__ void __launch_bounds__(32 * kWarpsPerCta) direct_kernel(const DirectArgs a) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t gwarp = (uint64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  const uint64_t total = a.num_blocks * a.tiles * a.splits;
  if (gwarp >= total) return;  // warp-uniform
  if (a.guard) {  // exact recomputation only after a tripped rounding guard
    if (*(volatile const int*)a.guard == 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.repairs) atomicAdd(a.repairs, 1ull);
  }
  const uint32_t split = (uint32_t)(gwarp % a.splits);
  const uint64_t t2 = gwarp / a.splits;
  const uint32_t tile = (uint32_t)(t2 % a.tiles);
  const uint64_t blk = t2 / a.tiles;

  const uint32_t w_begin = split * a.words_per_split;
  uint32_t w_end = w_begin + a.words_per_split;
  if (w_end > a.nw_t) w_end = a.nw_t;

  const uint32_t* __restrict__ raw = a.raw + blk * a.raw_stride;
  uint32_t myword = direct_tile<R>(raw, a.nw_t, a.tail_mask, a.seed_rev, a.m, tile, w_begin, w_end, lane);
  if (lane < (uint32_t)R) {
    const uint32_t ow = tile * R + lane;
    if (ow < a.mw) {
      myword = finish_word(myword, ow, a.m, a.modified && split == 0, a.id_off, raw, a.raw_stride);
      uint32_t* dst = a.out + blk * a.out_stride + ow;
      if (a.splits > 1) atomicXor(dst, myword);
      else *dst = myword;
    }
  }
}

// Uneven requests, each with its own seed (one block per request), from one persistent launch:
// every warp repeatedly takes the next work item (request, output tile, raw-word split) from a
// global counter; items are numbered with the largest requests first so the tail stays short.
// Partial parities of the splits of one tile are XOR-combined in the zeroed output staging.
template <int R>
__global__ void __launch_bounds__(32 * kWarpsPerCta) batch_direct_kernel(const BatchReq* __restrict__ reqs,
                                                                          uint32_t nreq, uint64_t total_items,
                                                                          const uint32_t* __restrict__ raw_stage,
                                                                          const uint32_t* __restrict__ rev,
                                                                          uint32_t* __restrict__ out_stage,
                                                                          unsigned long long* __restrict__ counter) {
  const uint32_t lane = threadIdx.x & 31;
  while (true) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(counter, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total_items) return;
    // request r: the last one whose first item is <= item
    uint32_t lo = 0, hi = nreq - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (reqs[mid].item_begin <= item) lo = mid;
      else hi = mid - 1;
    }
    const BatchReq& q = reqs[lo];
    const uint64_t local = item - q.item_begin;
    const uint32_t split = (uint32_t)(local % q.splits);
    const uint32_t tile = (uint32_t)(local / q.splits);
    const uint32_t w_begin = split * kBatchWordsPerSplit;
    const uint32_t w_end = min(w_begin + kBatchWordsPerSplit, q.nw_t);
    const uint32_t* raw = raw_stage + q.raw_stage_off;
    uint32_t myword = direct_tile<R>(raw, q.nw_t, q.tail_mask, rev + q.rev_off, q.m, tile, w_begin, w_end, lane);
    if (lane < (uint32_t)R) {
      const uint32_t ow = tile * R + lane;
      if (ow < q.mw) {
        myword = finish_word(myword, ow, q.m, q.form == QRNG_FORM_MODIFIED && split == 0, q.id_off, raw,
                             q.raw_words);
        uint32_t* dst = out_stage + q.out_stage_off + ow;
        if (q.splits > 1) atomicXor(dst, myword);
        else *dst = myword;
      }
    }
  }
}

}  // namespace

int direct_outputs_per_warp() { return 32 * kR; }

cudaError_t launch_batch_direct(const BatchReq* reqs, uint32_t nreq, uint64_t total_items, const uint32_t* raw_stage,
                                const uint32_t* rev, uint32_t* out_stage, unsigned long long* counter, int num_sms,
                                cudaStream_t s, uint32_t* kernels) {
  const uint64_t want = ceil_div(total_items, kWarpsPerCta);
  const uint64_t cap = (uint64_t)num_sms * 8;  // persistent: a few resident CTAs per SM
  batch_direct_kernel<kR><<<(unsigned)(want < cap ? want : cap), 32 * kWarpsPerCta, 0, s>>>(
      reqs, nreq, total_items, raw_stage, rev, out_stage, counter);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_direct(const DirectArgs& a, cudaStream_t s, uint32_t* kernels) {
  const uint64_t warps = a.num_blocks * a.tiles * a.splits;
  const uint64_t ctas = ceil_div(warps, kWarpsPerCta);
  if (ctas > 0x7fffffffull) return cudaErrorInvalidConfiguration;
  direct_kernel<kR><<<(unsigned)ctas, 32 * kWarpsPerCta, 0, s>>>(a);
  ++*kernels;
  return cudaGetLastError();
}

}  // namespace qrng
