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

constexpr int kR = 16;           // output words per warp (= outputs per lane)
constexpr int kWarpsPerCta = 4;

template <int R>
__global__ void __launch_bounds__(32 * kWarpsPerCta) direct_kernel(const DirectArgs a) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t gwarp = (uint64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  const uint64_t total = a.num_blocks * a.tiles * a.splits;
  if (gwarp >= total) return;  // warp-uniform
  const uint32_t split = (uint32_t)(gwarp % a.splits);
  const uint64_t t2 = gwarp / a.splits;
  const uint32_t tile = (uint32_t)(t2 % a.tiles);
  const uint64_t blk = t2 / a.tiles;

  const uint32_t w_begin = split * a.words_per_split;
  uint32_t w_end = w_begin + a.words_per_split;
  if (w_end > a.nw_t) w_end = a.nw_t;

  const uint32_t* __restrict__ raw = a.raw + blk * a.raw_stride;
  const uint32_t* __restrict__ seed = a.seed_rev;

  // Padded reversed-seed bit of window (lane, t):  P(t) = c + 32 t, c = m-1-i0-lane + 32*front.
  const int64_t i0 = (int64_t)tile * 32 * R;
  const int64_t c = (int64_t)a.m - 1 - i0 - (int64_t)lane + 32 * (int64_t)kSeedFrontWords;
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

  const uint32_t nfull = (a.tail_mask == 0xffffffffu) ? a.nw_t : a.nw_t - 1;  // words needing no mask
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
        if (w == a.nw_t - 1) x &= a.tail_mask;
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

  // Epilogue: parities -> output words (lane k keeps word k of this tile).
  uint32_t myword = 0;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    uint32_t wrd = __ballot_sync(0xffffffffu, __popc(acc[k]) & 1u);
    if (lane == (uint32_t)k) myword = wrd;
  }
  if (lane < (uint32_t)R) {
    const uint32_t ow = tile * R + lane;
    if (ow < a.mw) {
      const uint32_t rem = a.m - 32 * ow;
      const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
      myword &= omask;
      if (a.modified && split == 0) {
        // identity block: raw bits [n-m + 32 ow, +32)
        const uint64_t bit = (uint64_t)a.id_off + 32ull * ow;
        const uint64_t rq = bit >> 5;
        const uint32_t rs = (uint32_t)(bit & 31);
        const uint32_t rlo = __ldg(raw + rq);
        const uint32_t rhi = (rs && rq + 1 < a.raw_stride) ? __ldg(raw + rq + 1) : 0u;
        myword ^= __funnelshift_r(rlo, rhi, rs) & omask;
      }
      uint32_t* dst = a.out + blk * a.out_stride + ow;
      if (a.splits > 1) atomicXor(dst, myword);
      else *dst = myword;
    }
  }
}

}  // namespace

int direct_outputs_per_warp() { return 32 * kR; }

cudaError_t launch_direct(const DirectArgs& a, cudaStream_t s, uint32_t* kernels) {
  const uint64_t warps = a.num_blocks * a.tiles * a.splits;
  const uint64_t ctas = ceil_div(warps, kWarpsPerCta);
  if (ctas > 0x7fffffffull) return cudaErrorInvalidConfiguration;
  direct_kernel<kR><<<(unsigned)ctas, 32 * kWarpsPerCta, 0, s>>>(a);
  ++*kernels;
  return cudaGetLastError();
}

}  // namespace qrng
