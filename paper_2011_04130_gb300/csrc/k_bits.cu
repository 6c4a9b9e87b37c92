// Bit-layout kernels around the extraction: the bit-reversed seed the Toeplitz windows are read
// from, and the conversions between the caller's bit-contiguous streams (Sec. III.E: block b at
// bit b*n, output b at bit b*m) and word-aligned per-block layouts.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qrng_internal.h"

namespace qrng {
namespace {

// Reads the 32 bits [bit, bit+32) of a byte buffer of `nbits` valid bits (zeros beyond).
__device__ __forceinline__ uint32_t read_bits32(const uint8_t* __restrict__ src, uint64_t nbits, uint64_t bit) {
  if (bit >= nbits) return 0;
  uint64_t byte0 = bit >> 3;
  uint64_t nbytes = (nbits + 7) >> 3;
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (byte0 + k < nbytes) acc |= (uint64_t)src[byte0 + k] << (8 * k);
  uint32_t v = (uint32_t)(acc >> (bit & 7));
  uint64_t left = nbits - bit;
  if (left < 32) v &= (1u << left) - 1u;
  return v;
}

// rev word (kSeedFrontWords + w), bit t  =  a[L-1-(32w+t)]  (zero outside the seed).
__global__ void seed_reverse_kernel(const uint8_t* __restrict__ seed, uint64_t L, uint32_t* __restrict__ rev,
                                    uint64_t rev_words) {
  uint64_t pw = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pw >= rev_words) return;
  int64_t w = (int64_t)pw - kSeedFrontWords;
  uint32_t out = 0;
  if (w >= 0) {
    // reversed bits u = 32w .. 32w+31 map to seed bits L-1-u, i.e. the 32 seed bits ending at L-1-32w.
    int64_t top = (int64_t)L - 1 - 32 * w;  // seed bit for t = 0
    if (top >= 0) {
      int64_t lo = top - 31;  // seed bit for t = 31 (may be negative)
      uint32_t x;
      if (lo >= 0) {
        x = read_bits32(seed, L, (uint64_t)lo);
      } else {
        // only seed bits [0, top] exist: place them at the top of the 32-bit window
        x = read_bits32(seed, L, 0) << (uint32_t)(-lo);
      }
      out = __brev(x);  // bit 31-s of x (seed bit lo+31-s... ) -> bit s: seed bit top-s
    }
  }
  rev[pw] = out;
}

// dst word (b, w) = bits [b*n + 32w, b*n + 32w + 32) of the stream, clipped to the block.
__global__ void repack_blocks_kernel(const uint8_t* __restrict__ src, uint64_t raw_bit_off, uint64_t n,
                                     uint64_t num_blocks, uint32_t* __restrict__ dst, uint64_t stride_w) {
  uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= num_blocks * stride_w) return;
  uint64_t b = idx / stride_w, w = idx - b * stride_w;
  uint64_t total = raw_bit_off + num_blocks * n;
  uint32_t v = 0;
  if (32 * w < n) {
    uint64_t bit = raw_bit_off + b * n + 32 * w;
    v = read_bits32(src, total, bit);
    uint64_t left = n - 32 * w;
    if (left < 32) v &= (1u << left) - 1u;
  }
  dst[idx] = v;
}

// Destination 32-bit word D of the packed output = global output bits [32D, 32D+32).
__global__ void pack_blocks_kernel(const uint32_t* __restrict__ src, uint64_t stride_w, uint64_t m,
                                   uint64_t num_blocks, uint8_t* __restrict__ dst) {
  uint64_t D = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t total = num_blocks * m;
  if (32 * D >= total) return;
  uint32_t v = 0;
  uint64_t g = 32 * D;
  const uint64_t gend = (32 * D + 32 < total) ? 32 * D + 32 : total;
  // the block of bit g: a 32-bit division when every index fits (the common case), else 64-bit
  uint64_t b = total < (1ull << 32) ? (uint64_t)((uint32_t)g / (uint32_t)m) : g / m;
  uint64_t i = g - b * m;
  while (g < gend) {
    uint32_t take = (uint32_t)((m - i) < (gend - g) ? (m - i) : (gend - g));  // bits from this block
    const uint32_t* row = src + b * stride_w;
    uint64_t q = i >> 5;
    uint32_t sh = (uint32_t)(i & 31);
    uint32_t lo = __ldg(row + q);
    uint32_t hi = (sh && q + 1 < stride_w) ? __ldg(row + q + 1) : 0u;
    uint32_t bits = __funnelshift_r(lo, hi, sh);
    if (take < 32) bits &= (1u << take) - 1u;
    v |= bits << (uint32_t)(g - 32 * D);
    g += take;
    ++b;  // the next bits, if any, start the next block
    i = 0;
  }
  const uint64_t nbytes = (total + 7) >> 3;
  uint8_t* p = dst + 4 * D;
  if (((reinterpret_cast<uintptr_t>(dst) & 3) == 0) && 4 * D + 4 <= nbytes) {
    *reinterpret_cast<uint32_t*>(p) = v;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (4 * D + k < nbytes) p[k] = (uint8_t)(v >> (8 * k));
  }
}

// Index of the request whose range [first(r), first(r+1)) holds idx (ranges are non-decreasing).
template <class F>
__device__ __forceinline__ uint32_t find_req(uint32_t nreq, uint64_t idx, F first) {
  uint32_t lo = 0, hi = nreq - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (first(mid) <= idx) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Raw staging word idx of the batch (each request one word-aligned block, bits beyond n zero).
__global__ void batch_repack_kernel(const BatchReq* __restrict__ reqs, uint32_t nreq, uint64_t total,
                                    uint32_t* __restrict__ dst) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const uint32_t r = find_req(nreq, idx, [&](uint32_t k) { return reqs[k].raw_stage_off; });
  const BatchReq& q = reqs[r];
  const uint64_t w = idx - q.raw_stage_off;
  uint32_t v = 0;
  if (32 * w < q.n) {
    v = read_bits32(q.raw, q.raw_bit_off + q.n, q.raw_bit_off + 32 * w);
    const uint64_t left = q.n - 32 * w;
    if (left < 32) v &= (1u << left) - 1u;
  }
  dst[idx] = v;
}

// Reversed, padded seed word idx of the batch (the layout of seed_reverse_kernel, per request).
__global__ void batch_seed_reverse_kernel(const BatchReq* __restrict__ reqs, uint32_t nreq, uint64_t total,
                                          uint32_t* __restrict__ rev) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const uint32_t r = find_req(nreq, idx, [&](uint32_t k) { return reqs[k].rev_off; });
  const BatchReq& q = reqs[r];
  const int64_t w = (int64_t)(idx - q.rev_off) - kSeedFrontWords;
  uint32_t out = 0;
  if (w >= 0) {
    const int64_t top = (int64_t)q.L_t - 1 - 32 * w;
    if (top >= 0) {
      const int64_t lo = top - 31;
      const uint32_t x = lo >= 0 ? read_bits32(q.seed, q.L_t, (uint64_t)lo)
                                 : read_bits32(q.seed, q.L_t, 0) << (uint32_t)(-lo);
      out = __brev(x);
    }
  }
  rev[idx] = out;
}

// Destination word idx of the batch: bits of one request's output moved to its bit offset in the
// caller's buffer. Words shared with other bits of the buffer are merged with atomics.
__global__ void batch_pack_kernel(const BatchReq* __restrict__ reqs, uint32_t nreq, uint64_t total,
                                  const uint32_t* __restrict__ src) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const uint32_t r = find_req(nreq, idx, [&](uint32_t k) { return reqs[k].dst_begin; });
  const BatchReq& q = reqs[r];
  const uint64_t W = q.dst_word0 + (idx - q.dst_begin);      // absolute 32-bit word index
  const uint64_t start = reinterpret_cast<uintptr_t>(q.out) * 8 + q.out_bit_off;  // absolute first output bit
  const uint64_t g0 = (32 * W > start) ? 32 * W : start;
  const uint64_t g1 = (32 * W + 32 < start + q.m) ? 32 * W + 32 : start + q.m;
  const uint32_t* row = src + q.out_stage_off;
  uint32_t val = 0, mask = 0;
  for (uint64_t g = g0; g < g1;) {
    const uint64_t i = g - start;  // output index within the request
    const uint64_t qw = i >> 5;
    const uint32_t sh = (uint32_t)(i & 31);
    const uint32_t take = (uint32_t)min((uint64_t)(32 - sh), g1 - g);
    const uint32_t lo = row[qw];
    const uint32_t hi = (sh && qw + 1 < q.mw) ? row[qw + 1] : 0u;
    uint32_t bits = __funnelshift_r(lo, hi, sh);
    const uint32_t tm = take >= 32 ? 0xffffffffu : ((1u << take) - 1u);
    const uint32_t pos = (uint32_t)(g - 32 * W);
    val |= (bits & tm) << pos;
    mask |= tm << pos;
    g += take;
  }
  uint32_t* dst = reinterpret_cast<uint32_t*>(W * 4);
  if (mask == 0xffffffffu) {
    *dst = val;
  } else {
    atomicAnd(dst, ~mask);
    atomicOr(dst, val);
  }
}

}  // namespace

cudaError_t launch_batch_layout(const BatchReq* reqs, uint32_t nreq, uint64_t raw_words_total, uint64_t rev_words_total,
                                uint32_t* raw_stage, uint32_t* rev, cudaStream_t s, uint32_t* kernels) {
  const int T = 256;
  batch_repack_kernel<<<(unsigned)ceil_div(raw_words_total, T), T, 0, s>>>(reqs, nreq, raw_words_total, raw_stage);
  batch_seed_reverse_kernel<<<(unsigned)ceil_div(rev_words_total, T), T, 0, s>>>(reqs, nreq, rev_words_total, rev);
  *kernels += 2;
  return cudaGetLastError();
}

cudaError_t launch_batch_pack(const BatchReq* reqs, uint32_t nreq, uint64_t dst_words_total, const uint32_t* out_stage,
                              cudaStream_t s, uint32_t* kernels) {
  const int T = 256;
  batch_pack_kernel<<<(unsigned)ceil_div(dst_words_total, T), T, 0, s>>>(reqs, nreq, dst_words_total, out_stage);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_seed_reverse(const uint8_t* seed, uint64_t L, uint32_t* rev, uint64_t rev_words, cudaStream_t s,
                                uint32_t* kernels) {
  const int T = 256;
  seed_reverse_kernel<<<(unsigned)ceil_div(rev_words, T), T, 0, s>>>(seed, L, rev, rev_words);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_repack_blocks(const uint8_t* src, uint64_t raw_bit_off, uint64_t n, uint64_t num_blocks,
                                 uint32_t* dst, uint64_t stride_w, cudaStream_t s, uint32_t* kernels) {
  const int T = 256;
  uint64_t total = num_blocks * stride_w;
  repack_blocks_kernel<<<(unsigned)ceil_div(total, T), T, 0, s>>>(src, raw_bit_off, n, num_blocks, dst, stride_w);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_pack_blocks(const uint32_t* src, uint64_t stride_w, uint64_t m, uint64_t num_blocks, uint8_t* dst,
                               cudaStream_t s, uint32_t* kernels) {
  const int T = 256;
  uint64_t words = ceil_div(num_blocks * m, 32);
  pack_blocks_kernel<<<(unsigned)ceil_div(words, T), T, 0, s>>>(src, stride_w, m, num_blocks, dst);
  ++*kernels;
  return cudaGetLastError();
}

}  // namespace qrng
