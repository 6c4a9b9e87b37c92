// Block Karatsuba over GF(2) for the block-batched Toeplitz product (Sec. III.B, III.E).
//
// The hash of every block is k = T x over GF(2) with T the m x n_t Toeplitz matrix of the shared
// seed, T[i][j] = a[n_t - 1 + i - j]. Pad T with zero seed bits to M x K (multiples of
// span = h << levels) and x with zero bits; cut T into h x h blocks: block (r, c) depends on
// d = c - r alone (T_d, itself Toeplitz). A 2 x 2 group of blocks [[T_d, T_d+1], [T_d-1, T_d]]
// times (x0, x1) needs three block products instead of four, because over GF(2)
//     y0 = T_d x0 + T_d+1 x1 = T_d (x0 ^ x1) + (T_d+1 ^ T_d) x1     (A + B)
//     y1 = T_d-1 x0 + T_d x1 = T_d (x0 ^ x1) + (T_d-1 ^ T_d) x0     (A + C).
// The grid of A products (and of B, of C) is again block Toeplitz, with blocks of every other
// diagonal, so the split repeats: after `levels` rounds there are 3^levels sub-products, each an
// mq x kq product (mq = M / 2^levels, kq = K / 2^levels). In the reversed-seed form the kernels use
// (rho(p) = a[L-1-p], zero outside [0, L)), T_d+1 ^ T_d is the Toeplitz matrix of
// rho(p) ^ rho(p + s) and T_d-1 ^ T_d that of rho(p) ^ rho(p - s), s = h << (level - 1). Sub-product
// z = (z_1 .. z_levels) in base 3 (0 = A, 1 = B, 2 = C, level 1 least significant) reads the XOR
// of raw h-blocks 2^levels C + q over the q whose bit l-1 is 0 or 1 for A, 1 for B, 0 for C, and
// output h-block 2^levels R + q is the XOR of the 2^levels sub-products whose digit l is A or (B if
// bit l-1 of q is 0, else C). Parities add, so each sub-product is one exact integer product whose
// parity is taken once; the combining pass XORs words.
//
// Work: 3^levels mq kq against m n_t multiply-adds per block (9/16 at two levels), for three
// cheap memory-bound passes: the derived seeds (3^levels short bit strings), the derived raw
// operands (3^levels x K/2^levels bits per block) and the combination (2^levels words read per
// output word), which writes the bit-contiguous output stream directly when its layout allows.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "qrng_internal.h"
#include "tc_util.cuh"

namespace qrng {
namespace {

constexpr int kThreads = 256;
constexpr int kPackThreads = 128;  // combine-and-pack CTAs (one block each; most of the work is the staging)
constexpr uint32_t kPackSmemWords = 12288;  // 48 KB of shared memory per combine-and-pack CTA
constexpr size_t kPackBulkMaxSmem = 112 * 1024;  // double-buffered combination: at least two CTAs per SM
constexpr uint64_t kDefaultWorkspace = 1ull << 30;  // derived operands + sub-product parities per pass

__host__ __device__ constexpr int pow3c(int l) { return l == 0 ? 1 : 3 * pow3c(l - 1); }

__host__ __device__ inline uint32_t pow3(uint32_t l) {
  uint32_t r = 1;
  for (uint32_t i = 0; i < l; ++i) r *= 3;
  return r;
}

// Derived reversed seeds: word w of seed z holds bits p = 32 (w - front) .. +31 of
// rho_z = XOR of rho shifted by the offsets that z's digits select.
__global__ void kara_seed_kernel(const uint32_t* __restrict__ rev, uint64_t rev_words, uint32_t levels, uint32_t hw,
                                 uint32_t front, uint64_t words, uint32_t* __restrict__ seeds, uint64_t stride) {
  const uint32_t z = blockIdx.y;
  int64_t offs[1 << kMaxLevels];
  uint32_t n = 1;
  offs[0] = 0;
  uint32_t zz = z;
  for (uint32_t l = 0; l < levels; ++l) {
    const uint32_t d = zz % 3;
    zz /= 3;
    const int64_t s = (int64_t)hw << l;
    if (d != 0) {
      for (uint32_t i = 0; i < n; ++i) offs[n + i] = offs[i] + (d == 1 ? s : -s);
      n *= 2;
    }
  }
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v = 0;
    for (uint32_t i = 0; i < n; ++i) {
      const int64_t q = (int64_t)w - (int64_t)front + offs[i] + kSeedFrontWords;
      if (q >= 0 && q < (int64_t)rev_words) v ^= __ldg(rev + q);
    }
    seeds[(uint64_t)z * stride + w] = v;
  }
}

// Derived raw operands: thread (b, c, w) reads word w of raw h-blocks 2^L c + q (zero past the
// Toeplitz part) and writes word c * hw + w of every sub-product's operand row z * nb + b.
template <int L>
__global__ void kara_split_kernel(const uint32_t* __restrict__ raw, uint64_t raw_stride, uint32_t nw_t,
                                  uint32_t tail_mask, uint64_t nb, uint32_t hw, uint32_t kblocks, uint64_t xk_words,
                                  uint32_t* __restrict__ xk) {
  constexpr int Q = 1 << L;
  constexpr int G = pow3c(L);
  uint32_t take[G];  // bit q: raw h-block q of the group enters sub-product z
#pragma unroll
  for (int z = 0; z < G; ++z) {
    uint32_t mask = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      bool in = true;
      int zz = z;
#pragma unroll
      for (int l = 0; l < L; ++l) {
        const int d = zz % 3;
        zz /= 3;
        const int bit = (q >> l) & 1;
        in = in && (d == 0 || (d == 1 && bit == 1) || (d == 2 && bit == 0));
      }
      if (in) mask |= 1u << q;
    }
    take[z] = mask;
  }
  const uint64_t total = nb * kblocks * hw;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t w = (uint32_t)(idx % hw);
    const uint64_t t = idx / hw;
    const uint32_t c = (uint32_t)(t % kblocks);
    const uint64_t b = t / kblocks;
    uint32_t src[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint64_t i = ((uint64_t)c << L) * hw + (uint64_t)q * hw + w;
      uint32_t v = i < nw_t ? __ldg(raw + b * raw_stride + i) : 0u;
      if (i == (uint64_t)nw_t - 1) v &= tail_mask;
      src[q] = v;
    }
#pragma unroll
    for (int z = 0; z < G; ++z) {
      uint32_t v = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if ((take[z] >> q) & 1u) v ^= src[q];
      xk[((uint64_t)z * nb + b) * xk_words + (uint64_t)c * hw + w] = v;
    }
  }
}

// Output words of block b at row-word position (R, lw): for each q < 2^L, word
// ow = ((R << L) + q) h/32 + lw (rows 32 ow .. 32 ow + 31, inside h-block (R << L) + q) is the XOR
// of the 2^L sub-product words of rows R h + 32 lw that q selects. The thread loads the 3^L
// sub-product words once and writes all 2^L outputs; then the tail mask and, for the modified
// form, the identity part x[n - m + i].
template <int L>
__global__ void kara_combine_kernel(const uint32_t* __restrict__ qpar, uint64_t mwq, uint32_t log2h, uint64_t nb,
                                    uint32_t rblocks, uint32_t* __restrict__ out, uint64_t out_stride, uint32_t mw,
                                    uint32_t m, int modified, uint32_t id_off, const uint32_t* __restrict__ raw,
                                    uint64_t raw_stride) {
  constexpr int G = pow3c(L);
  const uint32_t hw = 1u << (log2h - 5);
  const uint64_t total = nb * rblocks * hw;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t lw = (uint32_t)(idx % hw);
    const uint64_t t = idx / hw;
    const uint32_t R = (uint32_t)(t % rblocks);
    const uint64_t b = t / rblocks;
    const uint64_t row_word = (uint64_t)R * hw + lw;
    uint32_t qz[G];
#pragma unroll
    for (int z = 0; z < G; ++z) qz[z] = __ldg(qpar + (b * G + (uint64_t)z) * mwq + row_word);
    const uint32_t* rr = raw + b * raw_stride;
#pragma unroll
    for (int q = 0; q < (1 << L); ++q) {
      const uint32_t ow = (((R << L) + (uint32_t)q) << (log2h - 5)) + lw;
      if (ow >= mw) break;  // ow grows with q
      uint32_t acc = 0;
#pragma unroll
      for (int s = 0; s < (1 << L); ++s) {  // subset s of the levels whose digit is B or C
        int z = 0, p3 = 1;
#pragma unroll
        for (int l = 0; l < L; ++l) {
          if ((s >> l) & 1) z += (1 + ((q >> l) & 1)) * p3;
          p3 *= 3;
        }
        acc ^= qz[z];
      }
      const uint32_t v0 = 32u * ow;
      const uint32_t rem = m - v0;
      const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
      acc &= omask;
      if (modified) {
        const uint64_t bit = (uint64_t)id_off + v0;
        const uint64_t rq = bit >> 5;
        const uint32_t rs = (uint32_t)(bit & 31);
        const uint32_t rlo = __ldg(rr + rq);
        const uint32_t rhi = (rs && rq + 1 < raw_stride) ? __ldg(rr + rq + 1) : 0u;
        acc ^= __funnelshift_r(rlo, rhi, rs) & omask;
      }
      out[b * out_stride + ow] = acc;
    }
  }
}

// The same combination for one block per CTA, written straight into the bit-contiguous stream.
// The block's sub-product parities (G rows of mwq words, contiguous) are staged in shared memory
// with 16-byte loads, `cw` row words of every sub-product at a time; the block's output words are
// assembled in shared memory, then its bit range [b m, (b+1) m) is stored in place -- words inside
// the range with plain stores, the (at most two) words it shares with its neighbours with an AND
// that clears its own bits and an OR that sets them (the neighbours' bits are disjoint, so the
// order of the four operations does not matter). The stream's last block also clears the pad bits
// of the last word. Needs a 4-byte aligned stream whose byte length is a multiple of 4, m >= 64 (a
// word then holds bits of at most two blocks), and mwq and cw multiples of 4.
template <int L>
__global__ void __launch_bounds__(kPackThreads) kara_combine_pack_kernel(
    const uint32_t* __restrict__ qpar, uint64_t mwq, uint32_t log2h, uint32_t cw, uint32_t* __restrict__ stream,
    uint64_t block0, uint64_t total_blocks, uint32_t mw, uint32_t m, int modified, uint32_t id_off,
    const uint32_t* __restrict__ raw, uint64_t raw_stride) {
  constexpr int G = pow3c(L);
  extern __shared__ __align__(16) uint32_t smem_words[];
  uint32_t* qs = smem_words;           // [G][cw]: the staged parity row words
  uint32_t* sw = smem_words + G * cw;  // the block's mw output words
  const uint32_t hw = 1u << (log2h - 5);
  const uint64_t b = blockIdx.x;
  const uint32_t* qb = qpar + b * G * mwq;
  const uint32_t* rr = raw + b * raw_stride;
  for (uint32_t rw0 = 0; rw0 < (uint32_t)mwq; rw0 += cw) {
    const uint32_t n = (uint32_t)mwq - rw0 < cw ? (uint32_t)mwq - rw0 : cw;  // a multiple of 4
    const uint32_t nv = n / 4;
    for (uint32_t i = threadIdx.x; i < G * nv; i += blockDim.x) {
      const uint32_t z = i / nv, k = i - z * nv;
      reinterpret_cast<uint4*>(qs + z * cw)[k] = __ldcs(reinterpret_cast<const uint4*>(qb + z * mwq + rw0) + k);
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
      const uint32_t row_word = rw0 + t;  // = R * hw + lw
      const uint32_t R = row_word / hw, lw = row_word - R * hw;
#pragma unroll
      for (int q = 0; q < (1 << L); ++q) {
        const uint32_t ow = (((R << L) + (uint32_t)q) << (log2h - 5)) + lw;
        if (ow >= mw) break;
        uint32_t acc = 0;
#pragma unroll
        for (int s = 0; s < (1 << L); ++s) {  // subset s of the levels whose digit is B or C
          int z = 0, p3 = 1;
#pragma unroll
          for (int l = 0; l < L; ++l) {
            if ((s >> l) & 1) z += (1 + ((q >> l) & 1)) * p3;
            p3 *= 3;
          }
          acc ^= qs[z * cw + t];
        }
        const uint32_t v0 = 32u * ow;
        const uint32_t rem = m - v0;
        const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
        acc &= omask;
        if (modified) {
          const uint64_t bit = (uint64_t)id_off + v0;
          const uint64_t rq = bit >> 5;
          const uint32_t rs = (uint32_t)(bit & 31);
          const uint32_t rlo = __ldg(rr + rq);
          const uint32_t rhi = (rs && rq + 1 < raw_stride) ? __ldg(rr + rq + 1) : 0u;
          acc ^= __funnelshift_r(rlo, rhi, rs) & omask;
        }
        sw[ow] = acc;
      }
    }
    __syncthreads();
  }
  const uint64_t gb = block0 + b;
  const uint64_t bm = gb * m;
  const uint64_t d0 = bm >> 5, d1 = (bm + m - 1) >> 5;
  const bool last = gb + 1 == total_blocks;
  for (uint64_t D = d0 + threadIdx.x; D <= d1; D += blockDim.x) {
    const int64_t off = (int64_t)(32 * D) - (int64_t)bm;  // block bit of the word's bit 0
    uint32_t v, mask;
    if (off >= 0) {
      const uint32_t q = (uint32_t)(off >> 5), sh = (uint32_t)(off & 31);
      const uint32_t lo = sw[q], hi = (sh && q + 1 < mw) ? sw[q + 1] : 0u;
      v = __funnelshift_r(lo, hi, sh);
      const uint64_t rem = m - (uint64_t)off;
      mask = (rem >= 32 || last) ? 0xffffffffu : ((1u << rem) - 1u);  // the last block owns the pad bits
    } else {
      const uint32_t k0 = (uint32_t)(-off);  // 1..31: the word starts inside the previous block
      v = sw[0] << k0;
      mask = 0xffffffffu << k0;
    }
    v &= mask;
    if (mask == 0xffffffffu) {
      stream[D] = v;
    } else {
      atomicAnd(stream + D, ~mask);
      atomicOr(stream + D, v);
    }
  }
}

// The combination for blocks whose parities fit twice in shared memory: persistent CTAs loop over
// blocks; a block's 3^L parity rows (one contiguous run of G mwq words) arrive by one bulk copy into
// one of two buffers while the previous block is combined and written, so every CTA keeps a copy in
// flight through its compute and store phases. Same output as kara_combine_pack_kernel. Waits are
// bounded: on a timeout the CTA records `err`, waits (again bounded) for its copy in flight and
// returns.
template <int L>
__global__ void __launch_bounds__(kPackThreads) kara_combine_pack_bulk_kernel(
    const uint32_t* __restrict__ qpar, uint32_t mwq, uint32_t log2h, uint32_t* __restrict__ stream, uint64_t nb,
    uint64_t block0, uint64_t total_blocks, uint32_t mw, uint32_t m, int modified, uint32_t id_off,
    const uint32_t* __restrict__ raw, uint64_t raw_stride, int* err, const DevSpec* __restrict__ spec) {
  using namespace tc;
  constexpr int G = pow3c(L);
  if (spec != nullptr) {  // a speculative hash: m from the device, nothing written unless it stands
    if (spec->status != 0) return;
    m = (uint32_t)spec->m;
    mw = spec->mw;
  }
  extern __shared__ __align__(16) uint32_t smem_words[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ volatile int abort_flag;
  const uint32_t qwords = (uint32_t)G * mwq;  // a multiple of 8: 32-byte runs
  const uint32_t bytes = qwords * 4u;
  uint32_t* sw = smem_words + 2 * qwords;     // the block's mw output words
  const uint32_t hw = 1u << (log2h - 5);
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](uint64_t blk, uint32_t slot) {
    fence_proxy_async_smem();  // the buffer's earlier generic reads before the async-proxy write
    mbar_arrive_expect_tx(&full[slot], bytes);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_words + slot * qwords)),
        "l"(qpar + blk * qwords), "r"(bytes), "r"(smem_u32(&full[slot]))
        : "memory");
  };
  if (threadIdx.x == 0 && blockIdx.x < nb) issue(blockIdx.x, 0);
  uint32_t it = 0;
  for (uint64_t b = blockIdx.x; b < nb; b += gridDim.x, ++it) {
    const uint32_t slot = it & 1u;
    const uint64_t bn = b + gridDim.x;
    if (threadIdx.x == 0 && bn < nb) issue(bn, slot ^ 1u);  // that buffer's last reader passed the barrier below
    mbar_wait(&full[slot], (it >> 1) & 1u, &abort_flag, err, 11);
    __syncthreads();
    if (abort_flag) {  // the copies this CTA issued must land before it exits
      if (threadIdx.x == 0) {
        mbar_drain(&full[slot], (it >> 1) & 1u, err, 12);
        if (bn < nb) mbar_drain(&full[slot ^ 1u], ((it + 1) >> 1) & 1u, err, 12);
      }
      return;
    }
    const uint32_t* qs = smem_words + slot * qwords;
    const uint32_t* rr = raw + b * raw_stride;
    for (uint32_t t = threadIdx.x; t < mwq; t += blockDim.x) {
      const uint32_t R = t / hw, lw = t - R * hw;  // row word t = R * hw + lw
#pragma unroll
      for (int q = 0; q < (1 << L); ++q) {
        const uint32_t ow = (((R << L) + (uint32_t)q) << (log2h - 5)) + lw;
        if (ow >= mw) break;
        uint32_t acc = 0;
#pragma unroll
        for (int s = 0; s < (1 << L); ++s) {  // subset s of the levels whose digit is B or C
          int z = 0, p3 = 1;
#pragma unroll
          for (int l = 0; l < L; ++l) {
            if ((s >> l) & 1) z += (1 + ((q >> l) & 1)) * p3;
            p3 *= 3;
          }
          acc ^= qs[z * mwq + t];
        }
        const uint32_t v0 = 32u * ow;
        const uint32_t rem = m - v0;
        const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
        acc &= omask;
        if (modified) {
          const uint64_t bit = (uint64_t)id_off + v0;
          const uint64_t rq = bit >> 5;
          const uint32_t rs = (uint32_t)(bit & 31);
          const uint32_t rlo = __ldg(rr + rq);
          const uint32_t rhi = (rs && rq + 1 < raw_stride) ? __ldg(rr + rq + 1) : 0u;
          acc ^= __funnelshift_r(rlo, rhi, rs) & omask;
        }
        sw[ow] = acc;
      }
    }
    __syncthreads();
    const uint64_t gb = block0 + b;
    const uint64_t bm = gb * m;
    const uint64_t d0 = bm >> 5, d1 = (bm + m - 1) >> 5;
    const bool last = gb + 1 == total_blocks;
    for (uint64_t D = d0 + threadIdx.x; D <= d1; D += blockDim.x) {
      const int64_t off = (int64_t)(32 * D) - (int64_t)bm;  // block bit of the word's bit 0
      uint32_t v, mask;
      if (off >= 0) {
        const uint32_t q = (uint32_t)(off >> 5), sh = (uint32_t)(off & 31);
        const uint32_t lo = sw[q], hi = (sh && q + 1 < mw) ? sw[q + 1] : 0u;
        v = __funnelshift_r(lo, hi, sh);
        const uint64_t rem = m - (uint64_t)off;
        mask = (rem >= 32 || last) ? 0xffffffffu : ((1u << rem) - 1u);  // the last block owns the pad bits
      } else {
        const uint32_t k0 = (uint32_t)(-off);  // 1..31: the word starts inside the previous block
        v = sw[0] << k0;
        mask = 0xffffffffu << k0;
      }
      v &= mask;
      if (mask == 0xffffffffu) {
        stream[D] = v;
      } else {
        atomicAnd(stream + D, ~mask);
        atomicOr(stream + D, v);
      }
    }
    __syncthreads();  // sw and this buffer are free again
  }
}

unsigned grid_for(uint64_t items, int num_sms) {
  const uint64_t want = ceil_div(items, kThreads);
  const uint64_t cap = (uint64_t)(num_sms > 0 ? num_sms : 1) * 16;
  return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <int L>
void launch_split(unsigned grid, cudaStream_t s, const DirectArgs& dc, const DirectArgs& d, uint64_t nb, uint32_t hw,
                  uint32_t kblocks, uint64_t xk_words, KaraWorkspace& ws) {
  kara_split_kernel<L><<<grid, kThreads, 0, s>>>(dc.raw, d.raw_stride, d.nw_t, d.tail_mask, nb, hw, kblocks, xk_words,
                                                 ws.xk.as<uint32_t>());
}

template <int L>
void launch_combine_pack(uint64_t nb, size_t smem, cudaStream_t s, const PairKara& k, uint64_t mwq, uint32_t log2h,
                         uint32_t cw, uint32_t* stream, uint64_t b0, const DirectArgs& d, const DirectArgs& dc) {
  kara_combine_pack_kernel<L><<<(unsigned)nb, kPackThreads, smem, s>>>(
      k.qpar, mwq, log2h, cw, stream, b0, d.num_blocks, d.mw, d.m, d.modified, d.id_off, dc.raw, d.raw_stride);
}

KaraSplitKey split_key(const DirectArgs& dc, const DirectArgs& d, uint64_t nb, uint64_t xk_words, uint32_t hw,
                       uint32_t kblocks, uint32_t levels) {
  KaraSplitKey k;
  k.raw = dc.raw;
  k.raw_stride = d.raw_stride;
  k.blocks = nb;
  k.xk_words = xk_words;
  k.nw_t = d.nw_t;
  k.tail_mask = d.tail_mask;
  k.hw = hw;
  k.kblocks = kblocks;
  k.levels = levels;
  return k;
}

cudaError_t launch_split_levels(uint32_t levels, const DirectArgs& dc, const DirectArgs& d, uint64_t nb, uint32_t hw,
                                uint32_t kblocks, uint64_t xk_words, KaraWorkspace& ws, int num_sms,
                                cudaStream_t s) {
  const unsigned gs = grid_for(nb * kblocks * hw, num_sms);
  switch (levels) {
    case 1: launch_split<1>(gs, s, dc, d, nb, hw, kblocks, xk_words, ws); break;
    case 2: launch_split<2>(gs, s, dc, d, nb, hw, kblocks, xk_words, ws); break;
    case 3: launch_split<3>(gs, s, dc, d, nb, hw, kblocks, xk_words, ws); break;
    default: launch_split<4>(gs, s, dc, d, nb, hw, kblocks, xk_words, ws); break;
  }
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_combine_pack_bulk(unsigned grid, size_t smem, cudaStream_t s, const PairKara& k, uint32_t mwq,
                                     uint32_t log2h, uint32_t* stream, uint64_t nb, uint64_t b0, const DirectArgs& d,
                                     const DirectArgs& dc, int* err, const DevSpec* spec) {
  // the shared-memory attribute is set once per device and level count
  constexpr int kMaxDev = 64;
  static size_t set_to[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev || set_to[dev] < smem) {
    e = cudaFuncSetAttribute(kara_combine_pack_bulk_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPackBulkMaxSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDev) set_to[dev] = kPackBulkMaxSmem;
  }
  kara_combine_pack_bulk_kernel<L><<<grid, kPackThreads, smem, s>>>(k.qpar, mwq, log2h, stream, nb, b0, d.num_blocks,
                                                                     d.mw, d.m, d.modified, d.id_off, dc.raw,
                                                                     d.raw_stride, err, spec);
  return cudaGetLastError();
}

template <int L>
void launch_combine(unsigned grid, cudaStream_t s, const PairKara& k, uint64_t mwq, uint32_t log2h, uint64_t nb,
                    uint32_t rblocks, const DirectArgs& d, const DirectArgs& dc) {
  kara_combine_kernel<L><<<grid, kThreads, 0, s>>>(k.qpar, mwq, log2h, nb, rblocks, dc.out, d.out_stride, d.mw, d.m,
                                                   d.modified, d.id_off, dc.raw, d.raw_stride);
}

}  // namespace

KaraPlan karatsuba_plan(uint64_t n_t, uint64_t m, uint64_t num_blocks, int num_sms, int forced_levels,
                        uint64_t forced_h, uint64_t max_workspace) {
  KaraPlan best;
  if (n_t == 0 || m == 0 || num_blocks == 0 || n_t > kGemmMaxColumns) return best;
  const uint64_t budget = max_workspace ? max_workspace : kDefaultWorkspace;
  const double clusters = (double)(num_sms / 2 > 0 ? num_sms / 2 : 1);
  for (uint32_t L = 1; L <= kMaxLevels; ++L) {
    if (forced_levels && (uint32_t)forced_levels != L) continue;
    for (uint32_t lg = 8; lg <= 13; ++lg) {
      const uint64_t h = 1ull << lg;
      if (forced_h ? forced_h != h : lg > 12) continue;
      const uint64_t span = h << L;
      const uint32_t G = pow3(L);
      // h = 256: pair tiles take two row blocks, so their number is rounded up to even
      const uint64_t rblocks = h == 256 ? ceil_div(m, 2 * span) * 2 : ceil_div(m, span);
      const uint64_t mq = rblocks * h, kq = ceil_div(n_t, span) * h;
      const uint64_t per_block = (uint64_t)G * (mq + kq) / 8;
      uint64_t chunk = budget / per_block;
      // whole tile widths of the product kernel; never fewer than one (224 blocks), even when the
      // budget is smaller than that needs
      chunk = chunk >= 224 ? chunk / 224 * 224 : 224;
      if (chunk > num_blocks) chunk = num_blocks;
      while ((uint64_t)G * chunk >= (1ull << 31)) chunk /= 2;
      if (chunk == 0) continue;
      // pair tiles of 512 sub-product rows x 224 blocks over whole rounds of one tile per cluster;
      // a tile takes kq/256 product steps (0.477 us each on GB300) plus one build-only step per K
      // block (about half a step; one per tile when h = 256) and its accumulator hand-back (about
      // 2.8 steps); the passes around it (derived operands written and read, parities written and
      // read once, the raw bits and the output) move their bytes at ~6 TB/s, part of them in L2
      // a pair whose second output tile holds no needed row issues half the MMAs (about 0.6 of a
      // full pair's time, its fixed per-tile part included)
      const uint64_t passes = ceil_div(num_blocks, chunk);
      const uint64_t live_tiles = ceil_div(ceil_div(m, span) * h, 256);
      const double pair_share = ((double)(live_tiles / 2) + 0.6 * (double)(live_tiles % 2)) / (double)(mq / 512);
      const double tiles = (double)G * (double)(mq / 512) * std::ceil((double)chunk / 224.0);
      const double steps = (double)(kq / 256) + 0.5 * (double)(h == 256 ? 1 : kq / h) + 2.8;
      const double kernel_s = (double)passes * std::ceil(tiles * pair_share / clusters) * steps * 0.477e-6;
      const double bytes =
          (double)num_blocks * ((double)n_t / 8 + 2.0 * G * (double)kq / 8 + 2.0 * G * (double)mq / 8 + (double)m / 8);
      const double t = kernel_s + bytes / 6e12 + (double)passes * 2e-5;
      if (best.levels == 0 || t < best.model_s) {
        best.levels = L;
        best.h = h;
        best.span = span;
        best.groups = G;
        best.mq = mq;
        best.kq = kq;
        best.seed_front = (uint32_t)(2 * span / 32 + 16);
        best.seed_stride = best.seed_front + ceil_div(m + ceil_div(n_t, span) * span, 32) + 16;
        best.chunk_blocks = chunk;
        best.model_s = t;
      }
    }
  }
  return best;
}

namespace {
// shared memory of the double-buffered combination: two blocks' parity rows and one output block
size_t bulk_smem_bytes(const KaraPlan& p, uint64_t mw) {
  return ((size_t)2 * p.groups * (p.mq / 32) + mw) * sizeof(uint32_t);
}
}  // namespace

bool kara_speculation_fits(const KaraPlan& p, uint64_t m_cap, uint64_t num_blocks) {
  return p.levels >= 1 && p.levels <= kMaxLevels && p.chunk_blocks >= num_blocks && m_cap >= kSpecMinBits &&
         m_cap <= kKaraPackMaxBits && bulk_smem_bytes(p, ceil_div(m_cap, 32)) <= kPackBulkMaxSmem;
}

cudaError_t launch_kara_seeds(const DirectArgs& d, const KaraPlan& p, KaraWorkspace& ws, cudaStream_t s,
                              uint32_t* kernels) {
  if (p.levels < 1 || p.levels > kMaxLevels) return cudaErrorInvalidValue;
  cudaError_t e = ws.seeds.ensure((size_t)p.groups * p.seed_stride * 4);
  if (e != cudaSuccess) return e;
  const uint64_t L_t = d.n_t + d.m - 1;
  const uint64_t rev_words = kSeedFrontWords + ceil_div(L_t, 32) + kSeedBackWords;
  kara_seed_kernel<<<dim3((unsigned)ceil_div(p.seed_stride, kThreads), p.groups), kThreads, 0, s>>>(
      d.seed_rev, rev_words, p.levels, (uint32_t)(p.h / 32), p.seed_front, p.seed_stride, ws.seeds.as<uint32_t>(),
      p.seed_stride);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_gemm_karatsuba(const DirectArgs& d, const KaraPlan& p, KaraWorkspace& ws, int* err, int fault,
                                  int num_sms, cudaStream_t s, uint32_t* kernels, const TimingHook& hook,
                                  uint8_t* packed_out, const DevSpec* spec, bool seeds_done,
                                  cudaStream_t combine_stream, cudaEvent_t product_done) {
  if (p.levels < 1 || p.levels > kMaxLevels) return cudaErrorInvalidValue;
  if (spec && (!packed_out || !kara_speculation_fits(p, d.m, d.num_blocks))) return cudaErrorInvalidValue;
  if (combine_stream && (!product_done || !packed_out || p.chunk_blocks < d.num_blocks)) return cudaErrorInvalidValue;
  const uint32_t G = p.groups;
  const uint32_t hw = (uint32_t)(p.h / 32);
  uint32_t log2h = 0;
  while ((1ull << log2h) < p.h) ++log2h;
  const uint64_t xk_words = p.kq / 32, mwq = p.mq / 32;
  const uint64_t chunk = p.chunk_blocks < d.num_blocks ? p.chunk_blocks : d.num_blocks;
  cudaError_t e;
  if ((e = ws.xk.ensure((size_t)G * chunk * xk_words * 4)) != cudaSuccess) return e;
  if ((e = ws.qpar.ensure((size_t)G * chunk * mwq * 4)) != cudaSuccess) return e;
  if (!seeds_done && (e = launch_kara_seeds(d, p, ws, s, kernels)) != cudaSuccess) return e;

  PairKara k{};
  k.seeds = ws.seeds.as<uint32_t>();
  k.seed_stride = p.seed_stride;
  k.seed_front = p.seed_front;
  k.xk = ws.xk.as<uint32_t>();
  k.xk_words = xk_words;
  k.qpar = ws.qpar.as<uint32_t>();
  k.h = p.h;
  k.span = p.span;
  k.mq = p.mq;
  k.mq_live = ceil_div(d.m, p.span) * p.h;
  k.kq = p.kq;
  k.groups = G;
  k.skip = spec ? &spec->status : nullptr;
  const uint32_t kblocks = (uint32_t)(p.kq / p.h);
  for (uint64_t b0 = 0; b0 < d.num_blocks; b0 += chunk) {
    const uint64_t nb = d.num_blocks - b0 < chunk ? d.num_blocks - b0 : chunk;
    DirectArgs dc = d;
    dc.raw = d.raw + b0 * d.raw_stride;
    dc.out = d.out + b0 * d.out_stride;
    dc.num_blocks = nb;
    const KaraSplitKey key = split_key(dc, d, nb, xk_words, hw, kblocks, p.levels);
    const bool presplit = b0 == 0 && ws.xk_ready && ws.xk_key == key;
    ws.xk_ready = false;
    if (presplit) ++ws.presplits_used;
    if (!presplit) {
      if ((e = launch_split_levels(p.levels, dc, d, nb, hw, kblocks, xk_words, ws, num_sms, s)) != cudaSuccess)
        return e;
      ++*kernels;
    }
    hook.on_begin(s);
    e = launch_gemm_pair_kara(dc, k, err, fault, num_sms, s, kernels);
    hook.on_end(s);
    if (e != cudaSuccess) return e;
    const uint32_t rblocks = (uint32_t)ceil_div(d.m, p.span);
    cudaStream_t cs = s;  // the combination's stream
    if (combine_stream) {
      if ((e = cudaEventRecord(product_done, s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(combine_stream, product_done, 0)) != cudaSuccess) return e;
      cs = combine_stream;
    }
    if (packed_out) {  // combine and pack in one pass
      uint32_t* stream = reinterpret_cast<uint32_t*>(packed_out);
      const size_t bulk_smem = bulk_smem_bytes(p, d.mw);
      if (bulk_smem <= kPackBulkMaxSmem) {  // persistent CTAs, one bulk copy per block, double-buffered
        const uint64_t per_sm = (227 * 1024) / (bulk_smem + 1024);
        const uint64_t ctas = (uint64_t)(num_sms > 0 ? num_sms : 1) * (per_sm < 8 ? per_sm : 8);
        const unsigned grid = (unsigned)(ctas < nb ? ctas : nb);
        switch (p.levels) {
          case 1: e = launch_combine_pack_bulk<1>(grid, bulk_smem, cs, k, (uint32_t)mwq, log2h, stream, nb, b0, d, dc, err, spec); break;
          case 2: e = launch_combine_pack_bulk<2>(grid, bulk_smem, cs, k, (uint32_t)mwq, log2h, stream, nb, b0, d, dc, err, spec); break;
          case 3: e = launch_combine_pack_bulk<3>(grid, bulk_smem, cs, k, (uint32_t)mwq, log2h, stream, nb, b0, d, dc, err, spec); break;
          default: e = launch_combine_pack_bulk<4>(grid, bulk_smem, cs, k, (uint32_t)mwq, log2h, stream, nb, b0, d, dc, err, spec); break;
        }
        ++*kernels;
        if (e != cudaSuccess) return e;
        continue;
      }
      // one CTA per block, the parity rows staged in chunks
      // staged row words per sub-product: as many as fit beside the output words (multiples of 4)
      const uint32_t room = (kPackSmemWords - (uint32_t)d.mw) / (uint32_t)G;
      const uint32_t cw = (uint32_t)(mwq < (uint64_t)room ? mwq : (uint64_t)room) & ~3u;
      const size_t smem = ((size_t)G * cw + d.mw) * sizeof(uint32_t);
      switch (p.levels) {
        case 1: launch_combine_pack<1>(nb, smem, cs, k, mwq, log2h, cw, stream, b0, d, dc); break;
        case 2: launch_combine_pack<2>(nb, smem, cs, k, mwq, log2h, cw, stream, b0, d, dc); break;
        case 3: launch_combine_pack<3>(nb, smem, cs, k, mwq, log2h, cw, stream, b0, d, dc); break;
        default: launch_combine_pack<4>(nb, smem, cs, k, mwq, log2h, cw, stream, b0, d, dc); break;
      }
      ++*kernels;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      continue;
    }
    const unsigned gc = grid_for(nb * rblocks * hw, num_sms);
    switch (p.levels) {
      case 1: launch_combine<1>(gc, s, k, mwq, log2h, nb, rblocks, d, dc); break;
      case 2: launch_combine<2>(gc, s, k, mwq, log2h, nb, rblocks, d, dc); break;
      case 3: launch_combine<3>(gc, s, k, mwq, log2h, nb, rblocks, d, dc); break;
      default: launch_combine<4>(gc, s, k, mwq, log2h, nb, rblocks, d, dc); break;
    }
    ++*kernels;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_kara_presplit(const DirectArgs& d, const KaraPlan& p, KaraWorkspace& ws, int num_sms,
                                 cudaStream_t s, uint32_t* kernels) {
  ws.xk_ready = false;
  if (p.levels < 1 || p.levels > kMaxLevels) return cudaErrorInvalidValue;
  const uint32_t hw = (uint32_t)(p.h / 32);
  const uint64_t xk_words = p.kq / 32;
  const uint64_t chunk = p.chunk_blocks < d.num_blocks ? p.chunk_blocks : d.num_blocks;
  cudaError_t e = ws.xk.ensure((size_t)p.groups * chunk * xk_words * 4);
  if (e != cudaSuccess) return e;
  const uint32_t kblocks = (uint32_t)(p.kq / p.h);
  if ((e = launch_split_levels(p.levels, d, d, chunk, hw, kblocks, xk_words, ws, num_sms, s)) != cudaSuccess) return e;
  ++*kernels;
  ws.xk_key = split_key(d, d, chunk, xk_words, hw, kblocks, p.levels);
  ws.xk_ready = true;
  return cudaSuccess;
}

}  // namespace qrng
