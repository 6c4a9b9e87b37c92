// Exact convolution route to the Toeplitz hash with a number-theoretic transform.
//
// Same embedding as the paper's FFT route (Sec. III.B Thm. 1-2, Sec. III.D): the Toeplitz part of
// k is the slice c[n_t - 1 + i] of the linear convolution c = a * r, taken from a cyclic
// convolution of length P >= n_t + m - 1 and computed as F^-1(F a . F r). Here F is the discrete
// Fourier transform over the prime field Z_p, p = 15 * 2^27 + 1 (2013265921), whose multiplicative
// group has elements of every order 2^k, k <= 27. Every entry of c is an integer <= n_t < p, so the
// field result IS the integer: there is no rounding to guard, and the transform runs on the integer
// pipes (FP64 is the slowest unit of the GB300).
//
// Arithmetic: elements in [0, p); roots of unity in Montgomery form (w 2^32 mod p) so that one
// Montgomery product w (*) x = w x mod p returns an ordinary residue.
//
// Schedule (four-step, in shared memory): with P = N1 N2, N2 = 2^L (L <= 13), index n = N2 n1 + n2
// and frequency k = k1 + N1 k2,
//   columns: for every n2, the length-N1 transform over n1 (decimation in frequency, so row
//            position rr holds k1 = bitrev(rr)), on tiles of W adjacent columns in shared memory;
//   rows:    for every row, multiply by w^(n2 k1), the length-N2 transform over n2 (position pos
//            holds k2 = bitrev(pos)); then the pointwise product with the seed's spectrum (kept in
//            the same permuted order), the inverse row transform (decimation in time) and
//            w^(-n2 k1), all in one kernel;
//   columns: the inverse length-N1 transforms, back to natural order.
// Three passes over the block's P elements in global memory (plus packing and extraction) instead
// of one pass per radix-4 stage.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qrng_internal.h"

namespace qrng {
namespace {

constexpr uint32_t kP = 2013265921u;        // 15 * 2^27 + 1
constexpr uint32_t kPinvNeg = 2013265919u;  // -p^-1 mod 2^32
constexpr uint32_t kGen = 31u;              // a generator of Z_p^*

// For a, b < p: a + b < 2p < 2^32; min(s, s - p) over unsigned words subtracts p exactly when s >= p
// (otherwise s - p wraps above s). Likewise a - b wraps when a < b, and then d + p is the smaller.
__host__ __device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b) {
  const uint32_t s = a + b;
  const uint32_t t = s - kP;
  return t < s ? t : s;
}

__host__ __device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b) {
  const uint32_t d = a - b;
  const uint32_t t = d + kP;
  return t < d ? t : d;
}

// Montgomery product a b 2^-32 mod p, for a, b < p, in 32-bit words: with q = (a b mod 2^32)(-p^-1),
// the low word of a b + q p is 0 and carries exactly when a b mod 2^32 != 0, so
// (a b + q p) / 2^32 = hi(a b) + hi(q p) + carry < 2p.
__host__ __device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  const uint32_t lo = a * b;
  const uint32_t q = lo * kPinvNeg;
  const uint32_t u = __umulhi(a, b) + __umulhi(q, kP) + (lo != 0u ? 1u : 0u);
#else
  const uint64_t t = (uint64_t)a * b;
  const uint32_t q = (uint32_t)t * kPinvNeg;
  const uint32_t u = (uint32_t)((t + (uint64_t)q * kP) >> 32);
#endif
  const uint32_t r = u - kP;
  return r < u ? r : u;
}

uint32_t pow_mod(uint64_t b, uint64_t e) {
  uint64_t r = 1;
  b %= kP;
  while (e) {
    if (e & 1) r = r * b % kP;
    b = b * b % kP;
    e >>= 1;
  }
  return (uint32_t)r;
}

uint32_t to_mont(uint32_t x) { return (uint32_t)(((uint64_t)x << 32) % kP); }

// tw[q] = omega^q in Montgomery form, q < P/2, omega a primitive P-th root of unity.
__global__ void ntt_twiddle_kernel(uint32_t* __restrict__ tw, uint64_t half, uint32_t omega_m, uint32_t one_m,
                                   uint32_t step_m) {
  // thread j fills tw[j*S .. (j+1)*S) by repeated multiplication from omega^(jS)
  const uint64_t S = 256;
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j * S >= half) return;
  // omega^(jS): square-and-multiply in Montgomery form
  uint32_t base = step_m, acc = one_m;
  uint64_t e = j;
  while (e) {
    if (e & 1) acc = mont_mul(acc, base);
    base = mont_mul(base, base);
    e >>= 1;
  }
  for (uint64_t q = j * S; q < (j + 1) * S && q < half; ++q) {
    tw[q] = acc;
    acc = mont_mul(acc, omega_m);
  }
}

// omega^t in Montgomery form for 0 <= t < P, from the half table (omega^(P/2) = -1).
__device__ __forceinline__ uint32_t ntt_root(const uint32_t* __restrict__ tw, uint64_t half, uint64_t t) {
  return t < half ? __ldg(tw + t) : kP - __ldg(tw + (t - half));
}

// omega^(-t) for 0 <= t < P.
__device__ __forceinline__ uint32_t ntt_iroot(const uint32_t* __restrict__ tw, uint64_t half, uint64_t t) {
  return t == 0 ? __ldg(tw) : ntt_root(tw, half, 2 * half - t);
}

// Transform shape: P = 2^(H+L); column tiles of 2^H rows x 2^logW columns.
struct NttPlan {
  uint32_t logP, L, H, logW;
};

NttPlan ntt_plan(uint32_t logP) {
  NttPlan pl;
  pl.logP = logP;
  // rows of 2^12 entries (2^13 from P = 2^24 on, so that column tiles stay at least 8 columns wide)
  pl.L = logP < 12 ? logP : (logP >= 24 ? 13 : 12);
  pl.H = logP - pl.L;
  const uint32_t want = pl.H >= 14 ? 0u : 14u - pl.H;  // about 16384 elements (64 KB) per column tile
  pl.logW = want < pl.L ? want : pl.L;
  return pl;
}

// Stage roots for the radix-16/4/2 passes, in ordinary form with Shoup quotients: for t = 2^s + j
// (s < 16, j < 2^s), st[t] = w_(2^(s+1))^j, st[E + t] = floor(st[t] 2^32 / p), st[2E + t] and
// st[3E + t] the same for the inverse root (E = kStageEntries). w_(2^(s+1)) = g^((p-1)/2^(s+1)) is the
// same root as w_P^(P/2^(s+1)) for every transform length P; one stage reads contiguous runs.
constexpr uint32_t kStageLog = 16;
constexpr uint32_t kStageEntries = 1u << kStageLog;

__device__ __forceinline__ uint32_t pow_m(uint32_t b, uint32_t e, uint32_t one_m) {
  uint32_t acc = one_m;
  for (; e; e >>= 1) {
    if (e & 1) acc = mont_mul(acc, b);
    b = mont_mul(b, b);
  }
  return acc;
}

// g_m = g and one_m = 1 in Montgomery form (a Montgomery product with 1 returns the ordinary residue).
__global__ void ntt_stage_table_kernel(uint32_t* __restrict__ st, uint32_t g_m, uint32_t one_m) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0 || t >= kStageEntries) return;
  const uint32_t s = 31 - __clz(t), j = t - (1u << s);
  const uint32_t e = (kP - 1) >> (s + 1);
  const uint32_t w = mont_mul(pow_m(pow_m(g_m, e, one_m), j, one_m), 1u);
  const uint32_t wi = mont_mul(pow_m(pow_m(g_m, (kP - 1) - e, one_m), j, one_m), 1u);
  st[t] = w;
  st[kStageEntries + t] = (uint32_t)(((uint64_t)w << 32) / kP);
  st[2 * kStageEntries + t] = wi;
  st[3 * kStageEntries + t] = (uint32_t)(((uint64_t)wi << 32) / kP);
}

// x w mod p for a constant w < p with its Shoup quotient wq = floor(w 2^32 / p): q = floor(x wq / 2^32)
// is floor(x w / p) or one less, so x w - q p (exact in 32 bits) lies in [0, 2p).
__device__ __forceinline__ uint32_t shoup_mul(uint32_t x, uint32_t w, uint32_t wq) {
  const uint32_t r = x * w - __umulhi(x, wq) * kP;
  const uint32_t t = r - kP;
  return t < r ? t : r;
}

// Butterflies of one stage: forward (decimation in frequency) a' = a + b, b' = (a - b) w; inverse
// (decimation in time) t = b w^-1, a' = a + t, b' = a - t. The root index k selects w_(2^(s+1))^j.
template <bool kInverse>
__device__ __forceinline__ void bfly(uint32_t& a, uint32_t& b, const uint32_t* __restrict__ st, uint32_t k) {
  if (!kInverse) {
    const uint32_t w = __ldg(st + k), wq = __ldg(st + kStageEntries + k);
    const uint32_t s0 = add_mod(a, b);
    b = shoup_mul(sub_mod(a, b), w, wq);
    a = s0;
  } else {
    const uint32_t w = __ldg(st + 2 * kStageEntries + k), wq = __ldg(st + 3 * kStageEntries + k);
    const uint32_t t = shoup_mul(b, w, wq);
    b = sub_mod(a, t);
    a = add_mod(a, t);
  }
}

// One pass of R = 2^G stages s, s-1, .., s-G+1 on R elements x[q] = X[i0 + q h], h = 2^(s-G+1),
// j = i0 mod h: forward from the widest span down, inverse from the narrowest up. The stage of span
// 2^t pairs q with q + 2^(t-s+G-1) and uses root index 2^t + j + (q mod 2^(t-s+G-1)) h.
template <bool kInverse, int G>
__device__ __forceinline__ void radix_pass(uint32_t (&x)[1 << G], const uint32_t* __restrict__ st, uint32_t s,
                                           uint32_t j) {
  constexpr int R = 1 << G;
  const uint32_t h = 1u << (s - G + 1);
#pragma unroll
  for (int gi = 0; gi < G; ++gi) {
    const int g = kInverse ? gi : G - 1 - gi;  // local span 2^g
    const uint32_t base = (1u << (s - G + 1 + g)) + j;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (q & (1 << g)) continue;
      bfly<kInverse>(x[q], x[q + (1 << g)], st, base + (uint32_t)(q & ((1 << g) - 1)) * h);
    }
  }
}

// In-place length-2^K transforms of `cols` interleaved sequences in shared memory (element r of
// column c at x[(r << logC) | c]): forward = decimation in frequency (natural in, bit-reversed out),
// inverse = decimation in time with inverse roots (bit-reversed in, natural out). The stages are
// grouped from the widest span down into radix-16 passes, then one radix-4 and one radix-2 pass as
// needed; the inverse runs the same groups in the opposite order.
// Shared-memory position of element t in a padded row (one spare word after every 16): the
// elements 16 apart that the last radix-16 pass gives each thread then fall in distinct banks.
__device__ __forceinline__ uint32_t pad16(uint32_t t) { return t + (t >> 4); }

template <bool kInverse, int G, bool kPad>
__device__ __forceinline__ void smem_pass(uint32_t* __restrict__ x, uint32_t K, uint32_t logC, uint32_t s,
                                          const uint32_t* __restrict__ st) {
  constexpr int R = 1 << G;
  const uint32_t C = 1u << logC;
  const uint32_t lh = s - G + 1;  // log2 h
  for (uint32_t u = threadIdx.x; u < (1u << (K - G + logC)); u += blockDim.x) {
    const uint32_t c = u & (C - 1), v = u >> logC;
    const uint32_t j = v & ((1u << lh) - 1);
    const uint32_t r0 = ((v >> lh) << (s + 1)) | j;
    uint32_t a[R];
    if (kPad) {  // rows only (logC = 0)
#pragma unroll
      for (int q = 0; q < R; ++q) a[q] = x[pad16(r0 + ((uint32_t)q << lh))];
      radix_pass<kInverse, G>(a, st, s, j);
#pragma unroll
      for (int q = 0; q < R; ++q) x[pad16(r0 + ((uint32_t)q << lh))] = a[q];
    } else {
      uint32_t* p0 = x + ((r0 << logC) | c);
      const uint32_t dh = 1u << (lh + logC);
#pragma unroll
      for (int q = 0; q < R; ++q) a[q] = p0[q * dh];
      radix_pass<kInverse, G>(a, st, s, j);
#pragma unroll
      for (int q = 0; q < R; ++q) p0[q * dh] = a[q];
    }
  }
  __syncthreads();
}

template <bool kInverse, bool kPad = false>
__device__ __forceinline__ void smem_transform(uint32_t* __restrict__ x, uint32_t K, uint32_t logC,
                                               const uint32_t* __restrict__ st) {
  const uint32_t n16 = K / 4, rem = K % 4;  // radix-16 passes, then radix-4 (rem >= 2), radix-2 (odd)
  const uint32_t npass = n16 + (rem >= 2 ? 1u : 0u) + (rem & 1u);
  for (uint32_t it = 0; it < npass; ++it) {
    const uint32_t p = kInverse ? npass - 1 - it : it;  // pass p covers the p-th group from the top
    if (p < n16) {
      smem_pass<kInverse, 4, kPad>(x, K, logC, K - 1 - 4 * p, st);
    } else if (p == n16 && rem >= 2) {
      smem_pass<kInverse, 2, kPad>(x, K, logC, K - 1 - 4 * n16, st);
    } else {
      smem_pass<kInverse, 1, kPad>(x, K, logC, 0, st);
    }
  }
}

__device__ __forceinline__ uint32_t bit_at(const uint8_t* __restrict__ p, uint64_t bit) {
  return (p[bit >> 3] >> (bit & 7)) & 1u;
}

// Column I/O: entries in z both ways; raw bits in (forward: the block's bits become the entries,
// no packed copy); parity bits out (inverse: bit i of the block's parity array = entry i mod 2,
// stored a byte per 8 columns of a row, instead of the entries).
enum { kColsZ = 0, kColsFromBits = 1, kColsToParity = 2 };

struct ColsIO {
  const uint32_t* raw;   // kColsFromBits: block b's bits at raw + b stride (words), first n_t of them
  uint64_t stride;
  uint64_t n_t;
  uint64_t b0;           // block of entry 0
  uint64_t num_blocks;
  const BatchReq* reqs;  // kColsFromBits for uneven requests: entry 2r = request r's seed bits (L_t of
                         // them), entry 2r+1 its raw bits (n_t from raw_bit_off); replaces raw..num_blocks
  uint8_t* parity;       // kColsToParity: P / 8 bytes per launched entry
};

// Length-2^H transforms down the columns of entries ent_off, ent_off + ent_stride, ... (row stride
// 2^L); one CTA per tile of 2^H rows x 2^logW adjacent columns.
template <bool kInverse, int kIO>
__global__ void __launch_bounds__(512) ntt_cols_kernel(uint32_t* __restrict__ z, const uint32_t* __restrict__ st,
                                                       NttPlan pl, uint64_t ent_stride, uint64_t ent_off, ColsIO io) {
  extern __shared__ uint32_t col_sm[];
  const uint32_t tiles_per_ent = 1u << (pl.L - pl.logW);
  const uint64_t ent = (uint64_t)blockIdx.x >> (pl.L - pl.logW);
  const uint32_t c0 = (blockIdx.x & (tiles_per_ent - 1)) << pl.logW;
  const uint64_t eidx = ent * ent_stride + ent_off;
  uint32_t* zb = z + (eidx << pl.logP) + c0;
  const uint32_t W = 1u << pl.logW, n = 1u << (pl.H + pl.logW);
  if (kIO == kColsFromBits && io.reqs) {
    const BatchReq& q = io.reqs[eidx >> 1];
    const uint8_t* src = (eidx & 1) ? q.raw : q.seed;
    const uint64_t off = (eidx & 1) ? q.raw_bit_off : 0, len = (eidx & 1) ? q.n_t : q.L_t;
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
      const uint64_t i = ((uint64_t)(e >> pl.logW) << pl.L) + c0 + (e & (W - 1));
      col_sm[e] = i < len ? bit_at(src, off + i) : 0u;
    }
  } else if (kIO == kColsFromBits) {
    const uint64_t b = io.b0 + eidx;
    const uint32_t* rb = io.raw + b * io.stride;
    const bool live = b < io.num_blocks;
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
      const uint64_t i = ((uint64_t)(e >> pl.logW) << pl.L) + c0 + (e & (W - 1));
      col_sm[e] = (live && i < io.n_t) ? ((__ldg(rb + (i >> 5)) >> (i & 31)) & 1u) : 0u;
    }
  } else {
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x)
      col_sm[e] = zb[((uint64_t)(e >> pl.logW) << pl.L) + (e & (W - 1))];
  }
  __syncthreads();
  smem_transform<kInverse>(col_sm, pl.H, pl.logW, st);
  if (kIO == kColsToParity) {
    // the tile's W columns of row r are entries (r << L) + c0 .. + W - 1. A warp takes 32 consecutive
    // tile elements (rows of W >= 8 columns, in order) and gathers their parities with one ballot; the
    // lane at the start of each row's run (or of each 32 columns) stores that run's bits.
    uint8_t* pb = io.parity + (ent << (pl.logP - 3)) + (c0 >> 3);
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {  // n is a multiple of 32 when logW >= 3
      const uint32_t bits = __ballot_sync(0xffffffffu, col_sm[e] & 1u);
      const uint32_t r = e >> pl.logW, c = e & (W - 1);
      uint8_t* dst = pb + ((uint64_t)r << (pl.L - 3)) + (c >> 3);
      if (W >= 32) {
        if (lane == 0) *reinterpret_cast<uint32_t*>(dst) = bits;
      } else if (c == 0) {
        const uint32_t field = bits >> lane;  // this row's W bits
        if (W == 16) *reinterpret_cast<uint16_t*>(dst) = (uint16_t)field;
        else *dst = (uint8_t)field;
      }
    }
  } else {
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x)
      zb[((uint64_t)(e >> pl.logW) << pl.L) + (e & (W - 1))] = col_sm[e];
  }
}

// Multiplies row element n2 (padded layout) by w_P^(+-n2 k1): the power is built from two tables of
// the row, w^(k1 b) (b < 2^lob) and w^(2^lob k1 a), one Montgomery product apart.
__device__ __forceinline__ void ntt_row_twiddle(uint32_t* __restrict__ x, const uint32_t* __restrict__ tlo,
                                                const uint32_t* __restrict__ thi, uint32_t L, uint32_t lob) {
  for (uint32_t n2 = threadIdx.x; n2 < (1u << L); n2 += blockDim.x) {
    const uint32_t w = mont_mul(thi[n2 >> lob], tlo[n2 & ((1u << lob) - 1)]);
    x[pad16(n2)] = mont_mul(w, x[pad16(n2)]);
  }
  __syncthreads();
}

enum { kRowsForward = 0, kRowsConvolve = 1, kRowsPairs = 2 };

// Rows of entries (one CTA per row, 2^L elements):
//   kRowsForward:  twiddle + forward row transform (finishes a forward transform);
//   kRowsConvolve: the same, times the spectrum spec (same permuted order), inverse row transform,
//                  inverse twiddle;
//   kRowsPairs:    entries 2r and 2r+1 (a request's seed and raw bits) both forward, their product
//                  (*) factor, inverse row transform and twiddle, written to entry 2r+1.
template <int kMode>
__global__ void __launch_bounds__(256) ntt_rows_kernel(uint32_t* __restrict__ z, const uint32_t* __restrict__ spec,
                                                       const uint32_t* __restrict__ tw,
                                                       const uint32_t* __restrict__ st, NttPlan pl,
                                                       uint32_t factor_m) {
  extern __shared__ uint32_t row_sm[];
  const uint32_t Lr = 1u << pl.L;
  const uint32_t Lp = Lr + (Lr >> 4);  // padded row
  const uint32_t lob = pl.L < 6 ? pl.L : 6;
  uint32_t* tlo = row_sm + (kMode == kRowsPairs ? 2 : 1) * Lp;  // w^(+-k1 b), b < 2^lob
  uint32_t* thi = tlo + (1u << lob);                            // w^(+-2^lob k1 a)
  uint32_t* row2 = row_sm + Lp;                                 // kRowsPairs: the raw entry's row
  const uint64_t P = 1ull << pl.logP, half = P >> 1;
  const uint64_t ent = (uint64_t)blockIdx.x >> pl.H;
  const uint32_t rr = (uint32_t)(blockIdx.x & ((1u << pl.H) - 1));
  const uint32_t k1 = pl.H ? (__brev(rr) >> (32 - pl.H)) : 0u;
  const uint64_t e0 = (kMode == kRowsPairs) ? 2 * ent : ent;
  uint32_t* x = z + (e0 << pl.logP) + ((uint64_t)rr << pl.L);
  uint32_t* x2 = x + P;  // kRowsPairs: the raw entry
  for (uint32_t t = threadIdx.x; t < Lr; t += blockDim.x) {
    row_sm[pad16(t)] = x[t];
    if (kMode == kRowsPairs) row2[pad16(t)] = x2[t];
  }
  if (pl.H) {
    for (uint32_t t = threadIdx.x; t < (1u << lob) + (Lr >> lob); t += blockDim.x) {
      if (t < (1u << lob)) tlo[t] = ntt_root(tw, half, ((uint64_t)k1 * t) & (P - 1));
      else thi[t - (1u << lob)] = ntt_root(tw, half, (((uint64_t)k1 * (t - (1u << lob))) << lob) & (P - 1));
    }
  }
  __syncthreads();
  if (pl.H) {
    ntt_row_twiddle(row_sm, tlo, thi, pl.L, lob);
    if (kMode == kRowsPairs) ntt_row_twiddle(row2, tlo, thi, pl.L, lob);
  }
  smem_transform<false, true>(row_sm, pl.L, 0, st);
  if (kMode == kRowsPairs) smem_transform<false, true>(row2, pl.L, 0, st);
  if (kMode == kRowsForward) {
    for (uint32_t t = threadIdx.x; t < Lr; t += blockDim.x) x[t] = row_sm[pad16(t)];
    return;
  }
  const uint32_t* sp = spec + ((uint64_t)rr << pl.L);
  for (uint32_t t = threadIdx.x; t < Lr; t += blockDim.x) {
    const uint32_t pt = pad16(t);
    if (kMode == kRowsConvolve) row_sm[pt] = mont_mul(row_sm[pt], __ldg(sp + t));
    else row_sm[pt] = mont_mul(mont_mul(row_sm[pt], row2[pt]), factor_m);
  }
  if (pl.H) {  // inverse twiddle tables (the forward ones were last read before the stage barriers)
    for (uint32_t t = threadIdx.x; t < (1u << lob) + (Lr >> lob); t += blockDim.x) {
      if (t < (1u << lob)) tlo[t] = ntt_iroot(tw, half, ((uint64_t)k1 * t) & (P - 1));
      else thi[t - (1u << lob)] = ntt_iroot(tw, half, (((uint64_t)k1 * (t - (1u << lob))) << lob) & (P - 1));
    }
  }
  __syncthreads();
  smem_transform<true, true>(row_sm, pl.L, 0, st);
  if (pl.H) ntt_row_twiddle(row_sm, tlo, thi, pl.L, lob);
  uint32_t* dst = (kMode == kRowsPairs) ? x2 : x;
  for (uint32_t t = threadIdx.x; t < Lr; t += blockDim.x) dst[t] = row_sm[pad16(t)];
}

__global__ void ntt_seed_kernel(const uint8_t* __restrict__ seed, uint64_t L, uint32_t* __restrict__ z, uint64_t P) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  z[t] = t < L ? (uint32_t)((seed[t >> 3] >> (t & 7)) & 1u) : 0u;
}

// Seed spectrum A -> A P^-1 2^32 mod p, so that one Montgomery product with a block's spectrum
// yields (A . R) / P, the spectrum of the convolution with the inverse transform's 1/P folded in.
__global__ void ntt_scale_kernel(uint32_t* __restrict__ z, uint64_t P, uint32_t factor_m) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  z[t] = mont_mul(z[t], factor_m);
}

__global__ void ntt_pack_kernel(const uint32_t* __restrict__ raw, uint64_t stride, uint64_t n_t, uint64_t num_blocks,
                                uint64_t b0, uint64_t nb, uint32_t* __restrict__ z, uint32_t logP) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (nb << logP)) return;
  const uint64_t bl = idx >> logP, t = idx & ((1ull << logP) - 1);
  const uint64_t b = b0 + bl;
  z[idx] = (t < n_t && b < num_blocks) ? ((raw[b * stride + (t >> 5)] >> (t & 31)) & 1u) : 0u;
}

// Output word w of block b0+bl from the block's parity bits (bit i = entry i mod 2 of the inverse
// transform): bits n_t - 1 + 32 w .. + 31, one funnel shift of two words; identity bits for the
// modified form.
__global__ void ntt_parity_extract_kernel(const uint32_t* __restrict__ par, uint32_t logP, uint64_t n_t, uint64_t m,
                                          uint64_t mw, const uint32_t* __restrict__ raw, uint64_t stride,
                                          int modified, uint64_t id_off, uint64_t num_blocks, uint64_t b0,
                                          uint64_t nb, uint32_t* __restrict__ out, uint64_t out_stride) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nb * mw) return;
  const uint64_t bl = g / mw, w = g - bl * mw;
  const uint64_t b = b0 + bl;
  if (b >= num_blocks) return;
  const uint64_t words = 1ull << (logP - 5);
  const uint32_t* pb = par + bl * words;
  const uint64_t pos = n_t - 1 + 32 * w;
  const uint64_t q = pos >> 5;
  const uint32_t sh = (uint32_t)(pos & 31);
  const uint32_t lo = __ldg(pb + q);
  const uint32_t hi = (sh && q + 1 < words) ? __ldg(pb + q + 1) : 0u;
  uint32_t word = __funnelshift_r(lo, hi, sh);
  const uint64_t rem = m - 32 * w;
  const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
  word &= omask;
  if (modified) {
    const uint32_t* rr = raw + b * stride;
    const uint64_t ip = id_off + 32 * w;
    const uint64_t rq = ip >> 5;
    const uint32_t rs = (uint32_t)(ip & 31);
    const uint32_t rlo = __ldg(rr + rq);
    const uint32_t rhi = (rs && rq + 1 < stride) ? __ldg(rr + rq + 1) : 0u;
    word ^= __funnelshift_r(rlo, rhi, rs) & omask;
  }
  out[b * out_stride + w] = word;
}

// Output word w of block b0+bl: parities of c[n_t - 1 + i] (exact integers), identity bits.
__global__ void ntt_extract_kernel(const uint32_t* __restrict__ z, uint64_t P, uint64_t n_t, uint64_t m, uint64_t mw,
                                   const uint32_t* __restrict__ raw, uint64_t stride, int modified, uint64_t id_off,
                                   uint64_t num_blocks, uint64_t b0, uint64_t nb, uint32_t* __restrict__ out,
                                   uint64_t out_stride) {
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (gw >= nb * mw) return;
  const uint64_t bl = gw / mw, w = gw - bl * mw;
  const uint64_t b = b0 + bl;
  const uint64_t i = 32 * w + lane;
  const uint32_t bit = (i < m) ? (z[bl * P + n_t - 1 + i] & 1u) : 0u;
  uint32_t word = __ballot_sync(0xffffffffu, bit);
  if (lane == 0 && b < num_blocks) {
    const uint64_t rem = m - 32 * w;
    const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    word &= omask;
    if (modified) {
      const uint32_t* rr = raw + b * stride;
      const uint64_t pos = id_off + 32 * w;
      const uint64_t rq = pos >> 5;
      const uint32_t rs = (uint32_t)(pos & 31);
      const uint32_t lo = rr[rq];
      const uint32_t hi = (rs && rq + 1 < stride) ? rr[rq + 1] : 0u;
      word ^= __funnelshift_r(lo, hi, rs) & omask;
    }
    out[b * out_stride + w] = word;
  }
}

inline unsigned grid_for(uint64_t total, int threads) { return (unsigned)ceil_div(total, (uint64_t)threads); }

constexpr int kNttThreads = 512;     // column tiles
constexpr int kNttRowThreads = 256;  // rows: 2^12 elements, 256 radix-16 items

// Columns forward/inverse over the entries ent_off, ent_off + ent_stride, ... (num_ent of them).
template <bool kInverse, int kIO>
cudaError_t ntt_columns(uint32_t* z, const uint32_t* st, const NttPlan& pl, uint64_t num_ent, uint64_t ent_stride,
                        uint64_t ent_off, const ColsIO& io, cudaStream_t s, uint32_t* kernels) {
  if (pl.H == 0) return cudaSuccess;
  const size_t smem = ((size_t)1 << (pl.H + pl.logW)) * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(ntt_cols_kernel<kInverse, kIO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const uint64_t tiles = num_ent << (pl.L - pl.logW);
  ntt_cols_kernel<kInverse, kIO><<<(unsigned)tiles, kNttThreads, smem, s>>>(z, st, pl, ent_stride, ent_off, io);
  ++*kernels;
  return cudaGetLastError();
}

template <int kMode>
cudaError_t ntt_rows(uint32_t* z, const uint32_t* spec, const uint32_t* tw, const uint32_t* st, const NttPlan& pl,
                     uint64_t num_rows_ent, uint32_t factor_m, cudaStream_t s, uint32_t* kernels) {
  const uint32_t lob = pl.L < 6 ? pl.L : 6;
  const size_t padded = (1u << pl.L) + ((1u << pl.L) >> 4);
  const size_t smem =
      ((size_t)(kMode == kRowsPairs ? 2 : 1) * padded + (1u << lob) + (1u << (pl.L - lob))) * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(ntt_rows_kernel<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const uint64_t ctas = num_rows_ent << pl.H;
  ntt_rows_kernel<kMode><<<(unsigned)ctas, kNttRowThreads, smem, s>>>(z, spec, tw, st, pl, factor_m);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t ensure_twiddles(FftWorkspace& ws, uint64_t P, cudaStream_t s, uint32_t* kernels) {
  cudaError_t e;
  if (!ws.ntt_stage.p) {
    if ((e = ws.ntt_stage.ensure(4 * kStageEntries * sizeof(uint32_t))) != cudaSuccess) return e;
    ntt_stage_table_kernel<<<kStageEntries / 256, 256, 0, s>>>(ws.ntt_stage.as<uint32_t>(), to_mont(kGen),
                                                                 to_mont(1));
    ++*kernels;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ws.ntt_P == P) return cudaSuccess;
  if ((e = ws.ntt_tw.ensure((P / 2) * sizeof(uint32_t))) != cudaSuccess) return e;
  const uint32_t omega = pow_mod(kGen, (kP - 1) / P);  // primitive P-th root of unity
  ntt_twiddle_kernel<<<grid_for(ceil_div(P / 2, 256), 128), 128, 0, s>>>(ws.ntt_tw.as<uint32_t>(), P / 2,
                                                                        to_mont(omega), to_mont(1),
                                                                        to_mont(pow_mod(omega, 256)));
  ++*kernels;
  ws.ntt_P = P;
  return cudaGetLastError();
}

// ---- uneven batches: requests with their own seeds, grouped by transform length P ----


// Entry 2r of the chunk holds request r's seed bits [0, L_t), entry 2r+1 its raw bits [0, n_t),
// both zero-padded to P.
__global__ void ntt_batch_inputs_kernel(const BatchReq* __restrict__ reqs, uint64_t nr, uint32_t* __restrict__ z,
                                        uint32_t logP) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ((2 * nr) << logP)) return;
  const uint64_t e = idx >> logP, t = idx & ((1ull << logP) - 1);
  const BatchReq& q = reqs[e >> 1];
  uint32_t v = 0;
  if (e & 1) {
    if (t < q.n_t) v = bit_at(q.raw, q.raw_bit_off + t);
  } else {
    if (t < q.L_t) v = bit_at(q.seed, t);
  }
  z[idx] = v;
}

// Output word w of chunk request r (one warp per word): parities of c[n_t - 1 + i] (entry 2r+1),
// identity bits.
__global__ void ntt_batch_extract_kernel(const BatchReq* __restrict__ reqs, uint64_t nr, uint64_t max_mw,
                                         const uint32_t* __restrict__ c, uint64_t P, uint32_t* __restrict__ out_stage) {
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (gw >= nr * max_mw) return;
  const uint64_t r = gw / max_mw, w = gw - r * max_mw;
  const BatchReq& q = reqs[r];
  if (w >= q.mw) return;  // warp-uniform
  const uint64_t i = 32 * w + lane;
  const uint32_t bit = (i < q.m) ? (c[(2 * r + 1) * P + q.n_t - 1 + i] & 1u) : 0u;
  uint32_t word = __ballot_sync(0xffffffffu, bit);
  const uint32_t ident = (q.form == QRNG_FORM_MODIFIED && i < q.m) ? bit_at(q.raw, q.raw_bit_off + q.id_off + i) : 0u;
  word ^= __ballot_sync(0xffffffffu, ident);
  if (lane == 0) out_stage[q.out_stage_off + w] = word;
}

// nbits <= 32 bits of a byte buffer from bit `bit` on (LSB-first), reading only the bytes they span.
__device__ __forceinline__ uint32_t bits_at(const uint8_t* __restrict__ p, uint64_t bit, uint32_t nbits) {
  const uint8_t* b = p + (bit >> 3);
  const uint32_t sh = (uint32_t)(bit & 7);
  const uint32_t nbytes = (sh + nbits + 7) >> 3;  // <= 5
  uint64_t v = 0;
  for (uint32_t k = 0; k < nbytes; ++k) v |= (uint64_t)b[k] << (8 * k);
  v >>= sh;
  return nbits >= 32 ? (uint32_t)v : (uint32_t)v & ((1u << nbits) - 1u);
}

// Output word w of chunk request r from its parity bits (one thread per word): bits n_t - 1 + 32 w
// .. + 31 of the product's inverse transform, identity bits for the modified form.
__global__ void ntt_batch_parity_extract_kernel(const BatchReq* __restrict__ reqs, uint64_t nr, uint64_t max_mw,
                                                const uint32_t* __restrict__ par, uint32_t logP,
                                                uint32_t* __restrict__ out_stage) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nr * max_mw) return;
  const uint64_t r = g / max_mw, w = g - r * max_mw;
  const BatchReq& q = reqs[r];
  if (w >= q.mw) return;
  const uint64_t words = 1ull << (logP - 5);
  const uint32_t* pb = par + r * words;
  const uint64_t pos = q.n_t - 1 + 32 * w;
  const uint64_t qw = pos >> 5;
  const uint32_t sh = (uint32_t)(pos & 31);
  const uint32_t lo = __ldg(pb + qw);
  const uint32_t hi = (sh && qw + 1 < words) ? __ldg(pb + qw + 1) : 0u;
  const uint64_t rem = q.m - 32 * w;
  const uint32_t nb = rem >= 32 ? 32u : (uint32_t)rem;
  const uint32_t omask = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
  uint32_t word = __funnelshift_r(lo, hi, sh) & omask;
  if (q.form == QRNG_FORM_MODIFIED) word ^= bits_at(q.raw, q.raw_bit_off + q.id_off + 32 * w, nb);
  out_stage[q.out_stage_off + w] = word;
}

}  // namespace

cudaError_t ntt_prepare(FftWorkspace& ws, uint64_t P, cudaStream_t s, uint32_t* kernels) {
  return ensure_twiddles(ws, P, s, kernels);
}

cudaError_t launch_ntt_batch(const BatchReq* reqs_dev, uint64_t nr, uint64_t P,
                             uint64_t max_mw, FftWorkspace& ws, uint32_t* out_stage, cudaStream_t s,
                             uint32_t* kernels) {
  uint32_t logP = 0;
  while ((1ull << logP) < P) ++logP;
  const NttPlan pl = ntt_plan(logP);
  cudaError_t e;
  if ((e = ensure_twiddles(ws, P, s, kernels)) != cudaSuccess) return e;
  if ((e = ws.buf0.ensure(2 * nr * P * sizeof(uint32_t))) != cudaSuccess) return e;
  uint32_t* z = ws.buf0.as<uint32_t>();
  const uint32_t* tw = ws.ntt_tw.as<uint32_t>();
  const uint32_t* st = ws.ntt_stage.as<uint32_t>();
  const uint32_t factor_m = to_mont(to_mont(pow_mod(P % kP, kP - 2)));
  if (pl.H > 0 && pl.logW >= 3) {
    // every request's seed and raw bits straight into the forward columns; parity bits out of the
    // inverse columns of the products (entries 2r+1)
    if ((e = ws.buf1.ensure(nr * (P / 8))) != cudaSuccess) return e;
    ColsIO in{};
    in.reqs = reqs_dev;
    if ((e = ntt_columns<false, kColsFromBits>(z, st, pl, 2 * nr, 1, 0, in, s, kernels)) != cudaSuccess) return e;
    if ((e = ntt_rows<kRowsPairs>(z, nullptr, tw, st, pl, nr, factor_m, s, kernels)) != cudaSuccess) return e;
    ColsIO outp{};
    outp.parity = ws.buf1.as<uint8_t>();
    if ((e = ntt_columns<true, kColsToParity>(z, st, pl, nr, 2, 1, outp, s, kernels)) != cudaSuccess) return e;
    ntt_batch_parity_extract_kernel<<<grid_for(nr * max_mw, 256), 256, 0, s>>>(reqs_dev, nr, max_mw,
                                                                               ws.buf1.as<uint32_t>(), logP,
                                                                               out_stage);
    ++*kernels;
    return cudaGetLastError();
  }
  ntt_batch_inputs_kernel<<<grid_for(2 * nr * P, 256), 256, 0, s>>>(reqs_dev, nr, z, logP);
  ++*kernels;
  // both entries of every request forward, then per row: the product (*) P^-1 2^64, inverse row
  // transform into entry 2r+1, then the inverse columns of the odd entries
  const ColsIO none{};
  if ((e = ntt_columns<false, kColsZ>(z, st, pl, 2 * nr, 1, 0, none, s, kernels)) != cudaSuccess) return e;
  if ((e = ntt_rows<kRowsPairs>(z, nullptr, tw, st, pl, nr, factor_m, s, kernels)) != cudaSuccess) return e;
  if ((e = ntt_columns<true, kColsZ>(z, st, pl, nr, 2, 1, none, s, kernels)) != cudaSuccess) return e;
  ntt_batch_extract_kernel<<<grid_for(nr * max_mw * 32, 256), 256, 0, s>>>(reqs_dev, nr, max_mw, z, P, out_stage);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_ntt(const DirectArgs& d, const uint8_t* seed, uint64_t L_t, FftWorkspace& ws, cudaStream_t s,
                       uint32_t* kernels) {
  const uint64_t n_t = d.n_t;
  const uint64_t P = fft64_length(n_t, d.m);
  if (P > (1ull << 27)) return cudaErrorInvalidValue;
  uint32_t logP = 0;
  while ((1ull << logP) < P) ++logP;
  const NttPlan pl = ntt_plan(logP);
  cudaError_t e;
  if ((e = ensure_twiddles(ws, P, s, kernels)) != cudaSuccess) return e;
  uint64_t chunk = kFftWorkspaceBytes / (P * sizeof(uint32_t));
  if (chunk < 1) chunk = 1;
  if (chunk > d.num_blocks) chunk = d.num_blocks;
  if ((e = ws.buf0.ensure(chunk * P * sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = ws.spec.ensure(P * sizeof(uint32_t))) != cudaSuccess) return e;
  uint32_t* z = ws.buf0.as<uint32_t>();
  uint32_t* spec = ws.spec.as<uint32_t>();
  const uint32_t* tw = ws.ntt_tw.as<uint32_t>();

  // seed spectrum (permuted order of the row transforms), scaled by P^-1, in Montgomery form
  ntt_seed_kernel<<<grid_for(P, 256), 256, 0, s>>>(seed, L_t, spec, P);
  ++*kernels;
  const uint32_t* st = ws.ntt_stage.as<uint32_t>();
  const ColsIO none{};
  if ((e = ntt_columns<false, kColsZ>(spec, st, pl, 1, 1, 0, none, s, kernels)) != cudaSuccess) return e;
  if ((e = ntt_rows<kRowsForward>(spec, nullptr, tw, st, pl, 1, 0, s, kernels)) != cudaSuccess) return e;
  const uint32_t pinv = pow_mod(P % kP, kP - 2);
  const uint32_t factor_m = to_mont(to_mont(pinv));  // P^-1 2^64 mod p: one product leaves P^-1 2^32
  ntt_scale_kernel<<<grid_for(P, 256), 256, 0, s>>>(spec, P, factor_m);
  ++*kernels;

  // the block's raw bits go straight into the forward columns and the inverse columns write packed
  // parity bits, when the column tiles are at least a byte wide
  const bool fused = pl.H > 0 && pl.logW >= 3;
  if (fused && (e = ws.buf1.ensure(chunk * (P / 8))) != cudaSuccess) return e;
  for (uint64_t bb = 0; bb < d.num_blocks; bb += chunk) {
    const uint64_t nb = (d.num_blocks - bb) < chunk ? (d.num_blocks - bb) : chunk;
    if (fused) {
      ColsIO in{};
      in.raw = d.raw;
      in.stride = d.raw_stride;
      in.n_t = n_t;
      in.b0 = bb;
      in.num_blocks = d.num_blocks;
      if ((e = ntt_columns<false, kColsFromBits>(z, st, pl, nb, 1, 0, in, s, kernels)) != cudaSuccess) return e;
      if ((e = ntt_rows<kRowsConvolve>(z, spec, tw, st, pl, nb, 0, s, kernels)) != cudaSuccess) return e;
      ColsIO outp{};
      outp.parity = ws.buf1.as<uint8_t>();
      if ((e = ntt_columns<true, kColsToParity>(z, st, pl, nb, 1, 0, outp, s, kernels)) != cudaSuccess) return e;
      ntt_parity_extract_kernel<<<grid_for(nb * d.mw, 256), 256, 0, s>>>(
          ws.buf1.as<uint32_t>(), logP, n_t, d.m, d.mw, d.raw, d.raw_stride, d.modified, d.id_off, d.num_blocks, bb,
          nb, d.out, d.out_stride);
      ++*kernels;
      continue;
    }
    ntt_pack_kernel<<<grid_for(nb * P, 256), 256, 0, s>>>(d.raw, d.raw_stride, n_t, d.num_blocks, bb, nb, z, logP);
    ++*kernels;
    if ((e = ntt_columns<false, kColsZ>(z, st, pl, nb, 1, 0, none, s, kernels)) != cudaSuccess) return e;
    if ((e = ntt_rows<kRowsConvolve>(z, spec, tw, st, pl, nb, 0, s, kernels)) != cudaSuccess) return e;
    if ((e = ntt_columns<true, kColsZ>(z, st, pl, nb, 1, 0, none, s, kernels)) != cudaSuccess) return e;
    ntt_extract_kernel<<<grid_for(nb * d.mw * 32, 256), 256, 0, s>>>(z, P, n_t, d.m, d.mw, d.raw, d.raw_stride,
                                                                     d.modified, d.id_off, d.num_blocks, bb, nb,
                                                                     d.out, d.out_stride);
    ++*kernels;
  }
  return cudaGetLastError();
}

}  // namespace qrng
