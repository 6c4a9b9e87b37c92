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
// Arithmetic: elements in [0, p); twiddles in Montgomery form (w 2^32 mod p) so that one Montgomery
// product w (*) x = w x mod p returns ordinary residues. Radix-2 Stockham passes over global
// memory, one launch per pass over a chunk of blocks (the same schedule as the FP64 route, with
// 4-byte elements instead of 16).
#include <cuda_runtime.h>
#include <stdint.h>

#include "qrng_internal.h"

namespace qrng {
namespace {

constexpr uint32_t kP = 2013265921u;        // 15 * 2^27 + 1
constexpr uint32_t kPinvNeg = 2013265919u;  // -p^-1 mod 2^32
constexpr uint32_t kGen = 31u;              // a generator of Z_p^*

__host__ __device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b) {
  const uint32_t s = a + b;  // < 2p < 2^32
  return s >= kP ? s - kP : s;
}

__host__ __device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b) { return a >= b ? a - b : a + kP - b; }

// Montgomery product a b 2^-32 mod p, for a, b < p.
__host__ __device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b) {
  const uint64_t t = (uint64_t)a * b;
  const uint32_t q = (uint32_t)t * kPinvNeg;
  const uint64_t u = (t + (uint64_t)q * kP) >> 32;  // < 2p
  return u >= kP ? (uint32_t)(u - kP) : (uint32_t)u;
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

// One radix-2 Stockham pass (see the FP64 route): y[g 2L + k] = x[j] + w x[j+P/2],
// y[g 2L + k + L] = x[j] - w x[j+P/2], w = omega^(+-k P/(2L)); the inverse uses
// omega^-q = -omega^(P/2 - q).
__global__ void ntt_pass_kernel(const uint32_t* __restrict__ x, uint32_t* __restrict__ y,
                                const uint32_t* __restrict__ tw, uint64_t P, uint32_t logL, uint32_t logP, int inverse,
                                uint64_t total) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const uint64_t half = P >> 1;
  const uint64_t b = idx >> (logP - 1);
  const uint64_t j = idx & (half - 1);
  const uint64_t L = 1ull << logL;
  const uint64_t k = j & (L - 1);
  const uint64_t g = j >> logL;
  const uint64_t q = k << (logP - 1 - logL);
  uint32_t w;
  if (!inverse || q == 0) w = tw[q];
  else w = kP - tw[half - q];
  const uint32_t* xb = x + b * P;
  uint32_t* yb = y + b * P;
  const uint32_t a = xb[j];
  const uint32_t t = mont_mul(w, xb[j + half]);
  yb[(g << (logL + 1)) + k] = add_mod(a, t);
  yb[(g << (logL + 1)) + k + L] = sub_mod(a, t);
}

// omega^t in Montgomery form for 0 <= t < P, from the half table (omega^(P/2) = -1).
__device__ __forceinline__ uint32_t ntt_root(const uint32_t* __restrict__ tw, uint64_t half, uint64_t t) {
  return t < half ? tw[t] : kP - tw[t - half];
}

// One radix-4 Stockham pass: with a_q = x[j + q P/4] and b_q = omega^(+-q k P/(4L)) a_q,
// y[g 4L + k + r L] = sum_q b_q i^(qr), i = omega^(+-P/4) a primitive 4th root of unity.
__global__ void ntt_pass4_kernel(const uint32_t* __restrict__ x, uint32_t* __restrict__ y,
                                 const uint32_t* __restrict__ tw, uint64_t P, uint32_t logL, uint32_t logP,
                                 int inverse, uint64_t total) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const uint64_t quarter = P >> 2, half = P >> 1;
  const uint64_t b = idx >> (logP - 2);
  const uint64_t j = idx & (quarter - 1);
  const uint64_t L = 1ull << logL;
  const uint64_t k = j & (L - 1);
  const uint64_t g = j >> logL;
  const uint64_t stride = k << (logP - 2 - logL);  // k P / (4L)
  const uint32_t* xb = x + b * P;
  uint32_t bq[4];
  bq[0] = xb[j];
#pragma unroll
  for (int q = 1; q < 4; ++q) {
    const uint64_t t = (uint64_t)q * stride;
    const uint32_t w = inverse ? (t == 0 ? tw[0] : ntt_root(tw, half, P - t)) : ntt_root(tw, half, t);
    bq[q] = mont_mul(w, xb[j + q * quarter]);
  }
  const uint32_t im = inverse ? kP - tw[quarter] : tw[quarter];  // omega^(+-P/4)
  const uint32_t s02 = add_mod(bq[0], bq[2]), d02 = sub_mod(bq[0], bq[2]);
  const uint32_t s13 = add_mod(bq[1], bq[3]), d13 = mont_mul(im, sub_mod(bq[1], bq[3]));
  uint32_t* yb = y + b * P + (g << (logL + 2)) + k;
  yb[0] = add_mod(s02, s13);
  yb[L] = add_mod(d02, d13);
  yb[2 * L] = sub_mod(s02, s13);
  yb[3 * L] = sub_mod(d02, d13);
}

// The same radix-4 pass with four consecutive butterflies (k .. k+3, same g) per thread, moved as
// 16-byte vectors: four times the loads in flight per thread. Needs L >= 4 and P >= 16.
__global__ void ntt_pass4_vec_kernel(const uint32_t* __restrict__ x, uint32_t* __restrict__ y,
                                     const uint32_t* __restrict__ tw, uint64_t P, uint32_t logL, uint32_t logP,
                                     int inverse, uint64_t total4) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total4) return;
  const uint64_t quarter = P >> 2, half = P >> 1;
  const uint64_t b = idx >> (logP - 4);
  const uint64_t j0 = (idx & ((quarter >> 2) - 1)) << 2;
  const uint64_t L = 1ull << logL;
  const uint64_t k0 = j0 & (L - 1);
  const uint64_t g = j0 >> logL;
  const uint32_t* xb = x + b * P;
  uint4 v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = *reinterpret_cast<const uint4*>(xb + j0 + q * quarter);
  const uint32_t im = inverse ? kP - tw[quarter] : tw[quarter];
  uint32_t o[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const uint64_t stride = (k0 + e) << (logP - 2 - logL);
    uint32_t bq[4];
    bq[0] = (&v[0].x)[e];
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      const uint64_t t = (uint64_t)q * stride;
      const uint32_t w = inverse ? (t == 0 ? tw[0] : ntt_root(tw, half, P - t)) : ntt_root(tw, half, t);
      bq[q] = mont_mul(w, (&v[q].x)[e]);
    }
    const uint32_t s02 = add_mod(bq[0], bq[2]), d02 = sub_mod(bq[0], bq[2]);
    const uint32_t s13 = add_mod(bq[1], bq[3]), d13 = mont_mul(im, sub_mod(bq[1], bq[3]));
    o[0][e] = add_mod(s02, s13);
    o[1][e] = add_mod(d02, d13);
    o[2][e] = sub_mod(s02, s13);
    o[3][e] = sub_mod(d02, d13);
  }
  uint32_t* yb = y + b * P + (g << (logL + 2)) + k0;
#pragma unroll
  for (int r = 0; r < 4; ++r) *reinterpret_cast<uint4*>(yb + r * L) = make_uint4(o[r][0], o[r][1], o[r][2], o[r][3]);
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
                                uint64_t b0, uint64_t nb, uint32_t* __restrict__ z, uint64_t P) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * P) return;
  const uint64_t bl = idx / P, t = idx - bl * P;
  const uint64_t b = b0 + bl;
  z[idx] = (t < n_t && b < num_blocks) ? ((raw[b * stride + (t >> 5)] >> (t & 31)) & 1u) : 0u;
}

__global__ void ntt_mul_kernel(uint32_t* __restrict__ z, const uint32_t* __restrict__ A, uint64_t P, uint64_t total) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  z[idx] = mont_mul(z[idx], A[idx & (P - 1)]);
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

cudaError_t run_ntt(uint32_t* a, uint32_t* b, const uint32_t* tw, uint64_t P, uint32_t logP, uint64_t batch,
                    int inverse, cudaStream_t s, uint32_t* kernels, uint32_t** result) {
  uint32_t* x = a;
  uint32_t* y = b;
  for (uint32_t logL = 0; logL < logP;) {
    if (logP - logL >= 2) {  // radix 4 while two factors of 2 remain, then one radix-2 pass
      if (logL >= 2 && logP >= 4) {
        const uint64_t total4 = batch * (P >> 4);
        ntt_pass4_vec_kernel<<<grid_for(total4, 256), 256, 0, s>>>(x, y, tw, P, logL, logP, inverse, total4);
      } else {
        const uint64_t total = batch * (P >> 2);
        ntt_pass4_kernel<<<grid_for(total, 256), 256, 0, s>>>(x, y, tw, P, logL, logP, inverse, total);
      }
      logL += 2;
    } else {
      const uint64_t total = batch * (P >> 1);
      ntt_pass_kernel<<<grid_for(total, 256), 256, 0, s>>>(x, y, tw, P, logL, logP, inverse, total);
      logL += 1;
    }
    ++*kernels;
    uint32_t* t = x;
    x = y;
    y = t;
  }
  *result = x;
  return cudaGetLastError();
}

// ---- uneven batches: requests with their own seeds, grouped by transform length P ----

__device__ __forceinline__ uint32_t bit_at(const uint8_t* __restrict__ p, uint64_t bit) {
  return (p[bit >> 3] >> (bit & 7)) & 1u;
}

// Entry 2r of the chunk holds request r's seed bits [0, L_t), entry 2r+1 its raw bits [0, n_t),
// both zero-padded to P.
__global__ void ntt_batch_inputs_kernel(const BatchReq* __restrict__ reqs, uint64_t nr, uint32_t* __restrict__ z,
                                        uint64_t P) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * nr * P) return;
  const uint64_t e = idx / P, t = idx - e * P;
  const BatchReq& q = reqs[e >> 1];
  uint32_t v = 0;
  if (e & 1) {
    if (t < q.n_t) v = bit_at(q.raw, q.raw_bit_off + t);
  } else {
    if (t < q.L_t) v = bit_at(q.seed, t);
  }
  z[idx] = v;
}

// c_r = (S_2r (*) S_2r+1) (*) factor = A R / P  (Montgomery products; factor = P^-1 2^64 mod p).
__global__ void ntt_batch_mul_kernel(const uint32_t* __restrict__ z, uint32_t* __restrict__ c, uint64_t P, uint64_t nr,
                                     uint32_t factor_m) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nr * P) return;
  const uint64_t r = idx / P, t = idx - r * P;
  c[idx] = mont_mul(mont_mul(z[(2 * r) * P + t], z[(2 * r + 1) * P + t]), factor_m);
}

// Output word w of chunk request r (one warp per word): parities of c[n_t - 1 + i], identity bits.
__global__ void ntt_batch_extract_kernel(const BatchReq* __restrict__ reqs, uint64_t nr, uint64_t max_mw,
                                         const uint32_t* __restrict__ c, uint64_t P, uint32_t* __restrict__ out_stage) {
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (gw >= nr * max_mw) return;
  const uint64_t r = gw / max_mw, w = gw - r * max_mw;
  const BatchReq& q = reqs[r];
  if (w >= q.mw) return;  // warp-uniform
  const uint64_t i = 32 * w + lane;
  const uint32_t bit = (i < q.m) ? (c[r * P + q.n_t - 1 + i] & 1u) : 0u;
  uint32_t word = __ballot_sync(0xffffffffu, bit);
  const uint32_t ident = (q.form == QRNG_FORM_MODIFIED && i < q.m) ? bit_at(q.raw, q.raw_bit_off + q.id_off + i) : 0u;
  word ^= __ballot_sync(0xffffffffu, ident);
  if (lane == 0) out_stage[q.out_stage_off + w] = word;
}

}  // namespace

cudaError_t launch_ntt_batch(const BatchReq* reqs_dev, uint64_t nr, uint64_t P,
                             uint64_t max_mw, FftWorkspace& ws, uint32_t* out_stage, cudaStream_t s,
                             uint32_t* kernels) {
  uint32_t logP = 0;
  while ((1ull << logP) < P) ++logP;
  cudaError_t e;
  if (ws.ntt_P != P) {
    if ((e = ws.ntt_tw.ensure((P / 2) * sizeof(uint32_t))) != cudaSuccess) return e;
    const uint32_t omega = pow_mod(kGen, (kP - 1) / P);
    ntt_twiddle_kernel<<<grid_for(ceil_div(P / 2, 256), 128), 128, 0, s>>>(
        ws.ntt_tw.as<uint32_t>(), P / 2, to_mont(omega), to_mont(1), to_mont(pow_mod(omega, 256)));
    ++*kernels;
    ws.ntt_P = P;
  }
  if ((e = ws.buf0.ensure(2 * nr * P * sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = ws.buf1.ensure(2 * nr * P * sizeof(uint32_t))) != cudaSuccess) return e;
  uint32_t* b0p = ws.buf0.as<uint32_t>();
  uint32_t* b1p = ws.buf1.as<uint32_t>();
  ntt_batch_inputs_kernel<<<grid_for(2 * nr * P, 256), 256, 0, s>>>(reqs_dev, nr, b0p, P);
  ++*kernels;
  uint32_t* spec = nullptr;
  if ((e = run_ntt(b0p, b1p, ws.ntt_tw.as<uint32_t>(), P, logP, 2 * nr, 0, s, kernels, &spec)) != cudaSuccess)
    return e;
  uint32_t* other = (spec == b0p) ? b1p : b0p;
  const uint32_t factor_m = to_mont(to_mont(pow_mod(P % kP, kP - 2)));
  ntt_batch_mul_kernel<<<grid_for(nr * P, 256), 256, 0, s>>>(spec, other, P, nr, factor_m);
  ++*kernels;
  uint32_t* res = nullptr;
  if ((e = run_ntt(other, spec, ws.ntt_tw.as<uint32_t>(), P, logP, nr, 1, s, kernels, &res)) != cudaSuccess) return e;
  ntt_batch_extract_kernel<<<grid_for(nr * max_mw * 32, 256), 256, 0, s>>>(reqs_dev, nr, max_mw, res, P, out_stage);
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
  cudaError_t e;
  if (ws.ntt_P != P) {
    if ((e = ws.ntt_tw.ensure((P / 2) * sizeof(uint32_t))) != cudaSuccess) return e;
    const uint32_t omega = pow_mod(kGen, (kP - 1) / P);  // primitive P-th root of unity
    const uint32_t omega_m = to_mont(omega);
    const uint32_t step_m = to_mont(pow_mod(omega, 256));
    ntt_twiddle_kernel<<<grid_for(ceil_div(P / 2, 256), 128), 128, 0, s>>>(ws.ntt_tw.as<uint32_t>(), P / 2, omega_m,
                                                                          to_mont(1), step_m);
    ++*kernels;
    ws.ntt_P = P;
  }
  uint64_t chunk = kFftWorkspaceBytes / (2 * P * sizeof(uint32_t));
  if (chunk < 1) chunk = 1;
  if (chunk > d.num_blocks) chunk = d.num_blocks;
  if ((e = ws.buf0.ensure(chunk * P * sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = ws.buf1.ensure(chunk * P * sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = ws.spec.ensure(P * sizeof(uint32_t))) != cudaSuccess) return e;
  uint32_t* b0p = ws.buf0.as<uint32_t>();
  uint32_t* b1p = ws.buf1.as<uint32_t>();

  // seed spectrum, scaled by P^-1 and kept in Montgomery form
  uint32_t* res = nullptr;
  ntt_seed_kernel<<<grid_for(P, 256), 256, 0, s>>>(seed, L_t, b0p, P);
  ++*kernels;
  if ((e = run_ntt(b0p, b1p, ws.ntt_tw.as<uint32_t>(), P, logP, 1, 0, s, kernels, &res)) != cudaSuccess) return e;
  const uint32_t pinv = pow_mod(P % kP, kP - 2);
  const uint32_t factor_m = to_mont(to_mont(pinv));  // P^-1 2^64 mod p: one product leaves P^-1 2^32
  ntt_scale_kernel<<<grid_for(P, 256), 256, 0, s>>>(res, P, factor_m);
  ++*kernels;
  if ((e = cudaMemcpyAsync(ws.spec.p, res, P * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;

  for (uint64_t bb = 0; bb < d.num_blocks; bb += chunk) {
    const uint64_t nb = (d.num_blocks - bb) < chunk ? (d.num_blocks - bb) : chunk;
    ntt_pack_kernel<<<grid_for(nb * P, 256), 256, 0, s>>>(d.raw, d.raw_stride, n_t, d.num_blocks, bb, nb, b0p, P);
    ++*kernels;
    if ((e = run_ntt(b0p, b1p, ws.ntt_tw.as<uint32_t>(), P, logP, nb, 0, s, kernels, &res)) != cudaSuccess) return e;
    ntt_mul_kernel<<<grid_for(nb * P, 256), 256, 0, s>>>(res, ws.spec.as<uint32_t>(), P, nb * P);
    ++*kernels;
    uint32_t* other = (res == b0p) ? b1p : b0p;
    uint32_t* fin = nullptr;
    if ((e = run_ntt(res, other, ws.ntt_tw.as<uint32_t>(), P, logP, nb, 1, s, kernels, &fin)) != cudaSuccess)
      return e;
    ntt_extract_kernel<<<grid_for(nb * d.mw * 32, 256), 256, 0, s>>>(fin, P, n_t, d.m, d.mw, d.raw, d.raw_stride,
                                                                     d.modified, d.id_off, d.num_blocks, bb, nb,
                                                                     d.out, d.out_stride);
    ++*kernels;
  }
  return cudaGetLastError();
}

}  // namespace qrng
