// FFT routes to the Toeplitz hash (Sec. III.B Thm. 1-2 and Sec. III.D of the paper).
//
// The Toeplitz part of the hash is a slice of a linear convolution: with c = a * r,
//     k_i = c[n_t - 1 + i] mod 2,  n_t = n (standard) or n - m (modified, whose identity part
// I_m is XORed afterwards). Embedding a and r in a cyclic convolution of length P >= n_t + m - 1
// (the circulant of Sec. III.B) leaves every needed entry free of wrap-around, and the
// convolution theorem turns it into F^-1(F a . F r).
//
// FFT64 (the paper's route): one P-point FP64 transform per PAIR of blocks -- two real blocks are
// the real and imaginary parts of one complex vector, and because the seed spectrum is the
// transform of a real sequence, F^-1(F a . F(r1 + i r2)) = a*r1 + i a*r2 separates them with no
// extra work. Radix-2 Stockham passes run over global memory (one launch per pass over a chunk of
// pairs), with a cached FP64 twiddle table. The worst |s - round(s)| of every entry used is kept
// as evidence of exactness (FP64 with P <= 2^27 keeps it far below 1/2).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qrng_internal.h"

namespace qrng {
namespace {

struct cd {
  double x, y;
};

__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

// tw[k] = exp(-2 pi i k / P), k < P/2.
__global__ void twiddle_kernel(cd* __restrict__ tw, uint64_t P) {
  uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P / 2) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)P, &s, &c);
  tw[k] = {c, s};
}

// One radix-2 Stockham pass over `batch` transforms of length P (half-length L of the butterflies
// produced by this pass): y[g 2L + k] = x[j] + w x[j + P/2], y[g 2L + k + L] = x[j] - w x[j + P/2],
// j = g L + k, w = exp(-+ 2 pi i k / (2L)) = tw[k P / (2L)] (conjugated for the inverse).
__global__ void stockham_pass_kernel(const cd* __restrict__ x, cd* __restrict__ y, const cd* __restrict__ tw,
                                     uint64_t P, uint32_t logL, uint32_t logP, int inverse, uint64_t total) {
  uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const uint64_t half = P >> 1;
  const uint64_t b = idx >> (logP - 1);
  const uint64_t j = idx & (half - 1);
  const uint64_t L = 1ull << logL;
  const uint64_t k = j & (L - 1);
  const uint64_t g = j >> logL;
  cd w = tw[k << (logP - 1 - logL)];
  if (inverse) w.y = -w.y;
  const cd* xb = x + b * P;
  cd* yb = y + b * P;
  const cd a = xb[j];
  const cd t = cmul(w, xb[j + half]);
  yb[(g << (logL + 1)) + k] = {a.x + t.x, a.y + t.y};
  yb[(g << (logL + 1)) + k + L] = {a.x - t.x, a.y - t.y};
}

// exp(-2 pi i t / P) for 0 <= t < P, from the half table (the second half is the negated first).
__device__ __forceinline__ cd fft_root(const cd* __restrict__ tw, uint64_t half, uint64_t t) {
  if (t < half) return tw[t];
  const cd w = tw[t - half];
  return {-w.x, -w.y};
}

// One radix-4 Stockham pass: with a_q = x[j + q P/4] and b_q = w^(q k P/(4L)) a_q,
// y[g 4L + k + r L] = sum_q b_q (-+i)^(qr)  (w and -i conjugated for the inverse).
__global__ void stockham_pass4_kernel(const cd* __restrict__ x, cd* __restrict__ y, const cd* __restrict__ tw,
                                      uint64_t P, uint32_t logL, uint32_t logP, int inverse, uint64_t total) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const uint64_t quarter = P >> 2, half = P >> 1;
  const uint64_t b = idx >> (logP - 2);
  const uint64_t j = idx & (quarter - 1);
  const uint64_t L = 1ull << logL;
  const uint64_t k = j & (L - 1);
  const uint64_t g = j >> logL;
  const uint64_t stride = k << (logP - 2 - logL);
  const cd* xb = x + b * P;
  cd bq[4];
  bq[0] = xb[j];
#pragma unroll
  for (int q = 1; q < 4; ++q) {
    cd w = fft_root(tw, half, (uint64_t)q * stride);
    if (inverse) w.y = -w.y;
    bq[q] = cmul(w, xb[j + q * quarter]);
  }
  const cd s02 = {bq[0].x + bq[2].x, bq[0].y + bq[2].y}, d02 = {bq[0].x - bq[2].x, bq[0].y - bq[2].y};
  const cd s13 = {bq[1].x + bq[3].x, bq[1].y + bq[3].y};
  const cd t13 = {bq[1].x - bq[3].x, bq[1].y - bq[3].y};
  // (-i) t forward, (+i) t inverse
  const cd d13 = inverse ? cd{-t13.y, t13.x} : cd{t13.y, -t13.x};
  cd* yb = y + b * P + (g << (logL + 2)) + k;
  yb[0] = {s02.x + s13.x, s02.y + s13.y};
  yb[L] = {d02.x + d13.x, d02.y + d13.y};
  yb[2 * L] = {s02.x - s13.x, s02.y - s13.y};
  yb[3 * L] = {d02.x - d13.x, d02.y - d13.y};
}

// Zero-padded seed (first L_t bits) as the real part of one complex vector.
__global__ void seed_to_complex_kernel(const uint8_t* __restrict__ seed, uint64_t L, cd* __restrict__ z, uint64_t P) {
  uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  double v = 0.0;
  if (t < L) v = (double)((seed[t >> 3] >> (t & 7)) & 1u);
  z[t] = {v, 0.0};
}

// z_p[t] = r_{2p}[t] + i r_{2p+1}[t] for t < n_t, zero beyond (pairs p0 .. p0+npairs-1).
__global__ void pack_pairs_kernel(const uint32_t* __restrict__ raw, uint64_t stride, uint64_t n_t,
                                  uint64_t num_blocks, uint64_t p0, uint64_t npairs, cd* __restrict__ z, uint64_t P) {
  uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npairs * P) return;
  const uint64_t p = idx / P, t = idx - p * P;
  const uint64_t b0 = 2 * (p0 + p), b1 = b0 + 1;
  double re = 0.0, im = 0.0;
  if (t < n_t) {
    re = (double)((raw[b0 * stride + (t >> 5)] >> (t & 31)) & 1u);
    if (b1 < num_blocks) im = (double)((raw[b1 * stride + (t >> 5)] >> (t & 31)) & 1u);
  }
  z[idx] = {re, im};
}

// Z_p[k] *= A[k] / P  (the 1/P of the inverse transform folded in).
__global__ void spectrum_mul_kernel(cd* __restrict__ z, const cd* __restrict__ A, uint64_t P, uint64_t total) {
  uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const cd a = A[idx & (P - 1)];
  const double s = 1.0 / (double)P;
  cd v = cmul(z[idx], a);
  z[idx] = {v.x * s, v.y * s};
}

// Output word w (32 outputs) of both blocks of pair p: parities of round(c[n_t - 1 + i]), the
// identity bits for the modified form, and the worst rounding distance.
__global__ void extract_pairs_kernel(const cd* __restrict__ z, uint64_t P, uint64_t n_t, uint64_t m, uint64_t mw,
                                     const uint32_t* __restrict__ raw, uint64_t stride, int modified, uint64_t id_off,
                                     uint64_t num_blocks, uint64_t p0, uint64_t npairs, uint32_t* __restrict__ out,
                                     uint64_t out_stride, unsigned long long* __restrict__ worst) {
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // one warp per (pair, word)
  const uint32_t lane = threadIdx.x & 31;
  if (gw >= npairs * mw) return;
  const uint64_t p = gw / mw, w = gw - p * mw;
  const uint64_t i = 32 * w + lane;
  double err = 0.0;
  uint32_t bit0 = 0, bit1 = 0;
  if (i < m) {
    const cd v = z[p * P + n_t - 1 + i];
    const double r0 = rint(v.x), r1 = rint(v.y);
    err = fmax(fabs(v.x - r0), fabs(v.y - r1));
    bit0 = (uint32_t)((long long)r0 & 1);
    bit1 = (uint32_t)((long long)r1 & 1);
  }
  uint32_t w0 = __ballot_sync(0xffffffffu, bit0);
  uint32_t w1 = __ballot_sync(0xffffffffu, bit1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) err = fmax(err, __shfl_xor_sync(0xffffffffu, err, o));
  if (lane == 0) {
    atomicMax(worst, (unsigned long long)__double_as_longlong(err));
    const uint64_t rem = m - 32 * w;
    const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    const uint64_t bb[2] = {2 * (p0 + p), 2 * (p0 + p) + 1};
    const uint32_t ww[2] = {w0, w1};
    for (int h = 0; h < 2; ++h) {
      if (bb[h] >= num_blocks) continue;
      uint32_t word = ww[h] & omask;
      if (modified) {
        const uint32_t* rr = raw + bb[h] * stride;
        const uint64_t bit = id_off + 32 * w;
        const uint64_t rq = bit >> 5;
        const uint32_t rs = (uint32_t)(bit & 31);
        const uint32_t lo = rr[rq];
        const uint32_t hi = (rs && rq + 1 < stride) ? rr[rq + 1] : 0u;
        word ^= __funnelshift_r(lo, hi, rs) & omask;
      }
      out[bb[h] * out_stride + w] = word;
    }
  }
}

inline unsigned grid_for(uint64_t total, int threads) { return (unsigned)ceil_div(total, (uint64_t)threads); }

cudaError_t run_fft(cd* a, cd* b, const cd* tw, uint64_t P, uint32_t logP, uint64_t batch, int inverse,
                    cudaStream_t s, uint32_t* kernels, cd** result) {
  cd* x = a;
  cd* y = b;
  for (uint32_t logL = 0; logL < logP;) {
    if (logP - logL >= 2) {  // radix 4 while two factors of 2 remain, then one radix-2 pass
      const uint64_t total = batch * (P >> 2);
      stockham_pass4_kernel<<<grid_for(total, 256), 256, 0, s>>>(x, y, tw, P, logL, logP, inverse, total);
      logL += 2;
    } else {
      const uint64_t total = batch * (P >> 1);
      stockham_pass_kernel<<<grid_for(total, 256), 256, 0, s>>>(x, y, tw, P, logL, logP, inverse, total);
      logL += 1;
    }
    ++*kernels;
    cd* t = x;
    x = y;
    y = t;
  }
  *result = x;
  return cudaGetLastError();
}

}  // namespace

uint64_t fft64_length(uint64_t n_t, uint64_t m) {
  uint64_t need = n_t + m - 1, P = 2;
  while (P < need) P <<= 1;
  return P;
}

cudaError_t launch_fft64(const DirectArgs& d, const uint8_t* seed, uint64_t L_t, FftWorkspace& ws, cudaStream_t s,
                         uint32_t* kernels) {
  const uint64_t n_t = d.n_t;
  const uint64_t P = fft64_length(n_t, d.m);
  uint32_t logP = 0;
  while ((1ull << logP) < P) ++logP;
  cudaError_t e;
  if (ws.tw_P != P) {
    if ((e = ws.tw.ensure((P / 2) * sizeof(cd))) != cudaSuccess) return e;
    twiddle_kernel<<<grid_for(P / 2, 256), 256, 0, s>>>(ws.tw.as<cd>(), P);
    ++*kernels;
    ws.tw_P = P;
  }
  const uint64_t npairs_total = ceil_div(d.num_blocks, 2);
  // chunk of pairs so that the two ping-pong buffers stay within the workspace budget
  uint64_t chunk = kFftWorkspaceBytes / (2 * P * sizeof(cd));
  if (chunk < 1) chunk = 1;
  if (chunk > npairs_total) chunk = npairs_total;
  if ((e = ws.buf0.ensure(chunk * P * sizeof(cd))) != cudaSuccess) return e;
  if ((e = ws.buf1.ensure(chunk * P * sizeof(cd))) != cudaSuccess) return e;
  if ((e = ws.spec.ensure(P * sizeof(cd))) != cudaSuccess) return e;

  // seed spectrum A = F a
  cd* out_ptr = nullptr;
  seed_to_complex_kernel<<<grid_for(P, 256), 256, 0, s>>>(seed, L_t, ws.buf0.as<cd>(), P);
  ++*kernels;
  if ((e = run_fft(ws.buf0.as<cd>(), ws.buf1.as<cd>(), ws.tw.as<cd>(), P, logP, 1, 0, s, kernels, &out_ptr)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(ws.spec.p, out_ptr, P * sizeof(cd), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;

  for (uint64_t p0 = 0; p0 < npairs_total; p0 += chunk) {
    const uint64_t np = (npairs_total - p0) < chunk ? (npairs_total - p0) : chunk;
    pack_pairs_kernel<<<grid_for(np * P, 256), 256, 0, s>>>(d.raw, d.raw_stride, n_t, d.num_blocks, p0, np,
                                                            ws.buf0.as<cd>(), P);
    ++*kernels;
    if ((e = run_fft(ws.buf0.as<cd>(), ws.buf1.as<cd>(), ws.tw.as<cd>(), P, logP, np, 0, s, kernels, &out_ptr)) !=
        cudaSuccess)
      return e;
    spectrum_mul_kernel<<<grid_for(np * P, 256), 256, 0, s>>>(out_ptr, ws.spec.as<cd>(), P, np * P);
    ++*kernels;
    cd* other = (out_ptr == ws.buf0.as<cd>()) ? ws.buf1.as<cd>() : ws.buf0.as<cd>();
    cd* res = nullptr;
    if ((e = run_fft(out_ptr, other, ws.tw.as<cd>(), P, logP, np, 1, s, kernels, &res)) != cudaSuccess) return e;
    extract_pairs_kernel<<<grid_for(np * d.mw * 32, 256), 256, 0, s>>>(
        res, P, n_t, d.m, d.mw, d.raw, d.raw_stride, d.modified, d.id_off, d.num_blocks, p0, np, d.out, d.out_stride,
        ws.worst);
    ++*kernels;
  }
  return cudaGetLastError();
}


// ------------------------------------------------------------------------------------------------
// FP64 route for uneven batches (each request its own seed, all of one transform length P):
// z_r = a_r + i r_r carries request r's seed and raw bits in one complex vector; from Z = F z the
// two spectra are A = (Z_k + conj Z_-k)/2 and R = (Z_k - conj Z_-k)/(2i); C_r = A R / P is the
// spectrum of the real convolution, so two requests share one inverse: F^-1(C_r + i C_r') =
// c_r + i c_r'. One forward and half an inverse transform per request.
// ------------------------------------------------------------------------------------------------
namespace {

__device__ __forceinline__ double bit_at_f(const uint8_t* __restrict__ p, uint64_t bit) {
  return (double)((p[bit >> 3] >> (bit & 7)) & 1u);
}

__global__ void fft_batch_inputs_kernel(const BatchReq* __restrict__ reqs, uint64_t nr, cd* __restrict__ z, uint64_t P) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nr * P) return;
  const uint64_t r = idx / P, t = idx - r * P;
  const BatchReq& q = reqs[r];
  z[idx] = {t < q.L_t ? bit_at_f(q.seed, t) : 0.0, t < q.n_t ? bit_at_f(q.raw, q.raw_bit_off + t) : 0.0};
}

// W_pair[k] = C_{2 pair}[k] + i C_{2 pair + 1}[k],  C_r = A_r R_r / P.
__global__ void fft_batch_mul_kernel(const cd* __restrict__ Z, cd* __restrict__ W, uint64_t P, uint64_t nr) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t npairs = (nr + 1) / 2;
  if (idx >= npairs * P) return;
  const uint64_t pr = idx / P, k = idx - pr * P;
  const uint64_t km = (P - k) & (P - 1);
  const double s = 1.0 / (double)P;
  cd c[2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int h = 0; h < 2; ++h) {
    const uint64_t r = 2 * pr + h;
    if (r >= nr) break;
    const cd zk = Z[r * P + k], zm = Z[r * P + km];
    const cd a = {0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y)};   // (Z_k + conj Z_-k) / 2
    const cd rr = {0.5 * (zk.y + zm.y), -0.5 * (zk.x - zm.x)};  // (Z_k - conj Z_-k) / (2i)
    const cd v = cmul(a, rr);
    c[h] = {v.x * s, v.y * s};
  }
  W[idx] = {c[0].x - c[1].y, c[0].y + c[1].x};  // c0 + i c1
}

// Output word w of request r (one warp per word): parity of round(c_r[n_t - 1 + i]), identity bits.
__global__ void fft_batch_extract_kernel(const BatchReq* __restrict__ reqs, uint64_t nr, uint64_t max_mw,
                                         const cd* __restrict__ Wt, uint64_t P, uint32_t* __restrict__ out_stage,
                                         unsigned long long* __restrict__ worst) {
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (gw >= nr * max_mw) return;
  const uint64_t r = gw / max_mw, w = gw - r * max_mw;
  const BatchReq& q = reqs[r];
  if (w >= q.mw) return;  // warp-uniform
  const uint64_t i = 32 * w + lane;
  double err = 0.0;
  uint32_t bit = 0;
  if (i < q.m) {
    const cd v = Wt[(r / 2) * P + q.n_t - 1 + i];
    const double x = (r & 1) ? v.y : v.x;
    const double rx = rint(x);
    err = fabs(x - rx);
    bit = (uint32_t)((long long)rx & 1);
  }
  uint32_t word = __ballot_sync(0xffffffffu, bit);
  const uint32_t ident = (q.form == QRNG_FORM_MODIFIED && i < q.m)
                             ? (uint32_t)bit_at_f(q.raw, q.raw_bit_off + q.id_off + i) : 0u;
  word ^= __ballot_sync(0xffffffffu, ident);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) err = fmax(err, __shfl_xor_sync(0xffffffffu, err, o));
  if (lane == 0) {
    atomicMax(worst, (unsigned long long)__double_as_longlong(err));
    out_stage[q.out_stage_off + w] = word;
  }
}

}  // namespace

cudaError_t launch_fft64_batch(const BatchReq* reqs_dev, uint64_t nr, uint64_t P, uint64_t max_mw, FftWorkspace& ws,
                               uint32_t* out_stage, cudaStream_t s, uint32_t* kernels) {
  uint32_t logP = 0;
  while ((1ull << logP) < P) ++logP;
  cudaError_t e;
  if (ws.tw_P != P) {
    if ((e = ws.tw.ensure((P / 2) * sizeof(cd))) != cudaSuccess) return e;
    twiddle_kernel<<<grid_for(P / 2, 256), 256, 0, s>>>(ws.tw.as<cd>(), P);
    ++*kernels;
    ws.tw_P = P;
  }
  if ((e = ws.buf0.ensure(nr * P * sizeof(cd))) != cudaSuccess) return e;
  if ((e = ws.buf1.ensure(nr * P * sizeof(cd))) != cudaSuccess) return e;
  cd* b0p = ws.buf0.as<cd>();
  cd* b1p = ws.buf1.as<cd>();
  fft_batch_inputs_kernel<<<grid_for(nr * P, 256), 256, 0, s>>>(reqs_dev, nr, b0p, P);
  ++*kernels;
  cd* Z = nullptr;
  if ((e = run_fft(b0p, b1p, ws.tw.as<cd>(), P, logP, nr, 0, s, kernels, &Z)) != cudaSuccess) return e;
  cd* Wb = (Z == b0p) ? b1p : b0p;
  const uint64_t npairs = (nr + 1) / 2;
  fft_batch_mul_kernel<<<grid_for(npairs * P, 256), 256, 0, s>>>(Z, Wb, P, nr);
  ++*kernels;
  cd* res = nullptr;
  if ((e = run_fft(Wb, Z, ws.tw.as<cd>(), P, logP, npairs, 1, s, kernels, &res)) != cudaSuccess) return e;
  fft_batch_extract_kernel<<<grid_for(nr * max_mw * 32, 256), 256, 0, s>>>(reqs_dev, nr, max_mw, res, P, out_stage,
                                                                          ws.worst);
  ++*kernels;
  return cudaGetLastError();
}

}  // namespace qrng
