// Min-entropy estimate of an ADC sample stream (Sec. II of the paper):
//   1. exact histogram of the codes (warp-privatised shared-memory counters, one pass over HBM);
//   2. a one-CTA FP64 finaliser: H_min of the measured distribution (Sec. II.A), the Gaussian
//      model fixed by the measured mean and variance (Sec. II.B), the statistical distance d_U,
//      the finite-size term, Delta H_m and H_modify (Sec. II.C).
#include <cuda_runtime.h>
#include <math.h>
#include <math_constants.h>
#include <stdint.h>

#include "qrng_internal.h"

namespace qrng {
namespace {

constexpr int kHistThreads = 256;
constexpr int kHistWarps = kHistThreads / 32;

// bits <= 8: each warp owns 256 counters; codes >= 2^bits land in counters the merge step
// adds to the out-of-range total.
__global__ void __launch_bounds__(kHistThreads) hist_u8_kernel(const uint8_t* __restrict__ samples, uint64_t count,
                                                                int bits, unsigned long long* __restrict__ hist) {
  __shared__ uint32_t sh[kHistWarps][256];
  for (int i = threadIdx.x; i < kHistWarps * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  uint32_t* my = sh[threadIdx.x >> 5];

  // Bytes before the first 16-byte boundary, then 16-byte vectors, then the tail.
  const uint64_t head = (16 - (reinterpret_cast<uintptr_t>(samples) & 15)) & 15;
  const uint64_t nhead = head < count ? head : count;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  if (tid < nhead) atomicAdd(&my[samples[tid]], 1u);
  const uint64_t nvec = (count - nhead) / 16;
  const uint4* vec = reinterpret_cast<const uint4*>(samples + nhead);
  for (uint64_t v = tid; v < nvec; v += nthreads) {
    uint4 x = __ldcs(vec + v);
    uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int s = 0; s < 32; s += 8) atomicAdd(&my[(w[k] >> s) & 0xffu], 1u);
    }
  }
  const uint64_t tail0 = nhead + nvec * 16;
  if (tail0 + tid < count) atomicAdd(&my[samples[tail0 + tid]], 1u);
  __syncthreads();

  const uint32_t K = 1u << bits;
  for (int b = threadIdx.x; b < 256; b += blockDim.x) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kHistWarps; ++w) s += sh[w][b];
    if (s) atomicAdd(&hist[b < (int)K ? b : (int)K], (unsigned long long)s);
  }
}

// 9 <= bits <= 13: one shared histogram per CTA (<= 8192 counters + one out-of-range counter).
__global__ void __launch_bounds__(kHistThreads) hist_u16_smem_kernel(const uint16_t* __restrict__ samples,
                                                                      uint64_t count, int bits,
                                                                      unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t shc[];
  const uint32_t K = 1u << bits;
  for (uint32_t i = threadIdx.x; i <= K; i += blockDim.x) shc[i] = 0;
  __syncthreads();
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t s = tid; s < count; s += nthreads) {
    uint32_t v = __ldcs(samples + s);
    atomicAdd(&shc[v < K ? v : K], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b <= K; b += blockDim.x)
    if (shc[b]) atomicAdd(&hist[b], (unsigned long long)shc[b]);
}

// 14 <= bits <= 16: counters straight in global memory.
__global__ void __launch_bounds__(kHistThreads) hist_u16_global_kernel(const uint16_t* __restrict__ samples,
                                                                        uint64_t count, int bits,
                                                                        unsigned long long* __restrict__ hist) {
  const uint32_t K = 1u << bits;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t s = tid; s < count; s += nthreads) {
    uint32_t v = __ldcs(samples + s);
    atomicAdd(&hist[v < K ? v : K], 1ull);
  }
}

// ------------------------------------------------------------------------------------------------
// Finaliser: one CTA.
// ------------------------------------------------------------------------------------------------

constexpr int kFinThreads = 512;

typedef unsigned __int128 u128_t;

__device__ __forceinline__ u128_t shfl_down_u128(u128_t v, int d) {
  const uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)v, d);
  const uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)(v >> 64), d);
  return ((u128_t)hi << 64) | lo;
}

// Largest count, lowest code on ties (arg 0xffffffff = none).
__device__ __forceinline__ void max_arg_merge(unsigned long long& mx, uint32_t& arg, unsigned long long m2,
                                              uint32_t a2) {
  if (a2 != 0xffffffffu && (arg == 0xffffffffu || m2 > mx || (m2 == mx && a2 < arg))) {
    mx = m2;
    arg = a2;
  }
}

// Phi(hi) - Phi(lo) without cancellation: a cell on one side of the mean is a difference of the
// tails c = erfc(|z| / sqrt 2) of its boundaries (computed once per boundary); the one cell across
// the mean is a difference of central masses, erf(hi / sqrt 2) - erf(lo / sqrt 2). (One minus the
// two tails, or two CDF values near 1/2 subtracted, would lose ~1e-16 absolute, i.e. ~1e-12
// relative for the 6e-5 cells of a 16-bit ADC.)
__device__ __forceinline__ double cell_from_tails(double lo, double hi, double c_lo, double c_hi) {
  if (lo >= 0.0) return 0.5 * (c_lo - c_hi);
  if (hi <= 0.0) return 0.5 * (c_hi - c_lo);
  return 0.5 * (erf(hi * M_SQRT1_2) - erf(lo * M_SQRT1_2));
}

constexpr uint32_t kFinChunk = 2048;  // cells per shared-memory chunk of boundary tails

// Model cells of codes [0, K) under N(mu, sigma^2) (boundaries v +- 1/2, end codes take the tails):
// each boundary's tail is computed once per chunk; returns this thread's largest cell, its sum of
// |hist/N - P| (when dist) and, for code `want`, its cell in *p_want.
__device__ void model_cells(const unsigned long long* __restrict__ hist, uint32_t K, unsigned long long N, double mu,
                            double sigma, bool dist, uint32_t want, double* __restrict__ s_tail, double& pmax,
                            double& dsum, double* p_want) {
  for (uint32_t c0 = 0; c0 < K; c0 += kFinChunk) {
    const uint32_t ncell = (K - c0) < kFinChunk ? (K - c0) : kFinChunk;
    // s_tail[i] = tail of boundary c0 - 1 + i, i = 0 .. ncell (boundary j lies between codes j, j + 1)
    for (uint32_t i = threadIdx.x; i <= ncell; i += blockDim.x) {
      const int64_t j = (int64_t)c0 - 1 + i;
      const double z = (j < 0 || j >= (int64_t)K - 1) ? CUDART_INF : (((double)j + 0.5 - mu) / sigma);
      s_tail[i] = erfc(fabs(z) * M_SQRT1_2);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < ncell; i += blockDim.x) {
      const uint32_t v = c0 + i;
      const double lo = (v == 0) ? -CUDART_INF : ((double)v - 0.5 - mu) / sigma;
      const double hi = (v == K - 1) ? CUDART_INF : ((double)v + 0.5 - mu) / sigma;
      const double P = cell_from_tails(lo, hi, s_tail[i], s_tail[i + 1]);
      pmax = fmax(pmax, P);
      if (dist) dsum += fabs((double)hist[v] / (double)N - P);
      if (v == want) *p_want = P;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kFinThreads) hmin_finalize_kernel(const unsigned long long* __restrict__ hist,
                                                                     int bits, double eps,
                                                                     DevHminResult* __restrict__ out, double var_sub,
                                                                     double h_ref) {
  constexpr int kWarps = kFinThreads / 32;
  __shared__ unsigned long long w_n[kWarps], w_max[kWarps];
  __shared__ uint32_t w_arg[kWarps];
  __shared__ u128_t w_s1[kWarps], w_s2[kWarps];
  __shared__ double w_pmax[kWarps], w_pmax_full[kWarps], w_dsum[kWarps];
  __shared__ double s_tail[kFinChunk + 1];
  __shared__ double s_mu, s_sigma, s_sigma_q, s_pa;
  __shared__ unsigned long long s_N, s_max;
  __shared__ uint32_t s_arg;
  __shared__ int s_point, s_bad_sub;

  const uint32_t K = 1u << bits;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;

  // Pass 1: count, exact first and second moments, largest bin (lowest code on ties).
  unsigned long long n = 0, mx = 0;
  uint32_t arg = 0xffffffffu;
  u128_t s1 = 0, s2 = 0;
  for (uint32_t v = t; v < K; v += kFinThreads) {
    const unsigned long long h = hist[v];
    n += h;
    s1 += (u128_t)v * h;
    s2 += (u128_t)((unsigned long long)v * v) * h;
    if (arg == 0xffffffffu || h > mx) {  // codes visited in increasing order: ties keep the lowest
      mx = h;
      arg = v;
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    n += __shfl_down_sync(0xffffffffu, n, d);
    s1 += shfl_down_u128(s1, d);
    s2 += shfl_down_u128(s2, d);
    max_arg_merge(mx, arg, __shfl_down_sync(0xffffffffu, mx, d), __shfl_down_sync(0xffffffffu, arg, d));
  }
  if (lane == 0) {
    w_n[wid] = n; w_s1[wid] = s1; w_s2[wid] = s2; w_max[wid] = mx; w_arg[wid] = arg;
  }
  __syncthreads();
  if (t == 0) {
    unsigned long long N = 0, M = 0;
    uint32_t A = 0xffffffffu;
    u128_t S1 = 0, S2 = 0;
    for (int w = 0; w < kWarps; ++w) {
      N += w_n[w]; S1 += w_s1[w]; S2 += w_s2[w];
      max_arg_merge(M, A, w_max[w], w_arg[w]);
    }
    s_N = N; s_max = M; s_arg = A;
    if (N == 0) {
      out->status = QRNG_EINVAL;
    } else {
      const u128_t num = (u128_t)N * S2 - S1 * S1;  // N^2 * population variance, exact
      const double mu = (double)S1 / (double)N;
      const double var = (double)num / ((double)N * (double)N);
      s_mu = mu;
      s_sigma = sqrt(var);
      s_point = (num == 0);
      const double var_q = var - var_sub;
      s_bad_sub = (var_sub > 0.0) && !(var_q > 0.0);
      s_sigma_q = var_sub > 0.0 && var_q > 0.0 ? sqrt(var_q) : s_sigma;
      qrng_hmin_report& r = out->rep;
      r.count = N;
      r.max_count = M;
      r.argmax = A;
      r.bits = (uint32_t)bits;
      r.mean = mu;
      r.var = var;
      r.h_emp = -log2((double)M / (double)N);
      out->out_of_range = hist[K];
    }
  }
  __syncthreads();
  const unsigned long long N = s_N;
  if (N == 0) return;

  // Pass 2: model cells, their maximum, and the distance to the measured distribution.
  const double mu = s_mu, sigma = s_sigma;
  const bool sub = var_sub > 0.0 && !s_bad_sub;
  const uint32_t amax = s_arg;
  double pmax_full = 0.0, dsum = 0.0, pmax = 0.0;
  if (s_point) {  // every sample on one code: the model is that point mass
    for (uint32_t v = t; v < K; v += kFinThreads) {
      const double P = (v == amax) ? 1.0 : 0.0;
      pmax_full = fmax(pmax_full, P);
      dsum += fabs((double)hist[v] / (double)N - P);
    }
    if (t == 0) s_pa = 1.0;
    pmax = pmax_full;
  } else {
    double pa = 0.0;
    model_cells(hist, K, N, mu, sigma, true, amax, s_tail, pmax_full, dsum, &pa);
    if (amax % (uint32_t)kFinThreads == (uint32_t)t) s_pa = pa;  // the thread that visited code amax
    if (sub) {
      double unused_d = 0.0, unused_p = 0.0;
      model_cells(hist, K, N, mu, s_sigma_q, false, K, s_tail, pmax, unused_d, &unused_p);
    } else {
      pmax = pmax_full;
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    pmax = fmax(pmax, __shfl_down_sync(0xffffffffu, pmax, d));
    pmax_full = fmax(pmax_full, __shfl_down_sync(0xffffffffu, pmax_full, d));
    dsum += __shfl_down_sync(0xffffffffu, dsum, d);
  }
  if (lane == 0) {
    w_pmax[wid] = pmax; w_pmax_full[wid] = pmax_full; w_dsum[wid] = dsum;
  }
  __syncthreads();
  if (t == 0) {
    double PM = 0.0, PF = 0.0, DS = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      PM = fmax(PM, w_pmax[w]); PF = fmax(PF, w_pmax_full[w]); DS += w_dsum[w];
    }
    qrng_hmin_report& r = out->rep;
    r.h_model = -log2(PM);
    out->h_subtracted = -log2(PF) - h_ref;
    if (sub) r.var = s_sigma_q * s_sigma_q;
    r.d_u = 0.5 * DS;
    r.d_u_peak = 0.5 * fabs((double)s_max / (double)N - s_pa);
    r.delta_fs = 0.5 * sqrt(2.0 * ((double)K * M_LN2 + log(1.0 / eps)) / (double)N);
    r.delta_hm = log2((r.d_u + r.delta_fs) * ldexp(1.0, bits + 1) + 1.0);
    double h = r.h_model - r.delta_hm;
    r.h_modify = h > 0.0 ? h : 0.0;
    out->status = (out->out_of_range || s_bad_sub) ? QRNG_EINVAL : QRNG_OK;
  }
}

// Random subsample (any width): counters in shared memory for up to 2^13 codes, else global.
__global__ void __launch_bounds__(kHistThreads) hist_sampled_kernel(const void* __restrict__ samples, uint64_t count,
                                                                     int bits, uint64_t thr, uint64_t sel_seed,
                                                                     unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t shs[];
  const uint32_t K = 1u << bits;
  const bool smem = bits <= 13;
  if (smem) {
    for (uint32_t i = threadIdx.x; i <= K; i += blockDim.x) shs[i] = 0;
    __syncthreads();
  }
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t s = tid; s < count; s += nthreads) {
    // splitmix64 output s+1 of the generator started at sel_seed
    uint64_t z = sel_seed + (s + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    if ((z >> 11) >= thr) continue;
    const uint32_t v = bits <= 8 ? static_cast<const uint8_t*>(samples)[s] : static_cast<const uint16_t*>(samples)[s];
    const uint32_t c = v < K ? v : K;
    if (smem) atomicAdd(&shs[c], 1u);
    else atomicAdd(&hist[c], 1ull);
  }
  if (smem) {
    __syncthreads();
    for (uint32_t b = threadIdx.x; b <= K; b += blockDim.x)
      if (shs[b]) atomicAdd(&hist[b], (unsigned long long)shs[b]);
  }
}

}  // namespace

cudaError_t launch_histogram(const void* samples, uint64_t count, int bits, unsigned long long* hist, int num_sms,
                             cudaStream_t s, uint32_t* kernels) {
  const uint32_t K = 1u << bits;
  cudaError_t e = cudaMemsetAsync(hist, 0, (K + 1) * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const uint64_t per_cta = bits <= 8 ? 16ull * kHistThreads * 8 : (uint64_t)kHistThreads * 16;
  uint64_t want = ceil_div(count, per_cta);
  uint64_t cap = (uint64_t)num_sms * (bits <= 8 ? 6 : 4);
  int grid = (int)(want < cap ? (want ? want : 1) : cap);
  if (bits <= 8) {
    hist_u8_kernel<<<grid, kHistThreads, 0, s>>>(static_cast<const uint8_t*>(samples), count, bits, hist);
  } else if (bits <= 13) {
    hist_u16_smem_kernel<<<grid, kHistThreads, (K + 1) * sizeof(uint32_t), s>>>(
        static_cast<const uint16_t*>(samples), count, bits, hist);
  } else {
    hist_u16_global_kernel<<<grid, kHistThreads, 0, s>>>(static_cast<const uint16_t*>(samples), count, bits, hist);
  }
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_histogram_sampled(const void* samples, uint64_t count, int bits, uint64_t thr, uint64_t sel_seed,
                                     unsigned long long* hist, int num_sms, cudaStream_t s, uint32_t* kernels) {
  const uint32_t K = 1u << bits;
  cudaError_t e = cudaMemsetAsync(hist, 0, (K + 1) * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  uint64_t want = ceil_div(count, (uint64_t)kHistThreads * 16);
  uint64_t cap = (uint64_t)num_sms * 4;
  int grid = (int)(want < cap ? (want ? want : 1) : cap);
  const size_t smem = bits <= 13 ? (K + 1) * sizeof(uint32_t) : 0;
  hist_sampled_kernel<<<grid, kHistThreads, smem, s>>>(samples, count, bits, thr, sel_seed, hist);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_hmin_finalize(const unsigned long long* hist, int bits, double eps, DevHminResult* out,
                                 cudaStream_t s, uint32_t* kernels, double var_sub, double h_ref) {
  hmin_finalize_kernel<<<1, kFinThreads, 0, s>>>(hist, bits, eps, out, var_sub, h_ref);
  ++*kernels;
  return cudaGetLastError();
}

}  // namespace qrng
