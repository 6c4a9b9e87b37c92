// Min-entropy estimate of an ADC sample stream (Sec. II of the paper):
//   1. exact histogram of the codes (privatised shared-memory counters, one pass over HBM);
//   2. an FP64 finaliser in two kernels: exact integer moments, H_min of the measured distribution
//      (Sec. II.A) and the Gaussian model fixed by the measured mean and variance (Sec. II.B) in
//      one CTA; the model cells, the statistical distance d_U, the finite-size term, Delta H_m and
//      H_modify (Sec. II.C) over many CTAs (FP64 runs at a few operations per clock per SM).
#include <cooperative_groups.h>
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
// adds to the out-of-range total. One shared-memory atomic per sample: on GB300 the atomics, at
// about 9 per clock per SM, bound the kernel (copies per lane, which remove every bank conflict and
// every collision inside a warp, were measured slower: they cost occupancy and instructions).
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

// Sample i of a little-endian uint16 stream at any byte address (two byte loads when it is odd).
__device__ __forceinline__ uint32_t load_u16(const void* __restrict__ p, uint64_t i, bool odd) {
  if (!odd) return __ldcs(static_cast<const uint16_t*>(p) + i);
  const uint8_t* b = static_cast<const uint8_t*>(p) + 2 * i;
  return (uint32_t)__ldcs(b) | ((uint32_t)__ldcs(b + 1) << 8);
}

// 9 <= bits <= 13: one shared histogram per CTA (<= 8192 counters + one out-of-range counter).
__global__ void __launch_bounds__(kHistThreads) hist_u16_smem_kernel(const void* __restrict__ samples,
                                                                      uint64_t count, int bits,
                                                                      unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t shc[];
  const uint32_t K = 1u << bits;
  const bool odd = reinterpret_cast<uintptr_t>(samples) & 1;
  for (uint32_t i = threadIdx.x; i <= K; i += blockDim.x) shc[i] = 0;
  __syncthreads();
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t s = tid; s < count; s += nthreads) {
    uint32_t v = load_u16(samples, s, odd);
    atomicAdd(&shc[v < K ? v : K], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b <= K; b += blockDim.x)
    if (shc[b]) atomicAdd(&hist[b], (unsigned long long)shc[b]);
}

// 14 <= bits <= 16: every CTA counts all 2^bits codes in shared memory as 16-bit halves of 32-bit
// words (2^15 words for 16 bits), one atomic per sample. A half that wraps past 0xffff is fixed up
// at once: the atomic's old value shows the wrap, so exactly one thread takes the 2^16 out of the
// word (a carry into the upper half is subtracted) and adds it to the global counter. Two CTAs form
// a cluster: after a cluster barrier each adds one half of the codes over both CTAs' shared
// memory (distributed shared-memory loads) to the global histogram, so only one flush per pair of
// SMs reaches global atomics. No scratch beyond the 2^bits + 1 output counters.
constexpr int kH16Threads = 1024;

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kH16Threads, 1)
    hist_u16_cluster_kernel(const void* __restrict__ samples_v, uint64_t count, int bits,
                            unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t shw[];  // 2^(bits-1) words, codes 2w and 2w+1
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const uint32_t K = 1u << bits, W = K / 2;
  for (uint32_t i = threadIdx.x; i < W; i += blockDim.x) shw[i] = 0u;
  cluster.sync();
  unsigned long long bad = 0;
  auto add = [&](uint32_t v) {
    if (v >= K) {
      ++bad;
      return;
    }
    const uint32_t sh = (v & 1u) << 4;
    const uint32_t old = atomicAdd(&shw[v >> 1], 1u << sh);
    if (((old >> sh) & 0xffffu) == 0xffffu) {  // this add wrapped the half: move 2^16 to global memory
      if (sh == 0) atomicSub(&shw[v >> 1], 0x10000u);
      atomicAdd(&hist[v], 65536ull);
    }
  };
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  if (reinterpret_cast<uintptr_t>(samples_v) & 1) {  // an odd address: one sample from two bytes at a time
    for (uint64_t i = tid; i < count; i += nthreads) add(load_u16(samples_v, i, true));
    count = 0;
  }
  const uint16_t* samples = static_cast<const uint16_t*>(samples_v);
  const uint64_t head = ((16 - (reinterpret_cast<uintptr_t>(samples) & 15)) & 15) / 2;
  const uint64_t nhead = head < count ? head : count;
  if (tid < nhead) add(samples[tid]);
  const uint64_t nvec = (count - nhead) / 8;
  const uint4* vec = reinterpret_cast<const uint4*>(samples + nhead);
  for (uint64_t v = tid; v < nvec; v += 2 * nthreads) {
    const uint4 x0 = __ldcs(vec + v);
    const uint4 x1 = v + nthreads < nvec ? __ldcs(vec + v + nthreads) : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t w0[4] = {x0.x, x0.y, x0.z, x0.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      add(w0[q] & 0xffffu);
      add(w0[q] >> 16);
    }
    if (v + nthreads < nvec) {
      const uint32_t w1[4] = {x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        add(w1[q] & 0xffffu);
        add(w1[q] >> 16);
      }
    }
  }
  const uint64_t tail0 = nhead + nvec * 8;
  if (tail0 + tid < count) add(samples[tail0 + tid]);
  if (bad) atomicAdd(&hist[K], bad);
  cluster.sync();  // both CTAs' counts are complete
  const uint32_t r = cluster.block_rank(), per = W / 2;
  const uint32_t* mine = shw;
  const uint32_t* peer = cluster.map_shared_rank(shw, r ^ 1u);
  for (uint32_t i = threadIdx.x; i < per; i += blockDim.x) {
    const uint32_t wi = r * per + i;
    const uint32_t a = mine[wi], b = peer[wi];
    const uint32_t lo = (a & 0xffffu) + (b & 0xffffu), hi = (a >> 16) + (b >> 16);
    if (lo) atomicAdd(&hist[2 * wi], (unsigned long long)lo);
    if (hi) atomicAdd(&hist[2 * wi + 1], (unsigned long long)hi);
  }
  cluster.sync();  // the peer has read this CTA's counts before either exits
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

// Pass 1, one CTA: count, exact first and second moments (128-bit integers), largest bin (lowest
// code on ties), mean, population variance, the model's sigma (and the quantum model's), the
// report's integer and moment fields and its status; clears the accumulators of pass 2.
__global__ void __launch_bounds__(kFinThreads) hmin_moments_kernel(const unsigned long long* __restrict__ hist,
                                                                    int bits, DevHminResult* __restrict__ out,
                                                                    double var_sub) {
  constexpr int kWarps = kFinThreads / 32;
  __shared__ unsigned long long w_n[kWarps], w_max[kWarps];
  __shared__ uint32_t w_arg[kWarps];
  __shared__ u128_t w_s1[kWarps], w_s2[kWarps];
  const uint32_t K = 1u << bits;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
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
  if (t != 0) return;
  unsigned long long N = 0, M = 0;
  uint32_t A = 0xffffffffu;
  u128_t S1 = 0, S2 = 0;
  for (int w = 0; w < kWarps; ++w) {
    N += w_n[w]; S1 += w_s1[w]; S2 += w_s2[w];
    max_arg_merge(M, A, w_max[w], w_arg[w]);
  }
  out->n = N;
  out->out_of_range = hist[K];
  out->pmax_bits = 0;
  out->pmax_full_bits = 0;
  out->dsum_fixed = 0;
  out->p_argmax = 0.0;
  out->done = 0;
  if (N == 0) {
    out->status = QRNG_EINVAL;
    return;
  }
  const u128_t num = (u128_t)N * S2 - S1 * S1;  // N^2 * population variance, exact
  const double mu = (double)S1 / (double)N;
  const double var = (double)num / ((double)N * (double)N);
  const double var_q = var - var_sub;
  const int bad_sub = (var_sub > 0.0) && !(var_q > 0.0);
  out->mu = mu;
  out->sigma = sqrt(var);
  out->point = (num == 0);
  out->bad_sub = bad_sub;
  out->sigma_q = var_sub > 0.0 && var_q > 0.0 ? sqrt(var_q) : out->sigma;
  qrng_hmin_report& r = out->rep;
  r.count = N;
  r.max_count = M;
  r.argmax = A;
  r.bits = (uint32_t)bits;
  r.mean = mu;
  r.var = (var_sub > 0.0 && !bad_sub) ? var_q : var;
  r.h_emp = -log2((double)M / (double)N);
  out->status = (hist[K] || bad_sub) ? QRNG_EINVAL : QRNG_OK;
}

constexpr int kCellThreads = 64;  // model cells per CTA of pass 2

// Cell v = c0 + threadIdx.x of the model N(mu, sg^2) (boundaries v +- 1/2, end codes take the
// tails): the CTA's kCellThreads + 1 boundary tails are computed once into s_tail.
__device__ __forceinline__ double cta_cell(uint32_t c0, uint32_t K, double mu, double sg, double* s_tail) {
  for (uint32_t i = threadIdx.x; i <= (uint32_t)kCellThreads; i += blockDim.x) {
    const int64_t j = (int64_t)c0 - 1 + i;  // boundary j lies between codes j and j + 1
    const double z = (j < 0 || j >= (int64_t)K - 1) ? CUDART_INF : (((double)j + 0.5 - mu) / sg);
    s_tail[i] = erfc(fabs(z) * M_SQRT1_2);
  }
  __syncthreads();
  const uint32_t v = c0 + threadIdx.x;
  double P = 0.0;
  if (v < K) {
    const double lo = (v == 0) ? -CUDART_INF : ((double)v - 0.5 - mu) / sg;
    const double hi = (v == K - 1) ? CUDART_INF : ((double)v + 0.5 - mu) / sg;
    P = cell_from_tails(lo, hi, s_tail[threadIdx.x], s_tail[threadIdx.x + 1]);
  }
  __syncthreads();
  return P;
}

// Pass 2, ceil(K / kCellThreads) CTAs (the FP64 tails spread over the SMs): model cells, their
// maximum and the distance to the measured distribution, folded into the result by atomics (the
// distance as a 2^-62 fixed-point integer, so the sum does not depend on the order of the CTAs);
// the last CTA to finish completes the report.
__global__ void __launch_bounds__(kCellThreads) hmin_cells_kernel(const unsigned long long* __restrict__ hist,
                                                                   int bits, double eps,
                                                                   DevHminResult* __restrict__ out, double var_sub,
                                                                   double h_ref) {
  __shared__ double s_tail[kCellThreads + 1];
  __shared__ double s_pm[kCellThreads / 32], s_pf[kCellThreads / 32];
  __shared__ unsigned long long s_ds[kCellThreads / 32];
  __shared__ int s_last;
  const uint32_t K = 1u << bits;
  const unsigned long long N = out->n;
  if (N == 0) return;
  const double mu = out->mu, sigma = out->sigma;
  const uint32_t amax = out->rep.argmax;
  const bool sub = var_sub > 0.0 && !out->bad_sub;
  const uint32_t c0 = blockIdx.x * kCellThreads, v = c0 + threadIdx.x;
  double P;
  if (out->point) {  // every sample on one code: the model is that point mass
    P = (v < K && v == amax) ? 1.0 : 0.0;
  } else {
    P = cta_cell(c0, K, mu, sigma, s_tail);
  }
  double pf = P, pm = P;
  unsigned long long ds = 0;
  if (v < K) {
    ds = (unsigned long long)llrint(fabs((double)hist[v] / (double)N - P) * 0x1p62);
    if (v == amax) out->p_argmax = out->point ? 1.0 : P;
  }
  if (sub && !out->point) pm = cta_cell(c0, K, mu, out->sigma_q, s_tail);
  for (int d = 16; d > 0; d >>= 1) {
    pm = fmax(pm, __shfl_down_sync(0xffffffffu, pm, d));
    pf = fmax(pf, __shfl_down_sync(0xffffffffu, pf, d));
    ds += __shfl_down_sync(0xffffffffu, ds, d);
  }
  if ((threadIdx.x & 31) == 0) {
    s_pm[threadIdx.x >> 5] = pm;
    s_pf[threadIdx.x >> 5] = pf;
    s_ds[threadIdx.x >> 5] = ds;
  }
  __threadfence();  // p_argmax before the ticket
  __syncthreads();
  if (threadIdx.x == 0) {
    double PM = 0.0, PF = 0.0;
    unsigned long long DS = 0;
    for (int w = 0; w < kCellThreads / 32; ++w) {
      PM = fmax(PM, s_pm[w]);
      PF = fmax(PF, s_pf[w]);
      DS += s_ds[w];
    }
    atomicMax(&out->pmax_bits, (unsigned long long)__double_as_longlong(PM));  // non-negative doubles
    atomicMax(&out->pmax_full_bits, (unsigned long long)__double_as_longlong(PF));
    atomicAdd(&out->dsum_fixed, DS);
    __threadfence();
    s_last = atomicAdd(&out->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  const double PM = __longlong_as_double((long long)atomicAdd(&out->pmax_bits, 0ull));
  const double PF = __longlong_as_double((long long)atomicAdd(&out->pmax_full_bits, 0ull));
  const double DS = (double)atomicAdd(&out->dsum_fixed, 0ull) * 0x1p-62;
  const double pa = *(volatile double*)&out->p_argmax;
  qrng_hmin_report& r = out->rep;
  r.h_model = -log2(PM);
  out->h_subtracted = -log2(PF) - h_ref;
  r.d_u = 0.5 * DS;
  r.d_u_peak = 0.5 * fabs((double)r.max_count / (double)N - pa);
  r.delta_fs = 0.5 * sqrt(2.0 * ((double)K * M_LN2 + log(1.0 / eps)) / (double)N);
  r.delta_hm = log2((r.d_u + r.delta_fs) * ldexp(1.0, bits + 1) + 1.0);
  const double h = r.h_model - r.delta_hm;
  r.h_modify = h > 0.0 ? h : 0.0;
  // leave the accumulators at zero for the next finaliser on this buffer (the fused kernel below
  // does not clear them first)
  out->pmax_bits = 0;
  out->pmax_full_bits = 0;
  out->dsum_fixed = 0;
  out->done = 0;
}

// ------------------------------------------------------------------------------------------------
// Fused finaliser for up to 2^kSmallMaxBits codes: ceil(K / kSmallCells) CTAs of one warp. Every
// CTA recomputes the exact integer moments and the largest bin from the (small) histogram, so no
// second launch hands them over; lanes 0 .. kSmallCells evaluate the CTA's boundary tails at once,
// lanes below kSmallCells its cells. The accumulators (largest cells, distance sum, CTA count)
// are zero on entry -- every finaliser leaves them so -- and the last CTA completes the report
// with its final logarithms on separate lanes.
// ------------------------------------------------------------------------------------------------
constexpr int kSmallMaxBits = 10;
constexpr int kSmallCells = 16;

__device__ __forceinline__ u128_t shfl_xor_u128(u128_t v, int d) {
  const uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)v, d);
  const uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(v >> 64), d);
  return ((u128_t)hi << 64) | lo;
}

// Cell v = c0 + lane of N(mu, sg^2) for lanes below kSmallCells (boundaries v +- 1/2, end codes
// take the tails); lane i <= kSmallCells computes the tail of boundary c0 - 1 + i.
__device__ __forceinline__ double warp_cell(uint32_t c0, uint32_t K, double mu, double sg, uint32_t lane) {
  const int64_t j = (int64_t)c0 - 1 + lane;  // boundary j lies between codes j and j + 1
  const double z = (lane > (uint32_t)kSmallCells || j < 0 || j >= (int64_t)K - 1) ? CUDART_INF
                                                                                  : (((double)j + 0.5 - mu) / sg);
  const double t = erfc(fabs(z) * M_SQRT1_2);
  const double t_hi = __shfl_down_sync(0xffffffffu, t, 1);
  const uint32_t v = c0 + lane;
  double P = 0.0;
  if (lane < (uint32_t)kSmallCells && v < K) {
    const double lo = (v == 0) ? -CUDART_INF : ((double)v - 0.5 - mu) / sg;
    const double hi = (v == K - 1) ? CUDART_INF : ((double)v + 0.5 - mu) / sg;
    P = cell_from_tails(lo, hi, t, t_hi);
  }
  return P;
}

__global__ void __launch_bounds__(32) hmin_small_kernel(const unsigned long long* __restrict__ hist, int bits,
                                                        double eps, DevHminResult* __restrict__ out, double var_sub,
                                                        double h_ref) {
  const uint32_t K = 1u << bits;
  const uint32_t lane = threadIdx.x;
  // exact count, first and second moments (128-bit integers), largest bin (lowest code on ties)
  unsigned long long n = 0, mx = 0;
  uint32_t arg = 0xffffffffu;
  u128_t s1 = 0, s2 = 0;
  for (uint32_t v = lane; v < K; v += 32) {
    const unsigned long long h = hist[v];
    n += h;
    s1 += (u128_t)v * h;
    s2 += (u128_t)((unsigned long long)v * v) * h;
    if (arg == 0xffffffffu || h > mx) {  // codes visited in increasing order: ties keep the lowest
      mx = h;
      arg = v;
    }
  }
  for (int d = 16; d > 0; d >>= 1) {  // butterfly: every lane ends with the totals
    n += __shfl_xor_sync(0xffffffffu, n, d);
    s1 += shfl_xor_u128(s1, d);
    s2 += shfl_xor_u128(s2, d);
    max_arg_merge(mx, arg, __shfl_xor_sync(0xffffffffu, mx, d), __shfl_xor_sync(0xffffffffu, arg, d));
  }
  const unsigned long long N = n;
  const unsigned long long oor = hist[K];
  if (N == 0) {
    if (blockIdx.x == 0 && lane == 0) {
      out->n = 0;
      out->out_of_range = oor;
      out->status = QRNG_EINVAL;
    }
    return;
  }
  const u128_t num = (u128_t)N * s2 - s1 * s1;  // N^2 * population variance, exact
  const double mu = (double)s1 / (double)N;
  const double var = (double)num / ((double)N * (double)N);
  const double var_q = var - var_sub;
  const bool bad_sub = (var_sub > 0.0) && !(var_q > 0.0);
  const bool point = (num == 0);
  const double sigma = sqrt(var);
  const double sigma_q = var_sub > 0.0 && var_q > 0.0 ? sqrt(var_q) : sigma;
  const bool sub = var_sub > 0.0 && !bad_sub;
  const uint32_t c0 = blockIdx.x * kSmallCells, v = c0 + lane;

  double P;
  if (point)  // every sample on one code: the model is that point mass
    P = (lane < (uint32_t)kSmallCells && v < K && v == arg) ? 1.0 : 0.0;
  else
    P = warp_cell(c0, K, mu, sigma, lane);
  double pf = P, pm = P;
  unsigned long long ds = 0;
  if (lane < (uint32_t)kSmallCells && v < K) {
    ds = (unsigned long long)llrint(fabs((double)hist[v] / (double)N - P) * 0x1p62);
    if (v == arg) out->p_argmax = P;
  }
  if (sub && !point) pm = warp_cell(c0, K, mu, sigma_q, lane);
  // the finite-size term depends on N, K and eps only: computed before the hand-over
  const double delta_fs = 0.5 * sqrt(2.0 * ((double)K * M_LN2 + log(1.0 / eps)) / (double)N);
  for (int d = 16; d > 0; d >>= 1) {
    pm = fmax(pm, __shfl_xor_sync(0xffffffffu, pm, d));
    pf = fmax(pf, __shfl_xor_sync(0xffffffffu, pf, d));
    ds += __shfl_xor_sync(0xffffffffu, ds, d);
  }
  uint32_t last = 0;
  if (lane == 0) {
    atomicMax(&out->pmax_bits, (unsigned long long)__double_as_longlong(pm));  // non-negative doubles
    atomicMax(&out->pmax_full_bits, (unsigned long long)__double_as_longlong(pf));
    atomicAdd(&out->dsum_fixed, ds);
    __threadfence();
    last = atomicAdd(&out->done, 1u) == gridDim.x - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence();
  const double PM = __longlong_as_double((long long)*(volatile unsigned long long*)&out->pmax_bits);
  const double PF = __longlong_as_double((long long)*(volatile unsigned long long*)&out->pmax_full_bits);
  const double d_u = 0.5 * (double)*(volatile unsigned long long*)&out->dsum_fixed * 0x1p-62;
  const double pa = *(volatile double*)&out->p_argmax;
  // the four logarithms of the report at once, one per lane
  const double larg = lane == 0 ? PM : lane == 1 ? PF : lane == 2 ? (double)mx / (double)N
                                                                    : (d_u + delta_fs) * ldexp(1.0, bits + 1) + 1.0;
  const double lg = log2(larg);
  const double l_pm = __shfl_sync(0xffffffffu, lg, 0), l_pf = __shfl_sync(0xffffffffu, lg, 1);
  const double l_emp = __shfl_sync(0xffffffffu, lg, 2), l_hm = __shfl_sync(0xffffffffu, lg, 3);
  __syncwarp();
  if (lane != 0) return;
  qrng_hmin_report& r = out->rep;
  out->n = N;
  out->out_of_range = oor;
  out->mu = mu;
  out->sigma = sigma;
  out->sigma_q = sigma_q;
  out->point = point;
  out->bad_sub = bad_sub;
  r.count = N;
  r.max_count = mx;
  r.argmax = arg;
  r.bits = (uint32_t)bits;
  r.mean = mu;
  r.var = sub ? var_q : var;
  r.h_emp = -l_emp;
  r.h_model = -l_pm;
  out->h_subtracted = -l_pf - h_ref;
  r.d_u = d_u;
  r.d_u_peak = 0.5 * fabs((double)mx / (double)N - pa);
  r.delta_fs = delta_fs;
  r.delta_hm = l_hm;
  const double h = r.h_model - r.delta_hm;
  r.h_modify = h > 0.0 ? h : 0.0;
  out->status = (oor || bad_sub) ? QRNG_EINVAL : QRNG_OK;
  out->pmax_bits = 0;
  out->pmax_full_bits = 0;
  out->dsum_fixed = 0;
  out->done = 0;
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
    const uint32_t v = bits <= 8 ? static_cast<const uint8_t*>(samples)[s]
                                 : load_u16(samples, s, reinterpret_cast<uintptr_t>(samples) & 1);
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

// Output length of a pipeline call from the finaliser's report (Sec. III.B: m = n H / bits less
// the leftover-hash term), for a hash enqueued before the host reads the report. One thread; the
// operations are rounded one by one (no contraction), as in the host's computation of m, so both
// sides find the same m.
__global__ void pipeline_size_kernel(const DevHminResult* __restrict__ res, uint64_t n, int bits, double lhl_term,
                                     uint64_t m_cap, uint64_t seed_cap, uint64_t out_cap, uint64_t nb,
                                     DevSpec* __restrict__ spec) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int st = 0;
  uint64_t m = 0;
  if (res->out_of_range != 0 || res->status != 0) {
    st = 2;
  } else {
    const double x = __dsub_rn(__ddiv_rn(__dmul_rn((double)n, res->rep.h_modify), (double)bits), lhl_term);
    if (x > 0.0) m = (uint64_t)floor(x);
    if (m > n) m = n;
    if (m == 0 || seed_cap < n + m - 1 || out_cap < (nb * m + 7) / 8)
      st = 2;
    else if (m > m_cap || m < kSpecMinBits)
      st = 1;
  }
  spec->m = m;
  spec->mw = (uint32_t)((m + 31) / 32);
  spec->status = st;
}

}  // namespace

cudaError_t launch_histogram(const void* samples, uint64_t count, int bits, unsigned long long* hist, int num_sms,
                             cudaStream_t s, uint32_t* kernels) {
  const uint32_t K = 1u << bits;
  cudaError_t e = cudaMemsetAsync(hist, 0, (K + 1) * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (bits <= 8) {
    const uint64_t want = ceil_div(count, 16ull * kHistThreads * 8);
    const uint64_t cap = (uint64_t)num_sms * 6;
    const int grid = (int)(want < cap ? (want ? want : 1) : cap);
    hist_u8_kernel<<<grid, kHistThreads, 0, s>>>(static_cast<const uint8_t*>(samples), count, bits, hist);
    ++*kernels;
    return cudaGetLastError();
  }
  if (bits <= 13) {
    const uint64_t want = ceil_div(count, (uint64_t)kHistThreads * 16);
    const uint64_t cap = (uint64_t)num_sms * 4;
    const int grid = (int)(want < cap ? (want ? want : 1) : cap);
    hist_u16_smem_kernel<<<grid, kHistThreads, (K + 1) * sizeof(uint32_t), s>>>(samples, count, bits, hist);
    ++*kernels;
    return cudaGetLastError();
  }
  // 14..16 bits: one CTA per SM, clusters of two (an even grid)
  const size_t smem = (K / 2) * sizeof(uint32_t);
  if ((e = cudaFuncSetAttribute(hist_u16_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  const uint64_t want = ceil_div(count, (uint64_t)kH16Threads * 16);
  uint64_t grid = (uint64_t)(num_sms > 1 ? num_sms : 2) & ~1ull;
  if (want < grid) grid = want < 2 ? 2 : (want + 1) & ~1ull;
  hist_u16_cluster_kernel<<<(unsigned)grid, kH16Threads, smem, s>>>(samples, count, bits, hist);
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
  if (bits <= kSmallMaxBits) {
    const uint32_t ctas = (uint32_t)ceil_div(1u << bits, (uint64_t)kSmallCells);
    hmin_small_kernel<<<ctas, 32, 0, s>>>(hist, bits, eps, out, var_sub, h_ref);
    ++*kernels;
    return cudaGetLastError();
  }
  hmin_moments_kernel<<<1, kFinThreads, 0, s>>>(hist, bits, out, var_sub);
  ++*kernels;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint32_t K = 1u << bits;
  hmin_cells_kernel<<<(unsigned)ceil_div(K, (uint64_t)kCellThreads), kCellThreads, 0, s>>>(hist, bits, eps, out,
                                                                                            var_sub, h_ref);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_pipeline_size(const DevHminResult* res, uint64_t n, int bits, double lhl_term, uint64_t m_cap,
                                 uint64_t seed_capacity_bits, uint64_t out_capacity_bytes, uint64_t num_blocks,
                                 DevSpec* spec, cudaStream_t s, uint32_t* kernels) {
  pipeline_size_kernel<<<1, 32, 0, s>>>(res, n, bits, lhl_term, m_cap, seed_capacity_bits, out_capacity_bytes,
                                        num_blocks, spec);
  ++*kernels;
  return cudaGetLastError();
}

}  // namespace qrng
