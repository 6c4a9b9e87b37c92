// FFT32_SEG: the Toeplitz part of the hash (Sec. III.B-D) as a sum of short FP32 cyclic
// convolutions whose results are rounded to their exact integers and reduced to parities.
//
// Raw segment s holds raw bits r_s = r[sS, (s+1)S); output tile q holds outputs [qS, (q+1)S).
// The part of k_i (i = qS + i') that segment s contributes is (w_d * r_s)[i' + S - 1], where * is
// the linear convolution and w_d[v] = a[n_t - 1 + dS - S + 1 + v] (v < 2S - 1, zero outside the
// seed) is the seed window of d = q - s. A cyclic convolution of length N = 2S leaves those
// entries free of wrap-around, so with W_d and R_s the length-N spectra, tile q's sums are
// F^-1(sum_s W_{q-s} R_s) at [S-1, 2S-1): the sum over segments can be taken in the frequency
// domain, and each segment and each window is transformed once per call.
//
// Every real length-N transform is an S-point complex FFT of z[n] = x[2n] + i x[2n+1] plus one
// split step (X[k] = E[k] + e^{-2 pi i k / N} O[k] with E, O the spectra of the even and odd
// samples), so only the S half-spectrum bins are stored and multiplied (DC and Nyquist, both
// real, share bin 0 as its real and imaginary part); the inverse runs the same steps backwards.
//
// Exactness: for FP32 (unit roundoff u = 2^-24) and radix-2^k transforms with twiddles within
// beta = u/2, Percival's bound for FFT-based convolution puts every result within
// |x| |y| eps_k of its exact value, eps_k = (1+u)^{3k} (1+sqrt5 u)^{3k+1} (1+beta)^{3k} - 1, k =
// log2 N (the S-point transform and its split step make k levels). A window has at most 2S - 1
// ones and a segment at most S, so one product term is off by at most sqrt((2S-1) S) eps_k; T
// terms summed before one inverse add T sqrt((2S-1) S) (eps_k + T u). T is the largest count that
// keeps this below 0.45: every rounded sum is then the exact integer, and the parities of the
// ceil(NS / T) inverses of a tile XOR together into the hash (addition mod 2 is linear). Every
// launch also reduces the observed max |sum - round(sum)| (a sum of 2^20 or more, whose FP32
// spacing hides that distance, counts as 1); if it reaches 0.25 (possible only when a caller
// forces T past the bound) a flag makes the exact direct kernel recompute the call.
//
// Kernels: seg_spectra_kernel (the window spectra once per call; the segment spectra per chunk
// of blocks, written to workspace) and seg_mac_kernel (one CTA per block and group of Q tiles:
// T-term products accumulated in registers, then per tile the inverse transform in shared
// memory, rounding, parity, XOR into the tile's bits).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qrng_internal.h"

namespace qrng {
namespace {

constexpr float kGuard = 0.25f;

// Threads of a CTA for S = 2^LOG_S (one radix-16 butterfly each per pass), resident CTAs per SM,
// and the most tiles a multiply-and-inverse CTA accumulates at once (Q x BINS complex registers).
template <int LOG_S>
struct SegCfg {
  static constexpr int S = 1 << LOG_S;
  static constexpr int THREADS = S / 16;
  static constexpr int BINS = 16;
  static constexpr int MIN_CTAS = 512 / THREADS;  // 512 resident threads per SM: at most 128 registers each
  static constexpr int QMAX = 2;
};
constexpr uint64_t kSpecBudget = 256ull << 20;  // bytes of segment spectra per chunk of blocks

// Shared-memory index of transform entry i: one pad entry after every 32, so that the strided
// writes of the first Stockham passes (consecutive butterflies 16 entries apart) spread over the
// banks instead of landing on one. A buffer of S entries takes SPAD(S) slots.
__host__ __device__ constexpr int SPAD(int i) { return i + (i >> 5); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// (DIR i) * a
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
  return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// tw[t] = exp(-2 pi i t / N) for t < S (N = 2S), rounded once from FP64.
__global__ void seg_twiddle_kernel(float2* __restrict__ tw, int S) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S) return;
  double s, c;
  sincospi(-(double)t / (double)S, &s, &c);
  tw[t] = make_float2((float)c, (float)s);
}

// exp(DIR 2 pi i t / S) for 0 <= t < S from the length-N table.
template <int S, int DIR>
__device__ __forceinline__ float2 root_s(const float2* __restrict__ tw, int t) {
  float2 w = t < S / 2 ? __ldg(tw + 2 * t) : make_float2(-__ldg(tw + 2 * t - S).x, -__ldg(tw + 2 * t - S).y);
  return DIR > 0 ? cconj(w) : w;
}

template <int DIR>
__device__ __forceinline__ void dft2(float2* b) {
  const float2 t = b[1];
  b[1] = csub(b[0], t);
  b[0] = cadd(b[0], t);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2* b) {  // y[r] = sum_q b[q] exp(DIR 2 pi i q r / 4)
  const float2 s02 = cadd(b[0], b[2]), d02 = csub(b[0], b[2]);
  const float2 s13 = cadd(b[1], b[3]), d13 = mul_i<DIR>(csub(b[1], b[3]));
  b[0] = cadd(s02, s13);
  b[2] = csub(s02, s13);
  b[1] = cadd(d02, d13);
  b[3] = csub(d02, d13);
}

template <int DIR>
__device__ __forceinline__ void dft8(float2* b) {  // y[r] = sum_q b[q] exp(DIR 2 pi i q r / 8)
  float2 e[4] = {b[0], b[2], b[4], b[6]}, o[4] = {b[1], b[3], b[5], b[7]};
  dft4<DIR>(e);
  dft4<DIR>(o);
  const float h = 0.70710678118654752f;
  // o[r] *= exp(DIR 2 pi i r / 8)
  o[1] = make_float2(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
  o[2] = mul_i<DIR>(o[2]);
  o[3] = make_float2(h * (-o[3].x - DIR * o[3].y), h * (-o[3].y + DIR * o[3].x));
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    b[r] = cadd(e[r], o[r]);
    b[r + 4] = csub(e[r], o[r]);
  }
}

// y[r] = sum_q b[q] exp(DIR 2 pi i q r / 16) as 4 x 4: DFT4 over q1 of b[4 q1 + q2], times
// exp(DIR 2 pi i q2 r1 / 16), then DFT4 over q2 into y[r1 + 4 r2].
template <int DIR>
__device__ __forceinline__ void dft16(float2* b) {
  float2 c[4][4];
#pragma unroll
  for (int q2 = 0; q2 < 4; ++q2) {
    float2 t[4] = {b[q2], b[4 + q2], b[8 + q2], b[12 + q2]};
    dft4<DIR>(t);
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) c[q2][r1] = t[r1];
  }
  const float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  // exp(DIR 2 pi i k / 16) = (C_k, DIR S_k) for k = q2 r1 in {1, 2, 3, 4, 6, 9}
  auto rot = [](float2 a, float C, float Sd) { return make_float2(a.x * C - a.y * Sd, a.x * Sd + a.y * C); };
  c[1][1] = rot(c[1][1], c1, DIR * s1);
  c[1][2] = rot(c[1][2], h, DIR * h);
  c[1][3] = rot(c[1][3], s1, DIR * c1);
  c[2][1] = rot(c[2][1], h, DIR * h);
  c[2][2] = mul_i<DIR>(c[2][2]);
  c[2][3] = rot(c[2][3], -h, DIR * h);
  c[3][1] = rot(c[3][1], s1, DIR * c1);
  c[3][2] = rot(c[3][2], -h, DIR * h);
  c[3][3] = rot(c[3][3], -c1, -DIR * s1);
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) {
    float2 t[4] = {c[0][r1], c[1][r1], c[2][r1], c[3][r1]};
    dft4<DIR>(t);
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) b[r1 + 4 * r2] = t[r2];
  }
}

// One in-place Stockham pass of radix R over the S points in shared memory, L = length of the
// sub-transforms done so far: butterfly j = iL + k reads x[j + q S/R] (q < R), multiplies input q
// by exp(DIR 2 pi i q k / (R L)), and writes output r to x[i R L + k + r L]. Every thread reads all
// its inputs before the barrier and writes after it, so one buffer suffices.
template <int S, int THREADS, int R, int DIR>
__device__ __forceinline__ void stockham_pass(float2* x, const float2* __restrict__ tw, int L) {
  constexpr int NB = S / R;
  constexpr int PER = NB / THREADS;
  float2 v[PER][R];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int j = threadIdx.x + p * THREADS;
#pragma unroll
    for (int q = 0; q < R; ++q) v[p][q] = x[SPAD(j + q * NB)];
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int j = threadIdx.x + p * THREADS;
    const int k = j & (L - 1);
    const int i = j / L;
    const int step = k * (S / (R * L));
#pragma unroll
    for (int q = 1; q < R; ++q) v[p][q] = cmul(v[p][q], root_s<S, DIR>(tw, q * step));
    if (R == 16) dft16<DIR>(v[p]);
    else if (R == 8) dft8<DIR>(v[p]);
    else if (R == 4) dft4<DIR>(v[p]);
    else dft2<DIR>(v[p]);
    const int y0 = i * R * L + k;
#pragma unroll
    for (int r = 0; r < R; ++r) x[SPAD(y0 + r * L)] = v[p][r];
  }
  __syncthreads();
}

// Unnormalised S-point complex FFT in shared memory (natural order in and out); callers
// synchronise before it.
template <int S, int THREADS, int DIR>
__device__ void fft_s(float2* x, const float2* __restrict__ tw) {
  int L = 1;
#pragma unroll 1
  while (L < S) {
    const int rest = S / L;
    if (rest >= 16) {
      stockham_pass<S, THREADS, 16, DIR>(x, tw, L);
      L *= 16;
    } else if (rest == 8) {
      stockham_pass<S, THREADS, 8, DIR>(x, tw, L);
      L *= 8;
    } else if (rest == 4) {
      stockham_pass<S, THREADS, 4, DIR>(x, tw, L);
      L *= 4;
    } else {
      stockham_pass<S, THREADS, 2, DIR>(x, tw, L);
      L *= 2;
    }
  }
}

struct SpecArgs {
  // raw segments of blocks [0, nb) (item = b NS + s) or, with seed != null, seed windows
  // d = dmin + item
  const uint32_t* raw;
  uint64_t raw_stride;
  uint64_t n_t;
  uint32_t NS;
  const uint8_t* seed;
  uint64_t L;
  int64_t D;     // n_t - 1
  int64_t dmin;  // -(NS - 1)
  uint64_t items;
  float2* spec;  // row `item` of S bins
  const float2* tw;
};

// Bits [base, base + 2S - 1) of a seed of L bits (zero outside it) as z[n] = x[2n] + i x[2n+1]
// into sx: the bytes are staged in shared memory first (one load per byte).
template <int S, int THREADS, int BINS>
__device__ __forceinline__ void stage_window(const uint8_t* __restrict__ seed, uint64_t L, int64_t base, float2* sx,
                                             uint8_t* sb) {
  const int64_t byte0 = base >= 0 ? base / 8 : -((-base + 7) / 8);
  const int64_t lbytes = (int64_t)((L + 7) / 8);
  for (int i = threadIdx.x; i < S / 4 + 2; i += THREADS) {
    const int64_t bi = byte0 + i;
    sb[i] = (bi >= 0 && bi < lbytes) ? __ldg(seed + bi) : (uint8_t)0;
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < BINS; ++p) {
    const int n = threadIdx.x + p * THREADS;
    float v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = 2 * n + h;
      const int64_t xi = base + u;
      v[h] = (u < 2 * S - 1 && xi >= 0 && xi < (int64_t)L) ? (float)((sb[(xi >> 3) - byte0] >> (xi & 7)) & 1u) : 0.f;
    }
    sx[SPAD(n)] = make_float2(v[0], v[1]);
  }
}

template <int LOG_S>
__global__ void __launch_bounds__(SegCfg<LOG_S>::THREADS, SegCfg<LOG_S>::MIN_CTAS) seg_spectra_kernel(const SpecArgs a) {
  constexpr int S = SegCfg<LOG_S>::S, THREADS = SegCfg<LOG_S>::THREADS, BINS = SegCfg<LOG_S>::BINS;
  extern __shared__ float2 sx[];
  uint32_t* sw = reinterpret_cast<uint32_t*>(sx + SPAD(S));  // staged input bits
  const uint64_t item = blockIdx.x;
  if (item >= a.items) return;
  // z[n] = x[2n] + i x[2n+1] of the real length-2S input
  if (a.seed) {
    const int64_t base = a.D + (a.dmin + (int64_t)item) * S - S + 1;
    stage_window<S, THREADS, BINS>(a.seed, a.L, base, sx, reinterpret_cast<uint8_t*>(sw));
  } else {
    const uint64_t b = item / a.NS, s = item - b * a.NS;
    const uint32_t* row = a.raw + b * a.raw_stride;
    const uint64_t w0 = s * (S / 32);
    for (int w = threadIdx.x; w < S / 32; w += THREADS) sw[w] = w0 + w < a.raw_stride ? __ldg(row + w0 + w) : 0u;
    __syncthreads();
#pragma unroll
    for (int p = 0; p < BINS; ++p) {
      const int n = threadIdx.x + p * THREADS;
      float v[2] = {0.f, 0.f};
      if (2 * n < S) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int u = 2 * n + h;
          v[h] = s * S + u < a.n_t ? (float)((sw[u >> 5] >> (u & 31)) & 1u) : 0.f;
        }
      }
      sx[SPAD(n)] = make_float2(v[0], v[1]);
    }
  }
  __syncthreads();
  fft_s<S, THREADS, -1>(sx, a.tw);
  // split: E = (Z_k + conj Z_{S-k}) / 2, O = (Z_k - conj Z_{S-k}) / (2i), X_k = E + exp(-2 pi i k / N) O
  float2* out = a.spec + item * S;
#pragma unroll
  for (int p = 0; p < BINS; ++p) {
    const int k = threadIdx.x + p * THREADS;
    const float2 zk = sx[SPAD(k)];
    float2 X;
    if (k == 0) {
      X = make_float2(zk.x + zk.y, zk.x - zk.y);  // (DC, Nyquist)
    } else {
      const float2 zm = cconj(sx[SPAD(S - k)]);
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
      const float2 d = csub(zk, zm);
      const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);
      X = cadd(e, cmul(__ldg(a.tw + k), o));
    }
    out[k] = X;
  }
}

struct MacArgs {
  const float2* spec_raw;  // (b NS + s) rows of S bins, blocks of this chunk
  const float2* spec_win;  // (d - dmin) rows
  const float2* tw;
  uint32_t NS, NQ, NQG, T;
  int64_t dmin;
  uint64_t nb;             // blocks in this chunk
  const uint32_t* raw;     // this chunk's first block (for the identity part)
  uint64_t raw_stride;
  uint32_t* out;           // this chunk's first block's output words
  uint64_t out_stride;
  uint32_t m, mw;
  int modified;
  uint32_t id_off;
  unsigned long long* worst;
  int* guard_flag;
};

// Tiles q0 .. q0+nq-1 (nq <= Q) of one block: for every group of T segments the products
// W_{q-s} R_s are summed in registers (this thread's BINS bins), then per tile the inverse split,
// the inverse transform in shared memory (sx, S bins), rounding, parity and XOR into the tile's
// bits (Q x S/32 words in shared memory, zeroed by the caller). R_s is row s of `segs`, W_d row
// d + NS - 1 of `wins`. Returns this thread's largest rounding distance.
template <int LOG_S, int Q>
__device__ float mac_tiles(const float2* __restrict__ segs, const float2* __restrict__ wins, uint32_t NS,
                           uint32_t q0, uint32_t nq, uint32_t T, const float2* __restrict__ tw, float2* sx,
                           uint32_t* bits) {
  constexpr int S = SegCfg<LOG_S>::S, THREADS = SegCfg<LOG_S>::THREADS, BINS = SegCfg<LOG_S>::BINS,
                WORDS = S / 32;
  const uint32_t lane = threadIdx.x & 31;
  float err = 0.f;
#pragma unroll 1
  for (uint32_t g0 = 0; g0 < NS; g0 += T) {
    const uint32_t g1 = min(NS, g0 + T);
    float2 acc[Q][BINS];
#pragma unroll
    for (int j = 0; j < Q; ++j)
#pragma unroll
      for (int p = 0; p < BINS; ++p) acc[j][p] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (uint32_t s = g0; s < g1; ++s) {
      float2 rv[BINS];
      const float2* R = segs + (uint64_t)s * S;
#pragma unroll
      for (int p = 0; p < BINS; ++p) rv[p] = R[threadIdx.x + p * THREADS];
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        if ((uint32_t)j >= nq) break;
        const float2* Wd = wins + (uint64_t)(q0 + j + NS - 1 - s) * S;
#pragma unroll
        for (int p = 0; p < BINS; ++p) {
          const float2 w = __ldg(Wd + threadIdx.x + p * THREADS);
          if (p == 0 && threadIdx.x == 0) {  // DC and Nyquist are real
            acc[j][p].x += w.x * rv[p].x;
            acc[j][p].y += w.y * rv[p].y;
          } else {
            acc[j][p].x += w.x * rv[p].x - w.y * rv[p].y;
            acc[j][p].y += w.x * rv[p].y + w.y * rv[p].x;
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      if ((uint32_t)j >= nq) break;
#pragma unroll
      for (int p = 0; p < BINS; ++p) sx[SPAD(threadIdx.x + p * THREADS)] = acc[j][p];
      __syncthreads();
      // inverse split: Z_k = E_k + i O_k, E = (X_k + conj X_{S-k}) / 2, O = (X_k - conj X_{S-k}) / 2 e^{+2 pi i k / N}
      float2 zv[BINS];
#pragma unroll
      for (int p = 0; p < BINS; ++p) {
        const int k = threadIdx.x + p * THREADS;
        float2 xk, xm;
        if (k == 0) {
          xk = make_float2(sx[SPAD(0)].x, 0.f);
          xm = make_float2(sx[SPAD(0)].y, 0.f);  // the Nyquist bin, partner of DC
        } else {
          xk = sx[SPAD(k)];
          xm = sx[SPAD(S - k)];
        }
        xm = cconj(xm);
        const float2 e = make_float2(0.5f * (xk.x + xm.x), 0.5f * (xk.y + xm.y));
        const float2 d = make_float2(0.5f * (xk.x - xm.x), 0.5f * (xk.y - xm.y));
        const float2 o = cmul(d, cconj(__ldg(tw + k)));
        zv[p] = make_float2(e.x - o.y, e.y + o.x);
      }
      __syncthreads();
#pragma unroll
      for (int p = 0; p < BINS; ++p) sx[SPAD(threadIdx.x + p * THREADS)] = zv[p];
      __syncthreads();
      fft_s<S, THREADS, +1>(sx, tw);
      // c[t], t = S - 1 + i': even t in z[t/2].x, odd t in z[(t-1)/2].y (scale 1/S)
      uint32_t* tb = bits + j * WORDS;
#pragma unroll
      for (int p = 0; p < BINS; ++p) {
        const int ip = threadIdx.x + p * THREADS;
        const int t = S - 1 + ip;
        const float2 z = sx[SPAD(t >> 1)];
        const float v = ((t & 1) ? z.y : z.x) * (1.0f / (float)S);
        const float r = rintf(v);
        // a sum of 2^20 or more (FP32 spacing 1/8 and coarser) cannot show its rounding distance:
        // it counts as a guard trip (the proven T keeps every sum below T S <= 2^15)
        err = fmaxf(err, fabsf(r) >= 1048576.f ? 1.f : fabsf(v - r));
        const uint32_t word = __ballot_sync(0xffffffffu, ((int)r) & 1);
        if (lane == 0) tb[ip >> 5] ^= word;
      }
      __syncthreads();
    }
  }
  return err;
}

// Largest value of `err` over the CTA, reported to *worst (and to *guard_flag when it reaches the guard).
template <int THREADS>
__device__ void report_err(float err, unsigned long long* worst, int* guard_flag) {
  __shared__ float s_err[THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) err = fmaxf(err, __shfl_xor_sync(0xffffffffu, err, o));
  if ((threadIdx.x & 31) == 0) s_err[threadIdx.x >> 5] = err;
  __syncthreads();
  if (threadIdx.x == 0) {
    float e = 0.f;
    for (int w = 0; w < THREADS / 32; ++w) e = fmaxf(e, s_err[w]);
    atomicMax(worst, (unsigned long long)__double_as_longlong((double)e));
    if (guard_flag && e >= kGuard) atomicExch(guard_flag, 1);
  }
}

template <int LOG_S, int Q>
__global__ void __launch_bounds__(SegCfg<LOG_S>::THREADS, SegCfg<LOG_S>::MIN_CTAS) seg_mac_kernel(const MacArgs a) {
  constexpr int S = SegCfg<LOG_S>::S, THREADS = SegCfg<LOG_S>::THREADS, WORDS = S / 32;
  extern __shared__ float2 sx[];
  uint32_t* bits = reinterpret_cast<uint32_t*>(sx + SPAD(S));  // Q x WORDS tile bits
  const uint64_t b = blockIdx.x / a.NQG;
  const uint32_t q0 = (uint32_t)(blockIdx.x - b * a.NQG) * Q;
  const uint32_t nq = min((uint32_t)Q, a.NQ - q0);
  for (int w = threadIdx.x; w < Q * WORDS; w += THREADS) bits[w] = 0u;
  __syncthreads();
  const float err = mac_tiles<LOG_S, Q>(a.spec_raw + b * a.NS * (uint64_t)S, a.spec_win, a.NS, q0, nq, a.T, a.tw,
                                        sx, bits);
  report_err<THREADS>(err, a.worst, a.guard_flag);
  const uint32_t* row = a.raw + b * a.raw_stride;
  for (int w = threadIdx.x; w < (int)nq * WORDS; w += THREADS) {
    const uint64_t ow = (uint64_t)q0 * WORDS + w;
    if (ow >= a.mw) continue;
    const uint32_t rem = a.m - 32 * (uint32_t)ow;
    const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    uint32_t word = bits[w] & omask;
    if (a.modified) {
      const uint64_t bit = (uint64_t)a.id_off + 32ull * ow;
      const uint64_t rq = bit >> 5;
      const uint32_t rs = (uint32_t)(bit & 31);
      const uint32_t lo = __ldg(row + rq);
      const uint32_t hi = (rs && rq + 1 < a.raw_stride) ? __ldg(row + rq + 1) : 0u;
      word ^= __funnelshift_r(lo, hi, rs) & omask;
    }
    a.out[b * a.out_stride + ow] = word;
  }
}

// ---- uneven batches: every request its own seed, windows and segments ----

__device__ __forceinline__ uint32_t byte_bit(const uint8_t* __restrict__ p, uint64_t bit) {
  return (__ldg(p + (bit >> 3)) >> (bit & 7)) & 1u;
}

// nbits <= 32 bits from bit `bit` of a byte buffer (LSB-first), reading only the bytes they span.
__device__ __forceinline__ uint32_t byte_bits(const uint8_t* __restrict__ p, uint64_t bit, uint32_t nbits) {
  const uint8_t* b = p + (bit >> 3);
  const uint32_t sh = (uint32_t)(bit & 7);
  const uint32_t nbytes = (sh + nbits + 7) >> 3;
  uint64_t v = 0;
  for (uint32_t k = 0; k < nbytes; ++k) v |= (uint64_t)__ldg(b + k) << (8 * k);
  v >>= sh;
  return nbits >= 32 ? (uint32_t)v : (uint32_t)v & ((1u << nbits) - 1u);
}

// Request of a group holding item `x` of a prefix-summed numbering (the last one starting at or before it).
template <uint64_t BatchReq::*F>
__device__ __forceinline__ uint32_t find_request(const BatchReq* __restrict__ reqs, uint32_t nr, uint64_t x) {
  uint32_t lo = 0, hi = nr - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (reqs[mid].*F <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One CTA per spectra item of a group: request r's windows d = -(NS-1) .. NQ-1 first, then its
// segments, each into row spec_row + local item.
template <int LOG_S>
__global__ void __launch_bounds__(SegCfg<LOG_S>::THREADS, SegCfg<LOG_S>::MIN_CTAS)
    seg_batch_spectra_kernel(const BatchReq* __restrict__ reqs, uint32_t nr, float2* __restrict__ spec,
                             const float2* __restrict__ tw) {
  constexpr int S = SegCfg<LOG_S>::S, THREADS = SegCfg<LOG_S>::THREADS, BINS = SegCfg<LOG_S>::BINS;
  extern __shared__ float2 sx[];
  uint8_t* sb = reinterpret_cast<uint8_t*>(sx + SPAD(S));  // staged input bytes
  const uint64_t item = blockIdx.x;
  const BatchReq& q = reqs[find_request<&BatchReq::spec_item_begin>(reqs, nr, item)];
  const uint64_t local = item - q.spec_item_begin;
  const uint64_t nw = (uint64_t)q.seg_nq + q.seg_ns - 1;
  if (local < nw) {
    const int64_t base = (int64_t)q.n_t - 1 + ((int64_t)local - (int64_t)(q.seg_ns - 1)) * S - S + 1;
    stage_window<S, THREADS, BINS>(q.seed, q.L_t, base, sx, sb);
  } else {
    // the segment's bits: only the bytes holding raw bits [sg S, min(n_t, (sg+1) S)) are read
    const uint64_t sg = local - nw;
    const uint64_t bit0 = q.raw_bit_off + sg * S;
    const uint64_t end = q.raw_bit_off + (q.n_t < (sg + 1) * S ? q.n_t : (sg + 1) * S);
    const uint64_t byte0 = bit0 >> 3, byte_end = (end + 7) >> 3;
    for (uint64_t i = threadIdx.x; i < (uint64_t)S / 8 + 1; i += THREADS)
      sb[i] = byte0 + i < byte_end ? __ldg(q.raw + byte0 + i) : (uint8_t)0;
    __syncthreads();
#pragma unroll
    for (int p = 0; p < BINS; ++p) {
      const int n = threadIdx.x + p * THREADS;
      float v[2] = {0.f, 0.f};
      if (2 * n < S) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint64_t u = 2 * n + h;
          const uint64_t g = bit0 + u;
          v[h] = sg * S + u < q.n_t ? (float)((sb[(g >> 3) - byte0] >> (g & 7)) & 1u) : 0.f;
        }
      }
      sx[SPAD(n)] = make_float2(v[0], v[1]);
    }
  }
  __syncthreads();
  fft_s<S, THREADS, -1>(sx, tw);
  float2* out = spec + (q.spec_row + local) * S;
#pragma unroll
  for (int p = 0; p < BINS; ++p) {
    const int k = threadIdx.x + p * THREADS;
    const float2 zk = sx[SPAD(k)];
    float2 X;
    if (k == 0) {
      X = make_float2(zk.x + zk.y, zk.x - zk.y);
    } else {
      const float2 zm = cconj(sx[SPAD(S - k)]);
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
      const float2 d = csub(zk, zm);
      const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);
      X = cadd(e, cmul(__ldg(tw + k), o));
    }
    out[k] = X;
  }
}

// One CTA per (request, group of Q tiles) of a group; output words into the request's staging.
template <int LOG_S, int Q>
__global__ void __launch_bounds__(SegCfg<LOG_S>::THREADS, SegCfg<LOG_S>::MIN_CTAS) seg_batch_mac_kernel(const BatchReq* __restrict__ reqs,
                                                                               uint32_t nr, const float2* __restrict__ spec,
                                                                               const float2* __restrict__ tw, uint32_t T,
                                                                               uint32_t* __restrict__ out_stage,
                                                                               unsigned long long* __restrict__ worst) {
  constexpr int S = SegCfg<LOG_S>::S, THREADS = SegCfg<LOG_S>::THREADS, WORDS = S / 32;
  extern __shared__ float2 sx[];
  uint32_t* bits = reinterpret_cast<uint32_t*>(sx + SPAD(S));
  const BatchReq& q = reqs[find_request<&BatchReq::mac_cta_begin>(reqs, nr, blockIdx.x)];
  const uint32_t q0 = (uint32_t)(blockIdx.x - q.mac_cta_begin) * Q;
  const uint32_t nq = min((uint32_t)Q, q.seg_nq - q0);
  for (int w = threadIdx.x; w < Q * WORDS; w += THREADS) bits[w] = 0u;
  __syncthreads();
  const float2* wins = spec + q.spec_row * S;
  const uint64_t nw = (uint64_t)q.seg_nq + q.seg_ns - 1;
  const float err = mac_tiles<LOG_S, Q>(wins + nw * S, wins, q.seg_ns, q0, nq, T, tw, sx, bits);
  report_err<THREADS>(err, worst, nullptr);
  for (int w = threadIdx.x; w < (int)nq * WORDS; w += THREADS) {
    const uint64_t ow = (uint64_t)q0 * WORDS + w;
    if (ow >= q.mw) continue;
    const uint64_t rem = q.m - 32 * ow;
    const uint32_t nb = rem >= 32 ? 32u : (uint32_t)rem;
    const uint32_t omask = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
    uint32_t word = bits[w] & omask;
    if (q.form == QRNG_FORM_MODIFIED) word ^= byte_bits(q.raw, q.raw_bit_off + q.id_off + 32 * ow, nb);
    out_stage[q.out_stage_off + ow] = word;
  }
}

template <int LOG_S>
size_t mac_smem(int Q) {
  return (size_t)SPAD(1 << LOG_S) * sizeof(float2) + (size_t)Q * ((1 << LOG_S) / 32) * sizeof(uint32_t);
}

template <int LOG_S, int Q>
cudaError_t launch_mac(const MacArgs& m, unsigned ctas, cudaStream_t s) {
  const size_t smem = mac_smem<LOG_S>(Q);
  cudaError_t e = cudaFuncSetAttribute(seg_mac_kernel<LOG_S, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  seg_mac_kernel<LOG_S, Q><<<ctas, SegCfg<LOG_S>::THREADS, smem, s>>>(m);
  return cudaGetLastError();
}

// the transform buffer and the staged input bits (S/4 + 2 bytes of a seed window at most)
template <int LOG_S>
size_t spectra_smem() {
  return (size_t)SPAD(1 << LOG_S) * sizeof(float2) + (size_t)(1 << LOG_S) / 4 + 16;
}

template <int LOG_S>
cudaError_t launch_spectra(const SpecArgs& sa, cudaStream_t s) {
  const size_t smem = spectra_smem<LOG_S>();
  cudaError_t e = cudaFuncSetAttribute(seg_spectra_kernel<LOG_S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (sa.items > 0x7fffffffull) return cudaErrorInvalidConfiguration;
  seg_spectra_kernel<LOG_S><<<(unsigned)sa.items, SegCfg<LOG_S>::THREADS, smem, s>>>(sa);
  return cudaGetLastError();
}

// Tiles per multiply-and-inverse CTA: as many as its accumulators hold (each segment spectrum the
// CTA loads then serves that many tiles).
int pick_q(uint32_t NQ, int qmax) { return (int)(NQ < (uint32_t)qmax ? NQ : (uint32_t)qmax); }

template <int LOG_S>
cudaError_t run_fft32(const DirectArgs& d, const uint8_t* seed, uint64_t L_t, int T, FftWorkspace& ws,
                      int* guard_flag, cudaStream_t s, uint32_t* kernels) {
  constexpr int S = 1 << LOG_S;
  const uint32_t NS = (uint32_t)ceil_div(d.n_t, S), NQ = (uint32_t)ceil_div(d.m, S);
  const int64_t dmin = -(int64_t)(NS - 1);
  const uint64_t NW = (uint64_t)NQ + NS - 1;
  cudaError_t e;
  if (ws.tw32_S != S) {
    if ((e = ws.tw32.ensure((size_t)S * sizeof(float2))) != cudaSuccess) return e;
    seg_twiddle_kernel<<<(unsigned)ceil_div(S, 256), 256, 0, s>>>(ws.tw32.as<float2>(), S);
    ++*kernels;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ws.tw32_S = S;
  }
  const uint64_t row_bytes = (uint64_t)S * sizeof(float2);
  uint64_t chunk = kSpecBudget / ((uint64_t)NS * row_bytes);
  if (chunk < 1) chunk = 1;
  if (chunk > d.num_blocks) chunk = d.num_blocks;
  if ((e = ws.spec.ensure(NW * row_bytes)) != cudaSuccess) return e;
  if ((e = ws.buf0.ensure(chunk * NS * row_bytes)) != cudaSuccess) return e;

  SpecArgs wa{};
  wa.seed = seed;
  wa.L = L_t;
  wa.D = (int64_t)d.n_t - 1;
  wa.dmin = dmin;
  wa.items = NW;
  wa.spec = ws.spec.as<float2>();
  wa.tw = ws.tw32.as<float2>();
  if ((e = launch_spectra<LOG_S>(wa, s)) != cudaSuccess) return e;
  ++*kernels;

  const int Q = pick_q(NQ, SegCfg<LOG_S>::QMAX);
  const uint32_t NQG = (uint32_t)ceil_div(NQ, Q);
  for (uint64_t b0 = 0; b0 < d.num_blocks; b0 += chunk) {
    const uint64_t nb = d.num_blocks - b0 < chunk ? d.num_blocks - b0 : chunk;
    SpecArgs ra{};
    ra.raw = d.raw + b0 * d.raw_stride;
    ra.raw_stride = d.raw_stride;
    ra.n_t = d.n_t;
    ra.NS = NS;
    ra.items = nb * NS;
    ra.spec = ws.buf0.as<float2>();
    ra.tw = ws.tw32.as<float2>();
    if ((e = launch_spectra<LOG_S>(ra, s)) != cudaSuccess) return e;
    ++*kernels;
    MacArgs m{};
    m.spec_raw = ws.buf0.as<float2>();
    m.spec_win = ws.spec.as<float2>();
    m.tw = ws.tw32.as<float2>();
    m.NS = NS;
    m.NQ = NQ;
    m.NQG = NQG;
    m.T = (uint32_t)T;
    m.dmin = dmin;
    m.nb = nb;
    m.raw = d.raw + b0 * d.raw_stride;
    m.raw_stride = d.raw_stride;
    m.out = d.out + b0 * d.out_stride;
    m.out_stride = d.out_stride;
    m.m = d.m;
    m.mw = d.mw;
    m.modified = d.modified;
    m.id_off = d.id_off;
    m.worst = ws.worst;
    m.guard_flag = guard_flag;
    const uint64_t ctas = nb * NQG;
    if (ctas > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    if (Q == 2) e = launch_mac<LOG_S, 2>(m, (unsigned)ctas, s);
    else e = launch_mac<LOG_S, 1>(m, (unsigned)ctas, s);
    if (e != cudaSuccess) return e;
    ++*kernels;
  }
  return cudaSuccess;
}

template <int LOG_S, int Q>
cudaError_t launch_batch_mac(const BatchReq* reqs, uint32_t nr, uint64_t ctas, const float2* spec, const float2* tw,
                             int T, uint32_t* out_stage, unsigned long long* worst, cudaStream_t s) {
  const size_t smem = mac_smem<LOG_S>(Q);
  cudaError_t e =
      cudaFuncSetAttribute(seg_batch_mac_kernel<LOG_S, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  seg_batch_mac_kernel<LOG_S, Q><<<(unsigned)ctas, SegCfg<LOG_S>::THREADS, smem, s>>>(reqs, nr, spec, tw, (uint32_t)T,
                                                                                  out_stage, worst);
  return cudaGetLastError();
}

template <int LOG_S>
cudaError_t run_fft32_batch(const BatchReq* reqs, uint64_t nr, uint64_t spec_items, uint64_t mac_ctas, int T,
                            FftWorkspace& ws, uint32_t* out_stage, cudaStream_t s, uint32_t* kernels) {
  constexpr int S = 1 << LOG_S;
  if (spec_items > 0x7fffffffull || mac_ctas > 0x7fffffffull || nr > 0xffffffffull) return cudaErrorInvalidConfiguration;
  cudaError_t e;
  if (ws.tw32_S != S) {
    if ((e = ws.tw32.ensure((size_t)S * sizeof(float2))) != cudaSuccess) return e;
    seg_twiddle_kernel<<<(unsigned)ceil_div(S, 256), 256, 0, s>>>(ws.tw32.as<float2>(), S);
    ++*kernels;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ws.tw32_S = S;
  }
  const size_t smem = spectra_smem<LOG_S>();
  if ((e = cudaFuncSetAttribute(seg_batch_spectra_kernel<LOG_S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)) != cudaSuccess)
    return e;
  seg_batch_spectra_kernel<LOG_S><<<(unsigned)spec_items, SegCfg<LOG_S>::THREADS, smem, s>>>(
      reqs, (uint32_t)nr, ws.spec.as<float2>(), ws.tw32.as<float2>());
  ++*kernels;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  constexpr int Q = SegCfg<LOG_S>::QMAX;
  e = launch_batch_mac<LOG_S, Q>(reqs, (uint32_t)nr, mac_ctas, ws.spec.as<float2>(), ws.tw32.as<float2>(), T,
                                 out_stage, ws.worst, s);
  ++*kernels;
  return e;
}

}  // namespace

int fft32_batch_tiles(int) { return SegCfg<12>::QMAX; }

cudaError_t launch_fft32_batch(const BatchReq* reqs_dev, uint64_t nr, uint64_t spec_items, uint64_t mac_ctas,
                               int log_s, int T, FftWorkspace& ws, uint32_t* out_stage, cudaStream_t s,
                               uint32_t* kernels) {
  if (!fft32_log_s_ok(log_s) || T < 1 || nr == 0) return cudaErrorInvalidValue;
  switch (log_s) {
    case 11: return run_fft32_batch<11>(reqs_dev, nr, spec_items, mac_ctas, T, ws, out_stage, s, kernels);
    case 12: return run_fft32_batch<12>(reqs_dev, nr, spec_items, mac_ctas, T, ws, out_stage, s, kernels);
    default: return run_fft32_batch<13>(reqs_dev, nr, spec_items, mac_ctas, T, ws, out_stage, s, kernels);
  }
}

int fft32_terms_bound(int log_s) {
  const double u = ldexp(1.0, -24), beta = u / 2;
  const int k = log_s + 1;  // log2 N
  const double S = ldexp(1.0, log_s);
  const double eps_k = pow(1 + u, 3 * k) * pow(1 + sqrt(5.0) * u, 3 * k + 1) * pow(1 + beta, 3 * k) - 1;
  const double per_term = sqrt((2 * S - 1) * S);
  int T = 0;
  while (T + 1 <= 4096 && (T + 1) * per_term * (eps_k + (T + 1) * u) <= 0.45) ++T;
  return T;
}

bool fft32_log_s_ok(int log_s) { return log_s >= 11 && log_s <= 13; }

double fft32_model_seconds(uint64_t n_t, uint64_t m, uint64_t B, int log_s, int T) {
  // S-point transforms (about 5 S log2 S flops at ~25 TFLOP/s in shared memory), bin products
  // (8 flops per bin at ~30 TFLOP/s) and the spectra the products read (8 bytes per bin per
  // operand from L2 at ~12 TB/s, a segment's shared by the Q tiles of a CTA)
  const double S = ldexp(1.0, log_s);
  const double NS = (double)ceil_div(n_t, (uint64_t)S), NQ = (double)ceil_div(m, (uint64_t)S);
  const double Q = (double)pick_q((uint32_t)NQ, 2);
  const double ffts = NS + NQ * std::ceil(NS / (double)T);
  const double flops_fft = ffts * 5.0 * S * log_s;
  const double flops_mac = NQ * NS * S * 8.0;
  const double bytes = std::ceil(NQ / Q) * NS * (1.0 + Q) * S * 8.0;
  return (double)B * (flops_fft / 2.5e13 + flops_mac / 3e13 + bytes / 1.2e13) + 2e-5;
}

cudaError_t launch_fft32_seg(const DirectArgs& d, const uint8_t* seed, uint64_t L_t, int log_s, int T,
                             FftWorkspace& ws, int* guard_flag, cudaStream_t s, uint32_t* kernels) {
  if (!fft32_log_s_ok(log_s) || T < 1) return cudaErrorInvalidValue;
  switch (log_s) {
    case 11: return run_fft32<11>(d, seed, L_t, T, ws, guard_flag, s, kernels);
    case 12: return run_fft32<12>(d, seed, L_t, T, ws, guard_flag, s, kernels);
    default: return run_fft32<13>(d, seed, L_t, T, ws, guard_flag, s, kernels);
  }
}

}  // namespace qrng
