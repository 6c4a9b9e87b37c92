/*
 * Reference oracle for QRNG post-processing (min-entropy estimate + Toeplitz hashing).
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, obviously-correct CPU restatement of
 * what the paper defines. It is used by the test-suite, by the smoke check and by the timed
 * CPU baseline of the benchmark; the product library never links, loads or calls it, and it
 * shares no code, header, table or helper with the CUDA path.
 *
 * Conventions (0-based, shared with the product only as a *specification*):
 *   - bits are packed LSB-first: bit t of a packed buffer is bit (t % 8) of byte (t / 8);
 *   - raw block r[0..n), seed a[0..L), output k[0..m);
 *   - standard Toeplitz (Sec. III.B, the matrix T with T[i][j] = a_{n+i-j} in the paper's
 *     1-based indices):      k_i = ( sum_{j<n}     a[n-1+i-j]   * r[j] )            mod 2,
 *     seed length L = n+m-1;
 *   - modified Toeplitz (Sec. III.D, A_m = (A, I_m) with A[i][j] = a_{n-m+i-j}):
 *                           k_i = ( sum_{j<n-m}   a[n-m-1+i-j] * r[j] + r[n-m+i] ) mod 2,
 *     seed length L = n-1.
 *
 * Min-entropy (Sec. II): H_min = -log2 max_x P(x) (Sec. II.A); the ideal model is the
 * Gaussian fixed by the measured mean and variance (Sec. II.B), discretised the way an ADC
 * rounds and clips; the statistical distance d_U = 1/2 sum_{x in U} |P'(x) - P(x)| (Sec. II.C)
 * is taken over every code; the finite-size amplification that Sec. II.C asks for (without a
 * formula) is the L1 deviation bound of an empirical distribution,
 *   delta = 1/2 sqrt( 2 (K ln 2 + ln(1/eps)) / N ),  K = 2^bits;
 * the correction is Delta H_m = log2( (d_U + delta) / 2^(-bits-1) + 1 ) (Sec. II.C), and the
 * corrected entropy is H_modify = max(0, H_model - Delta H_m).
 *
 * Output length (Sec. III.B, leftover hash lemma): m = n H / N_bits - 2 log2(1/eps), floored,
 * 0 when negative.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

static int get_bit(const uint8_t* buf, uint64_t t) { return (buf[t >> 3] >> (t & 7)) & 1; }

static void put_bit(uint8_t* buf, uint64_t t, int v) {
  uint8_t mask = (uint8_t)(1u << (t & 7));
  if (v) buf[t >> 3] |= mask;
  else buf[t >> 3] &= (uint8_t)~mask;
}

/* The standard definition holds for any m >= 1 (an extractor uses m <= n, but the modified
 * form's block A is a standard matrix of n-m columns that may have more rows than columns);
 * the modified form needs at least one column in A, so m < n. */
static int check_shape(uint64_t n, uint64_t m, int form) {
  if (n == 0 || m == 0) return ORACLE_EINVAL;
  if (form == 0) return ORACLE_OK;
  if (form == 1) return m < n ? ORACLE_OK : ORACLE_EINVAL;
  return ORACLE_EINVAL;
}

uint64_t oracle_seed_bits(uint64_t n, uint64_t m, int form) { return form == 0 ? n + m - 1 : n - 1; }

/* One output bit k_i of one block, straight from the definition. */
static int toeplitz_bit(const uint8_t* r, const uint8_t* a, uint64_t n, uint64_t m, int form, uint64_t i) {
  uint64_t sum = 0;
  if (form == 0) {
    for (uint64_t j = 0; j < n; ++j) sum += (uint64_t)(a[n - 1 + i - j] & r[j]);
  } else {
    for (uint64_t j = 0; j < n - m; ++j) sum += (uint64_t)(a[n - m - 1 + i - j] & r[j]);
    sum += r[n - m + i];
  }
  return (int)(sum % 2);
}

/* Unpack n bits starting at bit offset `off` into one byte per bit. */
static uint8_t* unpack(const uint8_t* buf, uint64_t off, uint64_t n) {
  uint8_t* u = (uint8_t*)malloc(n ? n : 1);
  if (!u) return NULL;
  for (uint64_t t = 0; t < n; ++t) u[t] = (uint8_t)get_bit(buf, off + t);
  return u;
}

/*
 * Full Toeplitz hash of one block: n raw bits at bit offset raw_off of `raw`, seed bits at
 * bit offset 0 of `seed`, m output bits written at bit offset out_off of `out` (other bits of
 * `out` are left unchanged).
 */
int oracle_toeplitz(const uint8_t* raw, uint64_t raw_off, uint64_t n, uint64_t m, const uint8_t* seed,
                    int form, uint8_t* out, uint64_t out_off) {
  int st = check_shape(n, m, form);
  if (st) return st;
  uint64_t L = oracle_seed_bits(n, m, form);
  uint8_t* r = unpack(raw, raw_off, n);
  uint8_t* a = unpack(seed, 0, L);
  if (!r || !a) { free(r); free(a); return ORACLE_ENOMEM; }
  for (uint64_t i = 0; i < m; ++i) put_bit(out, out_off + i, toeplitz_bit(r, a, n, m, form, i));
  free(r);
  free(a);
  return ORACLE_OK;
}

/* Block splitting (Sec. III.E): block b is raw bits [b n, (b+1) n), output bits [b m, (b+1) m). */
int oracle_toeplitz_blocks(const uint8_t* raw, uint64_t n, uint64_t m, const uint8_t* seed, int form,
                           uint64_t num_blocks, uint8_t* out) {
  for (uint64_t b = 0; b < num_blocks; ++b) {
    int st = oracle_toeplitz(raw, b * n, n, m, seed, form, out, b * m);
    if (st) return st;
  }
  return ORACLE_OK;
}

/*
 * Selected output bits of one block (each one O(n)): bits_out[q] = k_{idx[q]} of the block whose
 * raw bits start at raw_off. Used to check outputs too large for the full product.
 */
int oracle_toeplitz_bits(const uint8_t* raw, uint64_t raw_off, uint64_t n, uint64_t m, const uint8_t* seed,
                         int form, const uint64_t* idx, uint64_t count, uint8_t* bits_out) {
  int st = check_shape(n, m, form);
  if (st) return st;
  uint64_t L = oracle_seed_bits(n, m, form);
  for (uint64_t q = 0; q < count; ++q)
    if (idx[q] >= m) return ORACLE_EINVAL;
  uint8_t* r = unpack(raw, raw_off, n);
  uint8_t* a = unpack(seed, 0, L);
  if (!r || !a) { free(r); free(a); return ORACLE_ENOMEM; }
  for (uint64_t q = 0; q < count; ++q) bits_out[q] = (uint8_t)toeplitz_bit(r, a, n, m, form, idx[q]);
  free(r);
  free(a);
  return ORACLE_OK;
}

/*
 * Freivalds-style probabilistic check of every block of a shared-seed product, 64 random test
 * vectors at a time (vector q lives in bit q of a 64-bit lane word).
 *
 * With M the full hashing matrix (T, or (A, I_m) for the modified form), k_b = M r_b (mod 2)
 * implies u^T k_b = (u^T M) r_b (mod 2) for every u. u_lanes[i] holds bit q = u^(q)_i for i < m.
 * The function forms w = u^T M column by column from the definition, then for every block
 * compares parity(u & k_b) with parity(w & r_b) in all 64 lanes; mismatch_out[b] is the XOR of
 * the two lane words (0 when the block passes). A wrong block escapes with probability 2^-64.
 */
int oracle_freivalds(const uint8_t* raw, uint64_t n, uint64_t m, const uint8_t* seed, int form,
                     uint64_t num_blocks, const uint8_t* out, const uint64_t* u_lanes,
                     uint64_t* mismatch_out) {
  int st = check_shape(n, m, form);
  if (st) return st;
  uint64_t L = oracle_seed_bits(n, m, form);
  uint8_t* a = unpack(seed, 0, L);
  uint64_t* w = (uint64_t*)calloc(n, sizeof(uint64_t));
  if (!a || !w) { free(a); free(w); return ORACLE_ENOMEM; }
  for (uint64_t j = 0; j < n; ++j) {
    uint64_t acc = 0;
    for (uint64_t i = 0; i < m; ++i) {
      int mij;
      if (form == 0) mij = a[n - 1 + i - j];
      else if (j < n - m) mij = a[n - m - 1 + i - j];
      else mij = (j == n - m + i);
      if (mij) acc ^= u_lanes[i];
    }
    w[j] = acc;
  }
  for (uint64_t b = 0; b < num_blocks; ++b) {
    uint64_t lhs = 0, rhs = 0;
    for (uint64_t i = 0; i < m; ++i)
      if (get_bit(out, b * m + i)) lhs ^= u_lanes[i];
    for (uint64_t j = 0; j < n; ++j)
      if (get_bit(raw, b * n + j)) rhs ^= w[j];
    mismatch_out[b] = lhs ^ rhs;
  }
  free(a);
  free(w);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Min-entropy (Sec. II)                                                                       */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  double h_modify;   /* max(0, h_model - delta_hm)                                   */
  double h_emp;      /* -log2(max_count / count): min-entropy of the measured P'     */
  double h_model;    /* -log2 max_v P_v: min-entropy of the ideal Gaussian model P   */
  double d_u;        /* 1/2 sum over all codes of |P'_v - P_v|                       */
  double d_u_peak;   /* the same sum over U = {argmax P'} only (reported)            */
  double delta_fs;   /* finite-size amplification term                               */
  double delta_hm;   /* log2((d_u + delta_fs) 2^(bits+1) + 1)                        */
  double mean;       /* sample mean                                                  */
  double var;        /* population variance                                          */
  uint64_t count;    /* number of samples                                            */
  uint64_t max_count;/* largest histogram bin                                        */
  uint32_t argmax;   /* lowest code with max_count                                   */
  uint32_t bits;
} oracle_hmin_report;

/* Exact histogram of `count` samples (uint8 when bits <= 8, little-endian uint16 otherwise). */
int oracle_histogram(const void* samples, uint64_t count, int bits, uint64_t* hist, uint64_t* out_of_range) {
  if (bits < 1 || bits > 16) return ORACLE_EINVAL;
  uint64_t K = 1ull << bits;
  memset(hist, 0, K * sizeof(uint64_t));
  *out_of_range = 0;
  for (uint64_t s = 0; s < count; ++s) {
    uint64_t v = bits <= 8 ? ((const uint8_t*)samples)[s] : ((const uint16_t*)samples)[s];
    if (v >= K) (*out_of_range)++;
    else hist[v]++;
  }
  return ORACLE_OK;
}

/* Mass of the standard normal law on (y, z], y < z, either end possibly infinite; this is
 * Phi(z) - Phi(y), written so that no two nearly equal numbers are subtracted: both ends above
 * the mean -> difference of upper-tail masses, both below -> difference of lower-tail masses,
 * ends on either side of the mean -> sum of two central masses. */
static double std_normal_mass(double y, double z) {
  const double r = sqrt(0.5);
  if (y >= 0.0) return 0.5 * (erfc(y * r) - erfc(z * r));
  if (z <= 0.0) return 0.5 * (erfc(-z * r) - erfc(-y * r));
  return 0.5 * (erf(z * r) - erf(y * r));
}

/* Model cells of a Gaussian of mean mu and variance var (> 0) discretised like the ADC: code v
 * collects the real line between v - 1/2 and v + 1/2, and the end codes also take the tails. */
static void gaussian_cells(double mu, double var, uint64_t K, double* P) {
  double sigma = sqrt(var);
  for (uint64_t v = 0; v < K; ++v) {
    double lo = (v == 0) ? -INFINITY : ((double)v - 0.5 - mu) / sigma;
    double hi = (v == K - 1) ? INFINITY : ((double)v + 0.5 - mu) / sigma;
    P[v] = std_normal_mass(lo, hi);
  }
}

/* Min-entropy report from an exact histogram (the steps of Sec. II in the paper's order). */
int oracle_minentropy_from_hist(const uint64_t* hist, int bits, double eps, oracle_hmin_report* rep) {
  if (bits < 1 || bits > 16 || !(eps > 0.0 && eps < 1.0)) return ORACLE_EINVAL;
  uint64_t K = 1ull << bits;
  memset(rep, 0, sizeof(*rep));
  rep->bits = (uint32_t)bits;

  /* Empirical distribution P' and its min-entropy (Sec. II.A). */
  uint64_t N = 0, maxc = 0;
  uint32_t argmax = 0;
  unsigned __int128 s1 = 0, s2 = 0;
  for (uint64_t v = 0; v < K; ++v) {
    N += hist[v];
    s1 += (unsigned __int128)v * hist[v];
    s2 += (unsigned __int128)v * v * hist[v];
    if (hist[v] > maxc) { maxc = hist[v]; argmax = (uint32_t)v; }
  }
  if (N == 0) return ORACLE_EINVAL;
  rep->count = N;
  rep->max_count = maxc;
  rep->argmax = argmax;
  rep->h_emp = -log2((double)maxc / (double)N);

  /* Moments: mean and population variance, the numerator N*S2 - S1^2 taken exactly. */
  double mu = (double)s1 / (double)N;
  unsigned __int128 num = (unsigned __int128)N * s2 - s1 * s1;
  double var = (double)num / ((double)N * (double)N);
  rep->mean = mu;
  rep->var = var;

  /* Ideal model P: the Gaussian of that mean and variance (Sec. II.B), rounded and clipped to codes. */
  double* P = (double*)malloc(K * sizeof(double));
  if (!P) return ORACLE_ENOMEM;
  if (num == 0) {
    for (uint64_t v = 0; v < K; ++v) P[v] = (v == argmax) ? 1.0 : 0.0;
  } else {
    gaussian_cells(mu, var, K, P);
  }
  double pmax = 0.0;
  for (uint64_t v = 0; v < K; ++v)
    if (P[v] > pmax) pmax = P[v];
  rep->h_model = -log2(pmax);

  /* Statistical distance between P' and P (Sec. II.C), over every code and over {argmax P'}. */
  double d = 0.0;
  for (uint64_t v = 0; v < K; ++v) d += fabs((double)hist[v] / (double)N - P[v]);
  rep->d_u = 0.5 * d;
  rep->d_u_peak = 0.5 * fabs((double)maxc / (double)N - P[argmax]);
  free(P);

  /* Finite-size amplification, then the correction term and the corrected entropy (Sec. II.C). */
  rep->delta_fs = 0.5 * sqrt(2.0 * ((double)K * log(2.0) + log(1.0 / eps)) / (double)N);
  rep->delta_hm = log2((rep->d_u + rep->delta_fs) / ldexp(1.0, -bits - 1) + 1.0);
  double h = rep->h_model - rep->delta_hm;
  rep->h_modify = h > 0.0 ? h : 0.0;
  return ORACLE_OK;
}

/*
 * Classical-noise subtraction (Sec. II.B): the laser-off stream holds the classical noise alone,
 * the quantum noise variance is sigma_q^2 = sigma_{q+c}^2 - sigma_c^2, and the ideal model of the
 * quantum part is the Gaussian of that variance around the laser-on mean, discretised like the ADC.
 * The report is the laser-on stream's (counts, moments, empirical entropy, distance to its own
 * Gaussian model, finite-size term, correction) except h_model = -log2 max of the quantum model,
 * h_modify = max(0, h_model - delta_hm) and var = sigma_q^2. *h_subtracted receives the paper's
 * H^{q+c} - H'^c: the model min-entropy of the laser-on stream minus that of the laser-off stream.
 */
int oracle_minentropy_quantum_from_hist(const uint64_t* hist_on, const uint64_t* hist_off, int bits, double eps,
                                        oracle_hmin_report* rep, double* h_subtracted) {
  oracle_hmin_report off;
  int st = oracle_minentropy_from_hist(hist_off, bits, eps, &off);
  if (st) return st;
  st = oracle_minentropy_from_hist(hist_on, bits, eps, rep);
  if (st) return st;
  double var_q = rep->var - off.var;
  if (!(var_q > 0.0)) return ORACLE_EINVAL;
  uint64_t K = 1ull << bits;
  double* P = (double*)malloc(K * sizeof(double));
  if (!P) return ORACLE_ENOMEM;
  gaussian_cells(rep->mean, var_q, K, P);
  double pmax = 0.0;
  for (uint64_t v = 0; v < K; ++v)
    if (P[v] > pmax) pmax = P[v];
  free(P);
  *h_subtracted = rep->h_model - off.h_model;
  rep->h_model = -log2(pmax);
  rep->var = var_q;
  double h = rep->h_model - rep->delta_hm;
  rep->h_modify = h > 0.0 ? h : 0.0;
  return ORACLE_OK;
}

/* splitmix64 (Steele, Lea and Flood, 2014): output number s (s >= 1) of the generator started at x0. */
uint64_t oracle_splitmix64(uint64_t x0, uint64_t s) {
  uint64_t z = x0 + s * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/*
 * Random subsample (Sec. II.C: the corrected entropy may be estimated from randomly selected
 * samples): sample i (0-based) is kept when output i+1 of splitmix64 started at sel_seed, shifted
 * right by 11 bits, is below floor(fraction * 2^53); fraction 1 keeps every sample.
 */
int oracle_histogram_sampled(const void* samples, uint64_t count, int bits, double fraction, uint64_t sel_seed,
                             uint64_t* hist, uint64_t* out_of_range) {
  if (bits < 1 || bits > 16 || !(fraction > 0.0 && fraction <= 1.0)) return ORACLE_EINVAL;
  uint64_t K = 1ull << bits;
  uint64_t thr = (uint64_t)floor(fraction * 9007199254740992.0);
  memset(hist, 0, K * sizeof(uint64_t));
  *out_of_range = 0;
  for (uint64_t s = 0; s < count; ++s) {
    if ((oracle_splitmix64(sel_seed, s + 1) >> 11) >= thr) continue;
    uint64_t v = bits <= 8 ? ((const uint8_t*)samples)[s] : ((const uint16_t*)samples)[s];
    if (v >= K) (*out_of_range)++;
    else hist[v]++;
  }
  return ORACLE_OK;
}

/* Min-entropy report straight from samples; returns EINVAL when a sample is >= 2^bits. */
int oracle_minentropy(const void* samples, uint64_t count, int bits, double eps, oracle_hmin_report* rep) {
  if (bits < 1 || bits > 16 || count == 0) return ORACLE_EINVAL;
  uint64_t K = 1ull << bits;
  uint64_t* hist = (uint64_t*)malloc(K * sizeof(uint64_t));
  if (!hist) return ORACLE_ENOMEM;
  uint64_t bad = 0;
  int st = oracle_histogram(samples, count, bits, hist, &bad);
  if (st == ORACLE_OK && bad) st = ORACLE_EINVAL;
  if (st == ORACLE_OK) st = oracle_minentropy_from_hist(hist, bits, eps, rep);
  free(hist);
  return st;
}

/* Output length of the extractor (Sec. III.B): floor(n H / bits - 2 log2(1/eps)), 0 if negative. */
uint64_t oracle_output_length(uint64_t n, double h_per_sample, int bits, double eps_lhl) {
  if (bits < 1 || !(eps_lhl > 0.0 && eps_lhl <= 1.0) || !(h_per_sample >= 0.0)) return 0;
  double m = (double)n * h_per_sample / (double)bits - 2.0 * log2(1.0 / eps_lhl);
  if (!(m > 0.0)) return 0;
  return (uint64_t)floor(m);
}
