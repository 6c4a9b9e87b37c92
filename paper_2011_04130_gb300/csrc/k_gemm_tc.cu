// Block-batched Toeplitz hashing on the tcgen05 tensor cores.
//
// All blocks of a stream share one seed (Sec. III.E), so hashing them is one matrix product
//     D[i][b] = sum_j T[i][j] X[b][j],   k_i(block b) = D[i][b] mod 2,
// with T the m x n Toeplitz matrix (Sec. III.B; the first n-m columns of (A, I_m) for the modified
// form of Sec. III.D, whose identity part is XORed in the epilogue) and X the raw blocks, one per
// row. GB300's tcgen05 has no integer (i8) kind, so 0/1 entries go through a floating-point kind
// with an FP32 accumulator in tensor memory; every sum is an integer count c <= n_t, exact in FP32,
// and its parity is read from the float in the epilogue (valid for c < 2^22, the launcher's limit
// on n_t). Two operand encodings share one kernel template:
//   FP8  (kind::f8f6f4): one E4M3 byte per entry, 2^-6 for a one (byte 0x08), so D = c * 2^-12;
//   FP4  (kind::mxf4, block-scaled): one E2M1 nibble per entry, 1.0 for a one (nibble 0x2), every
//        UE8M0 scale factor 2^0 (byte 0x7F), so D = c. Half the shared-memory bytes per entry of
//        FP8 and the FP4 tensor rate. The K order inside each 32-entry group is permuted (entry
//        4j+q of a packed word is nibble j of chunk word q), identically for T and X, which leaves
//        every dot product unchanged.
//
// CTA tile: 256 outputs (two UMMA M=128 halves sharing one B tile) x BN blocks (UMMA N; 256 for
// FP8, using all 512 TMEM columns; 224 for FP4, whose last 64 TMEM columns hold the scale
// factors), K step = one 128-byte swizzle row (128 FP8 or 256 FP4 entries).
//   warps 0-7   producers: each K step, thread t builds T row t (from a funnel-shifted window of
//               the bit-reversed seed) and X row t (from packed raw words that TMA already put
//               in shared memory) in the canonical K-major SWIZZLE_128B layout;
//   warp 8      TMA: cp.async.bulk.tensor loads of the packed raw tile (BN blocks x one K step),
//               running up to PK_STAGES K steps ahead;
//   warp 9      allocates tensor memory and issues tcgen05.mma (one elected lane);
//   warps 10-13 epilogue: tcgen05.ld of both accumulators, parity, __ballot_sync into output
//               words (32 outputs of one block per word), identity XOR for the modified form.
// Stages are handed over with mbarriers. Every wait is bounded (about one second of clock): on
// timeout the kernel records an error code, stops issuing work, waits for its own MMAs and TMA
// loads, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "qrng_internal.h"
#include "tc_util.cuh"

namespace qrng {
namespace {

using namespace tc;

constexpr int UM = 128;                 // UMMA M
constexpr int BM = 2 * UM;              // outputs per CTA tile
constexpr int ROW_BYTES = 128;          // one swizzle row per operand row and K step
constexpr int STAGES = 3;
constexpr int A_BYTES = BM * ROW_BYTES; // 32 KB
constexpr int PK_STAGES = 6;            // packed raw tiles in flight
constexpr int PRODUCER_WARPS = 8;
constexpr int PRODUCERS = PRODUCER_WARPS * 32;
constexpr int TMA_WARP = PRODUCER_WARPS;
constexpr int MMA_WARP = TMA_WARP + 1;
constexpr int EPI_WARP0 = MMA_WARP + 1;
constexpr int THREADS = (EPI_WARP0 + 4) * 32;  // 448
constexpr int TMEM_COLS = 512;
constexpr uint32_t kOneE4M3 = 0x08u;    // 2^-6
static_assert(PRODUCERS == BM, "one T row per producer thread");

// Per-encoding tile shape and instruction descriptor.
template <bool kFp4>
struct Cfg {
  static constexpr int BN = kFp4 ? 224 : 256;       // blocks per CTA tile (UMMA N)
  static constexpr int BK = kFp4 ? 256 : 128;       // K entries per step
  static constexpr int KW = BK / 32;                // packed raw words per row and step
  static constexpr int MMA_K = kFp4 ? 64 : 32;      // K entries per instruction (32 bytes either way)
  static constexpr int B_BYTES = BN * ROW_BYTES;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int PK_BYTES = BN * KW * 4;
  static constexpr uint32_t SFA_COL = 2 * BN;       // FP4: scale factors of A, then of B
  static constexpr uint32_t SFB_COL = 2 * BN + 32;
  // FP32 count from the accumulator: the FP8 encoding scales every product by 2^-12
  static constexpr float COUNT_SCALE = kFp4 ? 1.0f : 4096.0f;
  // kind::f8f6f4: D = F32 (bit 4), A = B = E4M3 (0), K-major, N >> 3 at bit 17, M >> 4 at bit 24.
  // kind::mxf4: scale-factor ids 0, A = B = E2M1 (1 at bits 7 and 10), K-major, N >> 3 at bit 17,
  //             UE8M0 scale factors (bit 23), M >> 7 at bit 27, dense K = 64.
  static constexpr uint32_t IDESC =
      kFp4 ? ((1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | (1u << 23) | ((uint32_t)(UM >> 7) << 27))
           : ((1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24));
  static_assert(BN % 32 == 0 && BN <= PRODUCERS && 2 * BN + (kFp4 ? 64 : 0) <= TMEM_COLS, "tile does not fit");
  static_assert(MMA_K * (kFp4 ? 1 : 2) == 64, "each instruction consumes 32 bytes of a row");
};

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(Cfg<false>::IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_f4(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t tmem_sfa,
                                       uint32_t tmem_sfb, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(Cfg<true>::IDESC), "r"(tmem_sfa), "r"(tmem_sfb), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Spreads 4 bits to 4 bytes: bit j -> byte j with value kOneE4M3 (the shifted copies x << 7k never
// overlap for a 4-bit x, so the multiply has no carries).
__device__ __forceinline__ uint32_t nib_to_e4m3(uint32_t nib) { return (nib * 0x01020408u) & 0x08080808u; }
static_assert(0x08080808u == kOneE4M3 * 0x01010101u, "spread mask must select the E4M3 encoding of one");

// Writes 32 bits (K elements 32w..32w+31 of one row) as two 16-byte chunks of the swizzled row.
__device__ __forceinline__ void store_word_e4m3(uint32_t row_addr, uint32_t row, uint32_t w, uint32_t x) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t y = x >> (16 * h);
    const uint32_t c = 2 * w + h;
    const uint32_t addr = row_addr + (((c ^ (row & 7u)) & 7u) << 4);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(nib_to_e4m3(y & 0xFu)),
                 "r"(nib_to_e4m3((y >> 4) & 0xFu)), "r"(nib_to_e4m3((y >> 8) & 0xFu)),
                 "r"(nib_to_e4m3((y >> 12) & 0xFu))
                 : "memory");
  }
}

struct GemmArgs {
  const uint32_t* raw;
  uint64_t raw_stride;
  uint32_t nw_t;
  uint32_t tail_mask;
  uint32_t m;
  uint32_t mw;
  const uint32_t* seed_rev;
  int modified;
  uint32_t id_off;
  uint32_t* out;
  uint64_t out_stride;
  uint64_t num_blocks;
  uint32_t mtiles;
  uint32_t ntiles;
  uint32_t ksteps;
  int* err;
  int fault_no_tma;  // test hook: the loader publishes no raw tile, so every consumer's bounded wait runs out
};

template <bool kFp4>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_tc_kernel(const GemmArgs a, const __grid_constant__ CUtensorMap raw_map) {
  using C = Cfg<kFp4>;
  constexpr int BN = C::BN;
  constexpr int KW = C::KW;
  extern __shared__ uint8_t dyn_smem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t pk_full_bar[PK_STAGES];
  __shared__ __align__(8) uint64_t pk_empty_bar[PK_STAGES];
  __shared__ __align__(8) uint64_t accum_full_bar;
  __shared__ __align__(8) uint64_t accum_empty_bar;
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t smem_base = (smem_u32(dyn_smem) + 1023u) & ~1023u;
  const uint32_t pk_base = smem_base + STAGES * C::STAGE_BYTES;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], PRODUCERS);
      mbar_init(&empty_bar[s], 1);
    }
    for (int s = 0; s < PK_STAGES; ++s) {
      mbar_init(&pk_full_bar[s], 1);
      mbar_init(&pk_empty_bar[s], PRODUCERS);
    }
    mbar_init(&accum_full_bar, 1);
    mbar_init(&accum_empty_bar, 4 * 32);
    mbar_init(&drain_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;
  if constexpr (kFp4) {
    // every scale factor is 2^0: fill the 64 scale-factor columns in all 128 lanes, whatever
    // cells the MMAs read there
    if (warp >= EPI_WARP0) {
      const uint32_t lanes = (32u * (warp & 3u)) << 16;
      tmem_fill32(tmem_base + lanes + C::SFA_COL, kScaleOne);
      tmem_fill32(tmem_base + lanes + C::SFB_COL, kScaleOne);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }

  const uint64_t ntile_total = (uint64_t)a.mtiles * a.ntiles;

  if (warp < PRODUCER_WARPS) {
    // ------------------------------------------------------------------ producers
    const uint32_t t = threadIdx.x;  // T row t and (t < BN) X row t of every K step
    uint32_t stage = 0, phase = 0, pstage = 0, pphase = 0;
    for (uint64_t tile = blockIdx.x; tile < ntile_total && !abort_flag; tile += gridDim.x) {
      const uint32_t mt = (uint32_t)(tile % a.mtiles);
      // T row i: reversed-seed bits m-1-i+BK*ks .. +BK-1 (front padding keeps the index >= 0)
      const int64_t i = (int64_t)mt * BM + t;
      const int64_t ubase = (int64_t)a.m - 1 - i + 32 * (int64_t)kSeedFrontWords;
      const uint32_t sh = (uint32_t)(ubase & 31);
      const uint32_t* seed_row = a.seed_rev + (ubase >> 5);
      for (uint32_t ks = 0; ks < a.ksteps; ++ks) {
        // packed raw words of X row t for this K step (delivered by TMA)
        if (!mbar_wait(&pk_full_bar[pstage], pphase, &abort_flag, a.err, 1)) break;
        uint32_t xw[KW];
        if (t < (uint32_t)BN) {
#pragma unroll
          for (int h = 0; h < KW / 4; ++h)
            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(xw[4 * h]), "=r"(xw[4 * h + 1]), "=r"(xw[4 * h + 2]), "=r"(xw[4 * h + 3])
                         : "r"(pk_base + pstage * C::PK_BYTES + t * (KW * 4) + 16 * h)
                         : "memory");
        }
        if (KW * ks + KW > a.nw_t - 1) {  // words past the Toeplitz part (zero-filled) and its partial last word
#pragma unroll
          for (int w = 0; w < KW; ++w)
            if (KW * ks + w == a.nw_t - 1) xw[w] &= a.tail_mask;
        }
        uint32_t sw[KW + 1];
#pragma unroll
        for (int k = 0; k <= KW; ++k) sw[k] = __ldg(seed_row + KW * ks + k);

        if (!mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag, a.err, 2)) break;
        const uint32_t sA = smem_base + stage * C::STAGE_BYTES;
        const uint32_t sB = sA + A_BYTES;
        const uint32_t rowA = sA + t * ROW_BYTES;
        const uint32_t rowB = sB + t * ROW_BYTES;
#pragma unroll
        for (int w = 0; w < KW; ++w) {
          const uint32_t tw = __funnelshift_r(sw[w], sw[w + 1], sh);
          if constexpr (kFp4) {
            store_word_e2m1(rowA, t, w, tw);
            if (t < (uint32_t)BN) store_word_e2m1(rowB, t, w, xw[w]);
          } else {
            store_word_e4m3(rowA, t, w, tw);
            store_word_e4m3(rowB, t, w, xw[w]);
          }
        }
        fence_proxy_async_smem();
        mbar_arrive(&full_bar[stage]);
        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        // The packed tile is released only now: its words have been consumed by the stores above.
        // An arrive issued straight after the ld.shared does not wait for those loads, and the next
        // TMA load into the slot could overwrite the words before they are read.
        mbar_arrive(&pk_empty_bar[pstage]);
        if (++pstage == PK_STAGES) { pstage = 0; pphase ^= 1u; }
      }
    }
  } else if (warp == TMA_WARP) {
    // ------------------------------------------------------------------ TMA loads of packed raw tiles
    uint32_t pstage = 0, pphase = 0, issued = 0;
    if (lane == 0) {
      for (uint64_t tile = blockIdx.x; tile < ntile_total && !abort_flag; tile += gridDim.x) {
        const uint32_t nt = (uint32_t)(tile / a.mtiles);
        for (uint32_t ks = 0; ks < a.ksteps; ++ks) {
          if (!mbar_wait(&pk_empty_bar[pstage], pphase ^ 1u, &abort_flag, a.err, 3)) break;
          if (!a.fault_no_tma) {
            mbar_arrive_expect_tx(&pk_full_bar[pstage], C::PK_BYTES);
            tma_load_2d(pk_base + pstage * C::PK_BYTES, &raw_map, (int)(KW * ks), (int)(nt * BN),
                        &pk_full_bar[pstage]);
            ++issued;
          }
          if (++pstage == PK_STAGES) { pstage = 0; pphase ^= 1u; }
        }
      }
      // the loads still in flight must land before the CTA exits: wait for the last PK_STAGES slots
      for (uint32_t k = 0; k < PK_STAGES && k < issued; ++k) {
        if (pstage == 0) { pstage = PK_STAGES; pphase ^= 1u; }
        --pstage;
        mbar_drain(&pk_full_bar[pstage], pphase, a.err, 4);
      }
    }
    __syncwarp();
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------------ MMA issuer
    uint32_t stage = 0, phase = 0, acc_phase = 0;
    bool issued = false;
    for (uint64_t tile = blockIdx.x; tile < ntile_total && !abort_flag; tile += gridDim.x) {
      // the epilogue must have drained the previous tile's accumulators
      if (tile != blockIdx.x && !mbar_wait(&accum_empty_bar, acc_phase ^ 1u, &abort_flag, a.err, 5)) break;
      for (uint32_t ks = 0; ks < a.ksteps; ++ks) {
        if (!mbar_wait(&full_bar[stage], phase, &abort_flag, a.err, 6)) break;
        tc_fence_after();
        if (lane == 0) {
          const uint32_t sA = smem_base + stage * C::STAGE_BYTES;
          const uint32_t sB = sA + A_BYTES;
#pragma unroll
          for (int k = 0; k < ROW_BYTES / 32; ++k) {
            const uint64_t bdesc = smem_desc_sw128(sB + 32 * k);
            const uint64_t adesc0 = smem_desc_sw128(sA + 32 * k);
            const uint64_t adesc1 = smem_desc_sw128(sA + UM * ROW_BYTES + 32 * k);
            if constexpr (kFp4) {
              mma_f4(tmem_base, adesc0, bdesc, tmem_base + C::SFA_COL, tmem_base + C::SFB_COL, (ks | k) != 0);
              mma_f4(tmem_base + BN, adesc1, bdesc, tmem_base + C::SFA_COL, tmem_base + C::SFB_COL, (ks | k) != 0);
            } else {
              mma_f8(tmem_base, adesc0, bdesc, (ks | k) != 0);
              mma_f8(tmem_base + BN, adesc1, bdesc, (ks | k) != 0);
            }
          }
          mma_commit(&empty_bar[stage]);  // frees the stage once these MMAs have read it
          issued = true;
        }
        __syncwarp();
        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
      }
      if (abort_flag) break;
      if (lane == 0) mma_commit(&accum_full_bar);
      __syncwarp();
      acc_phase ^= 1u;
    }
    // every MMA this CTA issued must finish before the tensor memory is released
    if (lane == 0 && issued) {
      mma_commit(&drain_bar);
      mbar_drain(&drain_bar, 0, a.err, 7);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------------ epilogue
    const uint32_t q = warp & 3u;  // TMEM lane quarter this warp may access
    uint32_t acc_phase = 0;
    for (uint64_t tile = blockIdx.x; tile < ntile_total && !abort_flag; tile += gridDim.x) {
      const uint32_t mt = (uint32_t)(tile % a.mtiles);
      const uint32_t nt = (uint32_t)(tile / a.mtiles);
      if (!mbar_wait(&accum_full_bar, acc_phase, &abort_flag, a.err, 8)) break;
      tc_fence_after();
      for (uint32_t half = 0; half < 2; ++half) {
        const uint32_t ow = mt * (BM / 32) + half * (UM / 32) + q;  // output word of every block in the tile
        const uint32_t rem = (ow < a.mw) ? a.m - 32 * ow : 0u;
        const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
        for (uint32_t g = 0; g < (uint32_t)BN / 32; ++g) {
          uint32_t v[32];
          tmem_load32(tmem_base + ((32u * q) << 16) + half * BN + 32u * g, v);
          uint32_t mine = 0;
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const uint32_t wrd = __ballot_sync(0xffffffffu, count_parity(v[c], C::COUNT_SCALE));
            if (lane == (uint32_t)c) mine = wrd;
          }
          const uint64_t b = (uint64_t)nt * BN + 32u * g + lane;
          if (ow < a.mw && b < a.num_blocks) {
            mine &= omask;
            if (a.modified) {
              const uint64_t bit = (uint64_t)a.id_off + 32ull * ow;
              const uint32_t* rr = a.raw + b * a.raw_stride;
              const uint64_t rq = bit >> 5;
              const uint32_t rs = (uint32_t)(bit & 31);
              const uint32_t rlo = __ldg(rr + rq);
              const uint32_t rhi = (rs && rq + 1 < a.raw_stride) ? __ldg(rr + rq + 1) : 0u;
              mine ^= __funnelshift_r(rlo, rhi, rs) & omask;
            }
            a.out[b * a.out_stride + ow] = mine;
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&accum_empty_bar);
      acc_phase ^= 1u;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace

typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <bool kFp4>
static size_t smem_bytes() {
  return (size_t)STAGES * Cfg<kFp4>::STAGE_BYTES + (size_t)PK_STAGES * Cfg<kFp4>::PK_BYTES + 1024;
}

bool gemm_tc_layout_ok(const DirectArgs& d) {
  return (reinterpret_cast<uintptr_t>(d.raw) & 15) == 0 && (d.raw_stride % 4) == 0;
}

template <bool kFp4>
static cudaError_t launch(const DirectArgs& d, int* err, int fault, int num_sms, cudaStream_t s, uint32_t* kernels) {
  using C = Cfg<kFp4>;
  if (!gemm_tc_layout_ok(d)) return cudaErrorInvalidValue;
  GemmArgs a{};
  a.raw = d.raw;
  a.raw_stride = d.raw_stride;
  a.nw_t = d.nw_t;
  a.tail_mask = d.tail_mask;
  a.m = d.m;
  a.mw = d.mw;
  a.seed_rev = d.seed_rev;
  a.modified = d.modified;
  a.id_off = d.id_off;
  a.out = d.out;
  a.out_stride = d.out_stride;
  a.num_blocks = d.num_blocks;
  a.mtiles = (uint32_t)ceil_div(d.m, BM);
  a.ntiles = (uint32_t)ceil_div(d.num_blocks, C::BN);
  a.ksteps = (uint32_t)ceil_div((uint64_t)d.nw_t * 32, C::BK);
  a.err = err;
  a.fault_no_tma = (fault == QRNG_FAULT_GEMM_NO_TMA);

  // Tensor map over the raw words: dim 0 = the Toeplitz part's words of a block (reads beyond it
  // are zero-filled), dim 1 = blocks (rows past the last block are zero-filled); box KW x BN
  // (16 or 32 bytes per row; every x coordinate is a multiple of KW words, so 16-byte aligned).
  // The driver's encoder is looked up at run time, so the library has no link-time libcuda dependency.
  static PFN_encodeTiled encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_encodeTiled>(fn);
  }
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)d.nw_t, (cuuint64_t)d.num_blocks};
  const cuuint64_t gstride[1] = {(cuuint64_t)d.raw_stride * 4};
  const cuuint32_t box[2] = {(cuuint32_t)C::KW, (cuuint32_t)C::BN};
  const cuuint32_t estride[2] = {1, 1};
  CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t*>(d.raw), gdim, gstride, box,
                      estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;

  const size_t smem = smem_bytes<kFp4>();
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<kFp4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const uint64_t tiles = (uint64_t)a.mtiles * a.ntiles;
  const int grid = (int)(tiles < (uint64_t)num_sms ? tiles : (uint64_t)num_sms);
  gemm_tc_kernel<kFp4><<<grid, THREADS, smem, s>>>(a, map);
  ++*kernels;
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const DirectArgs& d, bool fp4, int* err, int fault, int num_sms, cudaStream_t s,
                           uint32_t* kernels) {
  return fp4 ? launch<true>(d, err, fault, num_sms, s, kernels) : launch<false>(d, err, fault, num_sms, s, kernels);
}

}  // namespace qrng
