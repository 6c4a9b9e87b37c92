// Block-batched Toeplitz hashing on pairs of SMs (tcgen05 cta_group::2).
//
// The same exact GF(2) product as the single-SM tensor-core kernel,
//     D[i][b] = sum_j T[i][j] X[b][j],   k_i(block b) = D[i][b] mod 2
// (T the Toeplitz matrix of the shared seed, Sec. III.B / III.D; X the raw blocks, Sec. III.E), with
// block-scaled E2M1 operands (0/1 as 1.0, every UE8M0 scale factor 2^0), issued as UMMAs of M = 256
// that span a cluster of two CTAs on two SMs: each CTA holds 128 of the 256 T rows and half of the X
// rows of a tile, and the pair's tensor cores each read their own T half and both X halves.
//
// T is Toeplitz: T[i + 256][j + 256] = T[i][j], so the T tile of output tile mt+1 at K step ks is the
// T tile of output tile mt at K step ks-1. A pair tile therefore covers two output tiles (512 outputs,
// two accumulators) x 224 blocks, and every stage carries one new T tile: at step e the MMAs are
//     D0 += T(mt, e-1) X(e-1),   D1 += T(mt, e-2) X(e-1)      (e = 1 .. ksteps),
// the second reading the previous stage's T tile; step e = 0 only builds T(mt, -1). Per MAC this
// halves the operand bytes the producers write, the traffic that bounds the single-SM kernel.
//
// Pair tile: 512 outputs x 224 blocks, K step 256 entries (one 128-byte swizzle row), 6 stages.
//   warps 0-5   producers: warp s owns operand stage s and raw slot s, i.e. every 6th step; it
//               builds the 128 T rows of this CTA (funnel-shifted windows of the bit-reversed seed)
//               and its 112 X rows (from the packed raw tile TMA put in slot s). One arrival per
//               stage and CTA on the leader's barrier: the peer's is a cluster-scope release, whose
//               memory barrier then costs a warp once per 6 steps;
//   warp 6      TMA: packed raw tiles (112 blocks x 32 bytes) of this CTA's blocks, in step order;
//   warp 7      tensor memory allocation (both CTAs); in the leader CTA (rank 0) one lane issues the
//               cta_group::2 MMAs and multicasts their completion to both CTAs' barriers;
//   warps 8-15  epilogue: two warps per TMEM lane quarter, one per accumulator; each CTA reads its
//               128 rows of both accumulators (its outputs) from its own tensor memory in 32-column
//               loads double-buffered against the parity packing of the previous load (one add and
//               one funnel shift per count), hands the accumulators back as soon as its last load
//               has landed, and only then transposes the packed words (32 x 32 bits across the
//               warp) and stores them; identity XOR for the modified form.
// Both epilogues signal the leader's accumulator barrier. Every wait is bounded (about one second of
// clock): on timeout a CTA records an error code and stops; the leader still drains its MMAs, and
// both CTAs meet at a cluster barrier before tensor memory is released.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "qrng_internal.h"
#include "tc_util.cuh"

namespace qrng {
namespace {

using namespace tc;

constexpr int PM = 256;                  // outputs per output tile (UMMA M over the pair)
constexpr int HM = 128;                  // T rows per CTA
constexpr int BK = 256;                  // E2M1 entries per K step
constexpr int KW = BK / 32;              // packed words per row and step
constexpr int ROW_BYTES = 128;
constexpr int STAGES = 6;
constexpr int A_BYTES = HM * ROW_BYTES;  // 16 KB
constexpr int PK_STAGES = STAGES;
constexpr int PRODUCER_WARPS = STAGES;   // warp s builds every use of operand stage s
constexpr int T_ROWS = HM / 32;          // T rows lane + 32 j of a lane
constexpr int TMA_WARP = PRODUCER_WARPS;
constexpr int MMA_WARP = TMA_WARP + 1;
constexpr int EPI_WARP0 = MMA_WARP + 1;
constexpr int EPI_WARPS = 8;                           // two per TMEM lane quarter: one per accumulator
constexpr int THREADS = (EPI_WARP0 + EPI_WARPS) * 32;  // 512
constexpr int TMEM_COLS = 512;
constexpr uint32_t SFA_COL = 448;        // scale factors (all 2^0) of A, then of B
constexpr uint32_t SFB_COL = 480;
constexpr uint16_t kPairMask = 0x3;      // both CTAs of the cluster
static_assert(PK_STAGES == STAGES, "producer warp s owns operand stage s and raw slot s");

// Blocks per pair tile (UMMA N, 112 or 96 X rows per CTA); the launcher picks the width that wastes
// the fewest block columns over whole rounds of tiles.
template <int kPN>
struct PairShape {
  static constexpr int PN = kPN;
  static constexpr int HN = PN / 2;                      // X rows per CTA
  static constexpr int B_BYTES = HN * ROW_BYTES;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int PK_BYTES = HN * KW * 4;
  static constexpr int X_ROWS = (HN + 31) / 32;          // X rows lane + 32 j < HN of a lane
  static constexpr uint32_t D1_COL = PN;                 // second accumulator
  // kind::mxf4: A = B = E2M1 (1 at bits 7 and 10), K-major, N >> 3 at bit 17, UE8M0 scales (bit
  // 23), M >> 7 at bit 27 (M = 256 over the pair), dense K = 64.
  static constexpr uint32_t IDESC =
      (1u << 7) | (1u << 10) | ((uint32_t)(PN >> 3) << 17) | (1u << 23) | ((uint32_t)(PM >> 7) << 27);
  static_assert(STAGE_BYTES % 1024 == 0 && A_BYTES % 1024 == 0, "swizzle atoms must stay 1024-byte aligned");
  static_assert(HN % 8 == 0 && PN % 16 == 0 && 2 * PN <= (int)SFA_COL, "accumulators and scale factors must fit");
};

__device__ __forceinline__ void mma_pair(uint32_t tmem_d, uint32_t tmem_base, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(tmem_base + SFA_COL), "r"(tmem_base + SFB_COL), "r"(accumulate)
      : "memory");
}

// Arrives on the barrier at this offset in both CTAs once every MMA issued so far has completed.
__device__ __forceinline__ void commit_both(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(kPairMask)
      : "memory");
}

__device__ __forceinline__ void commit_local(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

struct PairArgs {
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
  uint32_t mpairs;   // pairs of output tiles
  uint32_t mtiles;   // output tiles holding needed rows: a pair's second tile at or past it gets no MMAs
  uint32_t ntiles;
  uint32_t ksteps;   // K steps per K block (plain product: all of them, one K block)
  int* err;
  int fault_no_tma;  // test hook: the loader publishes no raw tile, so every consumer's bounded wait runs out
  // block Karatsuba sub-products (kKara): group z of `groups` is the product of derived seed z
  // (seed_rev + z * seed_stride) with derived raw operand z (rows z * num_blocks + b of the raw
  // map); its rows and columns are the h-blocks of every span-th position of a Toeplitz matrix, so
  // each K block of h columns starts with a step that builds only the T tile left of it, and each
  // K block / row block shifts the seed window by span - h bits.
  uint32_t seed_front;   // front padding (words) of every seed buffer
  uint32_t seed_kstep;   // seed words per K step: KW, or span / 32 when every K step is one h-block
  uint32_t kblocks;      // K blocks of h columns (plain: 1)
  uint32_t seed_kshift;  // (span - h) / 32: seed words skipped per K block
  uint32_t xk_kwords;    // h / 32: raw-operand words per K block
  uint32_t log2h;
  uint32_t row_shift;    // span - h: seed bits skipped per row block
  uint32_t groups;
  uint64_t seed_stride;  // words per derived seed
  uint32_t* qpar;        // parities of the sub-products: word (b * groups + z) * mwq + row / 32
  uint32_t mwq;
  const int* skip;       // non-null: return at once unless *skip == 0 (written by an earlier kernel)
};

struct TileCoord {
  uint32_t mt;  // first output tile of the pair (rows mt*256 .. mt*256 + 511)
  uint32_t nt;  // block column tile
  uint32_t z;   // sub-product (Karatsuba groups; 0 otherwise)
};

// Row pairs fastest, then block tiles, then groups: tiles that run together share raw operand tiles.
template <bool kKara>
__device__ __forceinline__ TileCoord tile_coord(const PairArgs& a, uint64_t tile) {
  TileCoord t;
  t.mt = 2u * (uint32_t)(tile % a.mpairs);
  const uint64_t rest = tile / a.mpairs;
  if (kKara) {
    t.nt = (uint32_t)(rest % a.ntiles);
    t.z = (uint32_t)(rest / a.ntiles);
  } else {
    t.nt = (uint32_t)rest;
    t.z = 0;
  }
  return t;
}

template <int kPN, bool kKara>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_pair_kernel(const PairArgs a, const __grid_constant__ CUtensorMap raw_map) {
  using S = PairShape<kPN>;
  constexpr int PN = S::PN, HN = S::HN, STAGE_BYTES = S::STAGE_BYTES, PK_BYTES = S::PK_BYTES, X_ROWS = S::X_ROWS;
  constexpr uint32_t D1_COL = S::D1_COL;
  extern __shared__ uint8_t dyn_smem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];       // leader: the owning producer warp of both CTAs
  __shared__ __align__(8) uint64_t empty_bar[STAGES];      // both: the leader's MMA completion
  __shared__ __align__(8) uint64_t pk_full_bar[PK_STAGES];
  __shared__ __align__(8) uint64_t pk_empty_bar[PK_STAGES];
  __shared__ __align__(8) uint64_t accum_full_bar;         // both: the leader's MMA completion
  __shared__ __align__(8) uint64_t accum_empty_bar;        // leader: one arrival per epilogue warp of both CTAs
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ uint32_t epi_words[EPI_WARPS][kPN / 32][32];  // an epilogue warp's packed parity rows of a tile
  __shared__ volatile int abort_flag;

  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const uint32_t smem_base = (smem_u32(dyn_smem) + 1023u) & ~1023u;
  const uint32_t pk_base = smem_base + STAGES * STAGE_BYTES;

  // a hash enqueued before its output length was known: every thread of both CTAs reads the same
  // word (an earlier kernel wrote it), so the whole cluster leaves before any barrier or allocation
  if (a.skip != nullptr && *a.skip != 0) return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 2);  // the owning warp of each CTA
      mbar_init(&empty_bar[s], 1);
    }
    for (int s = 0; s < PK_STAGES; ++s) {
      mbar_init(&pk_full_bar[s], 1);
      mbar_init(&pk_empty_bar[s], 1);
    }
    mbar_init(&accum_full_bar, 1);
    mbar_init(&accum_empty_bar, 2 * EPI_WARPS);
    mbar_init(&drain_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster_sync();  // both CTAs' barriers exist before any remote arrival
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;
  if (warp >= EPI_WARP0 && warp < EPI_WARP0 + 4) {
    // every scale factor is 2^0: fill the 64 scale-factor columns in all 128 lanes, whatever cells
    // the MMAs read there
    const uint32_t lanes = (32u * (warp & 3u)) << 16;
    tmem_fill32(tmem_base + lanes + SFA_COL, kScaleOne);
    tmem_fill32(tmem_base + lanes + SFB_COL, kScaleOne);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync();  // both CTAs' scale factors are in place before the first MMA
  tc_fence_after();

  const uint64_t ntile_total = (uint64_t)a.mpairs * a.ntiles * (kKara ? a.groups : 1u);
  const uint64_t first_tile = blockIdx.x >> 1;
  const uint64_t tile_stride = gridDim.x >> 1;
  const uint32_t spb = a.ksteps + 1;  // steps per K block: the first builds T(mt, -1) of the block only
  const uint32_t nsteps = spb * (kKara ? a.kblocks : 1u);
  if (warp < PRODUCER_WARPS) {
    // ------------------------------------------------------------------ producers (warp = stage)
    const uint32_t st = warp;
    const uint32_t full_leader = mapa_shared(smem_u32(&full_bar[st]), 0);
    const uint32_t sA = smem_base + st * STAGE_BYTES;
    const uint32_t sB = sA + A_BYTES;
    const uint32_t pk = pk_base + st * PK_BYTES;
    uint32_t use = 0;   // uses of this stage so far
    uint32_t base = 0;  // index of the tile's step 0 modulo STAGES
    for (uint64_t tile = first_tile; tile < ntile_total && !abort_flag; tile += tile_stride) {
      const TileCoord tc = tile_coord<kKara>(a, tile);
      const uint32_t r0 = tc.mt * PM;
      // T row i = r0 + rank*128 + lane + 32 j at K step ks reads reversed-seed bits
      // m-1-i+BK*ks .. +BK-1 (Karatsuba: minus row_shift per row block, plus row_shift per K block);
      // rows 32 apart start one word apart at the same shift (the front padding keeps every index
      // >= 0, also for the window left of a K block)
      const int64_t vshift = kKara ? (int64_t)(r0 >> a.log2h) * a.row_shift : 0;
      const int64_t ubase = (int64_t)a.m - 1 - ((int64_t)r0 + rank * HM + lane) - vshift + 32 * (int64_t)a.seed_front;
      const uint32_t sh = (uint32_t)(ubase & 31);
      const uint32_t* seed_row = a.seed_rev + (kKara ? tc.z * a.seed_stride : 0) + (ubase >> 5);
      bool stop = false;
      for (uint32_t e = (st + STAGES - base) % STAGES; e < nsteps; e += STAGES) {
        const uint32_t ph = use & 1u;
        const uint32_t c = (kKara && a.kblocks > 1) ? e / spb : 0u;  // K block
        const uint32_t el = e - c * spb;          // step within it (0: the window left of the block)
        const uint32_t E = c * a.ksteps + el;     // K step of the X rows + 1 (el >= 1)
        // the seed words depend on no barrier: issue all of them first. Word k of row lane + 32 j is
        // the funnel shift of seed words win + k - j and win + k - j + 1, so the lane's T_ROWS rows
        // read KW + T_ROWS distinct words and share KW + T_ROWS - 1 shifted words.
        const uint32_t* win =
            seed_row + (int64_t)a.seed_kstep * ((int64_t)E - 1) + (kKara ? a.seed_kshift * c : 0u) - (T_ROWS - 1);
        uint32_t sw[KW + T_ROWS];
#pragma unroll
        for (int t = 0; t < KW + T_ROWS; ++t) sw[t] = __ldg(win + t);
        if (!mbar_wait(&pk_full_bar[st], ph, &abort_flag, a.err, 1)) { stop = true; break; }
        uint32_t xw[X_ROWS][KW];
        if (el > 0) {
          const uint32_t ks = E - 1;
#pragma unroll
          for (int j = 0; j < X_ROWS; ++j) {
            const uint32_t r = lane + 32u * j;
            if (r < (uint32_t)HN) {
#pragma unroll
              for (int h = 0; h < KW / 4; ++h)
                asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(xw[j][4 * h]), "=r"(xw[j][4 * h + 1]), "=r"(xw[j][4 * h + 2]),
                               "=r"(xw[j][4 * h + 3])
                             : "r"(pk + r * (KW * 4) + 16 * h)
                             : "memory");
            }
          }
          // words past the Toeplitz part (zero-filled) and its partial last word; the Karatsuba
          // operands are zero past it already
          if (!kKara && KW * ks + KW > a.nw_t - 1) {
#pragma unroll
            for (int w = 0; w < KW; ++w)
              if (KW * ks + w == a.nw_t - 1) {
#pragma unroll
                for (int j = 0; j < X_ROWS; ++j) xw[j][w] &= a.tail_mask;
              }
          }
        }
        if (!mbar_wait(&empty_bar[st], ph ^ 1u, &abort_flag, a.err, 2)) { stop = true; break; }
#pragma unroll
        for (int t = 0; t < KW + T_ROWS - 1; ++t) {  // shifted word t: word k = t - (T_ROWS - 1) + j of row j
          const E2m1Chunk ch = e2m1_chunk(__funnelshift_r(sw[t], sw[t + 1], sh));
#pragma unroll
          for (int j = 0; j < T_ROWS; ++j) {
            const int k = t - (T_ROWS - 1) + j;
            if (k >= 0 && k < KW) {
              const uint32_t r = lane + 32u * j;
              store_chunk_e2m1(sA + r * ROW_BYTES, r, (uint32_t)k, ch);
            }
          }
        }
        if (el > 0) {
#pragma unroll
          for (int j = 0; j < X_ROWS; ++j) {
            const uint32_t r = lane + 32u * j;
            if (r < (uint32_t)HN) {
#pragma unroll
              for (int w = 0; w < KW; ++w) store_word_e2m1(sB + r * ROW_BYTES, r, w, xw[j][w]);
            }
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&pk_empty_bar[st]);  // the raw words have been consumed by the stores above
          if (rank == 0)
            mbar_arrive(&full_bar[st]);
          else
            mbar_arrive_cluster(full_leader);
        }
        __syncwarp();
        ++use;
      }
      if (stop) break;
      base = (uint32_t)((base + nsteps) % STAGES);
    }
  } else if (warp == TMA_WARP) {
    // ------------------------------------------------------------------ TMA loads of packed raw tiles
    // one load per step (the first step of a K block loads the block's first tile as well,
    // unused), so that raw slot s and operand stage s advance together
    uint32_t pstage = 0, pphase = 0, issued = 0;
    if (lane == 0) {
      for (uint64_t tile = first_tile; tile < ntile_total && !abort_flag; tile += tile_stride) {
        const TileCoord tc = tile_coord<kKara>(a, tile);
        const int row = (int)((kKara ? (uint64_t)tc.z * a.num_blocks : 0ull) + (uint64_t)tc.nt * PN + rank * HN);
        for (uint32_t e = 0; e < nsteps; ++e) {
          const uint32_t c = (kKara && a.kblocks > 1) ? e / spb : 0u;
          const uint32_t el = e - c * spb;
          if (!mbar_wait(&pk_empty_bar[pstage], pphase ^ 1u, &abort_flag, a.err, 3)) break;
          if (!a.fault_no_tma) {
            mbar_arrive_expect_tx(&pk_full_bar[pstage], PK_BYTES);
            tma_load_2d(pk_base + pstage * PK_BYTES, &raw_map,
                        (int)((kKara ? c * a.xk_kwords : 0u) + KW * (el > 0 ? el - 1 : 0)), row,
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
    // ------------------------------------------------------------------ MMA issuer (leader CTA)
    // One thread runs the whole issue loop: the tensor pipe's queue is shallow, so every
    // instruction between two steps' MMAs can leave it idle (no warp-wide waits, no per-step
    // warp synchronisation, descriptors as per-stage bases plus 2 k).
    if (rank == 0 && lane == 0) {
      uint32_t stage = 0, phase = 0, acc_phase = 0, prev = 0;
      bool issued = false;
      for (uint64_t tile = first_tile; tile < ntile_total && !abort_flag; tile += tile_stride) {
        // both epilogues must have drained the previous tile's accumulators
        if (tile != first_tile && !mbar_wait<true>(&accum_empty_bar, acc_phase ^ 1u, &abort_flag, a.err, 5)) break;
        // a pair whose second output tile holds no needed row (an odd number of row tiles) issues
        // the first tile's MMAs only
        const bool d1_live = 2u * ((uint32_t)tile % a.mpairs) + 1u < a.mtiles;  // tile < 2^32
        bool done = true;
        uint32_t c = 0, el = 0;  // K block and step within it (0: the build-only step)
        for (uint32_t e = 0; e < nsteps; ++e) {
          if (!mbar_wait<true>(&full_bar[stage], phase, &abort_flag, a.err, 6)) { done = false; break; }
          tc_fence_after();
          if (e > 0) {
            if (el > 0) {
              const uint32_t E = c * a.ksteps + el;
              const uint32_t sA = smem_base + stage * STAGE_BYTES;  // T(mt, ks)
              const uint64_t dA = kDescSw128Hi | (uint64_t)((sA & 0x3FFFFu) >> 4);
              const uint64_t dB = kDescSw128Hi | (uint64_t)(((sA + A_BYTES) & 0x3FFFFu) >> 4);  // X(ks)
              const uint64_t dP = kDescSw128Hi | (uint64_t)(((smem_base + prev * STAGE_BYTES) & 0x3FFFFu) >> 4);
              if (d1_live) {
#pragma unroll
                for (int k = 0; k < ROW_BYTES / 32; ++k) {  // 32 bytes = 2 descriptor units per K chunk
                  const uint32_t acc = (E > 1 || k > 0) ? 1u : 0u;
                  mma_pair(tmem_base, tmem_base, dA + 2 * k, dB + 2 * k, S::IDESC, acc);
                  mma_pair(tmem_base + D1_COL, tmem_base, dP + 2 * k, dB + 2 * k, S::IDESC, acc);  // T(mt+1, ks)
                }
              } else {
#pragma unroll
                for (int k = 0; k < ROW_BYTES / 32; ++k)
                  mma_pair(tmem_base, tmem_base, dA + 2 * k, dB + 2 * k, S::IDESC, (E > 1 || k > 0) ? 1u : 0u);
              }
            }
            commit_both(&empty_bar[prev]);  // the previous stage's T tile is not read again
            issued = true;
          }
          prev = stage;
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
          if (++el == spb) { el = 0; ++c; }  // the next step's place in its K block
        }
        if (!done || abort_flag) break;
        commit_both(&empty_bar[prev]);  // the tile's last stage
        commit_both(&accum_full_bar);
        acc_phase ^= 1u;
      }
      // every MMA must finish before either CTA releases its tensor or shared memory
      if (issued) {
        commit_local(&drain_bar);
        mbar_drain(&drain_bar, 0, a.err, 7);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------------ epilogue
    // warp EPI_WARP0 + 4 hs + q drains accumulator hs (D0 or D1) in TMEM lanes 32 q .. 32 q + 31:
    // 32-column loads double-buffered against the parity packing of the previous load, and the
    // accumulator handed back to the MMA issuer as soon as its last load has landed; the
    // transposes (lane c ends with column c's word: one output word per lane and load) and the
    // global stores follow, overlapping the next tile's MMAs
    const uint32_t q = warp & 3u;  // TMEM lane quarter this warp may access
    const uint32_t hs = (warp - EPI_WARP0) >> 2;
    constexpr uint32_t NW = PN / 32;  // 32-column loads (output words) per accumulator
    const uint32_t accum_empty_leader = mapa_shared(smem_u32(&accum_empty_bar), 0);
    uint32_t* words = &epi_words[warp - EPI_WARP0][0][0];  // [word][lane]: packed rows until the transpose
    // transpose stage l (j = 2^l): a lane keeps the columns whose bit l equals its own lane bit l
    // and takes the others from lane ^ j, whose word is rotated by j towards them; the bits a
    // rotation wraps around fall in the kept columns
    uint32_t xkeep[5], xrot[5];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
      const uint32_t j = 1u << l;
      const uint32_t m = l == 4 ? 0x0000FFFFu : l == 3 ? 0x00FF00FFu : l == 2 ? 0x0F0F0F0Fu
                         : l == 1 ? 0x33333333u : 0x55555555u;  // columns with bit l clear
      xkeep[l] = (lane & j) ? ~m : m;
      xrot[l] = (lane & j) ? 32u - j : j;
    }
    uint32_t acc_phase = 0;
    for (uint64_t tile = first_tile; tile < ntile_total && !abort_flag; tile += tile_stride) {
      const TileCoord tc = tile_coord<kKara>(a, tile);
      const uint32_t nt = tc.nt;
      if (!mbar_wait(&accum_full_bar, acc_phase, &abort_flag, a.err, 8)) break;
      tc_fence_after();
      if (hs == 1 && tc.mt + 1 >= a.mtiles) {  // this pair's second tile got no MMAs: nothing to drain
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster_relaxed(accum_empty_leader);
        __syncwarp();
        acc_phase ^= 1u;
        continue;
      }
      const uint32_t ow = (tc.mt + hs) * (PM / 32) + rank * (HM / 32) + q;  // output word of every block
      const uint32_t rem = (ow < a.mw) ? a.m - 32 * ow : 0u;
      const uint32_t omask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
      const uint32_t taddr = tmem_base + ((32u * q) << 16) + hs * D1_COL;
      // Lane r packs the parities of its row for each 32-column load (bit c = column c) as soon as
      // the load lands, the next load in flight meanwhile; the accumulator goes back to the MMA
      // issuer when the last load has landed. Only then does a 32 x 32 bit transpose across the
      // warp leave column c's 32 rows in lane c (stage j exchanges bit j of the row and column
      // indices: one shuffle, one rotate and one select), for all NW words at once, so that the
      // shuffles of different words overlap and none of it delays the next tile's MMAs.
      auto release = [&]() {  // every TMEM load of this warp has completed (the values are in registers)
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster_relaxed(accum_empty_leader);
      };
      uint32_t va[32], vb[32];
      tmem_load32_async(taddr, va);
      tmem_wait_ld(va);
#pragma unroll 1
      for (uint32_t g = 0; g < NW; g += 2) {  // load g is in va and has landed
        if (g + 1 < NW)
          tmem_load32_async(taddr + 32u * (g + 1), vb);
        else
          release();
        words[g * 32 + lane] = pack_parities32(va);
        if (g + 1 < NW) {
          tmem_wait_ld(vb);
          if (g + 2 < NW)
            tmem_load32_async(taddr + 32u * (g + 2), va);
          else
            release();
          words[(g + 1) * 32 + lane] = pack_parities32(vb);
          if (g + 2 < NW) tmem_wait_ld(va);
        }
      }
      uint32_t xw[NW];
#pragma unroll
      for (uint32_t g = 0; g < NW; ++g) xw[g] = words[g * 32 + lane];
#pragma unroll
      for (int l = 4; l >= 0; --l) {
#pragma unroll
        for (uint32_t g = 0; g < NW; ++g) {
          const uint32_t t = __shfl_xor_sync(0xffffffffu, xw[g], 1u << l);
          const uint32_t r = __funnelshift_l(t, t, xrot[l]);
          xw[g] = (xw[g] & xkeep[l]) | (r & ~xkeep[l]);
        }
      }
#pragma unroll
      for (uint32_t g = 0; g < NW; ++g) {  // lane c: column 32 g + c of the tile
        const uint32_t word = xw[g];
        const uint64_t b = (uint64_t)nt * PN + 32u * g + lane;
        if (kKara) {  // every row of a sub-product is kept: the combining pass selects and masks
          if (b < a.num_blocks) a.qpar[((uint64_t)b * a.groups + tc.z) * a.mwq + ow] = word;
        } else if (ow < a.mw && b < a.num_blocks) {
          uint32_t w = word & omask;
          if (a.modified) {
            const uint64_t bit = (uint64_t)a.id_off + 32ull * ow;
            const uint32_t* rr = a.raw + b * a.raw_stride;
            const uint64_t rq = bit >> 5;
            const uint32_t rs = (uint32_t)(bit & 31);
            const uint32_t rlo = __ldg(rr + rq);
            const uint32_t rhi = (rs && rq + 1 < a.raw_stride) ? __ldg(rr + rq + 1) : 0u;
            w ^= __funnelshift_r(rlo, rhi, rs) & omask;
          }
          a.out[b * a.out_stride + ow] = w;
        }
      }
      __syncwarp();
      acc_phase ^= 1u;
    }
  }

  tc_fence_before();
  cluster_sync();  // the leader's MMAs have drained; neither CTA touches the other's memory after this
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
}

}  // namespace

typedef CUresult (*PFN_encodeTiled_pair)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                         const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                         CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                         CUtensorMapFloatOOBfill);

template <int kPN>
static size_t pair_smem_bytes() {
  return (size_t)STAGES * PairShape<kPN>::STAGE_BYTES + (size_t)PK_STAGES * PairShape<kPN>::PK_BYTES + 1024;
}

// Tensor map over 32-bit words: dim 0 = `words` words of a row (reads beyond them are zero-filled),
// dim 1 = `rows` rows `stride_words` apart (rows past the last are zero-filled); box 8 words x
// `box_rows` rows, every x coordinate a multiple of 8 words (32 bytes).
static cudaError_t encode_words_map(CUtensorMap* map, const uint32_t* base, uint64_t words, uint64_t rows,
                                    uint64_t stride_words, uint32_t box_rows) {
  static PFN_encodeTiled_pair encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_encodeTiled_pair>(fn);
  }
  const cuuint64_t gdim[2] = {(cuuint64_t)words, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)stride_words * 4};
  const cuuint32_t box[2] = {(cuuint32_t)KW, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t*>(base), gdim, gstride, box,
                      estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int kPN, bool kKara>
static cudaError_t launch_pair(const PairArgs& a0, const CUtensorMap& map, int num_sms, cudaStream_t s,
                               uint32_t* kernels) {
  using S = PairShape<kPN>;
  PairArgs a = a0;
  a.ntiles = (uint32_t)ceil_div(a.num_blocks, S::PN);
  const size_t smem = pair_smem_bytes<kPN>();
  // the shared-memory attribute and the number of co-resident clusters are set and queried once
  // per device (they do not change), so that the launch adds no driver round trips to a call
  constexpr int kMaxDev = 64;
  static int clusters_of[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < kMaxDev && clusters_of[dev] > 0;
  if (!cached) {
    e = cudaFuncSetAttribute(gemm_pair_kernel<kPN, kKara>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const uint64_t tiles = (uint64_t)a.mpairs * a.ntiles * (kKara ? a.groups : 1u);
  if (tiles >= (1ull << 32)) return cudaErrorInvalidValue;  // the issuer takes tile indices as 32-bit
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * (tiles < (uint64_t)num_sms / 2 ? tiles : (uint64_t)num_sms / 2)));
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // one cluster per co-resident pair of SMs: every tile loop stride then runs concurrently
  int clusters = cached ? clusters_of[dev] : 0;
  if (!cached) {
    cfg.gridDim = dim3((unsigned)(num_sms / 2 > 0 ? 2 * (num_sms / 2) : 2));
    e = cudaOccupancyMaxActiveClusters(&clusters, gemm_pair_kernel<kPN, kKara>, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorNotSupported;
    if (dev >= 0 && dev < kMaxDev) clusters_of[dev] = clusters;
  }
  const uint64_t pairs = tiles < (uint64_t)clusters ? tiles : (uint64_t)clusters;
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  e = cudaLaunchKernelEx(&cfg, gemm_pair_kernel<kPN, kKara>, a, map);
  if (e != cudaSuccess) return e;
  ++*kernels;
  return cudaGetLastError();
}

// Tile width: block columns computed over whole rounds of tiles (one round = one tile per cluster
// of the pairs that fit), the narrower tile's columns weighted by its measured cost per column
// (more operand bytes per MAC: 1.07x on the 2^29-bit laser stream).
static bool pair_prefers_192(uint64_t row_tiles, uint64_t num_blocks, int num_sms) {
  const uint64_t rounds_cap = (uint64_t)(num_sms / 2 > 0 ? num_sms / 2 : 1);
  auto cost = [&](uint64_t pn, double per_col) {
    const uint64_t tiles = row_tiles * ceil_div(num_blocks, pn);
    return (double)(ceil_div(tiles, rounds_cap) * pn) * per_col;
  };
  return cost(192, 1.07) < cost(224, 1.0);
}

static PairArgs pair_args_from(const DirectArgs& d, int* err, int fault) {
  PairArgs a{};
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
  a.err = err;
  a.fault_no_tma = (fault == QRNG_FAULT_GEMM_NO_TMA);
  a.seed_front = kSeedFrontWords;
  a.seed_kstep = KW;
  a.kblocks = 1;
  a.groups = 1;
  return a;
}

cudaError_t launch_gemm_pair(const DirectArgs& d, int* err, int fault, int num_sms, cudaStream_t s,
                             uint32_t* kernels) {
  if ((reinterpret_cast<uintptr_t>(d.raw) & 15) != 0 || (d.raw_stride % 4) != 0) return cudaErrorInvalidValue;
  PairArgs a = pair_args_from(d, err, fault);
  a.mtiles = (uint32_t)ceil_div(d.m, PM);
  a.mpairs = (uint32_t)ceil_div(a.mtiles, 2);
  a.ksteps = (uint32_t)ceil_div((uint64_t)d.nw_t * 32, BK);
  CUtensorMap map;
  const bool narrow = pair_prefers_192(a.mpairs, d.num_blocks, num_sms);
  cudaError_t e = encode_words_map(&map, d.raw, d.nw_t, d.num_blocks, d.raw_stride, narrow ? 96 : 112);
  if (e != cudaSuccess) return e;
  return narrow ? launch_pair<192, false>(a, map, num_sms, s, kernels)
                : launch_pair<224, false>(a, map, num_sms, s, kernels);
}

cudaError_t launch_gemm_pair_kara(const DirectArgs& d, const PairKara& k, int* err, int fault, int num_sms,
                                  cudaStream_t s, uint32_t* kernels) {
  if ((reinterpret_cast<uintptr_t>(k.xk) & 15) != 0 || (k.xk_words % 8) != 0 || k.h < 256 ||
      (k.h & (k.h - 1)) != 0 || k.mq % 512 != 0 || k.mq % k.h != 0 || k.kq % k.h != 0 || k.span % k.h != 0)
    return cudaErrorInvalidValue;
  if ((uint64_t)k.groups * d.num_blocks >= (1ull << 31)) return cudaErrorInvalidValue;
  PairArgs a = pair_args_from(d, err, fault);
  a.seed_rev = k.seeds;
  a.seed_front = k.seed_front;
  a.mpairs = (uint32_t)(k.mq / (2 * PM));
  a.mtiles = (uint32_t)ceil_div(k.mq_live, PM);
  if (k.h == BK) {
    // every tile row block and every K step is a whole h-block: block (R+1, c) = block (R, c-1), so
    // the two output tiles share T tiles along the block diagonal like the plain product, one K
    // sequence with the seed window moving span bits per step
    a.ksteps = (uint32_t)(k.kq / BK);
    a.kblocks = 1;
    a.seed_kshift = 0;
    a.seed_kstep = (uint32_t)(k.span / 32);
  } else {
    a.ksteps = (uint32_t)(k.h / BK);
    a.kblocks = (uint32_t)(k.kq / k.h);
    a.seed_kshift = (uint32_t)((k.span - k.h) / 32);
  }
  a.xk_kwords = (uint32_t)(k.h / 32);
  uint32_t lg = 0;
  while ((1ull << lg) < k.h) ++lg;
  a.log2h = lg;
  a.row_shift = (uint32_t)(k.span - k.h);
  a.groups = k.groups;
  a.seed_stride = k.seed_stride;
  a.qpar = k.qpar;
  a.mwq = (uint32_t)(k.mq / 32);
  a.skip = k.skip;
  CUtensorMap map;
  const bool narrow = pair_prefers_192((uint64_t)a.mpairs * k.groups, d.num_blocks, num_sms);
  cudaError_t e = encode_words_map(&map, k.xk, k.xk_words, (uint64_t)k.groups * d.num_blocks, k.xk_words,
                                   narrow ? 96 : 112);
  if (e != cudaSuccess) return e;
  return narrow ? launch_pair<192, true>(a, map, num_sms, s, kernels)
                : launch_pair<224, true>(a, map, num_sms, s, kernels);
}

}  // namespace qrng
