// Device helpers shared by the tensor-core extraction kernels: mbarriers with bounded waits,
// tcgen05 fences and tensor-memory moves, shared-memory matrix descriptors, TMA tile loads, the
// E2M1 operand encoding, and the cluster primitives of the SM-pair kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qrng {
namespace tc {

constexpr long long kWaitCycles = 2000000000ll;  // ~1 s at 2 GHz
constexpr uint32_t kOneE2M1 = 0x2u;              // 1.0
constexpr uint32_t kScaleOne = 0x7F7F7F7Fu;      // four UE8M0 scale factors 2^0

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Phase test; kCluster selects cluster-scope acquire (arrivals that come from the peer CTA).
template <bool kCluster = false>
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  if constexpr (kCluster) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return ok != 0;
}

// Bounded wait on phase `parity`; on timeout records `code` and raises the CTA abort flag.
template <bool kCluster = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code) {
  if (mbar_test<kCluster>(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (*abort_flag) return false;
    if (mbar_test<kCluster>(bar, parity)) return true;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      atomicCAS(err, 0, code);
      return false;
    }
  }
}

// Bounded wait that ignores the abort flag (used to drain the CTA's own asynchronous work).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity, int* err, int code) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicCAS(err, 0, code);
      return;
    }
  }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// K-major, SWIZZLE_128B shared-memory matrix descriptor (rows of 128 bytes, 8-row atoms 1024 B apart):
// every field but the start address (bits 0-13, address >> 4)
constexpr uint64_t kDescSw128Hi = ((uint64_t)(16u >> 4) << 16)     // leading byte offset (unused for swizzled K-major)
                                  | ((uint64_t)(1024u >> 4) << 32)  // stride byte offset: next 8-row atom
                                  | ((uint64_t)1 << 46)             // descriptor version
                                  | ((uint64_t)2 << 61);            // SWIZZLE_128B
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return kDescSw128Hi | (uint64_t)((addr & 0x3FFFFu) >> 4);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Fills 32 TMEM columns of this warp's 32 lanes with the value v.
__device__ __forceinline__ void tmem_fill32(uint32_t taddr, uint32_t v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
      "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(v)
      : "memory");
}

// Reads 32 TMEM columns of this warp's 32 lanes (one value per column) and waits for them.
__device__ __forceinline__ void tmem_load32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Starts reading 32 TMEM columns of this warp's 32 lanes into v; the values may be used only after
// tmem_wait_ld(v).
__device__ __forceinline__ void tmem_load32_async(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

// Waits for every TMEM load of this thread; v is passed through so that no use of the registers
// being loaded can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                 "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]),
                 "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]),
                 "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
               :
               : "memory");
}

// 16-column variants of the two above.
__device__ __forceinline__ void tmem_load16_async(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                 "+r"(v[15])
               :
               : "memory");
}

// Writes 32 bits of one row as one 16-byte chunk of E2M1 nibbles into a 128-byte SWIZZLE_128B row:
// chunk word q holds bits q, q+4, ..., q+28 (one shift and one mask each). T and X rows use the
// same permutation of K, which leaves every dot product unchanged.
__device__ __forceinline__ void store_word_e2m1(uint32_t row_addr, uint32_t row, uint32_t w, uint32_t x) {
  constexpr uint32_t kMask = kOneE2M1 * 0x11111111u;
  const uint32_t addr = row_addr + (((w ^ (row & 7u)) & 7u) << 4);
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"((x << 1) & kMask), "r"(x & kMask),
               "r"((x >> 1) & kMask), "r"((x >> 2) & kMask)
               : "memory");
}

// The same chunk computed once (e2m1_chunk) and stored to several rows (store_chunk_e2m1).
struct E2m1Chunk {
  uint32_t a, b, c, d;
};
__device__ __forceinline__ E2m1Chunk e2m1_chunk(uint32_t x) {
  constexpr uint32_t kMask = kOneE2M1 * 0x11111111u;
  return E2m1Chunk{(x << 1) & kMask, x & kMask, (x >> 1) & kMask, (x >> 2) & kMask};
}
__device__ __forceinline__ void store_chunk_e2m1(uint32_t row_addr, uint32_t row, uint32_t w, const E2m1Chunk& c) {
  const uint32_t addr = row_addr + (((w ^ (row & 7u)) & 7u) << 4);
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(c.a), "r"(c.b), "r"(c.c), "r"(c.d)
               : "memory");
}

// Parity of the integer count held (scaled by `scale`) in an FP32 accumulator: adding 1.5 * 2^23
// leaves the count, < 2^22, in the low mantissa bits.
__device__ __forceinline__ uint32_t count_parity(uint32_t acc_bits, float scale) {
  return __float_as_uint(__fmaf_rn(__uint_as_float(acc_bits), scale, 12582912.0f)) & 1u;
}

// The parities of 32 unscaled counts (FP32 accumulators, each an integer below 2^22) as one word,
// bit c = parity of v[c]. After the 1.5 * 2^23 addition the parity is bit 0 of the sum's encoding;
// a funnel shift by one moves it into the top of a word being filled, so each count costs one add
// and one shift. Four independent chains of 8 (columns 8k .. 8k+7 end in the top byte of chain k)
// keep the dependent shifts short; three byte permutations join them.
__device__ __forceinline__ uint32_t pack_parities32(const uint32_t (&v)[32]) {
  uint32_t c[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      c[k] = __funnelshift_r(c[k], __float_as_uint(__uint_as_float(v[8 * k + i]) + 12582912.0f), 1);
  }
  const uint32_t lo = __byte_perm(c[0], c[1], 0x0073);  // byte 3 of chain 0, byte 3 of chain 1
  const uint32_t hi = __byte_perm(c[2], c[3], 0x0073);
  return __byte_perm(lo, hi, 0x5410);
}

// ---- clusters of two CTAs (the SM-pair kernel) ----

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Address of the same shared-memory variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// The same arrival without release semantics, for a signal that publishes no memory: it does not
// wait until the thread's earlier global stores are visible cluster-wide (measured: about 1100
// clocks after a tile's output stores). Only for resources whose last use by this thread has
// already completed, e.g. tensor memory after tcgen05.wait::ld.
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// Every thread of both CTAs; orders everything before it against everything after it, cluster-wide.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

}  // namespace tc
}  // namespace qrng
