// Pipelined plan kernels: the persistent, warp-specialised form of the plain tile pass.
//
// One CTA per SM runs a ring of S shared-memory tile slots.  A producer warp streams
// tiles from HBM into free slots with TMA tensor copies (cp.async.bulk.tensor, eight
// 128-byte rows per copy, the copy engine's 128-byte swizzle) and signals each slot's
// "full" mbarrier through the copies' transaction count; G compute groups (2^(m-1-kpr)
// threads each) take the CTA's tiles in turn, run the pass's stages on the slot through
// registers (tile_pack.cuh), and hand the slot back on its "empty" mbarrier.  When the
// last stage's quarter warps hold whole 128-byte rows (its lane bits are tile bits 1..3),
// it stores straight from registers to HBM and releases the slot as soon as it has read
// it; otherwise it writes the tile back into the slot in memory order and the producer
// writes the slot out with TMA tensor stores before it reloads it.  So a group never waits
// for a tile read (each group owns S / G slots: one computes while the others load) and
// the copy engine, not the compute warps, moves the input (and, in the second case, the
// output).
//
// Every wait is bounded (kWaitNs): a wait that gives up makes the CTA stop, set the
// plan's error word and return.
#pragma once

#include "plan_dev.h"

namespace svk {
namespace tpipe {

// A CUtensorMap as the kernel receives it (128 bytes, 64-byte aligned, by value).
struct __align__(64) TmaDesc {
  unsigned long long w[16];
};

constexpr unsigned long long kWaitNs = 1000000000ull;  // give up a wait after 1 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of the given parity to complete; false if it did not within limit_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (global_ns() - t0 < limit_ns)
    if (mbar_try(bar, parity)) return true;
  return false;
}

// Barrier of the `count` threads of one compute group (named barrier `id` >= 1); returns
// whether any of them passed a true `pred` (all threads receive the same answer).
__device__ __forceinline__ bool group_any(int id, int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void group_sync(int id, int count) {
  asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Order this thread's generic-proxy shared-memory accesses before later async-proxy
// (TMA) accesses of the same slot.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One 5-d tensor copy: the box at coordinates (c0..c4) into shared memory at dst,
// completing `bar`'s transaction count.
__device__ __forceinline__ void tma_load_5d(void *dst, const TmaDesc *map, int c0, int c1, int c2, int c3, int c4,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

// The reverse: the box at dst's coordinates written from shared memory at src (one bulk
// group per commit; the source must not change until the group has been read).
__device__ __forceinline__ void tma_store_5d(const TmaDesc *map, int c0, int c1, int c2, int c3, int c4,
                                             const void *src) {
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(
          reinterpret_cast<unsigned long long>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until every committed bulk group has finished reading its shared-memory source.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Wait until every committed bulk group has completed (its writes are done).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// The tile of a CTA's turn i.  The CTAs take runs of 2^B neighbouring tile ids per turn
// of the grid (B = 0 when num_tiles is not a multiple of 2^B): turns i and i + 1 of a CTA
// are tiles t and t + 1, which differ in the lowest qubit outside the tile.  When that
// qubit is qubit 4, their 128-byte rows are the two halves of 256-byte blocks, read (and
// written) by one SM a turn apart instead of by two SMs whose turns drift apart over the
// sweep.  For a fixed CTA the runs' first tiles increase with i, and a run lies wholly
// below num_tiles or wholly at or above it.
template <int B>
__device__ __forceinline__ unsigned long long tile_of(unsigned long long i, unsigned long long num_tiles) {
  const int b = (num_tiles & ((1ull << B) - 1)) ? 0 : B;
  return ((blockIdx.x + (i >> b) * gridDim.x) << b) | (i & ((1ull << b) - 1));
}
// The number of tiles tile_of<B> gives this CTA.
template <int B>
__device__ __forceinline__ unsigned long long tiles_of_cta(unsigned long long num_tiles) {
  const int b = (num_tiles & ((1ull << B) - 1)) ? 0 : B;
  const unsigned long long runs = num_tiles >> b;
  return (blockIdx.x < runs ? (runs - blockIdx.x + gridDim.x - 1) / gridDim.x : 0ull) << b;
}

// Global index offset of group g's element 0 in a stage (the G half of the stage's
// group-addressing entries).
__device__ __forceinline__ uint64_t group_global(const DevPlanView &plan, uint32_t si, int g) {
  const svp::DevGroupEntry *t = plan.gtab + svp::kGroupEntries * si;
  return t[g & 15].G ^ t[16 + ((g >> 4) & 15)].G ^ t[32 + ((g >> 8) & 15)].G;
}

}  // namespace tpipe
}  // namespace svk
