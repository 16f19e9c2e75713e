// Bulk asynchronous copies (the TMA engine) and mbarrier completion, in inline
// PTX, for the 3D passes' streamed column and row tiles.
//
// A copy is issued by one thread; the bytes it moves are counted against an
// mbarrier in shared memory (expect_tx), and threads wait for the barrier's
// phase to complete before they read the tile.  Every wait is bounded: after
// kTmaSpinLimit unsuccessful polls it gives up and the caller records an error
// status for the host instead of spinning forever.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace bpm {

#define BPM_TMA __device__ __forceinline__

// Polls of one wait before it gives up (each mbarrier.try_wait itself blocks
// for a bounded, hardware-defined time; a completed copy is seen within a few
// polls).
constexpr uint32_t kTmaSpinLimit = 1u << 22;

// Status word values written by a pass that gave up on a wait.
constexpr int kStatusTmaTimeout = 0x7A;

BPM_TMA uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

BPM_TMA void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Makes initialised barriers visible to the async proxy (the copy engine).
BPM_TMA void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies (async proxy) into the same memory.
BPM_TMA void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of copies to complete this phase.
BPM_TMA void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Contiguous global -> shared copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing on `bar`.
BPM_TMA void bulk_load(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(smem_dst)), "l"(gmem_src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Tiled 2D tensor copy global -> shared of the box at element coordinates
// (x, y) of the tensor map (a __grid_constant__ kernel parameter), completing
// on `bar`.  x times the element size must be a multiple of 16 bytes.
BPM_TMA void tma_load_2d(void* smem_dst, const void* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_addr(smem_dst)), "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// Tiled 2D tensor copy shared -> global of the box at (x, y), x >= 0 and
// y >= 0, in the current bulk group of this thread.
BPM_TMA void tma_store_2d(const void* map, int x, int y, const void* smem_src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(map), "r"(x), "r"(y), "r"(smem_addr(smem_src))
               : "memory");
}

// Closes this thread's current bulk group of stores.
BPM_TMA void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Waits until every committed store group of this thread has read its shared
// memory (the source may then be rewritten).
BPM_TMA void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Waits until every committed store group of this thread is complete.
BPM_TMA void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

BPM_TMA bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase of parity `parity` to complete; false on time-out.
BPM_TMA bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kTmaSpinLimit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace bpm
