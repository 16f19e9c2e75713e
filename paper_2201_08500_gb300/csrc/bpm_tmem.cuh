// Tensor memory (TMEM) as per-thread table storage.
//
// TMEM is the 256 KB per-SM array (128 lanes x 512 columns of 32 bits) that
// tcgen05 instructions address.  Warp w of a block may access lanes
// 32 (w % 4) .. 32 (w % 4) + 31; each thread reads and writes its own lane.
// Here each thread keeps its propagator-table slice (hi/lo float4 per position
// and envelope, 128 columns) in its lane, so the table multiply of every step
// reads TMEM instead of shared memory or L2.  A block allocates its columns
// once (warp 0, a power of two >= 32), gives up the permit to allocate again,
// and frees them before it exits; every tcgen05 access of a thread is followed
// by the matching wait before its registers (or the location) are reused.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace bpm {

#define BPM_TM __device__ __forceinline__

// Warp-collective allocation of ncols columns; the TMEM address is written to
// *slot (shared memory) and visible to the block after tmem_sync().
template <int NCOLS>
BPM_TM void tmem_alloc(uint32_t* slot) {
  static_assert(NCOLS >= 32 && NCOLS <= 512 && (NCOLS & (NCOLS - 1)) == 0, "TMEM columns");
  const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(slot));
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(dst), "n"(NCOLS) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

template <int NCOLS>
BPM_TM void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOLS)
               : "memory");
}

// Block barrier ordered with the tcgen05 operations before and after it.
BPM_TM void tmem_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive 32-bit columns of the thread's lane.
BPM_TM void tmem_st16(uint32_t taddr, const float4 (&v)[4]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "f"(v[0].x), "f"(v[0].y), "f"(v[0].z), "f"(v[0].w), "f"(v[1].x), "f"(v[1].y), "f"(v[1].z),
      "f"(v[1].w), "f"(v[2].x), "f"(v[2].y), "f"(v[2].z), "f"(v[2].w), "f"(v[3].x), "f"(v[3].y),
      "f"(v[3].z), "f"(v[3].w)
      : "memory");
}

BPM_TM void tmem_ld16(uint32_t taddr, float4 (&v)[4]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[0].z), "=f"(v[0].w), "=f"(v[1].x), "=f"(v[1].y),
        "=f"(v[1].z), "=f"(v[1].w), "=f"(v[2].x), "=f"(v[2].y), "=f"(v[2].z), "=f"(v[2].w),
        "=f"(v[3].x), "=f"(v[3].y), "=f"(v[3].z), "=f"(v[3].w)
      : "r"(taddr)
      : "memory");
}

BPM_TM void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
BPM_TM void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace bpm
