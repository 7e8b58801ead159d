// Tensor Memory (TMEM) helpers for sm_103a: inline PTX for tcgen05 allocation, 32-column
// loads of a thread's own TMEM lane, and the waits and fences that order them.
//
// TMEM is 128 lanes x 512 columns of 32-bit cells per SM; warp w of a CTA reaches lanes
// 32*(w%4) .. 32*(w%4)+31 only.  The BF16 cross-term kernel keeps its FP32 accumulator tile
// there (row m of D in lane m) and reads it back row by row.
#pragma once
#include <stdint.h>

namespace nlemk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Whole warp: allocate ncols (power of two, 32..512) columns; the TMEM address is written to
// *dst (shared memory).  Blocks until the columns are free on this SM.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
// Whole warp: this CTA will allocate no more, so other CTAs' allocations may proceed.
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// Whole warp: free the columns (every thread's TMEM accesses must be complete).
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

#define NLEM_R8(i) "=r"(v[i]), "=r"(v[i + 1]), "=r"(v[i + 2]), "=r"(v[i + 3]), "=r"(v[i + 4]), "=r"(v[i + 5]), \
                   "=r"(v[i + 6]), "=r"(v[i + 7])
#define NLEM_W8(i) "+r"(v[i]), "+r"(v[i + 1]), "+r"(v[i + 2]), "+r"(v[i + 3]), "+r"(v[i + 4]), "+r"(v[i + 5]), \
                   "+r"(v[i + 6]), "+r"(v[i + 7])

// Start loading 32 consecutive columns of this thread's lane into v (asynchronous: the
// values may be read only after tmem_wait_ld(v)).  taddr must be warp-uniform.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : NLEM_R8(0), NLEM_R8(8), NLEM_R8(16), NLEM_R8(24)
      : "r"(taddr));
}
// Wait for every TMEM load this thread issued; v is passed through so that the compiler
// orders its uses after the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : NLEM_W8(0), NLEM_W8(8), NLEM_W8(16), NLEM_W8(24)::"memory");
}
#undef NLEM_R8
#undef NLEM_W8

}  // namespace nlemk
