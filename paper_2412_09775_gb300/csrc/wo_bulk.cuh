// wo_bulk.cuh - TMA bulk copies (cp.async.bulk) between global and shared
// memory, the mbarrier they complete on, and the device clock the kernels'
// bounded waits read.
//
// A bulk load moves `bytes` (a multiple of 16) from a 16-byte aligned global
// address to a 16-byte aligned shared address through the tensor memory
// accelerator and signals completion on an mbarrier as transaction bytes:
// one thread arms the barrier with the expected byte count
// (mbar_expect_tx), the copies complete it, and every thread waits for the
// phase to flip (mbar_try_wait, polled against a time budget by the caller).
#pragma once
#include <stdint.h>

namespace wo {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

// Makes an mbarrier's initialisation visible to the async proxy (the bulk
// copies that will complete on it).
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// One bulk copy global -> shared (both 16-byte aligned, bytes a multiple of
// 16), completing on `bar`.
__device__ __forceinline__ void bulk_load(void* smem, const void* gmem, unsigned bytes, uint64_t* bar) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s),
               "l"(gmem), "r"(bytes), "r"(b)
               : "memory");
}

// Prefetch `bytes` (a multiple of 16) from a 16-byte aligned global address
// into L2 (no completion to wait for).
__device__ __forceinline__ void bulk_prefetch_l2(const void* gmem, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gmem), "r"(bytes) : "memory");
}

}  // namespace wo
