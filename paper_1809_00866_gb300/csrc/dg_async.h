// Bulk asynchronous copies global -> shared memory (cp.async.bulk, completed on an mbarrier)
// with bounded waits: a wait that gives up returns false instead of spinning forever.
#pragma once

#include <cstdint>

namespace dg {

constexpr unsigned kBulkWaitLimit = 1u << 22;  // try_wait polls before a wait gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// one bulk copy global -> shared; both addresses and the size must be multiples of 16 bytes
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Hint: start bringing the 16-byte aligned part of [lo, hi) from global memory into L2 (no data
// is returned; the later loads of that range hit L2 instead of HBM). [lo, hi) must lie inside
// one allocation; the range is shrunk to 16-byte boundaries, so it never reaches outside it.
__device__ __forceinline__ void prefetch_l2(const void* lo, const void* hi) {
  const unsigned long long a = (reinterpret_cast<unsigned long long>(lo) + 15ull) & ~15ull;
  const unsigned long long b = reinterpret_cast<unsigned long long>(hi) & ~15ull;
  if (b > a) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(b - a)) : "memory");
}
// Order this thread's earlier generic-proxy accesses of shared memory (ordinary loads and
// stores) before later async-proxy accesses of it (a bulk copy that overwrites the same bytes).
// Every thread that wrote a buffer executes it before the barrier after which one thread
// issues a bulk copy into that buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// bounded wait for the phase with parity `parity` of the barrier (at most `limit` polls);
// false when it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit = kBulkWaitLimit) {
  for (unsigned it = 0; it < limit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

}  // namespace dg
