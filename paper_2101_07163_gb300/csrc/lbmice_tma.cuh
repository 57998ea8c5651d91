// Bulk-tensor (TMA) operations for sm_100-family GPUs (inline PTX), on tensor maps that the
// host encodes once per state buffer (cuTensorMapEncodeTiled) and keeps in device memory:
// prefetches from HBM into L2 (no completion to wait for, no shared memory), and box loads
// into shared memory that complete on an mbarrier, waited for with a bounded poll.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace lbmice {

// Prefetch one box of a tensor map into L2 (no shared memory, nothing to wait for).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}

}  // namespace lbmice

namespace lbmice {

// Bounded waits that gave up (mbar_wait): a device word the host reads at its health checks.
__device__ unsigned int wait_word;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// An mbarrier expecting one arrival per phase, made visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// The one arrival of the current phase, which then completes once `bytes` have landed.
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// Wait for the phase of the given parity to complete: polls that suspend the thread until
// the phase completes (it wakes then) or for at most 1 ms each (the suspend-time hint bounds
// the system-dependent limit), at most kMbarTries of them (about a second in all). Suspended
// warps leave their issue slots to the others. A wait that gives up sets wait_word and returns
// false (the data are then not to be trusted, and the host reports LBMICE_ETIMEOUT at its
// next check).
constexpr int kMbarTries = 1024;
constexpr uint32_t kMbarSuspendNs = 1000000;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (int i = 0; i < kMbarTries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kMbarSuspendNs)
        : "memory");
    if (done) return true;
  }
  atomicOr(&wait_word, 1u);
  return false;
}

// A wait that runs out on purpose (lbmice_debug_wait_selftest): an mbarrier phase that
// expects 16 bytes no copy delivers. Nothing is in flight when the CTA ends.
__global__ void wait_selftest_kernel() {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    mbar_expect(&bar, 16);
  }
  __syncthreads();
  mbar_wait(&bar, 0);
}

// One box of a 2D tensor map into shared memory (16-byte aligned destination, x a multiple
// of 4 floats), its bytes counted against the mbarrier's current phase.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace lbmice
