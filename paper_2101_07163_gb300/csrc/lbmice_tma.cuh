// Bulk-tensor (TMA) prefetches from HBM into L2 for sm_100-family GPUs (inline PTX). They
// read tensor maps that the host encodes once per state buffer (cuTensorMapEncodeTiled) and
// keeps in device memory. A prefetch has no completion to wait for, and touches no shared
// memory.
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
