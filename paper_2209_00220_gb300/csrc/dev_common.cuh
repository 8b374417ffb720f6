// Device helpers shared by the scan and lookup device code.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bs {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// Rows of a 32-row word that exist (bit i set iff row0 + i < n).
__device__ __forceinline__ uint32_t valid_mask(uint64_t row0, uint64_t n) {
    if (row0 + 32 <= n) return kFull;
    if (row0 >= n) return 0u;
    return (1u << (uint32_t)(n - row0)) - 1u;
}

// Asynchronous global -> shared copies (completion per thread through
// commit / wait groups; other lanes see the bytes after a __syncwarp).
__device__ __forceinline__ void cp_async16(uint32_t smem_addr, const uint8_t *g) {
    asm volatile("cp.async.cg.shared.global.L2::256B [%0], [%1], 16;" ::"r"(smem_addr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t smem_addr, const uint32_t *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace
}  // namespace bs
