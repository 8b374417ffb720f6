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

}  // namespace
}  // namespace bs
