// Bounded device-side waiting, shared by the batched kernel's grid barrier and
// the bounded-wait self-test.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bs {
namespace {

// Polls *p (acquire loads, a short sleep between polls) until it reaches
// target; after max_polls polls it gives up, records a timeout in the device
// status word (kStatusTimeout, bit value 2) and returns false instead of
// waiting forever.
__device__ __forceinline__ bool bounded_wait_geq(const uint32_t *p, uint32_t target, uint32_t max_polls,
                                                 uint32_t *status) {
    for (uint32_t polls = 0;; polls++) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= target) return true;
        if (polls >= max_polls) {
            atomicOr(status, 2u);
            return false;
        }
        __nanosleep(64);
    }
}

}  // namespace
}  // namespace bs
