// Self-test of the bounded device wait: failure handling checked without a
// device fault. One thread waits for a flag that nothing sets; the wait must
// give up after its poll limit, record a timeout in the device status word and
// return, leaving the context usable.
#include <cuda_runtime.h>

#include "kernels.h"
#include "wait_dev.cuh"

static_assert(bs::kStatusTimeout == 2u, "bounded_wait_geq records the timeout bit as 2");

namespace {

__global__ void wait_on_unset_flag(const uint32_t *flag, uint32_t max_polls, uint32_t *status, uint32_t *done) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *done = bs::bounded_wait_geq(flag, 1u, max_polls, status) ? 1u : 2u;
}

}  // namespace

extern "C" int bs_selftest_bounded_wait(uint32_t max_polls, int32_t *gave_up) {
    if (!gave_up || max_polls > (1u << 24)) return BS_ERR_INVALID_ARG;
    *gave_up = 0;
    uint32_t *status = bs::status_word();
    if (!status) return BS_ERR_CUDA;
    uint32_t *words = nullptr;  // [0] the flag (never set), [1] the outcome
    if (cudaMalloc(&words, 2 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_OOM;
    }
    int rc = BS_OK;
    uint32_t done = 0;
    if (cudaMemset(words, 0, 2 * sizeof(uint32_t)) != cudaSuccess) rc = BS_ERR_CUDA;
    if (rc == BS_OK) {
        wait_on_unset_flag<<<1, 32>>>(words, max_polls, status, words + 1);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(&done, words + 1, sizeof done, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = BS_ERR_CUDA;
    }
    cudaFree(words);
    if (rc == BS_OK) *gave_up = done == 2u ? 1 : 0;
    return rc;
}
