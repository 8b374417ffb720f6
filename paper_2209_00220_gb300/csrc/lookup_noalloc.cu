// bs_lookup_noalloc: the lookup of bs_lookup with its scratch in a fixed,
// library-owned device array instead of caller or runtime allocations.
//
// Some callers cannot allocate device memory at lookup time: code that runs
// while a CUDA graph is being built or replayed by someone else, hosts that
// hand out a fixed memory budget up front, or real-time paths that must not
// touch an allocator. This entry point allocates nothing. Its scratch (the
// lookup's 32-bit count per 16,384 rows and 64-bit offset per 131,072 rows,
// 1.25 MiB for the largest column) lives in the file-scope array below, so
// every GPU that loads the library holds these 2 MiB + 4 KiB until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (1u << 21) + 4096;  // 262,144 chunks: any column below 2^32 rows

static __device__ __align__(256) unsigned char g_lookup_scratch[kNoAllocScratchBytes];

// Host code cannot use g_lookup_scratch as an address (in host code the name
// is a host-side stand-in); the device address is looked up once per device.
void *scratch_on_current_device(int *err) {
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        *err = BS_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lookup_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            *err = BS_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = p;
    }
    return addr[dev];
}

}  // namespace

extern "C" int bs_lookup_noalloc(const bs_column *col, const uint32_t *d_bits, int32_t *d_out, uint64_t out_cap,
                                 uint64_t *d_count, void *stream) {
    if (!col) return BS_ERR_INVALID_ARG;
    const bs::Column &c = col->c;
    if (c.raw || !c.d_arena) return BS_ERR_UNSUPPORTED;
    if (c.n && !d_bits) return BS_ERR_INVALID_ARG;
    if (out_cap && !d_out) return BS_ERR_INVALID_ARG;
    const uint64_t need = bs::lookup_workspace_bytes(c);
    if (need > kNoAllocScratchBytes) return BS_ERR_CAPACITY;  // column too long for the fixed scratch
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return BS_ERR_CUDA;
    if (prev != c.device && cudaSetDevice(c.device) != cudaSuccess) return BS_ERR_CUDA;
    int rc = BS_OK;
    void *ws = scratch_on_current_device(&rc);
    if (ws) {
        // the array keeps the previous call's contents; the lookup's count
        // kernel writes every scratch word before anything reads it
        rc = bs::launch_lookup(c, d_bits, d_out, nullptr, out_cap, d_count, ws, (cudaStream_t)stream);
    }
    if (prev != c.device) cudaSetDevice(prev);
    return rc;
}
