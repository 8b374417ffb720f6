// Device residency of a column: one cudaMalloc arena holding the layout, the
// GPU index (PP-VBS group offsets) and the decode tables, plus the device
// status word shared by every kernel of the library.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "kernels.h"

namespace bs {

__device__ uint32_t g_bs_status;

int read_and_clear_status(uint32_t *status) {
    uint32_t v = 0, zero = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return BS_ERR_CUDA;
    if (cudaMemcpyFromSymbol(&v, g_bs_status, sizeof v) != cudaSuccess) return BS_ERR_CUDA;
    if (cudaMemcpyToSymbol(g_bs_status, &zero, sizeof zero) != cudaSuccess) return BS_ERR_CUDA;
    *status = v;
    return BS_OK;
}

uint32_t *status_word() {
    static std::mutex mu;
    static uint32_t *cache[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!cache[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bs_status) != cudaSuccess) return nullptr;
        cache[dev] = (uint32_t *)p;
    }
    return cache[dev];
}

int sm_count(int device) {
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> g(mu);
    if (device < 0 || device >= 64) return 1;
    if (!cache[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 1;
        cache[device] = v;
    }
    return cache[device];
}

int blocks_per_sm(const void *kernel, int threads, size_t smem, int device) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(kernel, device * 65536 + threads);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem) != cudaSuccess || v < 1) {
        cudaGetLastError();
        v = 1;
    }
    cache[key] = v;
    return v;
}

namespace {
struct Arena {
    size_t used = 0;
    size_t take(size_t bytes) {  // 256-byte aligned sub-buffers
        size_t at = (used + 255) & ~(size_t)255;
        used = at + bytes;
        return at;
    }
};
}  // namespace

void free_device(Column &c) {
    if (c.d_arena) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(c.device);
        cudaFree(c.d_arena);
        cudaSetDevice(prev);
    }
    c.d_arena = nullptr;
    c.d_bytes = 0;
}

int upload_column(Column &c) {
    Arena ar;
    size_t o_dense = 0, o_packed = 0, o_val2 = 0, o_leaf2 = 0, o_val1 = 0, o_dict = 0;
    size_t o_mask[kMaxCodeBytes + 1] = {0}, o_off[kMaxCodeBytes + 1] = {0}, o_deep[kMaxCodeBytes + 1] = {0};
    if (c.layout == BS_PPVBS || c.layout == BS_BYTESLICE) o_dense = ar.take(c.h_dense.size() + 16);
    if (c.layout == BS_PPVBS) {
        for (int j = 2; j <= c.K; j++) {
            o_mask[j] = ar.take(c.h_mask[j].size() * 4);
            o_off[j] = ar.take(c.h_off[j].size() * 4);
            o_deep[j] = ar.take(c.h_deep[j].size());
        }
        o_val2 = ar.take(c.val2.size() * 4 + 4);
        o_leaf2 = ar.take(c.leaf2.size() * 4 + 4);
        o_val1 = ar.take(c.val1.size() * 4 + 4);
    }
    if (c.layout == BS_BITPACKED) o_packed = ar.take(c.h_packed.size() * 4);
    o_dict = ar.take(c.dict.size() * 4 + 4);
    size_t total = ar.used + 256;

    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(c.device) != cudaSuccess) return BS_ERR_CUDA;
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaSetDevice(prev);
        return e == cudaErrorMemoryAllocation ? BS_ERR_OOM : BS_ERR_CUDA;
    }
    uint8_t *b = (uint8_t *)base;
    auto put = [&](size_t off, const void *src, size_t bytes) -> bool {
        if (!bytes) return true;
        return cudaMemcpy(b + off, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = cudaMemset(base, 0, total) == cudaSuccess;
    if (c.layout == BS_PPVBS || c.layout == BS_BYTESLICE) {
        ok = ok && put(o_dense, c.h_dense.data(), c.h_dense.size());
        c.d_dense = b + o_dense;
    }
    if (c.layout == BS_PPVBS) {
        for (int j = 2; j <= c.K; j++) {
            ok = ok && put(o_mask[j], c.h_mask[j].data(), c.h_mask[j].size() * 4);
            ok = ok && put(o_off[j], c.h_off[j].data(), c.h_off[j].size() * 4);
            ok = ok && put(o_deep[j], c.h_deep[j].data(), c.h_deep[j].size());
            c.d_mask[j] = (const uint32_t *)(b + o_mask[j]);
            c.d_off[j] = (const uint32_t *)(b + o_off[j]);
            c.d_deep[j] = b + o_deep[j];
        }
        ok = ok && put(o_val2, c.val2.data(), c.val2.size() * 4);
        ok = ok && put(o_leaf2, c.leaf2.data(), c.leaf2.size() * 4);
        c.d_val2 = (const int32_t *)(b + o_val2);
        c.d_leaf2 = (const uint32_t *)(b + o_leaf2);
        ok = ok && put(o_val1, c.val1.data(), c.val1.size() * 4);
        c.d_val1 = (const int32_t *)(b + o_val1);
    }
    if (c.layout == BS_BITPACKED) {
        ok = ok && put(o_packed, c.h_packed.data(), c.h_packed.size() * 4);
        c.d_packed = (const uint32_t *)(b + o_packed);
    }
    // the device dictionary is indexed by what a code decodes to: the value
    // position for Algorithm 1 and the fixed-width layouts, the frequency rank
    // for Algorithm 2
    const std::vector<int32_t> &ddict = c.categorical ? c.rank_dict : c.dict;
    ok = ok && put(o_dict, ddict.data(), ddict.size() * 4);
    c.d_dict = (const int32_t *)(b + o_dict);
    c.d_arena = base;
    c.d_bytes = total;
    cudaSetDevice(prev);
    if (!ok) {
        free_device(c);
        return BS_ERR_CUDA;
    }
    return BS_OK;
}

}  // namespace bs
