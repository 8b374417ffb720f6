// Lookup kernels for sm_103a (single query): count, offsets and gather, plus
// the row-id lookup, with their launchers. The device-side building blocks and
// their description are in lookup_dev.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "lookup_dev.cuh"

namespace bs {
namespace {

// ------------------------------------------------------------ 1. count
// Writes chunk_cnt[c] for every chunk c < n_chunks and group_off[g] for every
// group g < n_groups (one CTA per group), whatever the bits hold: the scan and
// gather kernels read nothing of the workspace that this kernel did not write
// in the same call, so the workspace is never cleared (bs_lookup_noalloc's
// shared scratch relies on this; a count kernel that skipped empty chunks
// would break it).
__global__ void __launch_bounds__(kLookupThreads) lookup_count_kernel(const LookK a) {
    __shared__ uint32_t part[kLookupWarps];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t chunk = (uint64_t)blockIdx.x * kGroupChunks + warp;
    const uint64_t nwords = (a.n + 31) / 32;
    uint32_t acc = 0;
    if (chunk < a.n_chunks) {
        // 512 words per chunk: lane reads 16 of them, as four 16-byte loads when
        // the words are complete (no bit at or past n) and the vector is aligned
        const uint64_t w0 = chunk * (uint64_t)kChunkTiles * kTileWords;
        const uint64_t full = a.n / 32;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const uint64_t w = w0 + (uint64_t)(i * 32 + lane) * 4;
            if (a.bits_vec && w + 4 <= full) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.bits + w));
                acc += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            } else {
                for (uint64_t x = w; x < w + 4 && x < nwords; x++)
                    acc += __popc(__ldg(a.bits + x) & valid_mask(x * 32u, a.n));
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) a.chunk_cnt[chunk] = acc;
    }
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t s = 0;
        for (int i = 0; i < kLookupWarps; i++) s += part[i];
        a.group_off[blockIdx.x] = s;
    }
}

// ------------------------------------------------------------ 2. scan
__global__ void __launch_bounds__(kScanBlock) lookup_scan_kernel(const LookK a) {
    __shared__ uint64_t warp_tot[kScanBlock / 32];
    __shared__ uint64_t carry;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < a.n_groups; base += kScanBlock) {
        const uint32_t i = base + tid;
        const uint64_t v = i < a.n_groups ? a.group_off[i] : 0;
        uint64_t incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t o = __shfl_up_sync(kFull, incl, d);
            if (lane >= (uint32_t)d) incl += o;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint64_t w = warp_tot[lane];
            uint64_t wi = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint64_t o = __shfl_up_sync(kFull, wi, d);
                if (lane >= (uint32_t)d) wi += o;
            }
            warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
        }
        __syncthreads();
        const uint64_t excl = carry + warp_tot[warp] + incl - v;
        if (i < a.n_groups) a.group_off[i] = excl;
        __syncthreads();
        if (tid == kScanBlock - 1) carry = excl + v;
        __syncthreads();
    }
    if (tid == 0 && a.count) *a.count = carry;
}

// ------------------------------------------------------------ 3. gather
// Work units are (chunk, part): a chunk's 16 tiles are split over a.parts
// warps (1 on columns with enough chunks to fill the GPU, up to 16 on short
// ones). With one part a CTA's 8 warps own the 8 chunks of one count group;
// CTAs walk the units persistently (blockIdx.x * 8 + warp, then + gridDim.x *
// 8, ...). A unit's first output slot is its group's offset plus the counts of
// the chunks before it in the group (plus, inside gather_chunk, the counts of
// the chunk's earlier tiles).
template <int LAYOUT, bool CODES, int KMAX>
__global__ void __launch_bounds__(kLookupThreads, 5) lookup_gather_kernel(const LookK a) {
    __shared__ WarpSmemT<KMAX> smem[kLookupWarps];
    __shared__ int32_t val1[256];  // PP-VBS: value of every one-byte code
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (LAYOUT == BS_PPVBS && !CODES && threadIdx.x < 256) val1[threadIdx.x] = __ldg(a.val2 + (threadIdx.x << 8));
    __syncthreads();
    const uint32_t parts = a.parts ? a.parts : 1u, span = (uint32_t)kChunkTiles / parts;
    const uint32_t units = a.n_chunks * parts;
    for (uint32_t u = blockIdx.x * kLookupWarps + warp; u < units; u += gridDim.x * kLookupWarps) {
        const uint32_t c = u / parts, p = u % parts;
        const uint32_t g = c / kGroupChunks, k = c % kGroupChunks;
        // chunk offset: group offset + counts of the earlier chunks of the group
        const uint32_t cc = lane < k ? __ldg(a.chunk_cnt + g * kGroupChunks + lane) : 0u;
        const uint64_t base = a.group_off[g] + warp_sum(cc);
        gather_chunk<LAYOUT, CODES, KMAX>(a, c, base, smem[warp], val1, lane, (int)(p * span),
                                          (int)((p + 1) * span));
    }
}

// ------------------------------------------------------- lookup by row ids
template <int LAYOUT>
__global__ void lookup_rowids_kernel(const LookK a, const uint32_t *rowids, uint64_t m) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t row = rowids[i];
        if (row >= a.n) {
            atomicOr(a.status, kStatusBounds);
            a.out_vals[i] = 0;
            continue;
        }
        const uint64_t t = row >> 10;
        const uint32_t q = row & 1023u;
        uint64_t code;
        int len;
        if (LAYOUT == BS_PPVBS) {
            code = __ldg(a.dense + t * kTileRows + tile_pos(q));
            len = 1;
            const uint64_t g = row >> 8, w = row >> 5;
            const uint32_t b = row & 31u;
            for (int j = 2; j <= a.K; j++) {
                const uint32_t mw = __ldg(a.mask[j] + w);
                if (!((mw >> b) & 1u)) break;
                uint64_t idx = __ldg(a.off[j] + g);
                for (uint64_t x = g * kGroupWords; x < w; x++) idx += __popc(__ldg(a.mask[j] + x));
                idx += __popc(mw & ((1u << b) - 1u));
                uint32_t byte = 0;
                if (idx < a.deep_len[j]) byte = __ldg(a.deep[j] + idx);
                else atomicOr(a.status, kStatusBounds);
                code = (code << 8) | byte;
                len = j;
            }
        } else {
            fetch_code<LAYOUT, 4>(a, t, q, 1, (const WarpSmemT<4> *)nullptr, false, code, len);
        }
        a.out_vals[i] = decode_value<LAYOUT>(a, code, len);
    }
}

// Launch shape of the gather for a column: warps per chunk (parts), grid and
// the resident CTAs the grid is capped at. Short columns split chunks over
// more warps until the resident warps have about two units each or every warp
// holds one tile.
struct GatherShape {
    uint32_t parts, grid, resident;
};

template <int LAYOUT, bool CODES, int KMAX>
GatherShape gather_shape_k(const LookK &a, int dev) {
    auto fn = lookup_gather_kernel<LAYOUT, CODES, KMAX>;
    if (KMAX > 2) {
        // codes of three or more bytes read BS_3.., the leaf table and the
        // dictionary through L1: ask for the 196 KB shared-memory configuration
        // (85 % of 228 KB, rounded up by the driver), which leaves 60 KB of L1
        // at four resident CTAs instead of 28 KB at five (on 2^28-row columns of
        // 3- to 5-byte codes: 1.1x to 2.2x faster at 50 and 90 % selected,
        // within 10 % at 10 %); once per device, before the occupancy query
        // that sizes the grid
        static std::atomic<uint64_t> done{0};
        const uint64_t bit = 1ull << (dev & 63);
        if (!(done.load() & bit)) {
            cudaFuncSetAttribute((const void *)fn, cudaFuncAttributePreferredSharedMemoryCarveout, 85);
            cudaGetLastError();  // a hint: ignore a refusal
            done.fetch_or(bit);
        }
    }
    GatherShape g;
    const uint64_t resident = (uint64_t)sm_count(dev) * blocks_per_sm((const void *)fn, kLookupThreads, 0, dev);
    g.resident = (uint32_t)resident;
    g.parts = 1;
    while (g.parts < (uint32_t)kChunkTiles && (uint64_t)a.n_chunks * g.parts * 2 <= resident * kLookupWarps)
        g.parts *= 2;
    const uint64_t ctas = ((uint64_t)a.n_chunks * g.parts + kLookupWarps - 1) / kLookupWarps;
    g.grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(ctas, resident));
    return g;
}

template <int LAYOUT, bool CODES, int KMAX>
void launch_gather_k(const LookK &a, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    const GatherShape g = gather_shape_k<LAYOUT, CODES, KMAX>(a, dev);
    LookK b = a;
    b.parts = g.parts;
    lookup_gather_kernel<LAYOUT, CODES, KMAX><<<g.grid, kLookupThreads, 0, s>>>(b);
}

template <int LAYOUT>
GatherShape gather_shape(const LookK &a, int dev) {
    if (LAYOUT == BS_PPVBS && a.K > 4) return gather_shape_k<LAYOUT, false, 8>(a, dev);
    if (a.K > 2) return gather_shape_k<LAYOUT, false, 4>(a, dev);
    return gather_shape_k<LAYOUT, false, 2>(a, dev);
}

template <int LAYOUT, bool CODES>
void launch_gather(const LookK &a, cudaStream_t s) {
    if (LAYOUT == BS_PPVBS && a.K > 4) launch_gather_k<LAYOUT, CODES, 8>(a, s);
    else if (a.K > 2) launch_gather_k<LAYOUT, CODES, 4>(a, s);
    else launch_gather_k<LAYOUT, CODES, 2>(a, s);
}

template <bool CODES>
void launch_kernels(const LookK &a, cudaStream_t s) {
    lookup_count_kernel<<<a.n_groups, kLookupThreads, 0, s>>>(a);
    lookup_scan_kernel<<<1, kScanBlock, 0, s>>>(a);
    switch (a.layout) {
    case BS_PPVBS: launch_gather<BS_PPVBS, CODES>(a, s); break;
    case BS_BYTESLICE: launch_gather<BS_BYTESLICE, CODES>(a, s); break;
    default: launch_gather<BS_BITPACKED, CODES>(a, s); break;
    }
}

}  // namespace

int lookup_shape(const Column &c, uint32_t *parts, uint32_t *grid, uint32_t *resident) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BS_ERR_CUDA;
    const LookK a = make_look_args(c);
    GatherShape g;
    switch (c.layout) {
    case BS_PPVBS: g = gather_shape<BS_PPVBS>(a, dev); break;
    case BS_BYTESLICE: g = gather_shape<BS_BYTESLICE>(a, dev); break;
    default: g = gather_shape<BS_BITPACKED>(a, dev); break;
    }
    if (parts) *parts = g.parts;
    if (grid) *grid = g.grid;
    if (resident) *resident = g.resident;
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

uint64_t lookup_workspace_bytes(const Column &c) {
    const uint64_t chunks = ((uint64_t)c.n_tiles + kChunkTiles - 1) / kChunkTiles;
    const uint64_t groups = (chunks + kGroupChunks - 1) / kGroupChunks;
    return ((chunks * 4 + 255) & ~255ull) + ((groups * 8 + 255) & ~255ull);
}

int launch_lookup(const Column &c, const uint32_t *d_bits, int32_t *d_vals, uint64_t *d_codes, uint64_t out_cap,
                  uint64_t *d_count, void *d_ws, cudaStream_t s, uint32_t *status) {
    LookK a = make_look_args(c);
    a.bits = d_bits;
    a.bits_vec = ((uintptr_t)d_bits & 15u) == 0;
    a.chunk_cnt = (uint32_t *)d_ws;
    a.group_off = (uint64_t *)((uint8_t *)d_ws + ((a.n_chunks * 4ull + 255) & ~255ull));
    a.out_vals = d_vals;
    a.out_codes = d_codes;
    a.out_cap = out_cap;
    a.count = d_count;
    a.status = status ? status : status_word();
    if (!a.status) return BS_ERR_CUDA;
    if (c.n == 0) {
        if (d_count && cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s) != cudaSuccess) return BS_ERR_CUDA;
        return BS_OK;
    }
    // every workspace word is written by the count kernel before it is read
    if (d_codes) launch_kernels<true>(a, s);
    else launch_kernels<false>(a, s);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

int launch_lookup_rowids(const Column &c, const uint32_t *d_rowids, uint64_t m, int32_t *d_out, cudaStream_t s) {
    if (m == 0) return BS_OK;
    LookK a = make_look_args(c);
    a.out_vals = d_out;
    a.status = status_word();
    if (!a.status) return BS_ERR_CUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t want = (m + 255) / 256;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sm_count(dev) * 16));
    switch (c.layout) {
    case BS_PPVBS: lookup_rowids_kernel<BS_PPVBS><<<grid, 256, 0, s>>>(a, d_rowids, m); break;
    case BS_BYTESLICE: lookup_rowids_kernel<BS_BYTESLICE><<<grid, 256, 0, s>>>(a, d_rowids, m); break;
    default: lookup_rowids_kernel<BS_BITPACKED><<<grid, 256, 0, s>>>(a, d_rowids, m); break;
    }
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

}  // namespace bs
