// Lookup kernels for sm_103a (Algorithm 4 and the lookups of Sections 2.3 and
// 2.5): result bit vector -> values of the selected rows in ascending row
// order, or zero-padded codes.
//
// Algorithm 4 walks the bit vector word by word with running slice indices
// I_j; on the GPU the output position of every selected row comes from a
// three-kernel compaction instead:
//   1. count:   popcount of the bit vector per chunk of 16 tiles (16K rows);
//   2. offsets: one CTA turns the chunk counts into exclusive offsets and
//               writes the total;
//   3. gather:  per tile, a warp prefix-sums its 32 word popcounts, lists the
//               selected rows in shared memory (ascending), then lanes take
//               list entries round-robin, so output writes are coalesced.
// For PP-VBS a warp loads, per level j, the mask words M_j of the 256-row
// groups whose selected rows have byte j-1 (the paper's per-block beta test),
// prefix-sums their popcounts into shared memory, and every selected row then
// finds its byte j at off_j[group] + prefix + rank. The code is decoded with the
// prefix-preserving tree: root and level-1 internal nodes map a slot sub-code
// to the dictionary index, a pointer sub-code to a child node or to a leaf
// whose values have consecutive dictionary indices.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"

namespace bs {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kChunkTiles = 16;
constexpr int kLookupThreads = 256;
constexpr int kLookupWarps = kLookupThreads / 32;
constexpr int kTilesPerWarp = kChunkTiles / kLookupWarps;
constexpr int kScanBlock = 1024;

struct LookK {
    int32_t layout;
    int32_t K;            // PP-VBS longest code / ByteSlice slices
    int32_t k;            // code bits (ByteSlice / Bit-Packed)
    int32_t identity;
    int64_t domain_min;
    int32_t root_leaf;
    uint32_t n_trie_nodes;
    uint64_t n;
    uint32_t n_tiles;
    uint32_t n_chunks;
    const uint8_t *dense;
    uint64_t slice_bytes;
    const uint32_t *mask[kMaxCodeBytes + 1];
    const uint32_t *off[kMaxCodeBytes + 1];
    const uint8_t *deep[kMaxCodeBytes + 1];
    uint64_t deep_len[kMaxCodeBytes + 1];
    const uint32_t *packed;
    const uint32_t *trie;
    const int32_t *dict;
    uint64_t dict_size;
    const uint32_t *bits;
    uint32_t *chunk;      // workspace: chunk counts, then exclusive offsets
    int32_t *out_vals;
    uint64_t *out_codes;
    uint64_t out_cap;
    uint64_t *count;
    uint32_t *status;
};

__device__ __forceinline__ uint32_t valid_mask(uint64_t row0, uint64_t n) {
    if (row0 + 32 <= n) return kFull;
    if (row0 >= n) return 0u;
    return (1u << (uint32_t)(n - row0)) - 1u;
}

__device__ __forceinline__ uint32_t tile_pos(uint32_t q) {
    const uint32_t lane = q >> 5, r = q & 31u, b = r >> 3, w = r & 7u;
    return (w >> 2) * 512u + lane * 16u + (w & 3u) * 4u + b;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

// ------------------------------------------------------------ 1. count
__global__ void __launch_bounds__(kLookupThreads) lookup_count_kernel(const LookK a) {
    __shared__ uint32_t part[kLookupWarps];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t chunk = blockIdx.x;
    uint32_t acc = 0;
    for (int i = 0; i < kTilesPerWarp; i++) {
        const uint64_t t = (uint64_t)chunk * kChunkTiles + warp * kTilesPerWarp + i;
        if (t < a.n_tiles) {
            const uint64_t w = t * kTileWords + lane;
            const uint32_t vm = valid_mask(w * 32u, a.n);  // never read past ceil(n/32) words
            if (vm) acc += __popc(__ldg(a.bits + w) & vm);
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int i = 0; i < kLookupWarps; i++) s += part[i];
        a.chunk[chunk] = s;
    }
}

// ------------------------------------------------------------ 2. offsets
__global__ void __launch_bounds__(kScanBlock) lookup_offsets_kernel(const LookK a) {
    __shared__ uint64_t sums[kScanBlock];
    const uint32_t tid = threadIdx.x;
    const uint32_t per = (a.n_chunks + kScanBlock - 1) / kScanBlock;
    const uint64_t b = (uint64_t)tid * per, e = (b + per < a.n_chunks) ? b + per : (uint64_t)a.n_chunks;
    uint64_t s = 0;
    for (uint64_t i = b; i < e; i++) s += a.chunk[i];
    sums[tid] = s;
    __syncthreads();
    // inclusive Hillis-Steele scan over the per-thread sums
    for (uint32_t d = 1; d < kScanBlock; d <<= 1) {
        uint64_t v = tid >= d ? sums[tid - d] : 0;
        __syncthreads();
        sums[tid] += v;
        __syncthreads();
    }
    uint64_t run = tid ? sums[tid - 1] : 0;
    for (uint64_t i = b; i < e; i++) {
        uint32_t c = a.chunk[i];
        a.chunk[i] = (uint32_t)run;
        run += c;
    }
    if (tid == kScanBlock - 1 && a.count) *a.count = sums[kScanBlock - 1];
}

// ------------------------------------------------------------ 3. gather
__device__ __forceinline__ int32_t decode_value(const LookK &a, uint64_t code, int len) {
    uint64_t idx;
    if (a.layout != BS_PPVBS) {
        if (a.identity) return (int32_t)((int64_t)code + a.domain_min);
        idx = code;
    } else if (a.root_leaf) {
        idx = code - 1;
    } else {
        uint32_t node = 0;
        int pos = 0;
        idx = ~0ull;
        for (int guard = 0; guard < kMaxCodeBytes; guard++) {
            const uint32_t b = (uint32_t)(code >> (8 * (len - 1 - pos))) & 0xFFu;
            const uint32_t *nd = a.trie + (uint64_t)node * kTrieNodeWords;
            if (pos == len - 1) { idx = __ldg(nd + b); break; }
            const uint32_t ch = __ldg(nd + 256 + b);
            pos++;
            if (ch & kTrieInternal) {
                node = ch & ~kTrieInternal;
                if (node >= a.n_trie_nodes) break;
                continue;
            }
            const uint64_t rest = code & ((8 * (len - pos) >= 64) ? ~0ull : ((1ull << (8 * (len - pos))) - 1));
            idx = (uint64_t)ch + rest - 1;
            break;
        }
    }
    if (idx >= a.dict_size) {
        atomicOr(a.status, kStatusBounds);
        return 0;
    }
    return __ldg(a.dict + idx);
}

struct WarpSmem {
    uint16_t list[kTileRows];
    uint32_t mask[kMaxCodeBytes + 1][kTileWords];
    uint32_t pref[kMaxCodeBytes + 1][kTileWords];
};

template <int LAYOUT, bool CODES>
__device__ __forceinline__ void gather_tile(const LookK &a, uint64_t t, uint64_t out_base, WarpSmem &sm,
                                            uint32_t lane) {
    const uint64_t w = t * kTileWords + lane;
    const uint32_t vm = valid_mask(w * 32u, a.n);
    const uint32_t sel = vm ? (__ldg(a.bits + w) & vm) : 0u;
    const uint32_t cnt = __popc(sel);
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t v = __shfl_up_sync(kFull, incl, d);
        if (lane >= (uint32_t)d) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    {
        uint32_t pos = incl - cnt, r = sel;
        while (r) {
            const uint32_t b = __ffs(r) - 1;
            r &= r - 1;
            sm.list[pos++] = (uint16_t)(lane * 32u + b);
        }
    }
    int levels = 1;
    if (LAYOUT == BS_PPVBS) {
        // mask words and BS_j prefixes for the groups whose selected rows reach byte j
        uint32_t reach = sel;  // selected rows that have byte j-1
        for (int j = 2; j <= a.K; j++) {
            const uint32_t bal = __ballot_sync(kFull, reach != 0u);
            if (!bal) break;
            const uint32_t gact = (bal >> (lane & 24u)) & 0xFFu;
            const uint32_t m = gact ? __ldg(a.mask[j] + w) : 0u;
            const uint32_t c = __popc(m);
            uint32_t inc = c;
#pragma unroll
            for (int d = 1; d < 8; d <<= 1) {
                uint32_t v = __shfl_up_sync(kFull, inc, d);
                if ((lane & 7u) >= (uint32_t)d) inc += v;
            }
            const uint32_t goff = gact ? __ldg(a.off[j] + t * kGroupsPerTile + (lane >> 3)) : 0u;
            sm.mask[j][lane] = m;
            sm.pref[j][lane] = goff + inc - c;
            reach = sel & m;
            levels = j;
        }
    }
    __syncwarp();
    for (uint32_t i = lane; i < total; i += 32) {
        const uint32_t q = sm.list[i];
        const uint64_t row = t * kTileRows + q;
        uint64_t code;
        int len;
        if (LAYOUT == BS_PPVBS) {
            code = __ldg(a.dense + t * kTileRows + tile_pos(q));
            len = 1;
            const uint32_t wq = q >> 5, bq = q & 31u;
            for (int j = 2; j <= levels; j++) {
                const uint32_t m = sm.mask[j][wq];
                if (!((m >> bq) & 1u)) break;
                const uint64_t idx = (uint64_t)sm.pref[j][wq] + __popc(m & ((1u << bq) - 1u));
                uint32_t byte = 0;
                if (idx < a.deep_len[j]) byte = __ldg(a.deep[j] + idx);
                else atomicOr(a.status, kStatusBounds);
                code = (code << 8) | byte;
                len = j;
            }
        } else if (LAYOUT == BS_BYTESLICE) {
            uint64_t aligned = 0;
            const uint64_t pos = t * kTileRows + tile_pos(q);
            for (int s = 0; s < a.K; s++) aligned = (aligned << 8) | __ldg(a.dense + (uint64_t)s * a.slice_bytes + pos);
            code = aligned >> (8 * a.K - a.k);
            len = a.K;
        } else {
            const uint64_t bit = row * (uint64_t)a.k;
            const uint32_t *p = a.packed + (bit >> 5);
            const uint32_t lo = __ldg(p), hi = __ldg(p + 1);
            code = __funnelshift_r(lo, hi, (uint32_t)(bit & 31u)) & (a.k == 32 ? kFull : ((1u << a.k) - 1u));
            len = (a.k + 7) / 8;
        }
        const uint64_t o = out_base + i;
        if (o < a.out_cap) {
            if (CODES) {
                a.out_codes[o] = (LAYOUT == BS_PPVBS) ? (code << (8 * (a.K - len))) : code;
            } else {
                a.out_vals[o] = decode_value(a, code, len);
            }
        }
    }
    __syncwarp();
}

template <int LAYOUT, bool CODES>
__global__ void __launch_bounds__(kLookupThreads) lookup_gather_kernel(const LookK a) {
    __shared__ WarpSmem smem[kLookupWarps];
    __shared__ uint32_t tile_cnt[kChunkTiles];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t chunk = blockIdx.x;
    for (int i = 0; i < kTilesPerWarp; i++) {
        const uint64_t t = (uint64_t)chunk * kChunkTiles + warp * kTilesPerWarp + i;
        uint32_t c = 0;
        if (t < a.n_tiles) {
            const uint64_t w = t * kTileWords + lane;
            const uint32_t vm = valid_mask(w * 32u, a.n);
            if (vm) c = __popc(__ldg(a.bits + w) & vm);
        }
        c = warp_sum(c);
        if (lane == 0) tile_cnt[warp * kTilesPerWarp + i] = c;
    }
    __syncthreads();
    uint64_t base = a.chunk[chunk];
    for (uint32_t i = 0; i < warp * kTilesPerWarp; i++) base += tile_cnt[i];
    for (int i = 0; i < kTilesPerWarp; i++) {
        const uint64_t t = (uint64_t)chunk * kChunkTiles + warp * kTilesPerWarp + i;
        if (t >= a.n_tiles) break;
        if (base < a.out_cap) gather_tile<LAYOUT, CODES>(a, t, base, smem[warp], lane);
        base += tile_cnt[warp * kTilesPerWarp + i];
    }
}

// ------------------------------------------------------- lookup by row ids
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
        if (a.layout == BS_PPVBS) {
            code = __ldg(a.dense + t * kTileRows + tile_pos(q));
            len = 1;
            const uint64_t g = row >> 8;
            const uint64_t w = row >> 5;
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
        } else if (a.layout == BS_BYTESLICE) {
            uint64_t aligned = 0;
            const uint64_t pos = t * kTileRows + tile_pos(q);
            for (int s = 0; s < a.K; s++) aligned = (aligned << 8) | __ldg(a.dense + (uint64_t)s * a.slice_bytes + pos);
            code = aligned >> (8 * a.K - a.k);
            len = a.K;
        } else {
            const uint64_t bit = (uint64_t)row * (uint64_t)a.k;
            const uint32_t *p = a.packed + (bit >> 5);
            code = __funnelshift_r(__ldg(p), __ldg(p + 1), (uint32_t)(bit & 31u)) &
                   (a.k == 32 ? kFull : ((1u << a.k) - 1u));
            len = (a.k + 7) / 8;
        }
        a.out_vals[i] = decode_value(a, code, len);
    }
}

LookK make_args(const Column &c) {
    LookK a{};
    a.layout = c.layout;
    a.K = c.layout == BS_PPVBS ? c.K : c.S;
    a.k = c.k;
    a.identity = c.identity ? 1 : 0;
    a.domain_min = c.domain_min;
    a.root_leaf = c.root_leaf ? 1 : 0;
    a.n_trie_nodes = (uint32_t)(c.trie.size() / kTrieNodeWords);
    a.n = c.n;
    a.n_tiles = c.n_tiles;
    a.n_chunks = (c.n_tiles + kChunkTiles - 1) / kChunkTiles;
    a.dense = c.d_dense;
    a.slice_bytes = c.dense_slice_bytes();
    for (int j = 2; j <= c.K && c.layout == BS_PPVBS; j++) {
        a.mask[j] = c.d_mask[j];
        a.off[j] = c.d_off[j];
        a.deep[j] = c.d_deep[j];
        a.deep_len[j] = c.deep_len[j];
    }
    a.packed = c.d_packed;
    a.trie = c.d_trie;
    a.dict = c.d_dict;
    a.dict_size = c.dict.size();
    return a;
}

template <bool CODES>
void launch_gather(const LookK &a, cudaStream_t s) {
    switch (a.layout) {
    case BS_PPVBS: lookup_gather_kernel<BS_PPVBS, CODES><<<a.n_chunks, kLookupThreads, 0, s>>>(a); break;
    case BS_BYTESLICE: lookup_gather_kernel<BS_BYTESLICE, CODES><<<a.n_chunks, kLookupThreads, 0, s>>>(a); break;
    default: lookup_gather_kernel<BS_BITPACKED, CODES><<<a.n_chunks, kLookupThreads, 0, s>>>(a); break;
    }
}

}  // namespace

uint64_t lookup_workspace_bytes(const Column &c) {
    const uint64_t chunks = ((uint64_t)c.n_tiles + kChunkTiles - 1) / kChunkTiles;
    return std::max<uint64_t>(256, (chunks * 4 + 255) & ~255ull);
}

int launch_lookup(const Column &c, const uint32_t *d_bits, int32_t *d_vals, uint64_t *d_codes, uint64_t out_cap,
                  uint64_t *d_count, void *d_ws, cudaStream_t s) {
    LookK a = make_args(c);
    a.bits = d_bits;
    a.chunk = (uint32_t *)d_ws;
    a.out_vals = d_vals;
    a.out_codes = d_codes;
    a.out_cap = out_cap;
    a.count = d_count;
    a.status = status_word();
    if (!a.status) return BS_ERR_CUDA;
    if (c.n == 0) {
        if (d_count && cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s) != cudaSuccess) return BS_ERR_CUDA;
        return BS_OK;
    }
    lookup_count_kernel<<<a.n_chunks, kLookupThreads, 0, s>>>(a);
    lookup_offsets_kernel<<<1, kScanBlock, 0, s>>>(a);
    if (d_codes) launch_gather<true>(a, s);
    else launch_gather<false>(a, s);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

int launch_lookup_rowids(const Column &c, const uint32_t *d_rowids, uint64_t m, int32_t *d_out, cudaStream_t s) {
    if (m == 0) return BS_OK;
    LookK a = make_args(c);
    a.out_vals = d_out;
    a.status = status_word();
    if (!a.status) return BS_ERR_CUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t want = (m + 255) / 256;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sm_count(dev) * 16));
    lookup_rowids_kernel<<<grid, 256, 0, s>>>(a, d_rowids, m);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

}  // namespace bs
