// Device code of the lookup kernels for sm_103a (shared by lookup.cu and
// batch.cu) (Algorithm 4 and the lookups of Sections 2.3 and
// 2.5): result bit vector -> values of the selected rows in ascending row
// order, or zero-padded codes.
//
// Algorithm 4 walks the bit vector word by word with running slice indices
// I_j. On the GPU the output position of every selected row comes from three
// kernels instead:
//   1. count:  one warp per chunk of 16 tiles (16K rows) popcounts its 2 KB of
//              the bit vector with 16-byte loads; each CTA (8 chunks) also
//              writes the total of its 8 chunks;
//   2. scan:   one CTA turns the CTA totals into exclusive offsets (coalesced
//              segments of 4096) and writes the selected-row count;
//   3. gather: persistent CTAs walk the groups of 8 chunks, one warp per
//              chunk; a chunk's offset is its group's offset plus the counts
//              of the chunks before it in the group. Per tile, a warp
//              prefix-sums its 32 word popcounts, lists the selected rows in
//              shared memory (ascending), and lanes take list entries
//              round-robin, four at a time, so output writes are coalesced and
//              many loads are in flight.
//
// For PP-VBS a warp loads, per level j, the mask words M_j of the 256-row
// groups whose selected rows have byte j-1 (the paper's per-block beta test)
// and prefix-sums their popcounts into shared memory; a selected row's length
// and the address of each of its bytes then come from shared memory alone, so
// all its byte loads are issued together. A tile with many selected rows first
// copies its 1 KB of BS_1 into shared memory with coalesced 16-byte loads;
// for columns whose codes have at most two bytes, or at most four bytes by
// Algorithm 1, it also stages its BS_2 segment and takes M_2.. and the BS_j
// group offsets in the same round of loads, so a slot costs shared-memory
// reads plus its own longer bytes.
// Codes of at most two bytes decode with one table load (value by first two
// bytes); longer codes sit in level-2 leaves whose values have consecutive
// dictionary indices, decoded as dict[leaf start + rest - 1].
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "dev_common.cuh"
#include "kernels.h"

namespace bs {
namespace {


constexpr int kChunkTiles = 16;
constexpr int kLookupThreads = 256;
constexpr int kLookupWarps = kLookupThreads / 32;
constexpr int kTilesPerWarp = kChunkTiles / kLookupWarps;
constexpr int kUnroll = 4;
constexpr int kGroupChunks = 8;       // chunks counted by one CTA of the count kernel
constexpr int kScanBlock = 1024;
constexpr uint32_t kStageMin = 64;    // selected rows from which a tile stages BS_1
constexpr uint32_t kSparseMax = 256;  // selected rows up to which a chunk is resolved row-parallel

struct LookK {
    int32_t layout;
    int32_t K;            // PP-VBS longest code / ByteSlice slices
    int32_t categorical;  // PP-VBS codes by Algorithm 2 (dict in frequency-rank order)
    int32_t cat_B;        // Algorithm 2: levels of the tree
    int32_t k;            // code bits (ByteSlice / Bit-Packed)
    int32_t identity;
    int64_t domain_min;
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
    const int32_t *val2;
    const uint32_t *leaf2;
    const int32_t *dict;
    uint64_t dict_size;
    const uint32_t *bits;
    int32_t bits_vec;     // bits is 16-byte aligned
    uint32_t n_groups;    // groups of kGroupChunks chunks
    uint32_t *chunk_cnt;  // workspace: count per chunk
    uint64_t *group_off;  // workspace: total per group, then exclusive offset
    int32_t *out_vals;
    uint64_t *out_codes;
    uint64_t out_cap;
    uint64_t *count;
    uint32_t *status;
    uint32_t parts;       // gather: warps sharing one chunk's tiles (1, 2, 4, 8, 16; 0 = 1)
};


__device__ __forceinline__ uint32_t tile_pos(uint32_t q) {
    const uint32_t lane = q >> 5, r = q & 31u, b = r >> 3, w = r & 7u;
    return (w >> 2) * 512u + lane * 16u + (w & 3u) * 4u + b;
}

// A lane's 32 slice bytes arrive as words x0..x7 with word w byte b = row
// 8b + w; two 4x4 byte transposes put them in row order (word k = rows
// 4k..4k+3): rows 8m..8m+3 are byte m of x0..x3, rows 8m+4..8m+7 byte m of
// x4..x7.
__device__ __forceinline__ void transpose4(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t &y0,
                                           uint32_t &y1, uint32_t &y2, uint32_t &y3) {
    const uint32_t t0 = __byte_perm(a, b, 0x5140), t1 = __byte_perm(a, b, 0x7362);
    const uint32_t t2 = __byte_perm(c, d, 0x5140), t3 = __byte_perm(c, d, 0x7362);
    y0 = __byte_perm(t0, t2, 0x5410);
    y1 = __byte_perm(t0, t2, 0x7632);
    y2 = __byte_perm(t1, t3, 0x5410);
    y3 = __byte_perm(t1, t3, 0x7632);
}

__device__ __forceinline__ void transpose_lane_bytes(const uint4 &v0, const uint4 &v1, uint4 &r0, uint4 &r1) {
    uint32_t e0, e1, e2, e3, o0, o1, o2, o3;  // even / odd row-order words
    transpose4(v0.x, v0.y, v0.z, v0.w, e0, e1, e2, e3);
    transpose4(v1.x, v1.y, v1.z, v1.w, o0, o1, o2, o3);
    r0 = make_uint4(e0, o0, e1, o1);
    r1 = make_uint4(e2, o2, e3, o3);
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

__device__ __forceinline__ int32_t dict_value(const LookK &a, uint64_t idx) {
    if (idx >= a.dict_size) {
        atomicOr(a.status, kStatusBounds);
        return 0;
    }
    return __ldg(a.dict + idx);
}

// Value of a code: PP-VBS via the two-byte tables, the others by rank or range.
template <int LAYOUT>
__device__ __forceinline__ int32_t decode_value(const LookK &a, uint64_t code, int len) {
    if (LAYOUT == BS_PPVBS) {
        const uint32_t c1 = (uint32_t)(code >> (8 * (len - 1))) & 0xFFu;
        const uint32_t c2 = len >= 2 ? (uint32_t)(code >> (8 * (len - 2))) & 0xFFu : 0u;
        const uint32_t key = (c1 << 8) | c2;
        if (len <= 2) return __ldg(a.val2 + key);
        if (a.categorical) {
            // Algorithm 2: the rank follows from the code's level and position
            // (levels above the last: pointer path * 255 + slot - 1; the last
            // level: (slot - 1) * 256^(B-1) + pointer path)
            uint64_t before = 0, level = 255;
            for (int b = 1; b < len; b++) {
                before += level;
                level <<= 8;
            }
            const uint64_t slot = code & 0xFFu, path = code >> 8;
            const uint64_t rank =
                len < a.cat_B ? before + path * 255 + (slot - 1) : before + (slot - 1) * (1ull << (8 * (len - 1))) + path;
            return dict_value(a, rank);
        }
        const uint64_t rest = code & ((1ull << (8 * (len - 2))) - 1);
        return dict_value(a, (uint64_t)__ldg(a.leaf2 + key) + rest - 1);
    }
    if (a.identity) return (int32_t)((int64_t)code + a.domain_min);
    return dict_value(a, code);
}

// 16-byte aligned: dense[] receives 16-byte vector stores, one struct per warp
template <int KMAX>
struct __align__(16) WarpSmemT {
    uint8_t dense[kTileRows];         // staged BS_1 of the tile
    uint32_t seg[KMAX <= 4 ? kTileRows / 4 + 4 : 4];  // staged BS_2 segment (dense tiles, codes <= 4 bytes)
    uint16_t list[kTileRows];         // selected rows of the tile (tile-local indices)
    uint32_t mask[KMAX - 1][kTileWords];  // level j (2..KMAX) at j - 2
    uint32_t pref[KMAX - 1][kTileWords];
};

static_assert(sizeof(WarpSmemT<2>) % 16 == 0 && sizeof(WarpSmemT<4>) % 16 == 0 && sizeof(WarpSmemT<8>) % 16 == 0,
              "per-warp shared memory must keep 16-byte alignment");

// Code (unpadded) and length of tile-local row q of tile t. PP-VBS reads the
// warp's per-level mask words and BS_j prefixes from sm, and BS_1 from sm.dense
// when the tile was staged. KMAX bounds the code length (template constant).
template <int LAYOUT, int KMAX>
__device__ __forceinline__ void fetch_code(const LookK &a, uint64_t t, uint32_t q, int levels,
                                           const WarpSmemT<KMAX> *sm,
                                           bool staged, uint64_t &code, int &len) {
    if (LAYOUT == BS_PPVBS) {
        const uint32_t wq = q >> 5, bq = q & 31u, below = (1u << bq) - 1u;
        len = 1;
#pragma unroll
        for (int j = 2; j <= KMAX; j++)
            if (j <= levels && len == j - 1 && ((sm->mask[j - 2][wq] >> bq) & 1u)) len = j;
        uint32_t b[KMAX + 1];
        b[1] = staged ? (uint32_t)sm->dense[q] : (uint32_t)__ldg(a.dense + t * kTileRows + tile_pos(q));
#pragma unroll
        for (int j = 2; j <= KMAX; j++) {
            b[j] = 0;
            if (j <= len) {
                const uint64_t idx = (uint64_t)sm->pref[j - 2][wq] + __popc(sm->mask[j - 2][wq] & below);
                if (idx < a.deep_len[j]) b[j] = __ldg(a.deep[j] + idx);
                else atomicOr(a.status, kStatusBounds);
            }
        }
        code = b[1];
#pragma unroll
        for (int j = 2; j <= KMAX; j++)
            if (j <= len) code = (code << 8) | b[j];
    } else if (LAYOUT == BS_BYTESLICE) {
        const uint64_t pos = t * kTileRows + tile_pos(q);
        uint32_t b[KMAX];
#pragma unroll
        for (int s = 0; s < KMAX; s++) b[s] = s < a.K ? __ldg(a.dense + (uint64_t)s * a.slice_bytes + pos) : 0u;
        uint64_t aligned = 0;
#pragma unroll
        for (int s = 0; s < KMAX; s++)
            if (s < a.K) aligned = (aligned << 8) | b[s];
        code = aligned >> (8 * a.K - a.k);
        len = a.K;
    } else {
        const uint64_t bit = (t * kTileRows + q) * (uint64_t)a.k;
        const uint32_t *p = a.packed + (bit >> 5);
        const uint32_t lo = __ldg(p), hi = __ldg(p + 1);
        code = __funnelshift_r(lo, hi, (uint32_t)(bit & 31u)) & (a.k == 32 ? kFull : ((1u << a.k) - 1u));
        len = (a.k + 7) / 8;
    }
}

template <int LAYOUT, bool CODES, int KMAX>
__device__ __forceinline__ void gather_tile(const LookK &a, uint64_t t, uint32_t sel, uint64_t out_base,
                                            WarpSmemT<KMAX> &sm, const int32_t *val1, uint32_t lane) {
    const uint32_t cnt = __popc(sel);
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, d);
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
    // a dense tile copies its BS_1 bytes once, coalesced, instead of one load
    // per row, and stores them in plain row order (byte of row q at dense[q])
    const bool staged = LAYOUT == BS_PPVBS && total >= kStageMin;
    if (staged) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.dense + t * kTileRows);
        const uint4 v0 = __ldg(src + lane), v1 = __ldg(src + 32 + lane);
        uint4 r0, r1;
        transpose_lane_bytes(v0, v1, r0, r1);
        uint4 *dst = reinterpret_cast<uint4 *>(sm.dense + lane * 32u);
        dst[0] = r0;
        dst[1] = r1;
    }
    int levels = 1;
    if (LAYOUT == BS_PPVBS) {
        const uint64_t w = t * kTileWords + lane;
        uint32_t reach = sel;  // selected rows that have byte j-1
        for (int j = 2; j <= min(a.K, KMAX); j++) {
            const uint32_t bal = __ballot_sync(kFull, reach != 0u);
            if (!bal) break;
            const uint32_t gact = (bal >> (lane & 24u)) & 0xFFu;
            const uint32_t m = gact ? __ldg(a.mask[j] + w) : 0u;
            const uint32_t c = __popc(m);
            uint32_t inc = c;
#pragma unroll
            for (int d = 1; d < 8; d <<= 1) {
                const uint32_t v = __shfl_up_sync(kFull, inc, d);
                if ((lane & 7u) >= (uint32_t)d) inc += v;
            }
            const uint32_t goff = gact ? __ldg(a.off[j] + t * kGroupsPerTile + (lane >> 3)) : 0u;
            sm.mask[j - 2][lane] = m;
            sm.pref[j - 2][lane] = goff + inc - c;
            reach = sel & m;
            levels = j;
        }
    }
    __syncwarp();
    for (uint32_t i0 = 0; i0 < total; i0 += 32 * kUnroll) {
        uint64_t code[kUnroll];
        int len[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const uint32_t i = i0 + (uint32_t)u * 32u + lane;
            code[u] = 0;
            len[u] = 1;
            if (i < total) fetch_code<LAYOUT, KMAX>(a, t, sm.list[i], levels, &sm, staged, code[u], len[u]);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const uint32_t i = i0 + (uint32_t)u * 32u + lane;
            const uint64_t o = out_base + i;
            if (i < total && o < a.out_cap) {
                if (CODES) a.out_codes[o] = LAYOUT == BS_PPVBS ? (code[u] << (8 * (a.K - len[u]))) : code[u];
                else a.out_vals[o] = decode_value<LAYOUT>(a, code[u], len[u]);
            }
        }
    }
    __syncwarp();
}

// Code of one row with no shared-memory help: PP-VBS finds byte j at
// off_j[group] + popcounts of the group's earlier mask words + rank in its word
// (all within one 32-byte sector of M_j).
template <int LAYOUT, int KMAX>
__device__ __forceinline__ void row_code(const LookK &a, uint64_t row, uint64_t &code, int &len) {
    const uint64_t t = row >> 10;
    const uint32_t q = (uint32_t)(row & 1023u);
    if (LAYOUT == BS_PPVBS) {
        code = __ldg(a.dense + t * kTileRows + tile_pos(q));
        len = 1;
        const uint64_t g = row >> 8, w = row >> 5;
        const uint32_t b = (uint32_t)(row & 31u), below = (1u << b) - 1u;
        for (int j = 2; j <= min(a.K, KMAX); j++) {
            const uint32_t mw = __ldg(a.mask[j] + w);
            if (!((mw >> b) & 1u)) break;
            uint64_t idx = __ldg(a.off[j] + g) + __popc(mw & below);
            for (uint64_t x = g * kGroupWords; x < w; x++) idx += __popc(__ldg(a.mask[j] + x));
            uint32_t byte = 0;
            if (idx < a.deep_len[j]) byte = __ldg(a.deep[j] + idx);
            else atomicOr(a.status, kStatusBounds);
            code = (code << 8) | byte;
            len = j;
        }
    } else {
        fetch_code<LAYOUT, KMAX>(a, t, q, 1, (const WarpSmemT<KMAX> *)nullptr, false, code, len);
    }
}

// Dense PP-VBS tile whose codes have at most two bytes: the off_2 entries of
// the whole chunk come with the chunk (goff, seg_lo, seg_hi: the lane's group
// offset and the tile's BS_2 segment bounds), so the lane's 32 BS_1 bytes, its
// M_2 word and the tile's BS_2 segment are all loaded in one round; the
// two-byte decode table follows. Each lane walks its
// own selected rows in order and leaves a 16-bit key (first two code bytes) per
// output slot; the warp then decodes the keys and stores them coalesced.
__device__ __forceinline__ void gather_dense_k2(const LookK &a, uint64_t t, uint32_t sel, uint64_t out_base,
                                                uint32_t goff, uint32_t seg_lo, uint32_t seg_hi, WarpSmemT<2> &sm,
                                                const int32_t *val1, uint32_t lane) {
    // one round of independent loads: BS_1, M_2 and (below) the BS_2 segment
    const uint4 *src = reinterpret_cast<const uint4 *>(a.dense + t * kTileRows);
    uint4 v0, v1;
    {
        uint64_t pol;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
        asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=r"(v0.x), "=r"(v0.y), "=r"(v0.z), "=r"(v0.w) : "l"(src + lane), "l"(pol));
        asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=r"(v1.x), "=r"(v1.y), "=r"(v1.z), "=r"(v1.w) : "l"(src + 32 + lane), "l"(pol));
    }
    const bool has2 = a.K >= 2;
    const uint32_t m2 = has2 ? __ldg(a.mask[2] + t * kTileWords + lane) : 0u;
    // ALU while they fly: output positions of this lane's rows
    const uint32_t cnt = __popc(sel);
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, d);
        if (lane >= (uint32_t)d) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t c2 = __popc(m2);
    uint32_t inc2 = c2;
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, inc2, d);
        if ((lane & 7u) >= (uint32_t)d) inc2 += v;
    }
    // the tile's BS_2 bytes (contiguous)
    if (has2) {
        const uint32_t w0 = seg_lo >> 2, w1 = (seg_hi + 3) >> 2;
        const uint32_t *s32 = reinterpret_cast<const uint32_t *>(a.deep[2]);
        constexpr uint32_t kSegWords = sizeof(sm.seg) / 4;
        // up to four words per lane in flight at once (a segment of up to
        // 512 bytes, the usual case, is one round)
        const uint32_t nseg = min(w1 - w0, kSegWords);
        for (uint32_t i0 = 0; i0 < nseg; i0 += 32u * kUnroll) {
            uint32_t r[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const uint32_t i = i0 + (uint32_t)u * 32u + lane;
                r[u] = i < nseg ? __ldg(s32 + w0 + i) : 0u;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const uint32_t i = i0 + (uint32_t)u * 32u + lane;
                if (i < nseg) sm.seg[i] = r[u];
            }
        }
    }
    uint4 r0, r1;
    transpose_lane_bytes(v0, v1, r0, r1);
    uint4 *rows = reinterpret_cast<uint4 *>(sm.dense + lane * 32u);
    rows[0] = r0;
    rows[1] = r1;
    // per lane word: its M_2 bits and its first BS_2 byte, relative to the
    // staged segment
    sm.mask[0][lane] = m2;
    sm.pref[0][lane] = goff + inc2 - c2 - seg_lo;
    // the lane's selected rows, in row order, at its output positions
    uint32_t pos = incl - cnt, r = sel;
    while (r) {
        const uint32_t b = __ffs(r) - 1;
        r &= r - 1;
        sm.list[pos++] = (uint16_t)(lane * 32u + b);
    }
    __syncwarp();
    // every output slot by the lanes in turn: its row's first byte, the BS_2
    // byte at the row's rank among its word's two-byte rows (read
    // unconditionally: the rank stays inside the staged segment; kept only if
    // the row's M_2 bit is set), then the value of the two-byte key
    const uint8_t *seg = reinterpret_cast<const uint8_t *>(sm.seg) + (seg_lo & 3u);
    const uint64_t room = a.out_cap > out_base ? a.out_cap - out_base : 0;
    const uint32_t lim = (uint32_t)(room < total ? room : total);
    int32_t *dst = a.out_vals + out_base;
    auto value_of = [&](uint32_t i) -> int32_t {
        const uint32_t q = sm.list[i], w = q >> 5, b = q & 31u;
        const uint32_t mw = sm.mask[0][w];
        const uint32_t c1 = sm.dense[q];
        const uint32_t c2b = seg[sm.pref[0][w] + __popc(mw & ((1u << b) - 1u))];
        const uint32_t c2 = ((mw >> b) & 1u) ? c2b : 0u;  // 0: a one-byte code
        return c2 ? __ldg(a.val2 + ((c1 << 8) | c2)) : val1[c1];
    };
    // whole rounds of 32 * kUnroll slots (kUnroll loads in flight per lane),
    // then the remaining slots 32 at a time
    uint32_t i0 = 0;
    for (; i0 + 32u * kUnroll <= lim; i0 += 32u * kUnroll) {
        int32_t v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) v[u] = value_of(i0 + (uint32_t)u * 32u + lane);
#pragma unroll
        for (int u = 0; u < kUnroll; u++) dst[i0 + (uint32_t)u * 32u + lane] = v[u];
    }
    for (uint32_t i = i0 + lane; i < lim; i += 32u) dst[i] = value_of(i);
    __syncwarp();
}

// Dense PP-VBS tile of a column with codes of three or four bytes (Algorithm
// 1): as for two-byte codes, BS_1 and the tile's BS_2 segment are staged and
// every slot is resolved from shared memory up to its second byte; M_3 / M_4
// and the group offsets of BS_3 / BS_4 come with the same round of loads, so a
// longer code adds only its own byte loads. Codes of up to two bytes decode by
// the one- and two-byte tables, longer ones as dict[leaf2[first two bytes] +
// rest - 1] (indices clamped into the arrays whatever the bytes hold).
__device__ __forceinline__ void gather_dense_k4(const LookK &a, uint64_t t, uint32_t sel, uint64_t out_base,
                                                WarpSmemT<4> &sm, const int32_t *val1, uint32_t lane) {
    const uint4 *src = reinterpret_cast<const uint4 *>(a.dense + t * kTileRows);
    const uint4 v0 = __ldg(src + lane), v1 = __ldg(src + 32 + lane);
    const uint64_t w = t * kTileWords + lane, g = t * kGroupsPerTile;
    const bool has4 = a.K >= 4;
    const uint32_t m2 = __ldg(a.mask[2] + w), m3 = __ldg(a.mask[3] + w), m4 = has4 ? __ldg(a.mask[4] + w) : 0u;
    const uint32_t seg_lo = __ldg(a.off[2] + g), seg_hi = __ldg(a.off[2] + g + kGroupsPerTile);
    const uint32_t go2 = __ldg(a.off[2] + g + (lane >> 3)), go3 = __ldg(a.off[3] + g + (lane >> 3));
    const uint32_t go4 = has4 ? __ldg(a.off[4] + g + (lane >> 3)) : 0u;
    const uint32_t cnt = __popc(sel);
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, d);
        if (lane >= (uint32_t)d) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    // exclusive prefix of the mask popcounts inside each 256-row group
    auto group_excl = [&](uint32_t m) -> uint32_t {
        const uint32_t c = __popc(m);
        uint32_t inc = c;
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, inc, d);
            if ((lane & 7u) >= (uint32_t)d) inc += v;
        }
        return inc - c;
    };
    const uint32_t p2 = go2 + group_excl(m2) - seg_lo, p3 = go3 + group_excl(m3), p4 = go4 + group_excl(m4);
    {
        const uint32_t w0 = seg_lo >> 2, w1 = (seg_hi + 3) >> 2;
        const uint32_t *s32 = reinterpret_cast<const uint32_t *>(a.deep[2]);
        constexpr uint32_t kSegWords = sizeof(sm.seg) / 4;
        const uint32_t nseg = min(w1 - w0, kSegWords);
        for (uint32_t i0 = 0; i0 < nseg; i0 += 32u * kUnroll) {
            uint32_t r[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const uint32_t i = i0 + (uint32_t)u * 32u + lane;
                r[u] = i < nseg ? __ldg(s32 + w0 + i) : 0u;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const uint32_t i = i0 + (uint32_t)u * 32u + lane;
                if (i < nseg) sm.seg[i] = r[u];
            }
        }
    }
    uint4 r0, r1;
    transpose_lane_bytes(v0, v1, r0, r1);
    uint4 *rows = reinterpret_cast<uint4 *>(sm.dense + lane * 32u);
    rows[0] = r0;
    rows[1] = r1;
    sm.mask[0][lane] = m2;
    sm.pref[0][lane] = p2;
    sm.mask[1][lane] = m3;
    sm.pref[1][lane] = p3;
    sm.mask[2][lane] = m4;
    sm.pref[2][lane] = p4;
    uint32_t pos = incl - cnt, r = sel;
    while (r) {
        const uint32_t b = __ffs(r) - 1;
        r &= r - 1;
        sm.list[pos++] = (uint16_t)(lane * 32u + b);
    }
    __syncwarp();
    const uint8_t *seg = reinterpret_cast<const uint8_t *>(sm.seg) + (seg_lo & 3u);
    const uint64_t room = a.out_cap > out_base ? a.out_cap - out_base : 0;
    const uint32_t lim = (uint32_t)(room < total ? room : total);
    int32_t *dst = a.out_vals + out_base;
    const uint64_t l3 = a.deep_len[3] ? a.deep_len[3] - 1 : 0, l4 = a.deep_len[4] ? a.deep_len[4] - 1 : 0;
    const uint64_t dmax = a.dict_size ? a.dict_size - 1 : 0;
    // no branches: every load is predicated on the row's length, so the
    // kUnroll slots of a lane issue theirs together (byte 3 / 4, the two-byte
    // table or the leaf start, then the dictionary)
    auto value_of = [&](uint32_t i) -> int32_t {
        const uint32_t q = sm.list[i], wq = q >> 5, b = q & 31u, below = (1u << b) - 1u;
        const uint32_t c1 = sm.dense[q], mw2 = sm.mask[0][wq], mw3 = sm.mask[1][wq], mw4 = sm.mask[2][wq];
        const bool has2 = (mw2 >> b) & 1u, has3 = (mw3 >> b) & 1u, has4 = (mw4 >> b) & 1u;
        // the BS_2 index stays inside the staged segment even for a row
        // without byte 2, so the read needs no guard of its own
        const uint32_t key = (c1 << 8) | (has2 ? (uint32_t)seg[sm.pref[0][wq] + __popc(mw2 & below)] : 0u);
        const uint64_t i3 = (uint64_t)sm.pref[1][wq] + __popc(mw3 & below);
        const uint64_t i4 = (uint64_t)sm.pref[2][wq] + __popc(mw4 & below);
        const uint32_t b3 = has3 ? __ldg(a.deep[3] + (i3 < l3 ? i3 : l3)) : 0u;
        const uint32_t b4 = has4 ? __ldg(a.deep[4] + (i4 < l4 ? i4 : l4)) : 0u;
        const int32_t v2 = has2 && !has3 ? __ldg(a.val2 + key) : 0;
        const uint32_t leaf = has3 ? __ldg(a.leaf2 + key) : 0u;
        const uint64_t di = (uint64_t)leaf + (has4 ? ((b3 << 8) | b4) : b3) - 1;
        const int32_t vd = has3 ? __ldg(a.dict + (di < dmax ? di : dmax)) : 0;
        return has3 ? vd : (has2 ? v2 : val1[c1]);
    };
    uint32_t i0 = 0;
    for (; i0 + 32u * kUnroll <= lim; i0 += 32u * kUnroll) {
        int32_t v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) v[u] = value_of(i0 + (uint32_t)u * 32u + lane);
#pragma unroll
        for (int u = 0; u < kUnroll; u++) dst[i0 + (uint32_t)u * 32u + lane] = v[u];
    }
    for (uint32_t i = i0 + lane; i < lim; i += 32u) dst[i] = value_of(i);
    __syncwarp();
}

// One warp resolves tiles [tt0, tt1) of chunk c (16 tiles) whose first output
// slot is `base` (the whole chunk by default).
// It reads the chunk's 512 bit vector words at once. A sparse chunk (at most
// kSparseMax selected rows) lists its rows in shared memory and resolves them
// all in parallel across lanes; a dense chunk goes tile by tile.
// HOIST: dense two-byte PP-VBS chunks hold the chunk's off_2 entries in
// registers (more registers); without it each dense tile loads its own.
template <int LAYOUT, bool CODES, int KMAX, bool HOIST = true>
__device__ __forceinline__ void gather_chunk(const LookK &a, uint32_t c, uint64_t base, WarpSmemT<KMAX> &sm,
                                             const int32_t *val1, uint32_t lane, int tt0 = 0,
                                             int tt1 = kChunkTiles) {
    const uint64_t nwords = (a.n + 31) / 32;
    // the chunk's words: block i (4 tiles) holds words i*128 + 4L + 0..3 at lane L
    const uint64_t w0 = (uint64_t)c * kChunkTiles * kTileWords;
    uint32_t wv[4][4];
    uint32_t cnt[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        cnt[i] = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint64_t w = w0 + (uint64_t)(i * 128 + 4 * lane + k);
            const uint32_t vm = w < nwords ? valid_mask(w * 32u, a.n) : 0u;
            wv[i][k] = vm ? (__ldg(a.bits + w) & vm) : 0u;
            cnt[i] += __popc(wv[i][k]);
        }
    }
    const uint32_t chunk_total = warp_sum(cnt[0] + cnt[1] + cnt[2] + cnt[3]);
    if (chunk_total == 0) return;
    if (chunk_total <= kSparseMax) {
        if (tt0 != 0) return;  // a sparse chunk is resolved whole, by the warp of its first tiles
        // list the selected rows (row offset inside the chunk) in row order
        uint32_t pos0 = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            uint32_t incl = cnt[i];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t v = __shfl_up_sync(kFull, incl, d);
                if (lane >= (uint32_t)d) incl += v;
            }
            uint32_t pos = pos0 + incl - cnt[i];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                uint32_t r = wv[i][k];
                while (r) {
                    const uint32_t b = __ffs(r) - 1;
                    r &= r - 1;
                    sm.list[pos++] = (uint16_t)((i * 128 + 4 * lane + k) * 32 + b);
                }
            }
            pos0 += __shfl_sync(kFull, incl, 31);
        }
        __syncwarp();
        const uint64_t row0 = (uint64_t)c * kChunkTiles * kTileRows;
        for (uint32_t i0 = 0; i0 < chunk_total; i0 += 32 * kUnroll) {
            uint64_t code[kUnroll];
            int len[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const uint32_t i = i0 + (uint32_t)u * 32u + lane;
                code[u] = 0;
                len[u] = 1;
                if (i < chunk_total) row_code<LAYOUT, KMAX>(a, row0 + sm.list[i], code[u], len[u]);
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const uint32_t i = i0 + (uint32_t)u * 32u + lane;
                const uint64_t o = base + i;
                if (i < chunk_total && o < a.out_cap) {
                    if (CODES) a.out_codes[o] = LAYOUT == BS_PPVBS ? (code[u] << (8 * (a.K - len[u]))) : code[u];
                    else if (LAYOUT == BS_PPVBS && len[u] == 1) a.out_vals[o] = val1[code[u] & 0xFFu];
                    else a.out_vals[o] = decode_value<LAYOUT>(a, code[u], len[u]);
                }
            }
        }
        __syncwarp();
        return;
    }
    // dense chunk: tile by tile (tile 4i + j is lanes 8j..8j+7 of block i)
    uint32_t tcnt[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        uint32_t v = cnt[i];
        v += __shfl_xor_sync(kFull, v, 1);
        v += __shfl_xor_sync(kFull, v, 2);
        v += __shfl_xor_sync(kFull, v, 4);
        tcnt[i] = v;  // count of tile 4i + (lane >> 3)
    }
    // PP-VBS, codes <= 2 bytes: the chunk's 65 off_2 entries, two per lane
    // (entry e of the chunk at lane e / 2, the last one in every lane)
    constexpr bool kK2 = LAYOUT == BS_PPVBS && !CODES && KMAX == 2;
    constexpr bool kK4 = LAYOUT == BS_PPVBS && !CODES && KMAX == 4;
    constexpr bool kHoist = HOIST && kK2;
    uint32_t offa = 0, offb = 0, offz = 0;
    const uint64_t e0 = (uint64_t)c * kChunkTiles * kGroupsPerTile;
    if (kHoist && a.K >= 2) {
        const uint64_t nent = (uint64_t)a.n_tiles * kGroupsPerTile + 1;
        const uint64_t ea = e0 + 2 * lane;
        offa = ea < nent ? __ldg(a.off[2] + ea) : 0u;
        offb = ea + 1 < nent ? __ldg(a.off[2] + ea + 1) : 0u;
        offz = e0 + 64 < nent ? __ldg(a.off[2] + e0 + 64) : 0u;
    }
    auto off_entry = [&](uint32_t e) -> uint32_t {  // warp-wide call; e <= 64
        if (!kHoist) return a.K >= 2 ? __ldg(a.off[2] + e0 + e) : 0u;
        const uint32_t x = __shfl_sync(kFull, offa, (e >> 1) & 31u), y = __shfl_sync(kFull, offb, (e >> 1) & 31u);
        return e >= 64u ? offz : ((e & 1u) ? y : x);
    };
    // hoisted: lane i < 16 holds the selected-row count of tile i of the chunk
    uint32_t tcl = 0;
    if constexpr (kHoist) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t v = __shfl_sync(kFull, tcnt[i], j * 8);
                if (lane == (uint32_t)(4 * i + j)) tcl = v;
            }
        }
    }
    for (int tt = 0; tt < tt1; tt++) {
        uint32_t tc;
        if constexpr (kHoist) tc = __shfl_sync(kFull, tcl, tt);
        else tc = __shfl_sync(kFull, tcnt[tt >> 2], (tt & 3) * 8);
        if (tt < tt0) {  // tiles of another warp of this chunk: only their slots
            base += tc;
            continue;
        }
        const uint64_t t = (uint64_t)c * kChunkTiles + tt;
        if (tc && t < a.n_tiles && base < a.out_cap) {
            const uint64_t w = t * kTileWords + lane;
            const uint32_t vm = valid_mask(w * 32u, a.n);
            const uint32_t sel = vm ? (__ldg(a.bits + w) & vm) : 0u;
            if (kK2 && tc >= kStageMin) {
                const uint32_t e = (uint32_t)tt * kGroupsPerTile;
                const uint32_t goff = off_entry(e + (lane >> 3));
                const uint32_t lo = off_entry(e), hi = off_entry(e + kGroupsPerTile);
                gather_dense_k2(a, t, sel, base, goff, lo, hi, reinterpret_cast<WarpSmemT<2> &>(sm), val1, lane);
            } else if (kK4 && tc >= kStageMin && !a.categorical) {
                gather_dense_k4(a, t, sel, base, reinterpret_cast<WarpSmemT<4> &>(sm), val1, lane);
            } else {
                gather_tile<LAYOUT, CODES, KMAX>(a, t, sel, base, sm, val1, lane);
            }
        }
        base += tc;
    }
}

// One tile with `tc` selected rows (sel: the lane's word) whose first output
// slot is `base`, by the same per-tile paths as a dense chunk of
// gather_chunk: staged BS_1 / BS_2 for dense PP-VBS tiles of codes up to two
// (or, numerical, four) bytes, the listed-rows path otherwise. The tile's
// off_2 entries are loaded here (gather_chunk can hold a chunk's in registers).
template <int LAYOUT, int KMAX>
__device__ __forceinline__ void gather_one_tile(const LookK &a, uint64_t t, uint32_t sel, uint32_t tc, uint64_t base,
                                                WarpSmemT<KMAX> &sm, const int32_t *val1, uint32_t lane) {
    constexpr bool kK2 = LAYOUT == BS_PPVBS && KMAX == 2;
    constexpr bool kK4 = LAYOUT == BS_PPVBS && KMAX == 4;
    if (kK2 && tc >= kStageMin) {
        const uint64_t e = t * kGroupsPerTile;
        const bool has2 = a.K >= 2;
        const uint32_t goff = has2 ? __ldg(a.off[2] + e + (lane >> 3)) : 0u;
        const uint32_t lo = has2 ? __ldg(a.off[2] + e) : 0u, hi = has2 ? __ldg(a.off[2] + e + kGroupsPerTile) : 0u;
        gather_dense_k2(a, t, sel, base, goff, lo, hi, reinterpret_cast<WarpSmemT<2> &>(sm), val1, lane);
    } else if (kK4 && tc >= kStageMin && !a.categorical) {
        gather_dense_k4(a, t, sel, base, reinterpret_cast<WarpSmemT<4> &>(sm), val1, lane);
    } else {
        gather_tile<LAYOUT, false, KMAX>(a, t, sel, base, sm, val1, lane);
    }
}

// LookK view of a column (the per-call fields are filled by the caller).
inline LookK make_look_args(const Column &c) {
    LookK a{};
    a.layout = c.layout;
    a.K = c.layout == BS_PPVBS ? c.K : c.S;
    a.categorical = c.categorical ? 1 : 0;
    a.cat_B = c.cat_B;
    a.k = c.k;
    a.identity = c.identity ? 1 : 0;
    a.domain_min = c.domain_min;
    a.n = c.n;
    a.n_tiles = c.n_tiles;
    a.n_chunks = (c.n_tiles + kChunkTiles - 1) / kChunkTiles;
    a.n_groups = (a.n_chunks + kGroupChunks - 1) / kGroupChunks;
    a.dense = c.d_dense;
    a.slice_bytes = c.dense_slice_bytes();
    for (int j = 2; j <= c.K && c.layout == BS_PPVBS; j++) {
        a.mask[j] = c.d_mask[j];
        a.off[j] = c.d_off[j];
        a.deep[j] = c.d_deep[j];
        a.deep_len[j] = c.deep_len[j];
    }
    a.packed = c.d_packed;
    a.val2 = c.d_val2;
    a.leaf2 = c.d_leaf2;
    a.dict = c.d_dict;
    a.dict_size = c.dict.size();
    return a;
}

// Largest code length the gather must handle, as a template constant.
inline int kmax_for(const LookK &a) { return (a.layout == BS_PPVBS && a.K > 4) ? 8 : (a.K > 2 ? 4 : 2); }

}  // namespace
}  // namespace bs
