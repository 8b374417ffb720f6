// Device code of the scan kernels for sm_103a (shared by the single-query
// kernels of scan.cu and the batched kernel of batch.cu): PP-VBS (Algorithm 3), ByteSlice (Section 2.5) and
// Bit-Packed (Section 2.3), with optional seeding by a previous result bit
// vector (the pipelined conjunction of Section 3.3.1).
//
// One warp owns one 1024-row tile at a time (grid-stride over tiles); lane L
// owns rows 32L..32L+31 of the tile and produces result word L.
//
// Byte compare (the counterpart of the paper's cmpgt/cmpeq + movemask): each
// 32-bit word holds 4 row bytes. With r = x & 0x7f7f7f7f, adding
// 0x80 - (k & 0x7f) to every byte puts "low 7 bits >= k's low 7 bits" into bit
// 7 without carries between bytes; AND-ing (k >= 0x80) or OR-ing (k < 0x80)
// with x's own bit 7 then gives "x >= k" unsigned in bit 7 of every byte (one
// LOP3 when the high bit of k is a template constant). "x == c" is
// ge(c) & ~ge(c+1) (c + 1 = 256 never matches). The dense slices are stored so
// that word w byte b of a lane's 32 bytes is row 8b + w, hence OR-ing word w
// shifted right by 7 - w gathers the 32 flags of a lane into a row-ordered
// result word.
//
// Early stop (Section 2.5, Lemma 1): after byte 1 a lane keeps, per literal,
// LT (decided smaller) and EQ (equal so far) masks. Deeper bytes are touched
// only while some lane of the warp still has EQ rows (__any_sync). For PP-VBS a
// row's byte j exists iff bit j of mask M_j is set; the mask words are read
// only for 256-row groups (one 32-byte sector of M_j) that contain pending
// rows, and each pending row's byte is fetched from the packed slice BS_j at
// off_j[group] + (popcounts of the group's earlier mask words) + rank in its
// word. Rows that end before the literal are smaller, rows that continue past
// it are larger (the code tail after a shared prefix is never zero).
// When the predicate only needs "smaller" for a literal (v < c, v >= c and the
// lower end of BETWEEN), rows still equal after the literal's last byte are
// settled (equal or larger: never smaller), so level l + 1 is not read; with a
// one-byte literal the EQ mask is not even formed.
//
// Unseeded scans stream slice 1 through a cp.async ring in shared memory per
// warp (two slots in the single-query kernel: the next tile is in flight while
// one is resolved; kStages in the batched kernel). Each lane reads back only
// the 32 bytes it copied itself, so no barrier is needed beyond
// cp.async.wait_group.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dev_common.cuh"
#include "kernels.h"

namespace bs {
namespace {


constexpr uint32_t kMsb = 0x80808080u;
constexpr uint32_t kLow7 = 0x7F7F7F7Fu;
constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / 32;
constexpr int kStages = 3;  // ring slots per warp in the batched kernel (default; 2..kStagesMax)
constexpr int kStagesMax = 4;

struct DLit {
    uint32_t len;      // bytes in the literal code
    int32_t jend;      // deepest level whose masks/bytes can change the result
    uint64_t left;     // code left-aligned in 64 bits: byte j (1-based) = left >> (64 - 8j)
};

struct ScanK {
    const uint8_t *dense;      // BS_1 (PP-VBS) or slice 1 (ByteSlice)
    uint64_t slice_bytes;      // ByteSlice: distance between slices
    const uint32_t *mask[kMaxCodeBytes + 1];
    const uint32_t *off[kMaxCodeBytes + 1];
    const uint8_t *deep[kMaxCodeBytes + 1];
    uint64_t deep_len[kMaxCodeBytes + 1];
    const uint32_t *packed;
    uint64_t n;
    uint32_t n_tiles;
    int32_t K;                 // PP-VBS longest code; ByteSlice slice count
    int32_t k;                 // Bit-Packed code bits
    int32_t op;
    int32_t fill_all;          // fill kernel: 1 = every valid (seeded) row, 0 = none
    DLit lit[2];
    uint64_t lo, hi;           // Bit-Packed: code range of the predicate
    int32_t invert;            // Bit-Packed: result = !(lo <= code <= hi)
    uint32_t fin_l, fin_e, fin_i;  // one literal: result = ((LT & fin_l) | (EQ & fin_e)) ^ (valid & fin_i), all-ones or zero each
    uint32_t stop_all;         // early-stop granularity: 0 = a deeper level is read per 256-row group
                               // (PP-VBS) or lane (ByteSlice) with pending rows, 1 = for the whole
                               // 1024-row tile once any of its rows is pending
    const uint32_t *seed;
    uint32_t *out;
    uint32_t *status;
};

__device__ __forceinline__ uint4 ld_stream_v4(const uint8_t *p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ void st_stream(uint32_t *p, uint32_t v) {
    asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}



__device__ __forceinline__ uint32_t lit_byte(const DLit &l, int j) {  // j = 1..8
    return (uint32_t)(l.left >> (64 - 8 * j)) & 0xFFu;
}

// threshold constants for "byte >= k", k in 0..256
__device__ __forceinline__ uint32_t thr_add(uint32_t k) { return k >= 256u ? 0u : (0x80u - (k & 0x7Fu)) * 0x01010101u; }
__device__ __forceinline__ bool thr_hi(uint32_t k) { return k >= 128u; }

template <bool HI>
__device__ __forceinline__ uint32_t ge_msb(uint32_t x, uint32_t x7, uint32_t add) {
    const uint32_t y = x7 + add;
    return HI ? (y & x & kMsb) : ((y | x) & kMsb);
}

__device__ __forceinline__ uint32_t ge_msb_rt(uint32_t x, uint32_t x7, uint32_t add, uint32_t sel) {
    const uint32_t y = x7 + add;
    return ((y & x) | ((y | x) & sel)) & kMsb;
}

__device__ __forceinline__ uint32_t gather8(const uint32_t m[8]) {
    return (m[0] >> 7) | (m[1] >> 6) | (m[2] >> 5) | (m[3] >> 4) | (m[4] >> 3) | (m[5] >> 2) | (m[6] >> 1) | m[7];
}

// Byte 1 against literal byte c with compile-time high bits of c and c + 1.
// GE = rows with byte >= c; EQ = rows with byte == c (only if NEED_EQ).
template <bool HI0, bool HI1, bool NEED_EQ>
__device__ __forceinline__ void cmp32_fast(const uint32_t x[8], uint32_t add0, uint32_t add1, uint32_t &GE,
                                           uint32_t &EQ) {
    uint32_t ge[8], eq[8];
#pragma unroll
    for (int w = 0; w < 8; w++) {
        const uint32_t x7 = x[w] & kLow7;
        ge[w] = ge_msb<HI0>(x[w], x7, add0);
        if (NEED_EQ) eq[w] = ge[w] & ~ge_msb<HI1>(x[w], x7, add1);
    }
    GE = gather8(ge);
    if (NEED_EQ) EQ = gather8(eq);
}

// Runtime-constant variant (deeper ByteSlice slices, BETWEEN's upper literal).
__device__ __forceinline__ void cmp32_rt(const uint32_t x[8], uint32_t c, uint32_t &LT, uint32_t &EQ) {
    const uint32_t a0 = thr_add(c), a1 = thr_add(c + 1);
    const uint32_t s0 = thr_hi(c) ? 0u : kFull, s1 = thr_hi(c + 1) ? 0u : kFull;
    uint32_t ge[8], eq[8];
#pragma unroll
    for (int w = 0; w < 8; w++) {
        const uint32_t x7 = x[w] & kLow7;
        ge[w] = ge_msb_rt(x[w], x7, a0, s0);
        eq[w] = ge[w] & ~ge_msb_rt(x[w], x7, a1, s1);
    }
    LT = ~gather8(ge);
    EQ = gather8(eq);
}

__device__ __forceinline__ void load_lane32(const uint8_t *tile, uint32_t lane, uint32_t x[8]) {
    uint4 v0 = ld_stream_v4(tile + lane * 16u);
    uint4 v1 = ld_stream_v4(tile + 512u + lane * 16u);
    x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
    x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
}

// ------------------------------------------------------- PP-VBS levels >= 2
template <int NLIT, bool PF>
__device__ __forceinline__ void vbs_deeper(const ScanK &a, uint32_t t, uint32_t lane, uint32_t m2_pre, uint32_t &LT1,
                                           uint32_t &EQ1, uint32_t &LT2, uint32_t &EQ2) {
    const int K = a.K;
    const int l1 = (int)a.lit[0].len, e1 = a.lit[0].jend;
    const int l2 = NLIT == 2 ? (int)a.lit[1].len : 0, e2 = NLIT == 2 ? a.lit[1].jend : 1;
    const int jend = max(e1, e2);
    const uint64_t wbase = (uint64_t)t * kTileWords;
    for (int j = 2; j <= jend; j++) {
        const bool act1 = j <= e1, act2 = NLIT == 2 && j <= e2;
        const uint32_t pend = (act1 ? EQ1 : 0u) | (act2 ? EQ2 : 0u);
        if (!__any_sync(kFull, pend != 0u)) break;
        // M_j only for 256-row groups (8 lanes) holding a pending row; M_2 may
        // already be in shared memory (prefetched with the tile)
        uint32_t mj;
        if (PF && j == 2) {
            mj = m2_pre;
        } else {
            const uint32_t bal = __ballot_sync(kFull, pend != 0u);
            const uint32_t gact = a.stop_all ? bal : ((bal >> (lane & 24u)) & 0xFFu);
            mj = gact ? __ldg(a.mask[j] + wbase + lane) : 0u;
        }
        if (act1) {
            if (j <= l1) { LT1 |= EQ1 & ~mj; EQ1 &= mj; }   // row ends first: smaller
            else EQ1 &= ~mj;                               // row continues: larger; else equal
        }
        if (act2) {
            if (j <= l2) { LT2 |= EQ2 & ~mj; EQ2 &= mj; }
            else EQ2 &= ~mj;
        }
        const uint32_t need = (act1 && j <= l1 ? EQ1 : 0u) | (act2 && j <= l2 ? EQ2 : 0u);
        if (!__any_sync(kFull, need != 0u)) continue;
        // rank of each byte in BS_j: exclusive prefix of popcounts inside the group
        const uint32_t cnt = __popc(mj);
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, d);
            if ((lane & 7u) >= (uint32_t)d) incl += v;
        }
        if (need) {
            const uint64_t base = (uint64_t)__ldg(a.off[j] + (uint64_t)t * kGroupsPerTile + (lane >> 3)) + (incl - cnt);
            const uint8_t *deep = a.deep[j];
            const uint64_t dlen = a.deep_len[j];
            const uint32_t c1 = lit_byte(a.lit[0], j);
            const uint32_t c2 = NLIT == 2 ? lit_byte(a.lit[1], j) : 0u;
            // collect "less" and "differs" against each literal over the
            // lane's pending rows, then apply them once to the rows still
            // equal to that literal (the lane's BS_j bytes are the run
            // [base, base + cnt))
            if (base + cnt <= dlen) {
                const uint8_t *run = deep + base;
                uint32_t bits = need, lt1 = 0u, ne1 = 0u, lt2 = 0u, ne2 = 0u;
                while (bits) {
                    const uint32_t bit = bits & (0u - bits);
                    bits ^= bit;
                    const uint32_t byte = __ldg(run + __popc(mj & (bit - 1u)));
                    lt1 |= byte < c1 ? bit : 0u;
                    ne1 |= byte != c1 ? bit : 0u;
                    if (NLIT == 2) {
                        lt2 |= byte < c2 ? bit : 0u;
                        ne2 |= byte != c2 ? bit : 0u;
                    }
                }
                if (NLIT == 1) {  // every pending row is still equal to the literal
                    LT1 |= lt1;
                    EQ1 &= ~ne1;
                } else {
                    const uint32_t d1 = act1 && j <= l1 ? EQ1 & need : 0u;
                    const uint32_t d2 = act2 && j <= l2 ? EQ2 & need : 0u;
                    LT1 |= lt1 & d1;
                    EQ1 &= ~(ne1 & d1);
                    LT2 |= lt2 & d2;
                    EQ2 &= ~(ne2 & d2);
                }
            } else {
                atomicOr(a.status, kStatusBounds);
            }
        }
    }
    // a literal longer than every stored code: an equal prefix means a shorter row
    if (l1 > K) { LT1 |= EQ1; EQ1 = 0; }
    if (NLIT == 2 && l2 > K) { LT2 |= EQ2; EQ2 = 0; }
}

// ---------------------------------------------------- ByteSlice slices >= 2
template <int NLIT>
__device__ __forceinline__ void bsl_deeper(const ScanK &a, uint32_t t, uint32_t lane, uint32_t &LT1, uint32_t &EQ1,
                                        uint32_t &LT2, uint32_t &EQ2) {
    for (int j = 2; j <= a.K; j++) {
        const uint32_t pend = EQ1 | EQ2;
        if (!__any_sync(kFull, pend != 0u)) break;
        if (pend || a.stop_all) {
            uint32_t x[8];
            load_lane32(a.dense + (uint64_t)(j - 1) * a.slice_bytes + (uint64_t)t * kTileRows, lane, x);
            uint32_t lt, eq;
            cmp32_rt(x, lit_byte(a.lit[0], j), lt, eq);
            LT1 |= EQ1 & lt;
            EQ1 &= eq;
            if (NLIT == 2) {
                cmp32_rt(x, lit_byte(a.lit[1], j), lt, eq);
                LT2 |= EQ2 & lt;
                EQ2 &= eq;
            }
        }
    }
}

// One tile whose lane bytes are in x: byte 1, deeper levels, result word.
// HI23 (BETWEEN): bit 1 / bit 0 = high bit of the upper literal's first byte
// c2 / of c2 + 1 as compile-time constants (add2, add3 its thresholds), or -1
// to compare against c2 with run-time thresholds.
template <bool VBS, int NLIT, bool HI0, bool HI1, bool NEED_EQ, bool PF, int HI23 = -1>
__device__ __forceinline__ uint32_t scan_tile(const ScanK &a, uint32_t t, uint32_t lane, const uint32_t x[8],
                                          uint32_t sd, uint32_t add0, uint32_t add1, uint32_t m2_pre,
                                          uint32_t add2 = 0u, uint32_t add3 = 0u) {
    uint32_t GE1, EQ1 = 0, LT2 = 0, EQ2 = 0;
    cmp32_fast<HI0, HI1, NEED_EQ>(x, add0, add1, GE1, EQ1);
    uint32_t LT1 = sd & ~GE1;
    EQ1 &= sd;
    if (NLIT == 2) {
        if constexpr (HI23 >= 0) {
            uint32_t GE2;
            cmp32_fast<(HI23 & 2) != 0, (HI23 & 1) != 0, true>(x, add2, add3, GE2, EQ2);
            LT2 = ~GE2;
        } else {
            cmp32_rt(x, lit_byte(a.lit[1], 1), LT2, EQ2);
        }
        LT2 &= sd;
        EQ2 &= sd;
    }
    if (NEED_EQ || NLIT == 2) {
        if (__any_sync(kFull, (EQ1 | EQ2) != 0u)) {
            if (VBS) vbs_deeper<NLIT, PF>(a, t, lane, m2_pre, LT1, EQ1, LT2, EQ2);
            else bsl_deeper<NLIT>(a, t, lane, LT1, EQ1, LT2, EQ2);
        }
    }
    const uint64_t w = (uint64_t)t * kTileWords + lane;
    // the op from the fully resolved (LT, EQ) masks: BETWEEN keeps rows not
    // below c1 and not above c2; one literal picks LT and/or EQ and, for >, >=
    // and !=, complements within the valid rows (LT and EQ are subsets of them)
    const uint32_t res = NLIT == 2 ? (sd & ~LT1 & (LT2 | EQ2)) : (((LT1 & a.fin_l) | (EQ1 & a.fin_e)) ^ (sd & a.fin_i));
    if (a.out && w * 32u < a.n) st_stream(a.out + w, res);
    return res;
}

// ------------------------------------------------------------ Bit-Packed
// Lane L owns codes 32L..32L+31 of a tile; as 32 codes of k bits fill exactly k
// words, its codes are the k stream words starting at tile word L*k, loaded
// with 16-, 8- or 4-byte vector loads (k % 4 == 0, k even, k odd). With k a
// template constant every code is extracted with constant shifts; the range
// test (code - lo) <= span (unsigned) replaces the paper's cmpgt_epi32.
// Tiles are processed two at a time for k <= 16 so twice the words are in
// flight per warp.
template <int KB>
__device__ __forceinline__ void load_packed(const uint32_t *p, uint32_t w[KB]) {
    if (KB % 4 == 0) {
#pragma unroll
        for (int i = 0; i < KB / 4; i++) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p) + i);
            w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
        }
    } else if (KB % 2 == 0) {
#pragma unroll
        for (int i = 0; i < KB / 2; i++) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p) + i);
            w[2 * i] = v.x; w[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < KB; i++) w[i] = __ldg(p + i);
    }
}

template <int KB>
__device__ __forceinline__ uint32_t packed_bits(const uint32_t w[KB], uint32_t lo, uint32_t span) {
    constexpr uint32_t kMask = KB == 32 ? 0xFFFFFFFFu : ((1u << KB) - 1u);
    uint32_t res = 0;
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int bit = i * KB, wi = bit >> 5, sh = bit & 31;
        uint32_t code = w[wi] >> sh;
        if (sh + KB > 32) code |= w[wi + 1] << (32 - sh);
        code &= kMask;
        res |= (uint32_t)((code - lo) <= span) << i;
    }
    return res;
}


// ------------------------------------------------------------ host planning
inline DLit make_dlit(const LitCode &l) {
    DLit d{};
    d.len = l.len;
    d.left = l.len >= 8 ? l.code : (l.code << (8 * (8 - l.len)));
    return d;
}

// Which kernel variant runs a predicate, and with which constants.
struct ScanPlan {
    enum Kind : int32_t { kFill = 0, kPacked = 1, kDense = 2 };
    int32_t kind;
    int32_t k;        // Bit-Packed code bits
    bool vbs;         // dense: PP-VBS (else ByteSlice)
    int32_t nlit;     // 2 for BETWEEN
    bool hi0, hi1;    // high bits of the first literal byte c and of c + 1
    bool hi2, hi3;    // BETWEEN: the same for the upper literal's first byte
    bool eq1;         // the EQ mask of byte 1 is needed
    bool pf;          // PP-VBS: prefetch M_2 with every tile
};

// Fills the column and predicate fields of `a` (not out / status) and picks the
// variant. allow_pf: the caller's kernel can prefetch M_2 (the single-query ring).
inline void plan_scan(const Column &c, const KPred &p, const uint32_t *d_seed, bool allow_pf, ScanK &a,
                      ScanPlan &plan) {
    a = ScanK{};
    plan = ScanPlan{};
    a.n = c.n;
    a.n_tiles = c.n_tiles;
    a.seed = d_seed;
    a.op = p.op;
    {  // < : LT; <= : LT|EQ; > : valid & ~(LT|EQ); >= : valid & ~LT; = : EQ; != : valid & ~EQ
        const bool L = p.op == BS_LT || p.op == BS_LE || p.op == BS_GT || p.op == BS_GE;
        const bool E = p.op == BS_LE || p.op == BS_GT || p.op == BS_EQ || p.op == BS_NE;
        const bool I = p.op == BS_GT || p.op == BS_GE || p.op == BS_NE;
        a.fin_l = L ? 0xFFFFFFFFu : 0u;
        a.fin_e = E ? 0xFFFFFFFFu : 0u;
        a.fin_i = I ? 0xFFFFFFFFu : 0u;
    }
    if (p.mode != Pred::kNormal) {
        a.fill_all = p.mode == Pred::kAll;
        plan.kind = ScanPlan::kFill;
        return;
    }
    const int nlit = p.op == BS_BETWEEN ? 2 : 1;
    plan.nlit = nlit;
    if (c.layout == BS_BITPACKED) {
        plan.kind = ScanPlan::kPacked;
        plan.k = c.k;
        a.packed = c.d_packed;
        a.k = c.k;
        const uint64_t c1 = p.lit[0].code, c2 = p.lit[1].code;
        const uint64_t top = (c.k >= 64) ? ~0ull : ((1ull << c.k) - 1);
        a.invert = 0;
        switch (p.op) {
        case BS_LT:
            if (c1 == 0) { a.lo = 1; a.hi = 0; }  // empty range
            else { a.lo = 0; a.hi = c1 - 1; }
            break;
        case BS_LE: a.lo = 0; a.hi = c1; break;
        case BS_GT: a.lo = c1 + 1; a.hi = top; break;
        case BS_GE: a.lo = c1; a.hi = top; break;
        case BS_EQ: a.lo = c1; a.hi = c1; break;
        case BS_NE: a.lo = c1; a.hi = c1; a.invert = 1; break;
        default: a.lo = c1; a.hi = c2; break;
        }
        return;
    }
    plan.kind = ScanPlan::kDense;
    plan.vbs = c.layout == BS_PPVBS;
    a.dense = c.d_dense;
    a.slice_bytes = c.dense_slice_bytes();
    LitCode l0 = p.lit[0], l1 = nlit == 2 ? p.lit[1] : p.lit[0];
    const int K = c.layout == BS_PPVBS ? c.K : c.S;
    if (c.layout == BS_BYTESLICE) {
        // ByteSlice bytes are those of the code left-aligned in S bytes
        l0.code <<= (8 * c.S - c.k);
        l1.code <<= (8 * c.S - c.k);
        l0.len = l1.len = (uint32_t)c.S;
    }
    a.lit[0] = make_dlit(l0);
    a.lit[1] = make_dlit(l1);
    a.K = K;
    // does the result depend on "equal after the literal's last byte"?
    const bool need_eq0 = !(p.op == BS_LT || p.op == BS_GE || p.op == BS_BETWEEN);
    a.lit[0].jend = need_eq0 ? std::min((int)l0.len + 1, K) : std::min((int)l0.len, K);
    a.lit[1].jend = nlit == 2 ? std::min((int)l1.len + 1, K) : 1;  // BETWEEN's upper end: v <= c2
    // the EQ mask of byte 1 matters if a deeper level can still decide
    // "smaller", or if the predicate reads it directly
    // (BETWEEN: the lower end needs it only when its literal has a second
    // byte; rows equal to a one-byte lower literal are settled, not smaller)
    plan.eq1 = need_eq0 || l0.len >= 2;
    if (c.layout == BS_PPVBS) {
        for (int j = 2; j <= c.K; j++) {
            a.mask[j] = c.d_mask[j];
            a.off[j] = c.d_off[j];
            a.deep[j] = c.d_deep[j];
            a.deep_len[j] = c.deep_len[j];
        }
    }
    const uint32_t cb = (uint32_t)(a.lit[0].left >> 56);
    plan.hi0 = cb >= 128u;
    plan.hi1 = cb + 1 >= 128u;
    const uint32_t cb2 = (uint32_t)(a.lit[1].left >> 56);
    plan.hi2 = nlit == 2 && cb2 >= 128u;
    plan.hi3 = nlit == 2 && cb2 + 1 >= 128u;
    // prefetch M_2 with every tile when rows sharing the literal's first byte are
    // common enough that most tiles have some (more than one per tile on
    // average; 2^30-row columns of 12 to 20 bits: 3-9 % faster `<` and `=`
    // scans than a threshold of four per tile, BETWEEN unchanged)
    if (allow_pf && c.layout == BS_PPVBS && c.K >= 2 && (plan.eq1 || nlit == 2) && !d_seed) {
        if (c.first_byte_rows.size() == 256) {
            const uint32_t b1 = (uint32_t)(a.lit[1].left >> 56);
            const uint64_t share = c.first_byte_rows[cb] + (nlit == 2 && b1 != cb ? c.first_byte_rows[b1] : 0);
            plan.pf = share * (uint64_t)kTileRows > c.n;
        } else {
            plan.pf = true;  // raw-code column: no statistics
        }
    }
}

}  // namespace
}  // namespace bs
