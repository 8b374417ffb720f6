// Device code shared by the kernels that evaluate whole predicates tile by
// tile inside one launch (the batched kernel in batch.cu and the fused
// scan + lookup kernel in fused.cu): one predicate of any layout on one
// 1024-row tile, restricted to the rows of a seed word (the pipelined bit
// vectors of Section 3.3.1 held in registers), with the predicate's kernel
// variant chosen at run time from its host plan.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "scan_dev.cuh"

namespace bs {
namespace {

struct BPred {
    ScanK a;
    ScanPlan plan;
};

// ---------------------------------------------------------- predicate tile
template <int KB>
__device__ __forceinline__ uint32_t packed_tile(const ScanK &a, uint32_t t, uint32_t lane, uint32_t sd) {
    uint32_t w[KB];
    load_packed<KB>(a.packed + ((uint64_t)t * kTileWords + lane) * KB, w);
    uint32_t res = a.lo > a.hi ? 0u : packed_bits<KB>(w, (uint32_t)a.lo, (uint32_t)(a.hi - a.lo));
    if (a.invert) res = ~res;
    return res & sd;
}

__device__ __noinline__ uint32_t packed_dispatch(const ScanK &a, int k, uint32_t t, uint32_t lane, uint32_t sd) {
    switch (k) {
#define BS_PK(K) \
    case K: return packed_tile<K>(a, t, lane, sd);
        BS_PK(1) BS_PK(2) BS_PK(3) BS_PK(4) BS_PK(5) BS_PK(6) BS_PK(7) BS_PK(8)
        BS_PK(9) BS_PK(10) BS_PK(11) BS_PK(12) BS_PK(13) BS_PK(14) BS_PK(15) BS_PK(16)
        BS_PK(17) BS_PK(18) BS_PK(19) BS_PK(20) BS_PK(21) BS_PK(22) BS_PK(23) BS_PK(24)
        BS_PK(25) BS_PK(26) BS_PK(27) BS_PK(28) BS_PK(29) BS_PK(30) BS_PK(31) BS_PK(32)
#undef BS_PK
    default: return 0u;
    }
}

template <bool VBS, int NLIT>
__device__ __noinline__ uint32_t dense_dispatch(const ScanK &a, const ScanPlan &pl, uint32_t t, uint32_t lane,
                                                const uint32_t x[8], uint32_t sd) {
    const uint32_t c0 = lit_byte(a.lit[0], 1);
    const uint32_t add0 = thr_add(c0), add1 = thr_add(c0 + 1);
    const int sel = (pl.hi0 ? 4 : 0) | (pl.hi1 ? 2 : 0) | (pl.eq1 ? 1 : 0);
    switch (sel) {
    case 0: return scan_tile<VBS, NLIT, false, false, false, false>(a, t, lane, x, sd, add0, add1, 0u);
    case 1: return scan_tile<VBS, NLIT, false, false, true, false>(a, t, lane, x, sd, add0, add1, 0u);
    case 2: return scan_tile<VBS, NLIT, false, true, false, false>(a, t, lane, x, sd, add0, add1, 0u);
    case 3: return scan_tile<VBS, NLIT, false, true, true, false>(a, t, lane, x, sd, add0, add1, 0u);
    case 4: return scan_tile<VBS, NLIT, true, false, false, false>(a, t, lane, x, sd, add0, add1, 0u);
    case 5: return scan_tile<VBS, NLIT, true, false, true, false>(a, t, lane, x, sd, add0, add1, 0u);
    case 6: return scan_tile<VBS, NLIT, true, true, false, false>(a, t, lane, x, sd, add0, add1, 0u);
    default: return scan_tile<VBS, NLIT, true, true, true, false>(a, t, lane, x, sd, add0, add1, 0u);
    }
}

// A dense-slice predicate on one tile whose lane bytes x are already loaded.
__device__ __forceinline__ uint32_t dense_pred(const BPred &P, uint32_t t, uint32_t lane, const uint32_t x[8],
                                               uint32_t sd) {
    const ScanPlan &pl = P.plan;
    if (pl.vbs) return pl.nlit == 2 ? dense_dispatch<true, 2>(P.a, pl, t, lane, x, sd)
                                    : dense_dispatch<true, 1>(P.a, pl, t, lane, x, sd);
    return pl.nlit == 2 ? dense_dispatch<false, 2>(P.a, pl, t, lane, x, sd)
                        : dense_dispatch<false, 1>(P.a, pl, t, lane, x, sd);
}

// One predicate on one tile, restricted to the rows of sd (warp-wide call).
__device__ __forceinline__ uint32_t pred_tile(const BPred &P, uint32_t t, uint32_t lane, uint32_t sd) {
    const ScanPlan &pl = P.plan;
    const ScanK &a = P.a;
    if (pl.kind == ScanPlan::kFill) return a.fill_all ? sd : 0u;
    if (pl.kind == ScanPlan::kPacked) return sd ? packed_dispatch(a, pl.k, t, lane, sd) : 0u;
    uint32_t x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (sd) load_lane32(a.dense + (uint64_t)t * kTileRows, lane, x);
    return dense_pred(P, t, lane, x, sd);
}

__device__ __forceinline__ uint32_t claim(uint32_t *ctr, uint32_t lane) {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(ctr, 1u);
    return __shfl_sync(kFull, u, 0);
}

}  // namespace
}  // namespace bs
