// Fused scan + lookup for sm_103a: a conjunction of 1..4 predicates (Section
// 3.3.1's pipelined bit vectors) followed by the lookup of a projected column
// (Section 2.2's query shape, Algorithm 4), in one persistent kernel with no
// round trip of the result bit vector through memory.
//
// Work units are runs of four 1024-row tiles, claimed in order from an atomic
// ticket. Per unit a warp
//   1. evaluates the predicates on its tiles (the first predicate's dense
//      slice streamed through a two-slot cp.async ring, the others seeded by
//      the running result held in registers), optionally storing the result
//      bit vector words;
//   2. publishes the unit's selected-row count and finds the unit's first
//      output slot by a decoupled look-back over the descriptors of earlier
//      units (each descriptor is one 64-bit word: a state in the top two bits,
//      "count of this unit" or "inclusive prefix up to this unit", and the
//      value below, so a reader never sees a state without its value);
//      then publishes its inclusive prefix;
//   3. gathers the projected column's values of the selected rows of its
//      tiles with the lookup's per-tile code (lookup_dev.cuh).
// Steps 2 and 3 of a unit come after step 1 of the warp's next unit (see the
// main loop), so that look-backs rarely wait. The ring and the gather's
// scratch share a warp's shared memory (the next tiles are copied in after
// the gather), which with at most 51 registers a thread keeps five CTAs (40
// warps) of the specialised variant resident per SM. The gather reads a
// tile's BS_1 bytes again, a unit or two after the scan copied them: the
// scan's copies ask L2 to keep those lines (evict_last) and the gather's reads
// let them go (evict_first), so the second read is mostly an L2 hit rather
// than a second trip to DRAM.
// Measured and dropped (2^30 rows, v < c at 13.7 %): one tile per unit with
// the tile held in shared memory from scan to gather (no second read, but a
// look-back per tile: with ~5,000 warps claiming, the walk to the nearest
// published prefix outgrew its 128-descriptor window: 1.67 ms); units of 8
// or 16 tiles (1.31 / 2.20 ms: the second read of BS_1 misses L2 more).
// Because units are claimed in order, every unit a look-back waits for has
// been claimed by a running warp, so the wait always ends; it is bounded
// anyway (a timeout is recorded in the status word and the warp goes on).
//
// The single-predicate query whose projection is the predicate's own PP-VBS
// column (the bench's query) runs a specialised variant with the predicate's
// first-byte thresholds as compile-time constants, as the single-query scan
// kernel does; everything else runs the generic variant.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <utility>

#include "lookup_dev.cuh"
#include "pred_dev.cuh"
#include "scan_dev.cuh"

namespace bs {
namespace {

constexpr int kFuseTiles = 4;  // tiles per work unit (one look-back each)
constexpr int kFuseThreads = 256;
constexpr int kFuseWarps = kFuseThreads / 32;
constexpr uint64_t kDescAgg = 1ull << 62;  // descriptor holds the unit's own count
constexpr uint64_t kDescInc = 2ull << 62;  // descriptor holds the inclusive prefix
constexpr uint64_t kDescVal = kDescAgg - 1;
constexpr uint32_t kLookbackPolls = 1u << 21;
constexpr uint32_t kFuseWsHead = 256;  // workspace: ticket counter, then the descriptors

struct FuseK {
    BPred pred[BS_MAX_CONJ];
    int32_t npred;
    LookK look;            // projection column and outputs
    const int32_t *val1;   // projection PP-VBS: values of the one-byte codes
    uint32_t *bits;        // optional: the result bit vector
    uint32_t n_units;
    uint32_t *ticket;      // workspace, zeroed per call
    uint64_t *desc;        // workspace, zeroed per call: one descriptor per unit
    uint32_t *status;
};

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix of unit u (u > 0): the warp reads a window of the 128
// descriptors before `pos` (entry e = 32k + lane is unit pos-1-e, four loads
// in flight per lane); the nearest one holding an inclusive prefix ends the
// walk, and the counts of the units after it are added; a window of counts
// only moves the walk 128 units back. A window with an unpublished descriptor
// before that point is read again, at most kLookbackPolls times.
__device__ uint64_t lookback(const FuseK &f, uint32_t u, uint32_t lane) {
    constexpr int kW = 4;  // descriptors per lane and window
    uint64_t excl = 0;
    int64_t pos = u;
    uint32_t polls = 0;
    while (pos > 0) {
        uint64_t d[kW];
#pragma unroll
        for (int k = 0; k < kW; k++) {
            const int64_t idx = pos - 1 - (int64_t)(k * 32 + lane);
            d[k] = idx >= 0 ? ld_relaxed(f.desc + idx) : kDescInc;  // before unit 0: prefix 0
        }
        int kk = kW;         // the first group of 32 entries holding an inclusive prefix
        uint32_t upto = 31;  // and the lane of the nearest one in it
        bool blocked = false;
#pragma unroll
        for (int k = 0; k < kW; k++) {
            const uint32_t state = (uint32_t)(d[k] >> 62);
            const uint32_t inc = __ballot_sync(kFull, state == 2u);
            const uint32_t empty = __ballot_sync(kFull, state == 0u);
            if (kk == kW) {
                const uint32_t up = inc ? (uint32_t)(__ffs(inc) - 1) : 31u;
                const uint32_t need = up == 31u ? kFull : ((2u << up) - 1u);
                blocked |= (empty & need) != 0u;
                if (inc) {
                    kk = k;
                    upto = up;
                }
            }
        }
        if (blocked) {
            if (++polls >= kLookbackPolls) {
                if (lane == 0) atomicOr(f.status, kStatusTimeout);
                return excl;
            }
            __nanosleep(64);
            continue;
        }
        uint64_t v = 0;
#pragma unroll
        for (int k = 0; k < kW; k++)
            if (k < kk || (k == kk && lane <= upto)) v += d[k] & kDescVal;
        excl += warp_sum64(v);
        if (kk < kW) break;
        pos -= 32 * kW;
    }
    return excl;
}

// Step 2 for unit u of `tot` selected rows (its count already published):
// its first output slot, published as its inclusive prefix. The last unit's
// warp also writes the total count.
__device__ __forceinline__ uint64_t unit_offset(const FuseK &f, uint32_t u, uint32_t tot, uint32_t lane) {
    uint64_t excl = 0;
    if (u > 0) {
        excl = lookback(f, u, lane);
        if (lane == 0) st_relaxed(f.desc + u, kDescInc | (excl + tot));
    }
    if (u == f.n_units - 1 && lane == 0 && f.look.count) *f.look.count = excl + tot;
    return excl;
}

template <int KMAX>
__device__ __forceinline__ void gather_any_tile(const LookK &a, uint64_t t, uint32_t sel, uint32_t tc, uint64_t base,
                                                WarpSmemT<KMAX> &sm, const int32_t *val1, uint32_t lane) {
    switch (a.layout) {
    case BS_PPVBS: gather_one_tile<BS_PPVBS, KMAX>(a, t, sel, tc, base, sm, val1, lane); break;
    case BS_BYTESLICE: gather_one_tile<BS_BYTESLICE, KMAX>(a, t, sel, tc, base, sm, val1, lane); break;
    default: gather_one_tile<BS_BITPACKED, KMAX>(a, t, sel, tc, base, sm, val1, lane); break;
    }
}

// Shared memory: per warp the ring's two slices, sharing their bytes with the
// gather's scratch; after the warps, the values of the 256 one-byte PP-VBS
// codes.
template <int KMAX>
struct FuseSmem {
    static constexpr size_t warp = sizeof(WarpSmemT<KMAX>) > 2 * kTileRows ? sizeof(WarpSmemT<KMAX>) : 2 * kTileRows;
    static constexpr size_t total = kFuseWarps * warp + 256 * sizeof(int32_t);
};

// SPEC >= 0: one PP-VBS predicate with one literal on the projection column
// itself, SPEC = (HI0 << 2) | (HI1 << 1) | NEED_EQ as in the scan kernel;
// SPEC < 0: any predicates and projection (run-time dispatch).
template <int KMAX, int SPEC>
__global__ void __launch_bounds__(kFuseThreads, SPEC >= 0 ? 5 : 4) fused_kernel(const FuseK f) {
    extern __shared__ __align__(16) unsigned char fsm[];
    constexpr bool kSpec = SPEC >= 0;
    constexpr bool HI0 = (SPEC & 4) != 0, HI1 = (SPEC & 2) != 0, NEED_EQ = (SPEC & 1) != 0;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint8_t *ring = fsm + warp * FuseSmem<KMAX>::warp;
    WarpSmemT<KMAX> &sm = *reinterpret_cast<WarpSmemT<KMAX> *>(ring);
    int32_t *val1 = reinterpret_cast<int32_t *>(fsm + kFuseWarps * FuseSmem<KMAX>::warp);
    const LookK &L = f.look;
    if (L.layout == BS_PPVBS && threadIdx.x < 256) val1[threadIdx.x] = __ldg(f.val1 + threadIdx.x);
    __syncthreads();

    const BPred &P0 = f.pred[0];
    const bool ring_on = kSpec || P0.plan.kind == ScanPlan::kDense;
    const uint8_t *slice = P0.a.dense;
    const uint32_t rbase = (uint32_t)__cvta_generic_to_shared(ring);
    const uint32_t n_tiles = L.n_tiles;
    const uint64_t n = L.n;
    uint64_t pol_keep;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_keep));
    auto issue = [&](uint32_t t, int stage) {
        if (ring_on && t < n_tiles) {
            const uint8_t *g = slice + (uint64_t)t * kTileRows;
            const uint32_t s = rbase + (uint32_t)stage * kTileRows;
            asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s + lane * 16u),
                         "l"(g + lane * 16u), "l"(pol_keep) : "memory");
            asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s + 512u + lane * 16u),
                         "l"(g + 512u + lane * 16u), "l"(pol_keep) : "memory");
        }
        cp_async_commit();  // one group per slot, empty or not
    };
    uint32_t add0 = 0, add1 = 0;
    if (kSpec) {
        const uint32_t c0 = lit_byte(P0.a.lit[0], 1);
        add0 = thr_add(c0);
        add1 = thr_add(c0 + 1);
    }

    // 1. the predicates on the tiles of unit u: result words in sel, per-tile
    // counts in tc (warp-wide), total returned. Tiles come through the ring in
    // order: the unit's first two are in flight on entry; consuming tile i
    // issues tile i + 2 of the unit (or an empty group), so the wait is always
    // for all but the most recent group.
    auto scan_unit = [&](uint32_t u, uint32_t *sel, uint32_t *tc) -> uint32_t {
        const uint32_t t0 = u * kFuseTiles;
        uint32_t tot = 0;
#pragma unroll
        for (int i = 0; i < kFuseTiles; i++) {
            const uint32_t t = t0 + (uint32_t)i;
            sel[i] = 0;
            cp_async_wait<1>();
            if (t < n_tiles) {
                const uint64_t w = (uint64_t)t * kTileWords + lane;
                uint32_t sd = valid_mask(w * 32u, n);
                if (ring_on) {
                    const uint4 *sp = reinterpret_cast<const uint4 *>(ring + (i & 1) * kTileRows);
                    const uint4 v0 = sp[lane], v1 = sp[32 + lane];
                    const uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                    if (kSpec) sd = scan_tile<true, 1, HI0, HI1, NEED_EQ, false>(P0.a, t, lane, x, sd, add0, add1, 0u);
                    else sd = dense_pred(P0, t, lane, x, sd);
                    issue(i + 2 < kFuseTiles ? t + 2 : n_tiles, i & 1);  // slot i & 1 is free again
                } else {
                    cp_async_commit();
                    sd = pred_tile(P0, t, lane, sd);
                }
                if (!kSpec) {
                    for (int p = 1; p < f.npred; p++) {
                        if (!__any_sync(kFull, sd != 0u)) break;  // every row of the tile decided
                        sd = pred_tile(f.pred[p], t, lane, sd);
                    }
                }
                if (f.bits && w * 32u < n) st_stream(f.bits + w, sd);
                sel[i] = sd;
            } else {
                cp_async_commit();
            }
            tc[i] = warp_sum(__popc(sel[i]));
            tot += tc[i];
        }
        return tot;
    };
    auto start_unit = [&](uint32_t u) {
        if (u < f.n_units) {
            issue(u * kFuseTiles, 0);
            issue(u * kFuseTiles + 1, 1);
        }
    };
    // 2 + 3 run one unit behind 1: a unit's look-back comes after the warp has
    // scanned its next unit, when the units before it have mostly published
    // their prefixes, so it usually ends at the first window. A unit's count is
    // published right after its scan, and nothing between a unit's claim and
    // that scan waits for another warp (a gather never waits), so every
    // look-back wait is bounded by one gather and one scan of another warp.
    uint32_t cur = claim(f.ticket, lane);
    uint32_t sel_c[kFuseTiles], tc_c[kFuseTiles], tot_c = 0;
    if (cur < f.n_units) {
        start_unit(cur);
        tot_c = scan_unit(cur, sel_c, tc_c);
        if (lane == 0) st_relaxed(f.desc + cur, (cur == 0 ? kDescInc : kDescAgg) | tot_c);
    }
    uint32_t nxt = claim(f.ticket, lane);
    start_unit(nxt);
    while (cur < f.n_units) {
        uint32_t sel_n[kFuseTiles], tc_n[kFuseTiles], tot_n = 0;
        if (nxt < f.n_units) {
            tot_n = scan_unit(nxt, sel_n, tc_n);
            if (lane == 0) st_relaxed(f.desc + nxt, (nxt == 0 ? kDescInc : kDescAgg) | tot_n);
        }
        uint64_t base = unit_offset(f, cur, tot_c, lane);
        const uint32_t nn = claim(f.ticket, lane);
        const uint32_t t0 = cur * kFuseTiles;
#pragma unroll
        for (int i = 0; i < kFuseTiles; i++) {
            if (tc_c[i] && base < L.out_cap) {
                if (kSpec) gather_one_tile<BS_PPVBS, KMAX>(L, t0 + i, sel_c[i], tc_c[i], base, sm, val1, lane);
                else gather_any_tile<KMAX>(L, t0 + i, sel_c[i], tc_c[i], base, sm, val1, lane);
            }
            base += tc_c[i];
        }
        __syncwarp();
        start_unit(nn);  // the ring shares the gather's shared memory: refilled after the gather
        cur = nxt;
        tot_c = tot_n;
#pragma unroll
        for (int i = 0; i < kFuseTiles; i++) {
            sel_c[i] = sel_n[i];
            tc_c[i] = tc_n[i];
        }
        nxt = nn;
    }
    cp_async_wait<0>();
}

using FuseFn = void (*)(const FuseK);

template <int KMAX>
FuseFn pick_spec(int spec) {
    switch (spec) {
    case 0: return fused_kernel<KMAX, 0>;
    case 1: return fused_kernel<KMAX, 1>;
    case 2: return fused_kernel<KMAX, 2>;
    case 3: return fused_kernel<KMAX, 3>;
    case 6: return fused_kernel<KMAX, 6>;
    case 7: return fused_kernel<KMAX, 7>;
    default: return fused_kernel<KMAX, -1>;  // (no literal byte has HI0 without HI1)
    }
}

// Kernel, dynamic shared memory and resident CTAs of a variant; the shared
// memory limit is raised once per kernel and device.
struct FusePick {
    FuseFn fn;
    size_t smem;
};

// spec >= 0 (kmax 2 or 4): the variant specialised for one literal on the
// projection column; otherwise the generic one.
FusePick pick_kernel(int kmax, int spec) {
    if (kmax == 2) return {spec >= 0 ? pick_spec<2>(spec) : fused_kernel<2, -1>, FuseSmem<2>::total};
    if (kmax == 4) return {spec >= 0 ? pick_spec<4>(spec) : fused_kernel<4, -1>, FuseSmem<4>::total};
    return {fused_kernel<8, -1>, FuseSmem<8>::total};
}

int prepare(const FusePick &k, int dev) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    std::lock_guard<std::mutex> g(mu);
    const auto key = std::make_pair((const void *)k.fn, dev);
    if (done.count(key)) return BS_OK;
    if (cudaFuncSetAttribute((const void *)k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    done.insert(key);
    return BS_OK;
}

}  // namespace

uint64_t scan_lookup_workspace_bytes(const Column &c) {
    const uint64_t units = ((uint64_t)c.n_tiles + kFuseTiles - 1) / kFuseTiles;
    return kFuseWsHead + units * 8;
}

int launch_scan_lookup(const Column *const *cols, const KPred *kp, int npred, const Column &proj, uint32_t *d_bits,
                       int32_t *d_out, uint64_t out_cap, uint64_t *d_count, void *d_ws, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BS_ERR_CUDA;
    uint32_t *status = status_word();
    if (!status) return BS_ERR_CUDA;
    if (proj.n == 0) {
        if (d_count && cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s) != cudaSuccess) return BS_ERR_CUDA;
        return BS_OK;
    }
    FuseK f{};
    f.npred = npred;
    for (int p = 0; p < npred; p++) {
        plan_scan(*cols[p], kp[p], nullptr, false, f.pred[p].a, f.pred[p].plan);
        f.pred[p].a.out = nullptr;  // the kernel stores the final words itself
        f.pred[p].a.status = status;
    }
    f.look = make_look_args(proj);
    f.look.out_vals = d_out;
    f.look.out_cap = d_out ? out_cap : 0;
    f.look.count = d_count;
    f.look.status = status;
    f.val1 = proj.d_val1;
    f.bits = d_bits;
    f.n_units = (uint32_t)((proj.n_tiles + kFuseTiles - 1) / kFuseTiles);
    f.ticket = (uint32_t *)d_ws;
    f.desc = (uint64_t *)((uint8_t *)d_ws + kFuseWsHead);
    f.status = status;
    const int kmax = kmax_for(f.look);
    // the specialised variant: one single-literal PP-VBS predicate on the
    // projection column itself
    int spec = -1;
    const ScanPlan &pl = f.pred[0].plan;
    if (npred == 1 && cols[0] == &proj && pl.kind == ScanPlan::kDense && pl.vbs && pl.nlit == 1 && kmax <= 4)
        spec = (pl.hi0 ? 4 : 0) | (pl.hi1 ? 2 : 0) | (pl.eq1 ? 1 : 0);
    if (spec == 4 || spec == 5) spec = -1;
    const FusePick k = pick_kernel(kmax, spec);
    int rc = prepare(k, dev);
    if (rc) return rc;
    if (cudaMemsetAsync(d_ws, 0, scan_lookup_workspace_bytes(proj), s) != cudaSuccess) return BS_ERR_CUDA;
    const uint64_t resident = (uint64_t)sm_count(dev) * blocks_per_sm((const void *)k.fn, kFuseThreads, k.smem, dev);
    const uint64_t want = ((uint64_t)f.n_units + kFuseWarps - 1) / kFuseWarps;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, resident));
    k.fn<<<grid, kFuseThreads, k.smem, s>>>(f);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

}  // namespace bs
