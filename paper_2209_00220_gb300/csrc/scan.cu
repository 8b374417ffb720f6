// Scan kernels for sm_103a (single query): the dense kernel for PP-VBS and
// ByteSlice, the Bit-Packed kernel and the constant-result fill kernel, with
// their launch-time variant selection. The device-side building blocks and
// their description are in scan_dev.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "scan_dev.cuh"

namespace bs {
namespace {

// PF: the tile's M_2 words travel in the ring with its BS_1 bytes (chosen on
// the host when most tiles are expected to hold rows pending after byte 1).
template <bool VBS, int NLIT, bool HI0, bool HI1, bool NEED_EQ, bool PF, int HI23>
__global__ void __launch_bounds__(kScanThreads, 8) scan_dense_kernel(const ScanK a) {
    constexpr int kSlot = kTileRows + (PF ? kTileWords * 4 : 0);
    static_assert(kSlot % 16 == 0, "ring slots receive 16-byte cp.async copies");
    // two slots per warp: the tile being resolved and the next one in flight
    // (three measured 2-3 % slower: eight CTAs of three-slot rings take 221 KB
    // of the SM's shared memory, of two-slot rings 147 KB, and the rest serves
    // as L1 for the deeper bytes)
    __shared__ __align__(16) uint8_t ring[kScanWarps][2][kSlot];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t c0 = lit_byte(a.lit[0], 1);
    const uint32_t add0 = thr_add(c0), add1 = thr_add(c0 + 1);
    const uint32_t c2 = lit_byte(a.lit[1], 1);
    const uint32_t add2 = thr_add(c2), add3 = thr_add(c2 + 1);

    if (a.seed) {
        // seeded: lanes whose seed word is zero read nothing
        for (uint32_t t = gw; t < a.n_tiles; t += nw) {
            const uint64_t w = (uint64_t)t * kTileWords + lane;
            uint32_t sd = valid_mask(w * 32u, a.n);
            if (sd) sd &= __ldg(a.seed + w);
            uint32_t x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (sd) load_lane32(a.dense + (uint64_t)t * kTileRows, lane, x);
            scan_tile<VBS, NLIT, HI0, HI1, NEED_EQ, false, HI23>(a, t, lane, x, sd, add0, add1, 0u, add2, add3);
        }
        return;
    }
    // unseeded: 2-slot cp.async ring, the warp's next tile in flight while one is resolved
    uint8_t *my = &ring[warp][0][0];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(my);
    auto issue = [&](uint32_t t, int stage) {
        if (t < a.n_tiles) {
            const uint8_t *g = a.dense + (uint64_t)t * kTileRows;
            const uint32_t s = sbase + (uint32_t)stage * kSlot;
            cp_async16(s + lane * 16u, g + lane * 16u);
            cp_async16(s + 512u + lane * 16u, g + 512u + lane * 16u);
            if (PF) cp_async4(s + kTileRows + lane * 4u, a.mask[2] + (uint64_t)t * kTileWords + lane);
        }
        cp_async_commit();  // empty groups keep the group count uniform
    };
    issue(gw, 0);
    int stage = 0;
    const uint32_t full_tiles = (uint32_t)(a.n / kTileRows);
    for (uint32_t t = gw; t < a.n_tiles; t += nw) {
        issue(t + nw, stage ^ 1);
        cp_async_wait<1>();
        const uint8_t *slot = my + stage * kSlot;
        const uint4 *sp = reinterpret_cast<const uint4 *>(slot);
        const uint4 v0 = sp[lane], v1 = sp[32 + lane];
        const uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        const uint32_t m2 = PF ? reinterpret_cast<const uint32_t *>(slot + kTileRows)[lane] : 0u;
        const uint32_t sd = t < full_tiles ? kFull : valid_mask(((uint64_t)t * kTileWords + lane) * 32u, a.n);
        scan_tile<VBS, NLIT, HI0, HI1, NEED_EQ, PF, HI23>(a, t, lane, x, sd, add0, add1, m2, add2, add3);
        stage ^= 1;
    }
    cp_async_wait<0>();
}

template <int KB>
__global__ void __launch_bounds__(kScanThreads) scan_packed_kernel(const ScanK a) {
    constexpr int kPair = KB <= 16 ? 2 : 1;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t lo = (uint32_t)a.lo, span = (uint32_t)(a.hi - a.lo);
    const bool empty = a.lo > a.hi;
    for (uint32_t t0 = gw * kPair; t0 < a.n_tiles; t0 += nw * kPair) {
        uint32_t w[kPair][KB];
        uint32_t sd[kPair];
#pragma unroll
        for (int u = 0; u < kPair; u++) {
            const uint32_t t = t0 + (uint32_t)u;
            const uint64_t wd = (uint64_t)t * kTileWords + lane;
            sd[u] = t < a.n_tiles ? valid_mask(wd * 32u, a.n) : 0u;
            if (a.seed && sd[u]) sd[u] &= __ldg(a.seed + wd);
            if (sd[u]) load_packed<KB>(a.packed + ((uint64_t)t * kTileWords + lane) * KB, w[u]);
        }
#pragma unroll
        for (int u = 0; u < kPair; u++) {
            const uint32_t t = t0 + (uint32_t)u;
            const uint64_t wd = (uint64_t)t * kTileWords + lane;
            uint32_t res = 0;
            if (sd[u] && !empty) res = packed_bits<KB>(w[u], lo, span);
            if (a.invert) res = ~res;
            res &= sd[u];
            if (t < a.n_tiles && wd * 32u < a.n) st_stream(a.out + wd, res);
        }
    }
}

// Constant predicates (literal outside the dictionary): every valid seeded row,
// or none.
__global__ void scan_fill_kernel(const ScanK a) {
    const uint64_t nwords = (a.n + 31) / 32;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nwords;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        if (a.fill_all) {
            v = valid_mask(w * 32u, a.n);
            if (a.seed) v &= a.seed[w];
        }
        a.out[w] = v;
    }
}

// ---------------------------------------------------------------- host side
using KernelFn = void (*)(const ScanK);

int grid_for(KernelFn kernel, uint32_t n_tiles, int device) {
    const int per_sm = blocks_per_sm((const void *)kernel, kScanThreads, 0, device);
    const uint64_t want = ((uint64_t)n_tiles + kScanWarps - 1) / kScanWarps;
    const uint64_t cap = (uint64_t)sm_count(device) * (uint64_t)per_sm;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, cap));
}

template <bool VBS, int NLIT, bool PF>
KernelFn pick_dense(bool hi0, bool hi1, bool need_eq) {
    const int sel = (hi0 ? 4 : 0) | (hi1 ? 2 : 0) | (need_eq ? 1 : 0);
    switch (sel) {
    case 0: return scan_dense_kernel<VBS, NLIT, false, false, false, PF, -1>;
    case 1: return scan_dense_kernel<VBS, NLIT, false, false, true, PF, -1>;
    case 2: return scan_dense_kernel<VBS, NLIT, false, true, false, PF, -1>;
    case 3: return scan_dense_kernel<VBS, NLIT, false, true, true, PF, -1>;
    case 4: return scan_dense_kernel<VBS, NLIT, true, false, false, PF, -1>;
    case 5: return scan_dense_kernel<VBS, NLIT, true, false, true, PF, -1>;
    case 6: return scan_dense_kernel<VBS, NLIT, true, true, false, PF, -1>;
    default: return scan_dense_kernel<VBS, NLIT, true, true, true, PF, -1>;
    }
}

// BETWEEN: both literals' first-byte thresholds as compile-time constants,
// and whether the lower literal's byte-1 EQ mask is formed at all (EQ). The
// high bit of c + 1 is set whenever that of c is, so (true, false) never
// occurs for either pair.
template <bool VBS, bool PF, bool HI0, bool HI1, bool EQ>
KernelFn pick_between_hi(bool hi2, bool hi3) {
    if (hi2) return scan_dense_kernel<VBS, 2, HI0, HI1, EQ, PF, 3>;
    return hi3 ? scan_dense_kernel<VBS, 2, HI0, HI1, EQ, PF, 1> : scan_dense_kernel<VBS, 2, HI0, HI1, EQ, PF, 0>;
}

template <bool VBS, bool PF, bool EQ>
KernelFn pick_between_eq(bool hi0, bool hi1, bool hi2, bool hi3) {
    if (hi0) return pick_between_hi<VBS, PF, true, true, EQ>(hi2, hi3);
    return hi1 ? pick_between_hi<VBS, PF, false, true, EQ>(hi2, hi3)
               : pick_between_hi<VBS, PF, false, false, EQ>(hi2, hi3);
}

template <bool VBS, bool PF>
KernelFn pick_between(bool hi0, bool hi1, bool eq1, bool hi2, bool hi3) {
    return eq1 ? pick_between_eq<VBS, PF, true>(hi0, hi1, hi2, hi3) : pick_between_eq<VBS, PF, false>(hi0, hi1, hi2, hi3);
}

template <int... Ks>
KernelFn packed_table(int k, std::integer_sequence<int, Ks...>) {
    KernelFn fns[] = {scan_packed_kernel<Ks + 1>...};
    return (k >= 1 && k <= 32) ? fns[k - 1] : nullptr;
}

KernelFn packed_kernel_for(int k) { return packed_table(k, std::make_integer_sequence<int, 32>{}); }


}  // namespace

int launch_scan(const Column &c, const KPred &p, const uint32_t *d_seed, uint32_t *d_out, cudaStream_t s,
                uint32_t *status) {
    if (c.n == 0) return BS_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BS_ERR_CUDA;
    ScanK a{};
    ScanPlan plan{};
    plan_scan(c, p, d_seed, true, a, plan);
    a.out = d_out;
    a.status = status ? status : status_word();
    if (!a.status) return BS_ERR_CUDA;
    if (plan.kind == ScanPlan::kFill) {
        const uint64_t nwords = (c.n + 31) / 32;
        const int grid = (int)std::min<uint64_t>((nwords + 255) / 256, (uint64_t)sm_count(dev) * 8);
        scan_fill_kernel<<<std::max(grid, 1), 256, 0, s>>>(a);
        return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
    }
    if (plan.kind == ScanPlan::kPacked) {
        KernelFn fn = packed_kernel_for(c.k);
        if (!fn) return BS_ERR_INVALID_ARG;
        fn<<<grid_for(fn, (c.n_tiles + 1) / 2, dev), kScanThreads, 0, s>>>(a);
        return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
    }
    KernelFn fn;
    if (plan.vbs) {
        if (plan.pf)
            fn = plan.nlit == 2 ? pick_between<true, true>(plan.hi0, plan.hi1, plan.eq1, plan.hi2, plan.hi3)
                                : pick_dense<true, 1, true>(plan.hi0, plan.hi1, plan.eq1);
        else
            fn = plan.nlit == 2 ? pick_between<true, false>(plan.hi0, plan.hi1, plan.eq1, plan.hi2, plan.hi3)
                                : pick_dense<true, 1, false>(plan.hi0, plan.hi1, plan.eq1);
    } else {
        fn = plan.nlit == 2 ? pick_between<false, false>(plan.hi0, plan.hi1, plan.eq1, plan.hi2, plan.hi3)
                            : pick_dense<false, 1, false>(plan.hi0, plan.hi1, plan.eq1);
    }
    fn<<<grid_for(fn, c.n_tiles, dev), kScanThreads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

}  // namespace bs
