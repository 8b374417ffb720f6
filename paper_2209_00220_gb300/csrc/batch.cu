// Batched form: many scan + lookup requests in one persistent, cooperative,
// CUDA-graph-captured launch, and the serving loop built on it (the paper has
// no counterpart for either).
//
// One kernel, three phases separated by grid-wide barriers (cooperative
// launch, so every CTA is resident; the barrier is an arrival counter polled
// with acquire loads and an iteration cap that records a timeout instead of
// waiting forever):
//   1. scan   -- warps claim (request, chunk of 16 tiles) units from an atomic
//               counter, so columns of uneven length share the GPU evenly. Per
//               tile, the request's predicates run in order with the running
//               result as the seed held in registers (the pipelined bit vectors
//               of Section 3.3.1 without a round trip through memory; a tile
//               whose rows are all decided stops early). The first predicate's
//               dense slice streams through a 3-stage cp.async ring in the
//               warp's shared memory. The final bit vector word is stored, the
//               chunk's selected rows are counted and added to the total of its
//               segment (512 chunks).
//   2. offsets -- one warp per (request, segment): the earlier segments'
//               totals give the segment's base, a warp scan of its 512 chunk
//               counts the chunks' exclusive offsets; the last segment's warp
//               writes the request's selected-row count.
//   3. gather -- warps claim units again and run the lookup's chunk gather
//               (lookup_dev.cuh) at the chunk's offset.
// The host encodes every literal, uploads the request descriptors, sizes the
// scratch, picks the launch shape (threads per CTA, CTAs per SM -- timed on the
// batch itself when autotuning, with the winner cached per batch signature in a
// JSON-lines file) and captures the counter reset plus the kernel in a graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lookup_dev.cuh"
#include "pred_dev.cuh"
#include "scan_dev.cuh"
#include "wait_dev.cuh"

namespace bs {
namespace {

constexpr int kMaxPreds = BS_MAX_CONJ;
constexpr uint32_t kSegChunks = 512;  // chunks per offset segment: 16 per lane of a warp

struct BReq {
    BPred pred[kMaxPreds];
    int32_t npred;
    int32_t kmax;
    LookK look;             // projection column view + bits, outputs
    const int32_t *val1;    // projection is PP-VBS: one-byte code values
    uint32_t *bits;         // result bit vector (ceil(n/32) words)
    uint32_t *chunk_cnt;    // per chunk: selected rows (phase 1)
    uint64_t *chunk_off;    // per chunk: first output slot (phase 2)
    uint64_t *seg_tot;      // per segment of kSegChunks chunks: selected rows (zeroed before launch)
    uint32_t n_chunks;
    uint32_t n_segs;        // max(1, ceil(n_chunks / kSegChunks))
    uint32_t unit0;         // first chunk unit of this request
    uint32_t seg0;          // first segment of this request
};

struct BatchK {
    const BReq *reqs;
    const uint32_t *unit0;  // nreq + 1 entries: prefix of chunk counts
    const uint32_t *seg0;   // nreq + 1 entries: prefix of segment counts
    int32_t nreq;
    uint32_t total_units;
    uint32_t total_segs;
    uint32_t unit_chunks;   // chunks a warp takes per claim (1, 2 or 4; rows per claim = 16384 x this)
    uint32_t total_claims;  // ceil(total_units / unit_chunks)
    uint32_t *ctr;          // [0] scan units claimed, [1] gather units claimed, [2] barrier arrivals
    uint32_t *status;
};

union WarpSmemAny {
    WarpSmemT<2> k2;
    WarpSmemT<4> k4;
    WarpSmemT<8> k8;
    uint8_t ring[kStagesMax][kTileRows];  // phase 1: the first predicate's slice tiles in flight
};

// Largest r with prefix[r] <= u (prefix: nreq + 1 non-decreasing entries).
__device__ __forceinline__ uint32_t find_request(const uint32_t *prefix, int nreq, uint32_t u) {
    int lo = 0, hi = nreq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    return (uint32_t)lo;
}

template <int KMAX>
__device__ __forceinline__ void gather_any(const LookK &a, uint32_t c, uint64_t base, WarpSmemT<KMAX> &sm,
                                           const int32_t *val1, uint32_t lane) {
    switch (a.layout) {
    case BS_PPVBS: gather_chunk<BS_PPVBS, false, KMAX, false>(a, c, base, sm, val1, lane); break;
    case BS_BYTESLICE: gather_chunk<BS_BYTESLICE, false, KMAX, false>(a, c, base, sm, val1, lane); break;
    default: gather_chunk<BS_BITPACKED, false, KMAX, false>(a, c, base, sm, val1, lane); break;
    }
}

// Grid-wide barrier number `round` (1, 2, ...): every CTA adds one arrival and
// waits until all gridDim.x * round arrivals are in.
__device__ void grid_barrier(const BatchK &b, uint32_t round) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(b.ctr + 2, 1u);
        bounded_wait_geq(b.ctr + 2, gridDim.x * round, 1u << 24, b.status);
        __threadfence();
    }
    __syncthreads();
}

// 512-thread CTAs at two per SM at least: at most 64 registers a thread, so a
// 256-thread shape keeps 32 warps resident per SM. STAGES: slots of the
// phase-1 ring (tiles of the first predicate's slice in flight per warp).
template <int STAGES>
__global__ void __launch_bounds__(512, 2) batch_kernel(const BatchK b) {
    static_assert(STAGES >= 2 && STAGES <= kStagesMax, "ring slots");
    extern __shared__ __align__(16) unsigned char batch_smem[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    WarpSmemAny &sm = reinterpret_cast<WarpSmemAny *>(batch_smem)[warp];

    // ---- phase 1: scan every request's chunks, unit_chunks of them per claim
    uint8_t *ring = &sm.ring[0][0];
    const uint32_t rbase = (uint32_t)__cvta_generic_to_shared(ring);
    for (;;) {
        const uint32_t cl = claim(b.ctr + 0, lane);
        if (cl >= b.total_claims) break;
        for (uint32_t u = cl * b.unit_chunks; u < min((cl + 1) * b.unit_chunks, b.total_units); u++) {
        const uint32_t r = find_request(b.unit0, b.nreq, u);
        const BReq &R = b.reqs[r];
        const uint32_t c = u - R.unit0;
        const uint64_t n = R.look.n;
        const BPred &P0 = R.pred[0];
        const bool staged = P0.plan.kind == ScanPlan::kDense;
        const uint32_t t0 = c * (uint32_t)kChunkTiles;
        const uint32_t t1 = min(t0 + (uint32_t)kChunkTiles, R.look.n_tiles);
        // every dense slice holds whole tiles, so whole-tile copies stay in bounds;
        // each lane copies, and later reads, only its own 32 bytes of a tile
        auto issue = [&](uint32_t t, int stage) {
            if (t < t1) {
                const uint8_t *g = P0.a.dense + (uint64_t)t * kTileRows;
                const uint32_t sa = rbase + (uint32_t)stage * kTileRows;
                cp_async16(sa + lane * 16u, g + lane * 16u);
                cp_async16(sa + 512u + lane * 16u, g + 512u + lane * 16u);
            }
            cp_async_commit();
        };
        if (staged) {
#pragma unroll
            for (int s = 0; s < STAGES - 1; s++) issue(t0 + (uint32_t)s, s);
        }
        int stage = 0;
        uint32_t cnt = 0;
        for (uint32_t t = t0; t < t1; t++) {
            const uint64_t w = (uint64_t)t * kTileWords + lane;
            uint32_t sd = valid_mask(w * 32u, n);
            if (staged) {
                // the slot of tile t - 1 (read in the previous step) takes tile t + STAGES - 1
                issue(t + STAGES - 1, (stage + STAGES - 1) % STAGES);
                cp_async_wait<STAGES - 1>();
                const uint4 *sp = reinterpret_cast<const uint4 *>(ring + stage * kTileRows);
                const uint4 v0 = sp[lane], v1 = sp[32 + lane];
                const uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                sd = dense_pred(P0, t, lane, x, sd);
                stage = stage + 1 == STAGES ? 0 : stage + 1;
            } else {
                sd = pred_tile(P0, t, lane, sd);
            }
            for (int p = 1; p < R.npred; p++) {
                if (!__any_sync(kFull, sd != 0u)) break;  // every row of the tile decided
                sd = pred_tile(R.pred[p], t, lane, sd);
            }
            if (w * 32u < n) R.bits[w] = sd;
            cnt += __popc(sd);
        }
        if (staged) cp_async_wait<0>();
        cnt = warp_sum(cnt);
        if (lane == 0) {
            R.chunk_cnt[c] = cnt;
            if (cnt) atomicAdd((unsigned long long *)(R.seg_tot + c / kSegChunks), (unsigned long long)cnt);
        }
        }
    }
    grid_barrier(b, 1);

    // ---- phase 2: chunk offsets, one warp per (request, segment)
    {
        const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
        for (uint32_t u = gw; u < b.total_segs; u += nw) {
            const uint32_t r = find_request(b.seg0, b.nreq, u);
            const BReq &R = b.reqs[r];
            const uint32_t sg = u - R.seg0;
            uint64_t base = 0;
            for (uint32_t i = lane; i < sg; i += 32) base += __ldcg(R.seg_tot + i);
            base = warp_sum64(base);
            const uint32_t c0 = sg * kSegChunks + lane * (kSegChunks / 32);
            uint32_t v[kSegChunks / 32];
            uint64_t tot = 0;
#pragma unroll
            for (int i = 0; i < (int)(kSegChunks / 32); i++) {
                v[i] = c0 + i < R.n_chunks ? __ldcg(R.chunk_cnt + c0 + i) : 0u;
                tot += v[i];
            }
            uint64_t incl = tot;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint64_t o = __shfl_up_sync(kFull, incl, d);
                if (lane >= (uint32_t)d) incl += o;
            }
            uint64_t off = base + incl - tot;
#pragma unroll
            for (int i = 0; i < (int)(kSegChunks / 32); i++) {
                if (c0 + i < R.n_chunks) R.chunk_off[c0 + i] = off;
                off += v[i];
            }
            if (sg == R.n_segs - 1 && lane == 31 && R.look.count) *R.look.count = base + incl;
        }
    }
    grid_barrier(b, 2);

    // ---- phase 3: gather every request's chunks, unit_chunks of them per claim
    for (;;) {
        const uint32_t cl = claim(b.ctr + 1, lane);
        if (cl >= b.total_claims) break;
        for (uint32_t u = cl * b.unit_chunks; u < min((cl + 1) * b.unit_chunks, b.total_units); u++) {
            const uint32_t r = find_request(b.unit0, b.nreq, u);
            const BReq &R = b.reqs[r];
            const uint32_t c = u - R.unit0;
            const uint64_t base = __ldcg(R.chunk_off + c);
            if (base >= R.look.out_cap) continue;
            if (R.kmax == 2) gather_any<2>(R.look, c, base, sm.k2, R.val1, lane);
            else if (R.kmax == 4) gather_any<4>(R.look, c, base, sm.k4, R.val1, lane);
            else gather_any<8>(R.look, c, base, sm.k8, R.val1, lane);
        }
    }
}

using BatchFn = void (*)(const BatchK);

BatchFn batch_fn(int stages) {
    return stages == 2 ? batch_kernel<2> : (stages == 4 ? batch_kernel<4> : batch_kernel<3>);
}

// ------------------------------------------------------------ request plan
// Requests whose columns have at least this many tiles (2^28 rows) run as the
// single-query kernels (specialised per predicate, as the plain calls) ahead
// of the persistent kernel, which takes the others: one persistent launch pays
// off for many short and medium columns, while a column this long keeps the
// GPU busy alone and runs faster through the specialised kernels.
constexpr uint32_t kPlainTiles = 262144;

// A request run by the single-query kernels.
struct PlainReq {
    const Column *col[kMaxPreds];
    KPred kp[kMaxPreds];
    int npred;
    const Column *proj;
    int32_t *out;
    uint64_t cap;
    uint64_t *count;
    uint32_t *bits;  // scratch: result bit vector
    void *ws;        // scratch: lookup workspace
    uint32_t *status;  // device word the kernels report bounds / timeout flags into
};

// Validates request q and fills R's predicate and lookup fields and P
// (everything but the scratch pointers). device: -1 on entry for the first
// request.
int plan_request(const bs_request &q, BReq &R, PlainReq &P, int &device, int n_layout[3]) {
    if (q.npreds < 1 || q.npreds > kMaxPreds || !q.preds[0].col) return BS_ERR_INVALID_ARG;
    const bs_column *proj = q.proj ? q.proj : q.preds[0].col;
    const Column &pc = proj->c;
    if (pc.raw || !pc.d_arena) return BS_ERR_UNSUPPORTED;
    if (q.out_cap && !q.d_out) return BS_ERR_INVALID_ARG;
    if (device < 0) device = pc.device;
    if (pc.device != device) return BS_ERR_INVALID_ARG;
    R = BReq{};
    P = PlainReq{};
    R.npred = q.npreds;
    P.npred = q.npreds;
    for (int p = 0; p < q.npreds; p++) {
        const bs_column *col = q.preds[p].col;
        if (!col || col->c.n != pc.n || col->c.device != device) return BS_ERR_INVALID_ARG;
        if (col->c.raw || !col->c.d_arena) return BS_ERR_UNSUPPORTED;
        if (q.preds[p].op < BS_LT || q.preds[p].op > BS_BETWEEN) return BS_ERR_INVALID_ARG;
        const int rc = rewrite_literal(col->c, q.preds[p].op, q.preds[p].lit, q.preds[p].lit2, P.kp[p]);
        if (rc) return rc;
        P.col[p] = &col->c;
        plan_scan(col->c, P.kp[p], nullptr, false, R.pred[p].a, R.pred[p].plan);
        R.pred[p].a.out = nullptr;  // the batch kernel stores the final word itself
        if (n_layout) n_layout[col->c.layout]++;
    }
    R.look = make_look_args(pc);
    R.kmax = kmax_for(R.look);
    R.val1 = pc.d_val1;
    R.look.out_vals = q.d_out;
    R.look.out_cap = q.d_out ? q.out_cap : 0;
    R.look.count = q.d_count;
    R.n_chunks = R.look.n_chunks;
    R.n_segs = std::max<uint32_t>(1, (R.n_chunks + kSegChunks - 1) / kSegChunks);
    P.proj = &pc;
    P.out = q.d_out;
    P.cap = R.look.out_cap;
    P.count = q.d_count;
    return BS_OK;
}

bool runs_plain(const BReq &R) { return R.look.n_tiles >= kPlainTiles; }

// Scratch of one request: bit vector (unless supplied), per-chunk counts and
// offsets (together also the single-query lookup's workspace, which needs no
// more than one count per chunk and one offset per 8 chunks).
size_t scratch_part(uint64_t bytes) { return (std::max<uint64_t>(8, bytes) + 255) & ~(size_t)255; }

size_t request_scratch(const BReq &R, bool own_bits) {
    const uint64_t nw = (R.look.n + 31) / 32;
    return (own_bits ? scratch_part(nw * 4) : 0) + scratch_part((uint64_t)R.n_chunks * 4) +
           scratch_part((uint64_t)R.n_chunks * 8);
}

void bind_scratch(BReq &R, PlainReq &P, uint8_t *p, uint32_t *user_bits, uint32_t *status) {
    const uint64_t nw = (R.look.n + 31) / 32;
    if (user_bits) {
        R.bits = user_bits;
    } else {
        R.bits = (uint32_t *)p;
        p += scratch_part(nw * 4);
    }
    R.chunk_cnt = (uint32_t *)p;
    p += scratch_part((uint64_t)R.n_chunks * 4);
    R.chunk_off = (uint64_t *)p;
    R.look.bits = R.bits;
    R.look.status = status;
    for (int q = 0; q < R.npred; q++) R.pred[q].a.status = status;
    P.bits = R.bits;
    P.ws = R.chunk_cnt;
    P.status = status;
}

// The single-query kernels of one request: the conjunction's scans (each after
// the first seeded by, and overwriting, the running bit vector), then the lookup.
int launch_plain(const PlainReq &P, cudaStream_t s) {
    for (int p = 0; p < P.npred; p++) {
        const int rc = launch_scan(*P.col[p], P.kp[p], p ? P.bits : nullptr, P.bits, s, P.status);
        if (rc) return rc;
    }
    return launch_lookup(*P.proj, P.bits, P.out, nullptr, P.cap, P.count, P.ws, s, P.status);
}

// ------------------------------------------------------------- tuning cache
std::mutex g_tune_mu;

std::string tune_path(const bs_batch_opts &o) {
    if (o.tune_cache && *o.tune_cache) return o.tune_cache;
    const char *e = std::getenv("BS_TUNE_CACHE");
    return e ? std::string(e) : std::string();
}

// Launch shape of the persistent kernel: the candidates the tuner searches
// are threads per CTA {128, 256, 512} x CTAs per SM {1, 2, all that fit},
// then ring stages {2, 3, 4}, chunks per claim {1, 2, 4} and the early-stop
// granularity {256-row group, 1024-row tile}.
struct Shape {
    int threads = 256, bps = 0, stages = kStages, unit_chunks = 1, stop_all = 0;
};

bool tune_lookup(const std::string &path, const std::string &key, Shape &sh) {
    if (path.empty()) return false;
    std::lock_guard<std::mutex> g(g_tune_mu);
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        char k[512];
        Shape t;
        int stop_rows = 256;
        // {"key": "...", "threads": T, "blocks_per_sm": B, "stages": S, "unit_chunks": U, "stop_rows": R, ...}
        const int got = std::sscanf(line,
                                    " {\"key\": \"%511[^\"]\", \"threads\": %d, \"blocks_per_sm\": %d, \"stages\": "
                                    "%d, \"unit_chunks\": %d, \"stop_rows\": %d",
                                    k, &t.threads, &t.bps, &t.stages, &t.unit_chunks, &stop_rows);
        if (got >= 3 && key == k) {
            if (got < 6) t = Shape{t.threads, t.bps};  // an entry from before the wider search
            t.stop_all = stop_rows >= 1024 ? 1 : 0;
            sh = t;
            found = true;  // the last entry for a key wins
        }
    }
    std::fclose(f);
    return found;
}

void tune_store(const std::string &path, const std::string &key, const Shape &sh, double us) {
    if (path.empty()) return;
    std::lock_guard<std::mutex> g(g_tune_mu);
    FILE *f = std::fopen(path.c_str(), "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"threads\": %d, \"blocks_per_sm\": %d, \"stages\": %d, \"unit_chunks\": %d, "
                 "\"stop_rows\": %d, \"us\": %.2f}\n",
                 key.c_str(), sh.threads, sh.bps, sh.stages, sh.unit_chunks, sh.stop_all ? 1024 : 256, us);
    std::fclose(f);
}

size_t smem_bytes(int threads) { return (size_t)(threads / 32) * sizeof(WarpSmemAny); }

}  // namespace
}  // namespace bs

// ================================================================ host API
struct bs_batch {
    int device = 0;
    int nreq = 0;
    void *d_arena = nullptr;
    size_t zero_bytes = 0;  // counters and segment totals, cleared before every launch
    std::vector<bs::PlainReq> plain;  // requests run by the single-query kernels
    bs::BatchK k{};         // the others (k.nreq may be 0)
    std::vector<bs::BReq> hreqs;  // host copy of k.reqs (rewritten when the early-stop granularity changes)
    bs::Shape sh;           // launch shape (ctas follows from it)
    int threads = 256;
    int ctas = 0;
    bool use_graph = true;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    bool graph_ok = false;
};

namespace {

int launch_persistent(bs_batch *b, cudaStream_t s);

int launch_direct(bs_batch *b, cudaStream_t s) {
    for (const bs::PlainReq &P : b->plain) {
        const int rc = bs::launch_plain(P, s);
        if (rc) return rc;
    }
    return launch_persistent(b, s);
}

// The persistent kernel over the requests it takes (counters cleared first).
int launch_persistent(bs_batch *b, cudaStream_t s) {
    if (b->k.nreq == 0) return BS_OK;
    if (cudaMemsetAsync(b->k.ctr, 0, b->zero_bytes, s) != cudaSuccess) return BS_ERR_CUDA;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)b->ctas);
    cfg.blockDim = dim3((unsigned)b->threads);
    cfg.dynamicSmemBytes = bs::smem_bytes(b->threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, bs::batch_fn(b->sh.stages), b->k);
    return e == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

// Applies a launch shape: occupancy of the chosen kernel variant, the grid,
// the claim size, and the early-stop granularity written into the request
// descriptors (uploaded again when it changes).
int shape(bs_batch *b, const bs::Shape &sh) {
    if (sh.threads != 128 && sh.threads != 256 && sh.threads != 512) return BS_ERR_INVALID_ARG;
    if (sh.stages < 2 || sh.stages > bs::kStagesMax) return BS_ERR_INVALID_ARG;
    if (sh.unit_chunks != 1 && sh.unit_chunks != 2 && sh.unit_chunks != 4) return BS_ERR_INVALID_ARG;
    const bs::BatchFn fn = bs::batch_fn(sh.stages);
    const size_t smem = bs::smem_bytes(sh.threads);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, sh.threads, smem) != cudaSuccess || fit < 1) {
        cudaGetLastError();
        return BS_ERR_CUDA;
    }
    const int per_sm = sh.bps > 0 ? std::min(sh.bps, fit) : fit;
    if (b->k.nreq > 0 && (sh.stop_all != b->sh.stop_all || b->hreqs.empty())) {
        for (bs::BReq &R : b->hreqs)
            for (int p = 0; p < R.npred; p++) R.pred[p].a.stop_all = (uint32_t)sh.stop_all;
        if (cudaMemcpy((void *)b->k.reqs, b->hreqs.data(), sizeof(bs::BReq) * b->hreqs.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return BS_ERR_CUDA;
    }
    b->sh = sh;
    b->threads = sh.threads;
    b->ctas = per_sm * bs::sm_count(b->device);
    b->k.unit_chunks = (uint32_t)sh.unit_chunks;
    b->k.total_claims = (b->k.total_units + (uint32_t)sh.unit_chunks - 1) / (uint32_t)sh.unit_chunks;
    return BS_OK;
}

int capture(bs_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_ok = false;
    if (!b->use_graph) return BS_OK;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return BS_ERR_CUDA;
    int rc = BS_OK;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = BS_ERR_CUDA;
    if (rc == BS_OK) {
        const int lrc = launch_direct(b, s);
        const cudaError_t e = cudaStreamEndCapture(s, &b->graph);
        if (lrc != BS_OK || e != cudaSuccess) rc = BS_ERR_CUDA;
    }
    if (rc == BS_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = BS_ERR_CUDA;
    cudaStreamDestroy(s);
    if (rc != BS_OK) {
        // graph capture of the cooperative launch is not available: launch directly
        cudaGetLastError();
        if (b->graph) cudaGraphDestroy(b->graph);
        b->graph = nullptr;
        b->exec = nullptr;
        return BS_OK;
    }
    b->graph_ok = true;
    return BS_OK;
}

}  // namespace

extern "C" {

int bs_batch_create(const bs_request *reqs, int32_t nreq, const bs_batch_opts *opts, bs_batch **out) {
    using namespace bs;
    if (!out || !reqs || nreq < 1 || nreq > 65536) return BS_ERR_INVALID_ARG;
    *out = nullptr;
    bs_batch_opts o{};
    o.use_graph = 1;
    if (opts) o = *opts;
    // validate and plan on the host
    std::vector<BReq> h(nreq);
    std::vector<PlainReq> hp(nreq);
    int device = -1;
    size_t scratch = 0;
    std::vector<size_t> scratch_off(nreq, 0);
    auto take = [&](size_t bytes) {
        size_t at = (scratch + 255) & ~(size_t)255;
        scratch = at + bytes;
        return at;
    };
    uint64_t total_rows = 0;
    int n_layout[3] = {0, 0, 0};
    std::vector<int> batched;  // indexes of the requests the persistent kernel runs
    for (int r = 0; r < nreq; r++) {
        const bs_request &q = reqs[r];
        const int prc = plan_request(q, h[r], hp[r], device, n_layout);
        if (prc) return prc;
        total_rows += h[r].look.n;
        scratch_off[r] = take(request_scratch(h[r], q.d_bits == nullptr));
        if (!runs_plain(h[r])) batched.push_back(r);
    }
    const int nb = (int)batched.size();
    std::vector<uint32_t> unit0(nb + 1, 0), seg0(nb + 1, 0);
    for (int i = 0; i < nb; i++) {
        unit0[i + 1] = unit0[i] + h[batched[i]].n_chunks;
        seg0[i + 1] = seg0[i] + h[batched[i]].n_segs;
    }
    const size_t zero_bytes = 256 + (size_t)seg0[nb] * 8;  // counters, then segment totals
    const size_t o_ctr = take(zero_bytes);
    const size_t o_unit0 = take(unit0.size() * 4);
    const size_t o_seg0 = take(seg0.size() * 4);
    const size_t o_reqs = take(sizeof(BReq) * (size_t)std::max(nb, 1));
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return BS_ERR_CUDA;
    auto *b = new (std::nothrow) bs_batch;
    if (!b) return BS_ERR_OOM;
    b->device = device;
    b->nreq = nreq;
    b->zero_bytes = zero_bytes;
    b->use_graph = o.use_graph != 0;
    int rc = BS_OK;
    if (cudaMalloc(&b->d_arena, scratch) != cudaSuccess) {
        cudaGetLastError();
        rc = BS_ERR_OOM;
    }
    uint8_t *base = (uint8_t *)b->d_arena;
    std::vector<BReq> hb(std::max(nb, 1));
    if (rc == BS_OK) {
        uint32_t *status = status_word();
        if (!status) rc = BS_ERR_CUDA;
        for (int r = 0; r < nreq && rc == BS_OK; r++) {
            bind_scratch(h[r], hp[r], base + scratch_off[r], reqs[r].d_bits, status);
            if (runs_plain(h[r])) b->plain.push_back(hp[r]);
        }
        for (int i = 0; i < nb; i++) {
            hb[i] = h[batched[i]];
            hb[i].unit0 = unit0[i];
            hb[i].seg0 = seg0[i];
            hb[i].seg_tot = (uint64_t *)(base + o_ctr + 256) + seg0[i];
        }
        b->k.reqs = (const BReq *)(base + o_reqs);
        b->k.unit0 = (const uint32_t *)(base + o_unit0);
        b->k.seg0 = (const uint32_t *)(base + o_seg0);
        b->k.nreq = nb;
        b->k.total_units = unit0[nb];
        b->k.total_segs = seg0[nb];
        b->k.ctr = (uint32_t *)(base + o_ctr);
        b->k.status = status;
        if (rc == BS_OK && nb > 0 &&
            (cudaMemcpy(base + o_reqs, hb.data(), sizeof(BReq) * (size_t)nb, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(base + o_unit0, unit0.data(), unit0.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(base + o_seg0, seg0.data(), seg0.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess))
            rc = BS_ERR_CUDA;
    }
    // launch shape: explicit, cached, autotuned or the default
    Shape sh;
    if (o.threads > 0) sh.threads = o.threads;
    sh.bps = o.blocks_per_sm;
    if (o.stages > 0) sh.stages = o.stages;
    if (o.unit_chunks > 0) sh.unit_chunks = o.unit_chunks;
    if (o.stop_rows > 0) sh.stop_all = o.stop_rows >= 1024 ? 1 : 0;
    if (rc == BS_OK) {
        b->hreqs.assign(hb.begin(), hb.begin() + nb);
        cudaDeviceProp prop{};
        cudaGetDeviceProperties(&prop, device);
        char key[384];
        std::snprintf(key, sizeof key, "%s|nreq=%d|plain=%d|rows=2^%d|vbs=%d,bsl=%d,bp=%d", prop.name, nreq,
                      (int)b->plain.size(), total_rows ? 63 - __builtin_clzll(total_rows) : 0, n_layout[BS_PPVBS],
                      n_layout[BS_BYTESLICE], n_layout[BS_BITPACKED]);
        const std::string path = tune_path(o);
        const bool explicit_shape = o.threads > 0 || o.stages > 0 || o.unit_chunks > 0 || o.stop_rows > 0;
        if (!explicit_shape && !o.autotune) tune_lookup(path, key, sh);
        if (o.autotune && nb > 0) {
            // coordinate search on the batch itself: the CTA shape first, then
            // each of the ring stages, chunks per claim and early-stop
            // granularity around the best so far (the persistent kernel alone
            // is timed: the single-query kernels do not depend on the shape)
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            auto time_shape = [&](const Shape &c) -> double {
                if (shape(b, c) != BS_OK) return 1e30;
                if (launch_persistent(b, nullptr) != BS_OK) {
                    cudaGetLastError();
                    return 1e30;
                }
                cudaEventRecord(e0, nullptr);
                for (int rep = 0; rep < 3; rep++) launch_persistent(b, nullptr);
                cudaEventRecord(e1, nullptr);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = BS_ERR_CUDA;
                    return 1e30;
                }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                return ms * 1000.0 / 3;
            };
            Shape best_sh = sh;
            double best = 1e30;
            auto consider = [&](const Shape &c) {
                if (rc != BS_OK) return;
                const double us = time_shape(c);
                if (us < best) {
                    best = us;
                    best_sh = c;
                }
            };
            for (int t : {128, 256, 512})
                for (int bp : {1, 2, 0}) consider(Shape{t, bp, kStages, 1, 0});
            for (int st : {2, 4}) {
                Shape c = best_sh;
                c.stages = st;
                consider(c);
            }
            for (int uc : {2, 4}) {
                Shape c = best_sh;
                c.unit_chunks = uc;
                consider(c);
            }
            {
                Shape c = best_sh;
                c.stop_all = 1;
                consider(c);
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            sh = best_sh;
            if (rc == BS_OK) tune_store(path, key, sh, best);
        }
        if (rc == BS_OK) rc = shape(b, sh);
        if (rc == BS_OK) rc = capture(b);
    }
    cudaSetDevice(prev);
    if (rc != BS_OK) {
        bs_batch_free(b);
        return rc;
    }
    *out = b;
    return BS_OK;
}

int bs_batch_launch(bs_batch *b, void *stream) {
    if (!b) return BS_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != b->device && cudaSetDevice(b->device) != cudaSuccess) return BS_ERR_CUDA;
    int rc;
    if (b->graph_ok) rc = cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? BS_OK : BS_ERR_CUDA;
    else rc = launch_direct(b, (cudaStream_t)stream);
    if (prev != b->device) cudaSetDevice(prev);
    return rc;
}

int bs_batch_info(const bs_batch *b, int32_t *threads, int32_t *ctas, int32_t *graph) {
    if (!b) return BS_ERR_INVALID_ARG;
    if (threads) *threads = b->threads;
    if (ctas) *ctas = b->ctas;
    if (graph) *graph = b->graph_ok ? 1 : 0;
    return BS_OK;
}

int bs_batch_get_shape(const bs_batch *b, bs_batch_shape *out) {
    if (!b || !out) return BS_ERR_INVALID_ARG;
    out->threads = b->threads;
    out->blocks_per_sm = b->sh.bps;
    out->ctas = b->ctas;
    out->stages = b->sh.stages;
    out->unit_chunks = b->sh.unit_chunks;
    out->stop_rows = b->sh.stop_all ? 1024 : 256;
    out->graph = b->graph_ok ? 1 : 0;
    out->persistent_requests = b->k.nreq;
    out->single_query_requests = (int32_t)b->plain.size();
    return BS_OK;
}

void bs_batch_free(bs_batch *b) {
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_arena) cudaFree(b->d_arena);
    cudaSetDevice(prev);
    delete b;
}

}  // extern "C"

// ================================================================== server
// Dispatcher thread: completions first (events of the batches in flight),
// then admission in arrival order into every free slot, then a short spin.
namespace {

using Clock = std::chrono::steady_clock;

double us_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
}

// First-fit allocator over an offset range [0, cap) (256-byte granules).
class RangeAlloc {
  public:
    explicit RangeAlloc(size_t cap = 0) { reset(cap); }
    void reset(size_t cap) {
        free_.clear();
        if (cap) free_[0] = cap;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t &off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct QueryRec {
    bs::BReq plan;
    bs::PlainReq plain;           // the same query for the single-query kernels
    uint64_t bound = 0;           // upper bound of selected rows
    size_t out_bytes = 0, out_off = SIZE_MAX;
    size_t scratch_bytes = 0, scratch_off = SIZE_MAX;
    int state = 0;                // 0 queued, 1 running, 2 done
    int rc = 0;                   // BS_OK, or why the query failed (launch error, device check, timeout)
    uint64_t count = 0;
    Clock::time_point t_submit, t_launch, t_done;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t *d_desc = nullptr;    // BReq[max_batch] | unit0 | seg0 | ctr + segment totals | counts | status
    uint8_t *h_desc = nullptr;    // pinned mirror
    size_t desc_bytes = 0, o_unit0 = 0, o_seg0 = 0, o_ctr = 0, o_counts = 0, o_status = 0;
    std::vector<bs::PlainReq> plain;  // this batch's queries for the single-query kernels
    bool busy = false;
    std::vector<uint64_t> tickets;
};

}  // namespace

struct bs_server {
    bs_server_opts o{};
    int device = 0;
    uint8_t *d_result = nullptr, *d_scratch = nullptr;
    RangeAlloc result_alloc, scratch_alloc;
    std::vector<Slot> slots;
    int threads = 256, ctas = 1;
    uint32_t *status = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, QueryRec> recs;
    uint64_t next_ticket = 1;
    bs_server_stats stats{};
    uint64_t batched_queries = 0;
    int fail_launches = 0;        // test hook: batch launches still to fail on the host
    bool stop = false;
    std::thread th;
};

namespace {

// Launches the batch of `slot` (descriptors already in its pinned mirror).
// Launches the batch of `slot`: the single-query kernels of its long queries,
// then the persistent kernel over the others (descriptors already in the
// pinned mirror), then the read-back of all counts and the completion event.
int launch_slot(bs_server *S, Slot &sl, int nall, int nreq, uint32_t total_units, uint32_t total_segs) {
    using namespace bs;
    if (S->fail_launches > 0) {  // a launch failure faked on the host, before anything is enqueued
        S->fail_launches--;
        return BS_ERR_CUDA;
    }
    // the slot's own status word collects its kernels' bounds and timeout flags
    uint32_t *st = (uint32_t *)(sl.d_desc + sl.o_status);
    if (cudaMemsetAsync(st, 0, 8, sl.stream) != cudaSuccess) return BS_ERR_CUDA;
    for (const PlainReq &P : sl.plain) {
        const int rc = launch_plain(P, sl.stream);
        if (rc) return rc;
    }
    if (nreq > 0) {
        BatchK k{};
        k.reqs = (const BReq *)sl.d_desc;
        k.unit0 = (const uint32_t *)(sl.d_desc + sl.o_unit0);
        k.seg0 = (const uint32_t *)(sl.d_desc + sl.o_seg0);
        k.nreq = nreq;
        k.total_units = total_units;
        k.total_segs = total_segs;
        k.unit_chunks = 1;
        k.total_claims = total_units;
        k.ctr = (uint32_t *)(sl.d_desc + sl.o_ctr);
        k.status = st;
        if (cudaMemcpyAsync(sl.d_desc, sl.h_desc, sl.o_ctr, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            return BS_ERR_CUDA;
        if (cudaMemsetAsync(k.ctr, 0, 256 + (size_t)total_segs * 8, sl.stream) != cudaSuccess) return BS_ERR_CUDA;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)S->ctas);
        cfg.blockDim = dim3((unsigned)S->threads);
        cfg.dynamicSmemBytes = smem_bytes(S->threads);
        cfg.stream = sl.stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, batch_fn(kStages), k) != cudaSuccess) return BS_ERR_CUDA;
    }
    // counts and the status word in one copy (the status word follows the counts)
    if (cudaMemcpyAsync(sl.h_desc + sl.o_counts, sl.d_desc + sl.o_counts, sl.o_status + 8 - sl.o_counts,
                        cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
        return BS_ERR_CUDA;
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return BS_ERR_CUDA;
    return BS_OK;
}

void dispatcher(bs_server *S) {
    using namespace bs;
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool progress = false;
        // completions
        for (Slot &sl : S->slots) {
            if (!sl.busy || cudaEventQuery(sl.done) != cudaSuccess) continue;
            const auto now = Clock::now();
            const uint64_t *counts = (const uint64_t *)(sl.h_desc + sl.o_counts);
            // a bounds check or a bounded wait that failed in this batch's kernels
            // fails every query of the batch (their results cannot be trusted)
            const uint32_t dev_st = *(const uint32_t *)(sl.h_desc + sl.o_status);
            const int brc = (dev_st & kStatusTimeout) ? BS_ERR_TIMEOUT : (dev_st ? BS_ERR_DEVICE_CHECK : BS_OK);
            for (size_t i = 0; i < sl.tickets.size(); i++) {
                QueryRec &q = S->recs[sl.tickets[i]];
                q.count = brc == BS_OK ? counts[i] : 0;
                q.rc = brc;
                q.t_done = now;
                q.state = 2;
                S->scratch_alloc.release(q.scratch_off, q.scratch_bytes);
                q.scratch_off = SIZE_MAX;
                S->stats.completed++;
                if (brc != BS_OK) S->stats.failed++;
            }
            sl.tickets.clear();
            sl.busy = false;
            progress = true;
            S->cv_done.notify_all();
        }
        // admission and launch
        for (Slot &sl : S->slots) {
            if (sl.busy || S->queue.empty()) continue;
            const int maxb = S->o.max_batch;
            BReq *reqs = (BReq *)sl.h_desc;
            uint32_t *unit0 = (uint32_t *)(sl.h_desc + sl.o_unit0);
            uint32_t *seg0 = (uint32_t *)(sl.h_desc + sl.o_seg0);
            uint64_t *d_counts = (uint64_t *)(sl.d_desc + sl.o_counts);
            uint64_t *d_segs = (uint64_t *)(sl.d_desc + sl.o_ctr + 256);
            int nb = 0, nk = 0;  // queries in the batch, of which run by the persistent kernel
            uint32_t units = 0, segs = 0;
            sl.plain.clear();
            while (nb < maxb && !S->queue.empty()) {
                const uint64_t tk = S->queue.front();
                QueryRec &q = S->recs[tk];
                size_t ro = SIZE_MAX, so = SIZE_MAX;
                if (!S->result_alloc.alloc(q.out_bytes, ro)) break;        // wait for releases
                if (!S->scratch_alloc.alloc(q.scratch_bytes, so)) {         // wait for completions
                    S->result_alloc.release(ro, q.out_bytes);
                    break;
                }
                q.out_off = ro;
                q.scratch_off = so;
                BReq R = q.plan;
                PlainReq P = q.plain;
                R.look.out_vals = (int32_t *)(S->d_result + ro);
                R.look.out_cap = q.bound;
                R.look.count = d_counts + nb;
                bind_scratch(R, P, S->d_scratch + so, nullptr, (uint32_t *)(sl.d_desc + sl.o_status));
                P.out = R.look.out_vals;
                P.cap = q.bound;
                P.count = R.look.count;
                if (S->o.single_query_kernels || runs_plain(R)) {
                    sl.plain.push_back(P);
                    S->stats.single_query_queries++;
                } else {
                    R.unit0 = units;
                    unit0[nk] = units;
                    units += R.n_chunks;
                    R.seg0 = segs;
                    R.seg_tot = d_segs + segs;
                    seg0[nk] = segs;
                    segs += R.n_segs;
                    reqs[nk++] = R;
                    S->stats.persistent_queries++;
                }
                sl.tickets.push_back(tk);
                q.state = 1;
                S->queue.pop_front();
                nb++;
            }
            if (nb == 0) break;  // memory is full: wait for completions or releases
            unit0[nk] = units;
            seg0[nk] = segs;
            const auto now = Clock::now();
            for (uint64_t tk : sl.tickets) S->recs[tk].t_launch = now;
            const int lrc = launch_slot(S, sl, nb, nk, units, segs);
            if (lrc != BS_OK) {
                // whatever part of the batch was enqueued finishes before its
                // memory is handed out again; the queries complete with the
                // launch error as their status and no result
                cudaStreamSynchronize(sl.stream);
                cudaGetLastError();
                for (uint64_t tk : sl.tickets) {
                    QueryRec &q = S->recs[tk];
                    q.state = 2;
                    q.rc = lrc;
                    q.count = 0;
                    q.t_done = Clock::now();
                    S->scratch_alloc.release(q.scratch_off, q.scratch_bytes);
                    q.scratch_off = SIZE_MAX;
                    S->result_alloc.release(q.out_off, q.out_bytes);
                    q.out_off = SIZE_MAX;
                    S->stats.completed++;
                    S->stats.failed++;
                }
                sl.tickets.clear();
                S->cv_done.notify_all();
                continue;
            }
            sl.busy = true;
            S->stats.batches++;
            S->batched_queries += (uint64_t)nb;
            progress = true;
        }
        bool any_busy = false;
        for (Slot &sl : S->slots) any_busy |= sl.busy;
        if (S->stop && !any_busy) break;
        if (!progress) {
            if (any_busy) {
                // batches in flight: poll their events (a timed sleep would
                // oversleep by tens of microseconds)
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
            }
        }
    }
}

}  // namespace

extern "C" {

int bs_estimate_rows(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, uint64_t *out) {
    if (!col || !out || op < BS_LT || op > BS_BETWEEN) return BS_ERR_INVALID_ARG;
    *out = bs::estimate_rows(col->c, op, lit, lit2);
    return BS_OK;
}

int bs_server_create(const bs_server_opts *opts, bs_server **out) {
    using namespace bs;
    if (!out) return BS_ERR_INVALID_ARG;
    *out = nullptr;
    auto *S = new (std::nothrow) bs_server;
    if (!S) return BS_ERR_OOM;
    bs_server_opts o{};
    o.device = -1;
    if (opts) o = *opts;
    if (o.max_batch <= 0) o.max_batch = 64;
    if (o.slots <= 0) o.slots = 2;
    if (o.result_bytes == 0) o.result_bytes = 1ull << 30;
    if (o.scratch_bytes == 0) o.scratch_bytes = 4ull << 30;
    if (o.threads <= 0) o.threads = 256;
    if (o.max_batch > 4096 || o.slots > 16) {
        delete S;
        return BS_ERR_INVALID_ARG;
    }
    S->o = o;
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete S;
        return BS_ERR_CUDA;
    }
    S->device = dev;
    int prev = 0;
    cudaGetDevice(&prev);
    int rc = cudaSetDevice(dev) == cudaSuccess ? BS_OK : BS_ERR_CUDA;
    if (rc == BS_OK) {
        S->status = status_word();
        if (!S->status) rc = BS_ERR_CUDA;
    }
    if (rc == BS_OK && (cudaMalloc(&S->d_result, o.result_bytes) != cudaSuccess ||
                        cudaMalloc(&S->d_scratch, o.scratch_bytes) != cudaSuccess)) {
        cudaGetLastError();
        rc = BS_ERR_OOM;
    }
    S->result_alloc.reset(o.result_bytes);
    S->scratch_alloc.reset(o.scratch_bytes);
    if (rc == BS_OK) {
        // kernel shape: each slot's grid takes its share of the GPU, so batches
        // of different slots run side by side
        const size_t smem = smem_bytes(o.threads);
        int fit = 0;
        if (cudaFuncSetAttribute(batch_fn(kStages), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, batch_fn(kStages), o.threads, smem) != cudaSuccess ||
            fit < 1) {
            cudaGetLastError();
            rc = BS_ERR_CUDA;
        }
        S->threads = o.threads;
        S->ctas = std::max(1, fit * sm_count(dev) / o.slots);
    }
    S->slots.resize(o.slots);
    for (Slot &sl : S->slots) {
        if (rc != BS_OK) break;
        size_t at = 0;
        auto take = [&](size_t bytes) {
            size_t a = (at + 255) & ~(size_t)255;
            at = a + bytes;
            return a;
        };
        take(sizeof(BReq) * (size_t)o.max_batch);
        sl.o_unit0 = take(((size_t)o.max_batch + 1) * 4);
        sl.o_seg0 = take(((size_t)o.max_batch + 1) * 4);
        // counters, then up to 512 segment totals per query (n < 2^32 rows)
        sl.o_ctr = take(256 + (size_t)o.max_batch * 512 * 8);
        sl.o_counts = take((size_t)o.max_batch * 8);
        sl.o_status = sl.o_counts + (size_t)o.max_batch * 8;  // right after the counts (8-byte aligned)
        at = sl.o_status + 8;
        sl.desc_bytes = at;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&sl.d_desc, sl.desc_bytes) != cudaSuccess ||
            cudaMallocHost(&sl.h_desc, sl.desc_bytes) != cudaSuccess) {
            cudaGetLastError();
            rc = BS_ERR_OOM;
        }
    }
    cudaSetDevice(prev);
    if (rc != BS_OK) {
        bs_server_destroy(S);
        return rc;
    }
    S->th = std::thread(dispatcher, S);
    *out = S;
    return BS_OK;
}

int bs_server_submit(bs_server *S, const bs_query *q, uint64_t *ticket) {
    using namespace bs;
    if (!S || !q || !ticket) return BS_ERR_INVALID_ARG;
    QueryRec rec;
    bs_request r{};
    r.npreds = q->npreds;
    for (int i = 0; i < BS_MAX_CONJ; i++) r.preds[i] = q->preds[i];
    r.proj = q->proj;
    int device = S->device;
    int rc = plan_request(r, rec.plan, rec.plain, device, nullptr);
    if (rc) return rc;
    if (device != S->device) return BS_ERR_INVALID_ARG;
    uint64_t bound = rec.plan.look.n;
    for (int i = 0; i < q->npreds; i++)
        bound = std::min(bound, estimate_rows(q->preds[i].col->c, q->preds[i].op, q->preds[i].lit, q->preds[i].lit2));
    rec.bound = bound;
    rec.out_bytes = std::max<uint64_t>(256, bound * 4);
    rec.scratch_bytes = request_scratch(rec.plan, true);
    if (rec.out_bytes > S->o.result_bytes || rec.scratch_bytes > S->o.scratch_bytes) {
        std::lock_guard<std::mutex> g(S->mu);
        S->stats.rejected++;
        return BS_ERR_CAPACITY;
    }
    rec.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(S->mu);
        const uint64_t tk = S->next_ticket++;
        S->recs.emplace(tk, rec);
        S->queue.push_back(tk);
        S->stats.submitted++;
        *ticket = tk;
    }
    S->cv_work.notify_one();
    return BS_OK;
}

// A finished query reports its own status both in res->status and as the
// return value: BS_OK, or the launch error / device check / timeout that
// failed it (then count is 0 and d_values NULL).
static int fill_result(bs_server *S, const QueryRec &q, bs_query_result *res) {
    std::memset(res, 0, sizeof *res);
    if (q.state != 2) {
        res->status = BS_ERR_NOT_READY;
        return BS_ERR_NOT_READY;
    }
    res->status = q.rc;
    res->count = q.count;
    res->d_values = (q.rc != BS_OK || q.out_off == SIZE_MAX) ? nullptr : (const int32_t *)(S->d_result + q.out_off);
    res->queue_us = us_since(q.t_submit, q.t_launch);
    res->latency_us = us_since(q.t_submit, q.t_done);
    return q.rc;
}

int bs_server_poll(bs_server *S, uint64_t ticket, bs_query_result *res) {
    if (!S || !res) return BS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->recs.find(ticket);
    if (it == S->recs.end()) return BS_ERR_INVALID_ARG;
    return fill_result(S, it->second, res);
}

int bs_server_wait(bs_server *S, uint64_t ticket, int32_t timeout_ms, bs_query_result *res) {
    if (!S || !res) return BS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->recs.find(ticket);
    if (it == S->recs.end()) return BS_ERR_INVALID_ARG;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                        [&] { return S->recs[ticket].state == 2; });
    if (!ok) {
        std::memset(res, 0, sizeof *res);
        res->status = BS_ERR_NOT_READY;
        return BS_ERR_TIMEOUT;
    }
    return fill_result(S, S->recs[ticket], res);
}

int bs_server_copy_result(bs_server *S, uint64_t ticket, int32_t *dst, uint64_t cap, uint64_t *copied,
                          void *stream) {
    if (!S || (cap && !dst)) return BS_ERR_INVALID_ARG;
    const int32_t *src = nullptr;
    uint64_t n = 0;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->recs.find(ticket);
        if (it == S->recs.end()) return BS_ERR_INVALID_ARG;
        if (it->second.state != 2) return BS_ERR_NOT_READY;
        if (it->second.rc != BS_OK) return it->second.rc;
        if (it->second.out_off == SIZE_MAX) return BS_ERR_INVALID_ARG;
        src = (const int32_t *)(S->d_result + it->second.out_off);
        n = std::min(cap, it->second.count);
    }
    if (copied) *copied = n;
    if (n && cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDefault, (cudaStream_t)stream) != cudaSuccess)
        return BS_ERR_CUDA;
    return BS_OK;
}

int bs_server_release(bs_server *S, uint64_t ticket) {
    if (!S) return BS_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->recs.find(ticket);
        if (it == S->recs.end()) return BS_ERR_INVALID_ARG;
        if (it->second.state != 2) return BS_ERR_NOT_READY;
        if (it->second.out_off != SIZE_MAX) S->result_alloc.release(it->second.out_off, it->second.out_bytes);
        S->recs.erase(it);
    }
    S->cv_work.notify_one();
    return BS_OK;
}

int bs_server_get_stats(const bs_server *S, bs_server_stats *st) {
    if (!S || !st) return BS_ERR_INVALID_ARG;
    auto *M = const_cast<bs_server *>(S);
    std::lock_guard<std::mutex> g(M->mu);
    *st = S->stats;
    st->mean_batch = S->stats.batches ? (double)S->batched_queries / (double)S->stats.batches : 0.0;
    st->result_bytes_in_use = S->result_alloc.used();
    st->scratch_bytes_in_use = S->scratch_alloc.used();
    st->queued = S->queue.size();
    return BS_OK;
}

int bs_server_fail_next_launches(bs_server *S, int32_t n) {
    if (!S || n < 0) return BS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    S->fail_launches = n;
    return BS_OK;
}

void bs_server_destroy(bs_server *S) {
    if (!S) return;
    if (S->th.joinable()) {
        {
            std::lock_guard<std::mutex> g(S->mu);
            S->stop = true;
            S->queue.clear();  // queued queries are dropped; running batches finish
        }
        S->cv_work.notify_all();
        S->th.join();
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.d_desc) cudaFree(sl.d_desc);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
    }
    if (S->d_result) cudaFree(S->d_result);
    if (S->d_scratch) cudaFree(S->d_scratch);
    cudaSetDevice(prev);
    delete S;
}

}  // extern "C"
