// Column-layout advisor (Algorithm 5) and the C entry points of the
// effective-bytes counter.
//
// For one column: encode it as ByteSlice (dictionary codes) and as PP-VBS
// (Algorithm 1, or Algorithm 2 for a categorical column), pick 100 literals
// from the column whose selectivities span the feasible range -- numerical:
// `<` with the value at row quantile (i+0.5)/100, rounded up to the smallest
// value reaching it; categorical: `=` with the values at evenly spaced
// frequency ranks -- measure each scan on both layouts, integrate each
// (selectivity, cost) profile with the trapezoid rule and keep the layout with
// the smaller area; ties go to ByteSlice, as the algorithm's "Y <= Z" test
// does.
//   TIMED:       cost = median of 3 CUDA-event timings of bs_scan on the device.
//   BYTES_MODEL: cost = bytes the scan must move (effective-bytes counter), a
//                deterministic stand-in that needs no GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.h"

namespace {

using bs::Column;

double trapezoid(std::vector<std::pair<double, double>> pts) {
    std::stable_sort(pts.begin(), pts.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
    if (pts.empty()) return 0.0;
    if (pts.back().first - pts.front().first <= 0.0) {
        double s = 0;  // one distinct selectivity: the mean cost
        for (auto &p : pts) s += p.second;
        return s / (double)pts.size();
    }
    double auc = 0.0;
    for (size_t i = 1; i < pts.size(); i++)
        auc += (pts[i].first - pts[i - 1].first) * 0.5 * (pts[i].second + pts[i - 1].second);
    return auc;
}

}  // namespace

extern "C" {

int bs_scan_bytes(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, const uint32_t *h_seed,
                  bs_scan_bytes_t *out) {
    if (!col || !out || op < BS_LT || op > BS_BETWEEN) return BS_ERR_INVALID_ARG;
    bs::KPred p;
    int rc = bs::rewrite_literal(col->c, op, lit, lit2, p);
    if (rc) return rc;
    return bs::scan_bytes(col->c, p, h_seed, 1, out);
}

int bs_scan_bytes_sampled(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, const uint32_t *h_seed,
                          uint64_t tile_stride, bs_scan_bytes_t *out) {
    if (!col || !out || op < BS_LT || op > BS_BETWEEN || tile_stride == 0) return BS_ERR_INVALID_ARG;
    bs::KPred p;
    int rc = bs::rewrite_literal(col->c, op, lit, lit2, p);
    if (rc) return rc;
    return bs::scan_bytes(col->c, p, h_seed, tile_stride, out);
}

int bs_scan_lookup_bytes(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, const uint32_t *h_sel,
                         int32_t write_bits, bs_scan_bytes_t *out) {
    if (!col || !out || op < BS_LT || op > BS_BETWEEN || (col->c.n && !h_sel)) return BS_ERR_INVALID_ARG;
    bs::KPred p;
    int rc = bs::rewrite_literal(col->c, op, lit, lit2, p);
    if (rc) return rc;
    return bs::scan_lookup_bytes(col->c, p, h_sel, write_bits != 0, out);
}

int bs_lookup_bytes(const bs_column *col, const uint32_t *h_bits, bs_lookup_bytes_t *out) {
    if (!col || !out || (col->c.n && !h_bits)) return BS_ERR_INVALID_ARG;
    return bs::lookup_bytes(col->c, h_bits, out);
}

int bs_advise_layout_range(const int32_t *h_values, uint64_t n, int32_t mode, const bs_encode_opts *opts,
                           double sel_lo, double sel_hi, bs_advice *out) {
    if (!out || (n && !h_values) || (mode != BS_ADVISE_TIMED && mode != BS_ADVISE_BYTES_MODEL))
        return BS_ERR_INVALID_ARG;
    if (!(sel_lo >= 0.0 && sel_lo <= sel_hi && sel_hi <= 1.0)) return BS_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof *out);
    bs_encode_opts o;
    std::memset(&o, 0, sizeof o);
    o.device = -1;
    if (opts) o = *opts;
    if (mode == BS_ADVISE_BYTES_MODEL) {
        o.host_only = 1;
    } else {
        o.host_only = 0;
        o.keep_host = 0;
    }
    bs_column *bsl = nullptr, *vbs = nullptr;
    int rc = bs_encode_column(h_values, n, BS_BYTESLICE, &o, &bsl);
    if (rc) return rc;
    bs_encode_opts ov = o;
    ov.domain_bits = 0;
    ov.domain_values = nullptr;
    ov.n_domain = 0;
    rc = bs_encode_column(h_values, n, BS_PPVBS, &ov, &vbs);
    if (rc) {
        bs_column_free(bsl);
        return rc;
    }
    const Column &cv = vbs->c;
    const std::vector<uint64_t> &Q = cv.dcount;
    const int P = 100;
    std::vector<int32_t> lits(P);
    std::vector<double> sel(P);
    const bs_op op = o.categorical ? BS_EQ : BS_LT;
    if (o.categorical) {
        // categorical: `=` with values at evenly spaced frequency ranks among
        // those whose selectivity lies in [sel_lo, sel_hi] (the nearest rank
        // when none does; the whole range: from the most frequent value down)
        std::vector<uint32_t> order(Q.size());
        for (size_t i = 0; i < Q.size(); i++) order[i] = (uint32_t)i;
        std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return Q[x] > Q[y]; });
        size_t r0 = 0, r1 = order.empty() ? 0 : order.size() - 1;
        if (!order.empty() && n) {
            auto s_of = [&](size_t r) { return (double)Q[order[r]] / (double)n; };
            while (r0 < r1 && s_of(r0) > sel_hi) r0++;   // counts fall along the ranks
            while (r1 > r0 && s_of(r1) < sel_lo) r1--;
        }
        for (int i = 0; i < P; i++) {
            const size_t r = order.empty() ? 0 : r0 + (size_t)((double)i * (double)(r1 - r0) / (P - 1) + 0.5);
            const size_t u = order.empty() ? 0 : order[r];
            lits[i] = cv.dict.empty() ? 0 : cv.dict[u];
            sel[i] = n && !Q.empty() ? (double)Q[u] / (double)n : 0.0;
        }
    } else {
        // numerical: `<` with literals at row quantiles sel_lo + (i + 0.5) / 100
        // * (sel_hi - sel_lo) (the whole range: (i + 0.5) / 100)
        std::vector<uint64_t> cum(Q.size() + 1, 0);
        for (size_t i = 0; i < Q.size(); i++) cum[i + 1] = cum[i] + Q[i];
        for (int i = 0; i < P; i++) {
            const double target = (sel_lo + ((double)i + 0.5) / P * (sel_hi - sel_lo)) * (double)n;
            size_t u = 0;
            while (u + 1 < cum.size() && (double)cum[u] < target) u++;
            if (u >= cv.dict.size()) u = cv.dict.empty() ? 0 : cv.dict.size() - 1;
            lits[i] = cv.dict.empty() ? 0 : cv.dict[u];
            sel[i] = n ? (double)cum[u] / (double)n : 0.0;
        }
    }
    std::vector<double> cost_b(P, 0.0), cost_v(P, 0.0);
    if (mode == BS_ADVISE_BYTES_MODEL) {
        const uint64_t stride = std::max<uint64_t>(1, (uint64_t)cv.n_tiles / 4096);
        for (int i = 0; i < P && rc == BS_OK; i++) {
            bs::KPred pb, pv;
            bs_scan_bytes_t sb, sv;
            rc = bs::rewrite_literal(bsl->c, op, lits[i], 0, pb);
            if (!rc) rc = bs::rewrite_literal(vbs->c, op, lits[i], 0, pv);
            if (!rc) rc = bs::scan_bytes(bsl->c, pb, nullptr, stride, &sb);
            if (!rc) rc = bs::scan_bytes(vbs->c, pv, nullptr, stride, &sv);
            cost_b[i] = (double)sb.bytes;
            cost_v[i] = (double)sv.bytes;
        }
    } else {
        const uint64_t nw = (n + 31) / 32;
        uint32_t *d_bits = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaMalloc(&d_bits, std::max<uint64_t>(4, nw * 4)) != cudaSuccess) rc = BS_ERR_OOM;
        if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = BS_ERR_CUDA;
        auto time_scan = [&](const bs_column *c, int32_t lit, double &secs) -> int {
            float ms[3];
            int r = bs_scan(c, op, lit, 0, d_bits, nullptr);  // warm-up
            for (int k = 0; k < 3 && !r; k++) {
                cudaEventRecord(e0, nullptr);
                r = bs_scan(c, op, lit, 0, d_bits, nullptr);
                cudaEventRecord(e1, nullptr);
                if (cudaEventSynchronize(e1) != cudaSuccess) r = BS_ERR_CUDA;
                cudaEventElapsedTime(&ms[k], e0, e1);
            }
            std::sort(ms, ms + 3);
            secs = ms[1] * 1e-3;
            return r;
        };
        for (int i = 0; i < P && rc == BS_OK; i++) {
            rc = time_scan(bsl, lits[i], cost_b[i]);
            if (!rc) rc = time_scan(vbs, lits[i], cost_v[i]);
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (d_bits) cudaFree(d_bits);
    }
    bs_column_free(bsl);
    bs_column_free(vbs);
    if (rc) return rc;
    std::vector<std::pair<double, double>> pb, pv;
    for (int i = 0; i < P; i++) {
        pb.emplace_back(sel[i], cost_b[i]);
        pv.emplace_back(sel[i], cost_v[i]);
        out->selectivity[i] = sel[i];
        out->cost_byteslice[i] = cost_b[i];
        out->cost_ppvbs[i] = cost_v[i];
    }
    out->n_points = P;
    out->auc_byteslice = trapezoid(pb);
    out->auc_ppvbs = trapezoid(pv);
    out->layout = out->auc_byteslice <= out->auc_ppvbs ? BS_BYTESLICE : BS_PPVBS;
    return BS_OK;
}

int bs_advise_layout(const int32_t *h_values, uint64_t n, int32_t mode, const bs_encode_opts *opts,
                     bs_advice *out) {
    return bs_advise_layout_range(h_values, n, mode, opts, 0.0, 1.0, out);
}

}  // extern "C"
