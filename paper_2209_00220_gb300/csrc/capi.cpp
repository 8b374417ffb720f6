// extern "C" entry points of libbytestore (declared in include/bytestore.h):
// argument checking, literal rewriting and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "kernels.h"

using bs::Column;

namespace {

bs_encode_opts defaults() {
    bs_encode_opts o;
    std::memset(&o, 0, sizeof o);
    o.device = -1;
    return o;
}

bool valid_op(int op) { return op >= BS_LT && op <= BS_BETWEEN; }

void drop_host(Column &c) {
    std::vector<uint8_t>().swap(c.h_dense);
    for (int j = 0; j <= bs::kMaxCodeBytes; j++) {
        std::vector<uint32_t>().swap(c.h_mask[j]);
        std::vector<uint32_t>().swap(c.h_off[j]);
        std::vector<uint8_t>().swap(c.h_deep[j]);
    }
    std::vector<uint32_t>().swap(c.h_packed);
    c.has_host = false;
}

int finish_column(bs_column *col, const bs_encode_opts &o, int rc, bs_column **out) {
    if (rc != BS_OK) {
        delete col;
        return rc;
    }
    Column &c = col->c;
    if (!o.host_only) {
        rc = bs::upload_column(c);
        if (rc != BS_OK) {
            delete col;
            return rc;
        }
    }
    c.has_host = o.host_only || o.keep_host;
    if (!c.has_host) drop_host(c);
    *out = col;
    return BS_OK;
}

int pick_device(const bs_encode_opts &o, int &dev) {
    if (o.host_only) {
        dev = o.device >= 0 ? o.device : 0;
        return BS_OK;
    }
    if (o.device >= 0) {
        dev = o.device;
        return BS_OK;
    }
    return cudaGetDevice(&dev) == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bool on_device(const bs_column *col) { return col && col->c.d_arena != nullptr; }

// Scans and lookups run on the column's device; the caller's current device is
// restored afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

uint32_t host_row_byte1(const Column &c, uint64_t slice, uint64_t row) {
    const uint64_t t = row >> 10;
    return c.h_dense[slice * c.dense_slice_bytes() + t * bs::kTileRows + bs::tile_byte_pos((uint32_t)(row & 1023))];
}

}  // namespace

extern "C" {

int bs_encode_column(const int32_t *h_values, uint64_t n, bs_layout layout, const bs_encode_opts *opts,
                     bs_column **out) {
    if (!out) return BS_ERR_INVALID_ARG;
    *out = nullptr;
    if (layout != BS_PPVBS && layout != BS_BYTESLICE && layout != BS_BITPACKED) return BS_ERR_INVALID_ARG;
    bs_encode_opts o = opts ? *opts : defaults();
    auto *col = new (std::nothrow) bs_column;
    if (!col) return BS_ERR_OOM;
    int rc = pick_device(o, col->c.device);
    if (rc == BS_OK) rc = bs::encode_values(h_values, n, layout, o, col->c);
    return finish_column(col, o, rc, out);
}

int bs_column_from_codes(const uint64_t *h_codes, const uint8_t *h_lens, uint64_t n, bs_layout layout,
                         int32_t code_bits, const bs_encode_opts *opts, bs_column **out) {
    if (!out) return BS_ERR_INVALID_ARG;
    *out = nullptr;
    bs_encode_opts o = opts ? *opts : defaults();
    auto *col = new (std::nothrow) bs_column;
    if (!col) return BS_ERR_OOM;
    int rc = pick_device(o, col->c.device);
    if (rc == BS_OK) rc = bs::encode_raw(h_codes, h_lens, n, layout, code_bits, o, col->c);
    return finish_column(col, o, rc, out);
}

void bs_column_free(bs_column *col) {
    if (!col) return;
    bs::free_device(col->c);
    delete col;
}

int bs_column_get_info(const bs_column *col, bs_column_info *info) {
    if (!col || !info) return BS_ERR_INVALID_ARG;
    const Column &c = col->c;
    std::memset(info, 0, sizeof *info);
    info->n_rows = c.n;
    info->layout = c.layout;
    info->max_code_bytes = c.layout == BS_PPVBS ? c.K : c.S;
    info->code_bits = c.k;
    info->on_device = c.d_arena != nullptr;
    info->n_dict = c.dict.size();
    info->device_bytes = c.d_bytes;
    uint64_t lb = 0;
    if (c.layout == BS_PPVBS) {
        lb = c.n;
        for (int j = 2; j <= c.K; j++) lb += 4 * ((c.n + 31) / 32) + c.deep_len[j];
    } else if (c.layout == BS_BYTESLICE) {
        lb = (uint64_t)c.S * c.n;
    } else {
        lb = (c.n * (uint64_t)c.k + 7) / 8;
    }
    info->layout_bytes = lb;
    for (int l = 0; l <= bs::kMaxCodeBytes; l++) info->len_hist[l] = c.len_hist[l];
    return BS_OK;
}

int bs_column_row_codes(const bs_column *col, uint64_t row_begin, uint64_t count, uint64_t *h_codes,
                        uint8_t *h_lens) {
    if (!col || (count && (!h_codes || !h_lens))) return BS_ERR_INVALID_ARG;
    const Column &c = col->c;
    if (row_begin > c.n || count > c.n - row_begin) return BS_ERR_INVALID_ARG;
    if (!c.has_host) return BS_ERR_UNSUPPORTED;
    for (uint64_t i = 0; i < count; i++) {
        const uint64_t row = row_begin + i;
        uint64_t code = 0;
        uint32_t len = 0;
        if (c.layout == BS_PPVBS) {
            code = host_row_byte1(c, 0, row);
            len = 1;
            const uint64_t w = row >> 5, g = row >> 8;
            const uint32_t b = (uint32_t)(row & 31);
            for (int j = 2; j <= c.K; j++) {
                const uint32_t m = c.h_mask[j][w];
                if (!((m >> b) & 1u)) break;
                uint64_t idx = c.h_off[j][g];
                for (uint64_t x = g * bs::kGroupWords; x < w; x++) idx += (uint64_t)__builtin_popcount(c.h_mask[j][x]);
                idx += (uint64_t)__builtin_popcount(m & ((1u << b) - 1u));
                if (idx >= c.deep_len[j]) return BS_ERR_DEVICE_CHECK;
                code = (code << 8) | c.h_deep[j][idx];
                len = (uint32_t)j;
            }
        } else if (c.layout == BS_BYTESLICE) {
            uint64_t aligned = 0;
            for (int s = 0; s < c.S; s++) aligned = (aligned << 8) | host_row_byte1(c, (uint64_t)s, row);
            code = aligned >> (8 * c.S - c.k);
            len = (uint32_t)c.S;
        } else {
            const uint64_t bit = row * (uint64_t)c.k;
            const uint64_t lo = c.h_packed[bit >> 5], hi = c.h_packed[(bit >> 5) + 1];
            const uint64_t win = (hi << 32) | lo;
            code = (win >> (bit & 31)) & ((c.k >= 64) ? ~0ull : ((1ull << c.k) - 1));
            len = (uint32_t)c.S;
        }
        h_codes[i] = code;
        h_lens[i] = (uint8_t)len;
    }
    return BS_OK;
}

int bs_column_dictionary(const bs_column *col, int32_t *h_values, uint64_t *h_codes, uint8_t *h_lens,
                         uint64_t cap) {
    if (!col) return BS_ERR_INVALID_ARG;
    const Column &c = col->c;
    const uint64_t m = std::min<uint64_t>(cap, c.dict.size());
    for (uint64_t i = 0; i < m; i++) {
        if (h_values) h_values[i] = c.dict[i];
        if (h_codes) h_codes[i] = c.layout == BS_PPVBS ? c.dcode[i] : i;
        if (h_lens) h_lens[i] = c.layout == BS_PPVBS ? c.dlen[i] : (uint8_t)c.S;
    }
    return BS_OK;
}

static int scan_common(const bs_column *col, const bs::KPred &p, const uint32_t *d_seed, uint32_t *d_bits,
                       void *stream) {
    const Column &c = col->c;
    if (c.n && !d_bits) return BS_ERR_INVALID_ARG;
    DeviceGuard g(c.device);
    if (!g.ok) return BS_ERR_CUDA;
    return bs::launch_scan(c, p, d_seed, d_bits, (cudaStream_t)stream);
}

int bs_scan_seeded(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, const uint32_t *d_seed,
                   uint32_t *d_bits, void *stream) {
    if (!col || !valid_op(op)) return BS_ERR_INVALID_ARG;
    if (col->c.raw || !on_device(col)) return BS_ERR_UNSUPPORTED;
    bs::KPred p;
    int rc = bs::rewrite_literal(col->c, op, lit, lit2, p);
    if (rc) return rc;
    return scan_common(col, p, d_seed, d_bits, stream);
}

int bs_scan(const bs_column *col, bs_op op, int32_t lit, int32_t lit2, uint32_t *d_bits, void *stream) {
    return bs_scan_seeded(col, op, lit, lit2, nullptr, d_bits, stream);
}

int bs_scan_code(const bs_column *col, bs_op op, uint64_t code, int32_t len, uint64_t code2, int32_t len2,
                 const uint32_t *d_seed, uint32_t *d_bits, void *stream) {
    if (!col || !valid_op(op)) return BS_ERR_INVALID_ARG;
    if (!on_device(col)) return BS_ERR_UNSUPPORTED;
    bs::KPred p;
    int rc = bs::make_code_pred(col->c, op, code, len, code2, len2, p);
    if (rc) return rc;
    return scan_common(col, p, d_seed, d_bits, stream);
}

int bs_scan_conj(const bs_pred *preds, int32_t npreds, uint32_t *d_bits, void *stream) {
    if (!preds || npreds < 1 || npreds > 16 || !d_bits) return BS_ERR_INVALID_ARG;
    for (int i = 0; i < npreds; i++) {
        if (!preds[i].col || !valid_op(preds[i].op)) return BS_ERR_INVALID_ARG;
        if (preds[i].col->c.n != preds[0].col->c.n) return BS_ERR_INVALID_ARG;
        if (preds[i].col->c.device != preds[0].col->c.device) return BS_ERR_INVALID_ARG;
        if (preds[i].col->c.raw || !on_device(preds[i].col)) return BS_ERR_UNSUPPORTED;
    }
    for (int i = 0; i < npreds; i++) {
        int rc = bs_scan_seeded(preds[i].col, (bs_op)preds[i].op, preds[i].lit, preds[i].lit2,
                                i == 0 ? nullptr : d_bits, d_bits, stream);
        if (rc) return rc;
    }
    return BS_OK;
}

uint64_t bs_lookup_workspace_bytes(const bs_column *col) {
    if (!col) return 0;
    return bs::lookup_workspace_bytes(col->c);
}

static int lookup_common(const bs_column *col, const uint32_t *d_bits, int32_t *d_vals, uint64_t *d_codes,
                         uint64_t out_cap, uint64_t *d_count, void *d_ws, uint64_t ws_bytes, void *stream) {
    if (!col) return BS_ERR_INVALID_ARG;
    const Column &c = col->c;
    if (!on_device(col)) return BS_ERR_UNSUPPORTED;
    if (c.n && !d_bits) return BS_ERR_INVALID_ARG;
    if (out_cap && !d_vals && !d_codes) return BS_ERR_INVALID_ARG;
    DeviceGuard g(c.device);
    if (!g.ok) return BS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t need = bs::lookup_workspace_bytes(c);
    void *ws = d_ws;
    if (ws && ws_bytes < need) return BS_ERR_CAPACITY;
    bool own = false;
    if (!ws) {
        if (cudaMallocAsync(&ws, need, s) != cudaSuccess) {
            cudaGetLastError();
            return BS_ERR_OOM;
        }
        own = true;
    }
    int rc = bs::launch_lookup(c, d_bits, d_vals, d_codes, out_cap, d_count, ws, s);
    if (own) cudaFreeAsync(ws, s);
    return rc;
}

int bs_lookup(const bs_column *col, const uint32_t *d_bits, int32_t *d_out, uint64_t out_cap, uint64_t *d_count,
              void *d_workspace, uint64_t workspace_bytes, void *stream) {
    if (col && col->c.raw) return BS_ERR_UNSUPPORTED;
    return lookup_common(col, d_bits, d_out ? d_out : nullptr, nullptr, out_cap, d_count, d_workspace,
                         workspace_bytes, stream);
}

int bs_lookup_codes(const bs_column *col, const uint32_t *d_bits, uint64_t *d_codes, uint64_t out_cap,
                    uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes, void *stream) {
    if (out_cap && !d_codes) return BS_ERR_INVALID_ARG;
    return lookup_common(col, d_bits, nullptr, d_codes ? d_codes : nullptr, out_cap, d_count, d_workspace,
                         workspace_bytes, stream);
}

uint64_t bs_scan_lookup_workspace_bytes(const bs_column *proj) {
    if (!proj) return 0;
    return bs::scan_lookup_workspace_bytes(proj->c);
}

int bs_scan_lookup(const bs_pred *preds, int32_t npreds, const bs_column *proj, uint32_t *d_bits, int32_t *d_out,
                   uint64_t out_cap, uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes, void *stream) {
    if (!preds || npreds < 1 || npreds > BS_MAX_CONJ) return BS_ERR_INVALID_ARG;
    if (!proj) proj = preds[0].col;
    if (!proj) return BS_ERR_INVALID_ARG;
    if (proj->c.raw || !on_device(proj)) return BS_ERR_UNSUPPORTED;
    const Column *cols[BS_MAX_CONJ];
    bs::KPred kp[BS_MAX_CONJ];
    for (int i = 0; i < npreds; i++) {
        const bs_column *col = preds[i].col;
        if (!col || !valid_op(preds[i].op)) return BS_ERR_INVALID_ARG;
        if (col->c.n != proj->c.n || col->c.device != proj->c.device) return BS_ERR_INVALID_ARG;
        if (col->c.raw || !on_device(col)) return BS_ERR_UNSUPPORTED;
        const int rc = bs::rewrite_literal(col->c, preds[i].op, preds[i].lit, preds[i].lit2, kp[i]);
        if (rc) return rc;
        cols[i] = &col->c;
    }
    if (out_cap && !d_out) return BS_ERR_INVALID_ARG;
    DeviceGuard g(proj->c.device);
    if (!g.ok) return BS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t need = bs::scan_lookup_workspace_bytes(proj->c);
    void *ws = d_workspace;
    if (ws && workspace_bytes < need) return BS_ERR_CAPACITY;
    bool own = false;
    if (!ws) {
        if (cudaMallocAsync(&ws, need, s) != cudaSuccess) {
            cudaGetLastError();
            return BS_ERR_OOM;
        }
        own = true;
    }
    const int rc = bs::launch_scan_lookup(cols, kp, npreds, proj->c, d_bits, d_out, out_cap, d_count, ws, s);
    if (own) cudaFreeAsync(ws, s);
    return rc;
}

int bs_lookup_shape(const bs_column *col, int32_t *parts, int32_t *grid, int32_t *resident_ctas) {
    if (!col) return BS_ERR_INVALID_ARG;
    if (!on_device(col)) return BS_ERR_UNSUPPORTED;
    DeviceGuard g(col->c.device);
    if (!g.ok) return BS_ERR_CUDA;
    uint32_t p = 0, gr = 0, r = 0;
    const int rc = bs::lookup_shape(col->c, &p, &gr, &r);
    if (parts) *parts = (int32_t)p;
    if (grid) *grid = (int32_t)gr;
    if (resident_ctas) *resident_ctas = (int32_t)r;
    return rc;
}

int bs_lookup_rowids(const bs_column *col, const uint32_t *d_rowids, uint64_t m, int32_t *d_out, void *stream) {
    if (!col || (m && (!d_rowids || !d_out))) return BS_ERR_INVALID_ARG;
    if (col->c.raw || !on_device(col)) return BS_ERR_UNSUPPORTED;
    DeviceGuard g(col->c.device);
    if (!g.ok) return BS_ERR_CUDA;
    return bs::launch_lookup_rowids(col->c, d_rowids, m, d_out, (cudaStream_t)stream);
}

const char *bs_strerror(int status) {
    switch (status) {
    case BS_OK: return "ok";
    case BS_ERR_INVALID_ARG: return "invalid argument";
    case BS_ERR_OOM: return "out of memory";
    case BS_ERR_CUDA: return "CUDA runtime error";
    case BS_ERR_CAPACITY: return "output buffer too small";
    case BS_ERR_UNSUPPORTED: return "unsupported for this column";
    case BS_ERR_TIMEOUT: return "bounded wait expired";
    case BS_ERR_DEVICE_CHECK: return "device bounds check failed";
    case BS_ERR_NOT_READY: return "not ready";
    default: return "unknown status";
    }
}

int bs_last_device_error(void) {
    uint32_t st = 0;
    int rc = bs::read_and_clear_status(&st);
    if (rc) return rc;
    if (st & bs::kStatusTimeout) return BS_ERR_TIMEOUT;
    if (st & bs::kStatusBounds) return BS_ERR_DEVICE_CHECK;
    return BS_OK;
}

const char *bs_version(void) { return "bytestore-gb300 0.1 (sm_103a)"; }

}  // extern "C"
