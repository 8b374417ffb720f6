// Encoded columns to and from files (bs_column_save / bs_column_load): the
// encoder is the expensive step of ingestion, so an encoded column can be
// written once and read back instead of re-encoded. The file holds the
// dictionary side (values, codes, counts, decode tables) and the layout's
// byte arrays exactly as the column keeps them on the host; a column whose
// layout lives only on the device is read back from its device arena first.
//
// Format (little-endian, as the host writes it): the 8-byte magic
// "BSCOL\0\0\1", then the scalar fields, then every array as a uint64 element
// count followed by its elements.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "kernels.h"

namespace {

using bs::Column;

const char kMagic[8] = {'B', 'S', 'C', 'O', 'L', 0, 0, 1};

struct File {
    FILE *f = nullptr;
    bool ok = true;
    explicit File(FILE *fp) : f(fp) {}
    ~File() {
        if (f) std::fclose(f);
    }
    void put(const void *p, size_t n) {
        if (ok && n && std::fwrite(p, 1, n, f) != n) ok = false;
    }
    void get(void *p, size_t n) {
        if (ok && n && std::fread(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    void put(const T &v) {
        put(&v, sizeof v);
    }
    template <class T>
    void get(T &v) {
        get(&v, sizeof v);
    }
    template <class T>
    void put_vec(const std::vector<T> &v) {
        const uint64_t n = v.size();
        put(n);
        put(v.data(), n * sizeof(T));
    }
    template <class T>
    void get_vec(std::vector<T> &v, uint64_t max_elems) {
        uint64_t n = 0;
        get(n);
        if (!ok || n > max_elems) {
            ok = false;
            return;
        }
        v.resize(n);
        get(v.data(), n * sizeof(T));
    }
};

// device -> host copy of one layout array (when the column kept no host copy)
template <class T>
bool fetch(std::vector<T> &dst, const T *src, uint64_t n) {
    dst.resize(n);
    if (!n) return true;
    return cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost) == cudaSuccess;
}

}  // namespace

extern "C" {

int bs_column_save(const bs_column *col, const char *path) {
    if (!col || !path) return BS_ERR_INVALID_ARG;
    const Column &c = col->c;
    // the layout arrays: the host copy, or read back from the device arena
    std::vector<uint8_t> dense_tmp, deep_tmp[bs::kMaxCodeBytes + 1];
    std::vector<uint32_t> mask_tmp[bs::kMaxCodeBytes + 1], off_tmp[bs::kMaxCodeBytes + 1], packed_tmp;
    const std::vector<uint8_t> *dense = &c.h_dense;
    const std::vector<uint8_t> *deep[bs::kMaxCodeBytes + 1];
    const std::vector<uint32_t> *mask[bs::kMaxCodeBytes + 1], *off[bs::kMaxCodeBytes + 1], *packed = &c.h_packed;
    for (int j = 0; j <= bs::kMaxCodeBytes; j++) {
        deep[j] = &c.h_deep[j];
        mask[j] = &c.h_mask[j];
        off[j] = &c.h_off[j];
    }
    if (!c.has_host) {
        if (!c.d_arena) return BS_ERR_UNSUPPORTED;
        int prev = 0;
        cudaGetDevice(&prev);
        if (cudaSetDevice(c.device) != cudaSuccess) return BS_ERR_CUDA;
        bool ok = true;
        if (c.layout == BS_PPVBS || c.layout == BS_BYTESLICE) {
            const uint64_t slices = c.layout == BS_BYTESLICE ? (uint64_t)c.S : 1;
            ok = ok && fetch(dense_tmp, c.d_dense, slices * c.dense_slice_bytes());
            dense = &dense_tmp;
        }
        if (c.layout == BS_PPVBS) {
            for (int j = 2; j <= c.K; j++) {
                ok = ok && fetch(mask_tmp[j], c.d_mask[j], (uint64_t)c.n_tiles * bs::kTileWords);
                ok = ok && fetch(off_tmp[j], c.d_off[j], (uint64_t)c.n_tiles * bs::kGroupsPerTile + 1);
                ok = ok && fetch(deep_tmp[j], c.d_deep[j], c.deep_len[j] + 16);  // uploaded with 16 bytes of padding
                mask[j] = &mask_tmp[j];
                off[j] = &off_tmp[j];
                deep[j] = &deep_tmp[j];
            }
        }
        if (c.layout == BS_BITPACKED) {
            ok = ok && fetch(packed_tmp, c.d_packed, c.packed_words());
            packed = &packed_tmp;
        }
        cudaSetDevice(prev);
        if (!ok) return BS_ERR_CUDA;
    }
    File w(std::fopen(path, "wb"));
    if (!w.f) return BS_ERR_INVALID_ARG;
    w.put(kMagic, sizeof kMagic);
    w.put((int32_t)c.layout);
    w.put(c.n);
    w.put(c.n_tiles);
    w.put((uint8_t)c.raw);
    w.put((uint8_t)c.identity);
    w.put(c.domain_min);
    w.put((int32_t)c.k);
    w.put((int32_t)c.S);
    w.put((int32_t)c.K);
    w.put((uint8_t)c.categorical);
    w.put((int32_t)c.cat_B);
    w.put_vec(c.dict);
    w.put_vec(c.dcode);
    w.put_vec(c.dlen);
    w.put_vec(c.dcount);
    w.put_vec(c.dcum);
    w.put_vec(c.first_byte_rows);
    w.put_vec(c.val2);
    w.put_vec(c.leaf2);
    w.put_vec(c.val1);
    w.put_vec(c.rank_dict);
    w.put_vec(*dense);
    for (int j = 2; j <= bs::kMaxCodeBytes; j++) {
        w.put_vec(*mask[j]);
        w.put_vec(*off[j]);
        w.put_vec(*deep[j]);
        w.put(c.deep_len[j]);
    }
    w.put_vec(*packed);
    w.put(c.len_hist, sizeof c.len_hist);
    return w.ok ? BS_OK : BS_ERR_CUDA;
}

int bs_column_load(const char *path, const bs_encode_opts *opts, bs_column **out) {
    if (!path || !out) return BS_ERR_INVALID_ARG;
    *out = nullptr;
    bs_encode_opts o;
    std::memset(&o, 0, sizeof o);
    o.device = -1;
    if (opts) o = *opts;
    File r(std::fopen(path, "rb"));
    if (!r.f) return BS_ERR_INVALID_ARG;
    char magic[8];
    r.get(magic, sizeof magic);
    if (!r.ok || std::memcmp(magic, kMagic, sizeof kMagic) != 0) return BS_ERR_INVALID_ARG;
    std::unique_ptr<bs_column> col(new (std::nothrow) bs_column);
    if (!col) return BS_ERR_OOM;
    Column &c = col->c;
    int32_t layout = 0, k = 0, S = 0, K = 0, cat_B = 0;
    uint8_t raw = 0, identity = 0, categorical = 0;
    r.get(layout);
    r.get(c.n);
    r.get(c.n_tiles);
    r.get(raw);
    r.get(identity);
    r.get(c.domain_min);
    r.get(k);
    r.get(S);
    r.get(K);
    r.get(categorical);
    r.get(cat_B);
    if (!r.ok || layout < BS_BITPACKED || layout > BS_PPVBS || c.n >= (1ull << 32) ||
        c.n_tiles != (uint32_t)((c.n + bs::kTileRows - 1) / bs::kTileRows) || K < 1 || K > bs::kMaxCodeBytes ||
        k < 0 || k > 64 || S < 0 || S > bs::kMaxCodeBytes)
        return BS_ERR_INVALID_ARG;
    c.layout = (bs_layout)layout;
    c.raw = raw != 0;
    c.identity = identity != 0;
    c.k = k;
    c.S = S;
    c.K = K;
    c.categorical = categorical != 0;
    c.cat_B = cat_B;
    const uint64_t cap = (uint64_t)c.n_tiles * bs::kTileRows * bs::kMaxCodeBytes + (1ull << 20);  // bounds every array
    r.get_vec(c.dict, cap);
    r.get_vec(c.dcode, cap);
    r.get_vec(c.dlen, cap);
    r.get_vec(c.dcount, cap);
    r.get_vec(c.dcum, cap);
    r.get_vec(c.first_byte_rows, cap);
    r.get_vec(c.val2, cap);
    r.get_vec(c.leaf2, cap);
    r.get_vec(c.val1, cap);
    r.get_vec(c.rank_dict, cap);
    r.get_vec(c.h_dense, cap);
    for (int j = 2; j <= bs::kMaxCodeBytes; j++) {
        r.get_vec(c.h_mask[j], cap);
        r.get_vec(c.h_off[j], cap);
        r.get_vec(c.h_deep[j], cap);
        r.get(c.deep_len[j]);
    }
    r.get_vec(c.h_packed, cap);
    r.get(c.len_hist, sizeof c.len_hist);
    if (!r.ok) return BS_ERR_INVALID_ARG;
    // the sizes the kernels rely on
    bool sane = true;
    if (c.layout == BS_PPVBS) {
        sane = c.h_dense.size() == c.dense_slice_bytes() &&
               (c.raw || (c.val2.size() == 65536 && c.leaf2.size() == 65536 && c.val1.size() == 256 &&
                          c.dcode.size() == c.dict.size() && c.dlen.size() == c.dict.size()));
        for (int j = 2; j <= c.K && sane; j++)
            sane = c.h_mask[j].size() == (uint64_t)c.n_tiles * bs::kTileWords &&
                   c.h_off[j].size() == (uint64_t)c.n_tiles * bs::kGroupsPerTile + 1 &&
                   c.h_deep[j].size() >= c.deep_len[j] && c.h_off[j].back() == c.deep_len[j];
        for (int j = 2; j <= c.K && sane; j++) c.h_deep[j].resize(c.deep_len[j] + 16, 0);  // the encoder's padding
    } else if (c.layout == BS_BYTESLICE) {
        sane = c.h_dense.size() == (uint64_t)c.S * c.dense_slice_bytes();
    } else {
        sane = c.h_packed.size() == c.packed_words();
    }
    if (c.categorical && c.rank_dict.size() != c.dict.size()) sane = false;
    if (!sane) return BS_ERR_INVALID_ARG;
    c.has_host = true;
    if (o.host_only) {
        c.device = o.device >= 0 ? o.device : 0;
    } else {
        int dev = o.device;
        if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return BS_ERR_CUDA;
        c.device = dev;
        const int rc = bs::upload_column(c);
        if (rc != BS_OK) return rc;
        if (!o.keep_host) {
            std::vector<uint8_t>().swap(c.h_dense);
            for (int j = 0; j <= bs::kMaxCodeBytes; j++) {
                std::vector<uint32_t>().swap(c.h_mask[j]);
                std::vector<uint32_t>().swap(c.h_off[j]);
                std::vector<uint8_t>().swap(c.h_deep[j]);
            }
            std::vector<uint32_t>().swap(c.h_packed);
            c.has_host = false;
        }
    }
    *out = col.release();
    return BS_OK;
}

}  // extern "C"
