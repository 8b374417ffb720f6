// Host-side encoder of libbytestore: dictionary (Section 2.2), prefix-
// preserving encoding of numerical columns (Algorithm 1), the device layouts of
// PP-VBS (VBS, Section 3.2), ByteSlice (Section 2.5) and Bit-Packed
// (Section 2.3), the PP-VBS decode tables, and literal rewriting.
//
// Everything here is multithreaded with std::thread over row ranges; the
// result never depends on the thread count.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

#include <sched.h>

#include "bs_internal.h"

namespace bs {

int resolve_threads(int requested) {
    if (requested > 0) return std::min(requested, 256);
    cpu_set_t set;
    if (sched_getaffinity(0, sizeof set, &set) == 0) {
        int c = CPU_COUNT(&set);
        if (c > 0) return std::min(c, 256);
    }
    unsigned h = std::thread::hardware_concurrency();
    return h ? (int)std::min(h, 256u) : 1;
}

// Run fn(begin, end, thread_index) over [0, n) split into `threads` ranges.
static void parallel_for(uint64_t n, int threads, const std::function<void(uint64_t, uint64_t, int)> &fn,
                         uint64_t min_per_thread = 1 << 15) {
    if (n == 0) return;
    uint64_t t = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)threads, (n + min_per_thread - 1) / min_per_thread));
    if (t == 1) { fn(0, n, 0); return; }
    std::vector<std::thread> th;
    uint64_t chunk = (n + t - 1) / t;
    for (uint64_t i = 0; i < t; i++) {
        uint64_t b = std::min(n, i * chunk), e = std::min(n, b + chunk);
        th.emplace_back([=, &fn] { fn(b, e, (int)i); });
    }
    for (auto &x : th) x.join();
}

// ------------------------------------------------------------ dictionary
// Sorted distinct values A (out), counts Q (out) and, per row, the index of its
// value in A (ridx, out, n entries).
static int build_dictionary(const int32_t *v, uint64_t n, int threads, std::vector<int32_t> &A,
                            std::vector<uint64_t> &Q, std::vector<uint32_t> &ridx) {
    A.clear(); Q.clear();
    ridx.assign(n, 0);
    if (n == 0) return BS_OK;
    // value range
    int T = threads;
    std::vector<int32_t> lo(T, INT32_MAX), hi(T, INT32_MIN);
    parallel_for(n, T, [&](uint64_t b, uint64_t e, int t) {
        int32_t l = INT32_MAX, h = INT32_MIN;
        for (uint64_t i = b; i < e; i++) { l = std::min(l, v[i]); h = std::max(h, v[i]); }
        lo[t] = std::min(lo[t], l); hi[t] = std::max(hi[t], h);
    });
    int32_t mn = *std::min_element(lo.begin(), lo.end());
    int32_t mx = *std::max_element(hi.begin(), hi.end());
    uint64_t range = (uint64_t)((int64_t)mx - (int64_t)mn) + 1;

    if (range <= (1ull << 24) && range <= 8 * n + 4096) {
        // direct counting: per-thread histograms over the value range
        uint64_t tt = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)T, (n + (1 << 15) - 1) >> 15));
        if (tt * range * 4 > (2ull << 30)) tt = std::max<uint64_t>(1, (2ull << 30) / (range * 4));
        std::vector<std::vector<uint32_t>> part(tt);
        parallel_for(n, (int)tt, [&](uint64_t b, uint64_t e, int t) {
            auto &h = part[t];
            h.assign(range, 0);
            for (uint64_t i = b; i < e; i++) h[(uint32_t)((int64_t)v[i] - mn)]++;
        });
        std::vector<uint32_t> pos(range, UINT32_MAX);
        for (uint64_t x = 0; x < range; x++) {
            uint64_t q = 0;
            for (auto &h : part)
                if (!h.empty()) q += h[x];
            if (q) {
                pos[x] = (uint32_t)A.size();
                A.push_back((int32_t)((int64_t)mn + (int64_t)x));
                Q.push_back(q);
            }
        }
        parallel_for(n, T, [&](uint64_t b, uint64_t e, int) {
            for (uint64_t i = b; i < e; i++) ridx[i] = pos[(uint32_t)((int64_t)v[i] - mn)];
        });
        return BS_OK;
    }

    // general path: parallel LSD radix sort of the order-preserving keys
    std::vector<uint32_t> keys(n), tmp(n);
    parallel_for(n, T, [&](uint64_t b, uint64_t e, int) {
        for (uint64_t i = b; i < e; i++) keys[i] = (uint32_t)v[i] ^ 0x80000000u;
    });
    uint64_t tt = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)T, (n + (1 << 16) - 1) >> 16));
    uint64_t chunk = (n + tt - 1) / tt;
    std::vector<uint64_t> hist(tt * 256);
    for (int pass = 0; pass < 4; pass++) {
        int sh = pass * 8;
        std::fill(hist.begin(), hist.end(), 0);
        parallel_for(tt, (int)tt, [&](uint64_t b, uint64_t e, int) {
            for (uint64_t t = b; t < e; t++) {
                uint64_t rb = t * chunk, re = std::min(n, rb + chunk);
                uint64_t *h = &hist[t * 256];
                for (uint64_t i = rb; i < re; i++) h[(keys[i] >> sh) & 255u]++;
            }
        }, 1);
        uint64_t acc = 0;
        for (int d = 0; d < 256; d++)
            for (uint64_t t = 0; t < tt; t++) {
                uint64_t c = hist[t * 256 + d];
                hist[t * 256 + d] = acc;
                acc += c;
            }
        parallel_for(tt, (int)tt, [&](uint64_t b, uint64_t e, int) {
            for (uint64_t t = b; t < e; t++) {
                uint64_t rb = t * chunk, re = std::min(n, rb + chunk);
                uint64_t *h = &hist[t * 256];
                for (uint64_t i = rb; i < re; i++) tmp[h[(keys[i] >> sh) & 255u]++] = keys[i];
            }
        }, 1);
        keys.swap(tmp);
    }
    std::vector<uint32_t>().swap(tmp);
    std::vector<uint32_t> ukeys;
    for (uint64_t i = 0; i < n; i++) {
        if (i == 0 || keys[i] != keys[i - 1]) {
            ukeys.push_back(keys[i]);
            Q.push_back(1);
        } else {
            Q.back()++;
        }
    }
    std::vector<uint32_t>().swap(keys);
    A.resize(ukeys.size());
    for (size_t i = 0; i < ukeys.size(); i++) A[i] = (int32_t)(ukeys[i] ^ 0x80000000u);
    // row -> index: bucket on the top 16 key bits, then binary search
    std::vector<uint32_t> bstart(65537);
    {
        size_t j = 0;
        for (uint32_t bkt = 0; bkt <= 65536; bkt++) {
            uint64_t first = (uint64_t)bkt << 16;
            while (j < ukeys.size() && (uint64_t)ukeys[j] < first) j++;
            bstart[bkt] = (uint32_t)j;
        }
    }
    parallel_for(n, T, [&](uint64_t b, uint64_t e, int) {
        for (uint64_t i = b; i < e; i++) {
            uint32_t key = (uint32_t)v[i] ^ 0x80000000u;
            uint32_t bk = key >> 16;
            const uint32_t *f = ukeys.data() + bstart[bk], *l = ukeys.data() + bstart[bk + 1];
            ridx[i] = (uint32_t)(std::lower_bound(f, l, key) - ukeys.data());
        }
    });
    return BS_OK;
}

// ---------------------------------------------------------- Algorithm 1
// Codes are built top-down: every node knows the pointer path (prefix) that
// leads to it, so a value's code is prefix . slot (internal node) or prefix .
// beta-byte leaf number.
namespace {
struct PpeOut {
    std::vector<uint64_t> &C;
    std::vector<uint8_t> &L;
};

inline bool heavier(const std::vector<uint64_t> &Q, uint64_t a, uint64_t b) {
    return Q[a] > Q[b] || (Q[a] == Q[b] && a < b);
}

int beta_bytes(uint64_t count) {  // smallest beta with 256^beta >= count + 1
    int beta = 0;
    unsigned __int128 cap = 1;
    while (cap < (unsigned __int128)count + 1) { cap *= 256; beta++; }
    return beta;
}

void leaf(PpeOut &o, int b, uint64_t s, uint64_t e, uint64_t prefix) {
    int beta = beta_bytes(e - s);
    for (uint64_t i = s; i < e; i++) {
        o.C[i] = (prefix << (8 * beta)) | (i - s + 1);
        o.L[i] = (uint8_t)(b + beta);
    }
}

// indices of the 255 heaviest values in [s, e) (ties: smaller index), ascending
std::vector<uint64_t> top255(const std::vector<uint64_t> &Q, uint64_t s, uint64_t e, int threads) {
    auto cmp = [&](uint64_t a, uint64_t b) { return heavier(Q, a, b); };  // heap top = lightest kept
    uint64_t m = e - s;
    int T = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)threads, m / 65536));
    std::vector<std::vector<uint64_t>> part(T);
    uint64_t chunk = (m + T - 1) / T;
    auto work = [&](int t) {
        auto &h = part[t];
        uint64_t b = s + (uint64_t)t * chunk, en = std::min(e, b + chunk);
        for (uint64_t i = b; i < en; i++) {
            if (h.size() < 255) {
                h.push_back(i);
                std::push_heap(h.begin(), h.end(), cmp);
            } else if (heavier(Q, i, h.front())) {
                std::pop_heap(h.begin(), h.end(), cmp);
                h.back() = i;
                std::push_heap(h.begin(), h.end(), cmp);
            }
        }
    };
    if (T == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < T; t++) th.emplace_back(work, t);
        for (auto &x : th) x.join();
    }
    std::vector<uint64_t> all;
    for (auto &h : part) all.insert(all.end(), h.begin(), h.end());
    std::sort(all.begin(), all.end(), [&](uint64_t a, uint64_t b) { return heavier(Q, a, b); });
    all.resize(255);
    std::sort(all.begin(), all.end());
    return all;
}

// Encode an internal node over [s, e) at level b with pointer path `prefix`.
// Children that are internal are appended to `pending` (b + 1 < 2 only at the
// root).
struct Pending { int b; uint64_t s, e, prefix; };

void internal_node(PpeOut &o, const std::vector<uint64_t> &Q, int b, uint64_t s, uint64_t e, uint64_t prefix,
                   std::vector<Pending> &pending, int threads) {
    std::vector<uint64_t> I = top255(Q, s, e, threads);
    for (int t = 0; t < 255; t++) {
        o.C[I[t]] = (prefix << 8) | (uint64_t)(t + 1);
        o.L[I[t]] = (uint8_t)(b + 1);
    }
    auto sub = [&](uint32_t ptr, uint64_t cs, uint64_t ce) {
        uint64_t cp = (prefix << 8) | ptr;
        if (ce - cs < 256 || b + 1 >= 2) leaf(o, b + 1, cs, ce, cp);
        else pending.push_back({b + 1, cs, ce, cp});
    };
    sub(0, s, I[0]);
    for (int t = 0; t < 254; t++) sub((uint32_t)(t + 1), I[t] + 1, I[t + 1]);
    sub(255, I[254] + 1, e);
}
}  // namespace

static void ppe_numerical(const std::vector<uint64_t> &Q, std::vector<uint64_t> &C, std::vector<uint8_t> &L,
                          int threads) {
    uint64_t nd = Q.size();
    C.assign(nd, 0);
    L.assign(nd, 0);
    PpeOut o{C, L};
    if (nd < 256) {
        leaf(o, 0, 0, nd, 0);
        return;
    }
    std::vector<Pending> level1;
    internal_node(o, Q, 0, 0, nd, 0, level1, threads);
    // level-1 internal nodes are independent: encode them in parallel
    std::vector<std::vector<Pending>> none(level1.size());
    std::atomic<size_t> cursor{0};
    int T = std::max(1, std::min<int>(threads, (int)level1.size()));
    std::vector<std::thread> th;
    for (int t = 0; t < T; t++) {
        th.emplace_back([&] {
            for (size_t i; (i = cursor.fetch_add(1)) < level1.size();) {
                const Pending &p = level1[i];
                internal_node(o, Q, p.b, p.s, p.e, p.prefix, none[i], 1);
            }
        });
    }
    for (auto &x : th) x.join();
}

// Lookup decode tables for PP-VBS, indexed by the first two code bytes
// (c1 << 8 | c2, with c2 = 0 for one-byte codes): val2 holds the value of every
// code of at most two bytes; for longer codes -- which all sit in level-2 leaves
// whose values have consecutive dictionary indices and codes 1, 2, ... after
// the two-byte pointer path -- leaf2 holds the dictionary index of the leaf's
// first value, so value = dict[leaf2[c1 c2] + rest - 1].
// ---------------------------------------------------------- Algorithm 2
// The balanced tree of the categorical encoding, in closed form: levels
// 1..B-1 are full (level b holds 255 * 256^(b-1) codes: pointer path p, slot
// i = 1..255, code p * 256 + i, in that order); the last level B takes the
// remaining values slot-major (slot i outermost, then pointer path j), which
// spreads them evenly over the last-level nodes. B = ceil(log_256(nd + 1)).
static int categorical_levels(uint64_t nd) {
    int B = 1;
    uint64_t cap = 256;  // 256^B
    while (cap < nd + 1) {
        cap <<= 8;
        B++;
    }
    return B;
}

// code and length of the value with frequency rank r (0 = most frequent)
static void categorical_code(uint64_t r, int B, uint64_t &code, uint8_t &len) {
    uint64_t before = 0, level = 255;  // codes on the levels above, codes on this level
    for (int b = 1; b < B; b++) {
        if (r < before + level) {
            const uint64_t q = r - before;
            code = (q / 255) * 256 + (q % 255) + 1;
            len = (uint8_t)b;
            return;
        }
        before += level;
        level <<= 8;
    }
    const uint64_t q = r - before, paths = 1ull << (8 * (B - 1));  // 256^(B-1) last-level nodes
    code = (q % paths) * 256 + (q / paths) + 1;
    len = (uint8_t)B;
}

static void ppe_categorical(const std::vector<int32_t> &A, const std::vector<uint64_t> &Q, Column &c) {
    const uint64_t nd = A.size();
    std::vector<uint32_t> order(nd);
    for (uint64_t i = 0; i < nd; i++) order[i] = (uint32_t)i;
    // descending frequency; A is sorted, so a stable sort keeps ties by smaller value
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return Q[x] > Q[y]; });
    const int B = nd ? categorical_levels(nd) : 1;
    c.dcode.assign(nd, 0);
    c.dlen.assign(nd, 1);
    c.rank_dict.assign(nd, 0);
    for (uint64_t r = 0; r < nd; r++) {
        categorical_code(r, B, c.dcode[order[r]], c.dlen[order[r]]);
        c.rank_dict[r] = A[order[r]];
    }
    c.categorical = true;
    c.cat_B = B;
}

static void build_decode_tables(Column &c) {
    c.val2.assign(65536, 0);
    c.leaf2.assign(65536, 0);
    c.val1.assign(256, 0);
    for (size_t i = 0; i < c.dict.size(); i++) {
        const uint64_t C = c.dcode[i];
        const int L = c.dlen[i];
        if (L == 1) {
            c.val2[(size_t)(C << 8)] = c.dict[i];
            c.val1[(size_t)C] = c.dict[i];
        } else if (L == 2) {
            c.val2[(size_t)C] = c.dict[i];
        } else if (!c.categorical) {  // Algorithm 2's longer codes decode by arithmetic instead
            const uint64_t key = C >> (8 * (L - 2));
            const uint64_t rest = C & ((1ull << (8 * (L - 2))) - 1);
            c.leaf2[(size_t)key] = (uint32_t)(i - (rest - 1));
        }
    }
}

// ------------------------------------------------------------- layouts
// Row source: code (unpadded) and length in bytes of row i.
struct RowCodes {
    std::function<void(uint64_t, uint64_t &, uint32_t &)> get;
};

static inline uint8_t code_byte(uint64_t code, uint32_t len, int j) {  // j = 1..len
    return (uint8_t)(code >> (8 * (len - (uint32_t)j)));
}

template <class Get>
static void emit_vbs(Column &c, Get get, int T) {
    const uint64_t n = c.n;
    const uint32_t nt = c.n_tiles;
    const uint64_t nwords = (uint64_t)nt * kTileWords, ngroups = (uint64_t)nt * kGroupsPerTile;
    const int K = c.K;
    c.h_dense.assign((size_t)nt * kTileRows, 0);
    for (int j = 2; j <= K; j++) {
        c.h_mask[j].assign(nwords, 0);
        c.h_off[j].assign(ngroups + 1, 0);
    }
    std::vector<std::vector<uint64_t>> hist(T, std::vector<uint64_t>(kMaxCodeBytes + 1, 0));
    // BS_1 and the masks, tile by tile
    parallel_for(nt, T, [&](uint64_t tb, uint64_t te, int t) {
        for (uint64_t tile = tb; tile < te; tile++) {
            uint8_t *dst = &c.h_dense[tile * kTileRows];
            for (uint32_t q = 0; q < (uint32_t)kTileRows; q++) {
                uint64_t row = tile * kTileRows + q;
                if (row >= n) break;
                uint64_t code; uint32_t len;
                get(row, code, len);
                dst[tile_byte_pos(q)] = code_byte(code, len, 1);
                hist[t][len]++;
                for (int j = 2; j <= (int)len; j++) c.h_mask[j][row >> 5] |= 1u << (row & 31);
            }
        }
    }, 64);
    for (int l = 0; l <= kMaxCodeBytes; l++) {
        c.len_hist[l] = 0;
        for (int t = 0; t < T; t++) c.len_hist[l] += hist[t][l];
    }
    // group offsets into BS_j and the packed deeper bytes
    for (int j = 2; j <= K; j++) {
        auto &M = c.h_mask[j];
        auto &off = c.h_off[j];
        uint64_t acc = 0;
        for (uint64_t g = 0; g < ngroups; g++) {
            off[g] = (uint32_t)acc;
            for (int w = 0; w < kGroupWords; w++) acc += (uint64_t)__builtin_popcount(M[g * kGroupWords + w]);
        }
        off[ngroups] = (uint32_t)acc;
        c.deep_len[j] = acc;
        c.h_deep[j].assign(acc + 16, 0);
    }
    if (K >= 2) {
        parallel_for(ngroups, T, [&](uint64_t gb, uint64_t ge, int) {
            for (uint64_t g = gb; g < ge; g++) {
                uint64_t pos[kMaxCodeBytes + 1];
                for (int j = 2; j <= K; j++) pos[j] = c.h_off[j][g];
                for (uint64_t row = g * kGroupRows; row < std::min<uint64_t>(n, (g + 1) * kGroupRows); row++) {
                    uint64_t code; uint32_t len;
                    get(row, code, len);
                    for (int j = 2; j <= (int)len; j++) c.h_deep[j][pos[j]++] = code_byte(code, len, j);
                }
            }
        }, 256);
    }
}

template <class Get>
static void emit_byteslice(Column &c, Get get, int T) {
    const uint64_t sb = c.dense_slice_bytes();
    const int S = c.S, k = c.k;
    c.h_dense.assign((size_t)S * sb, 0);
    parallel_for(c.n_tiles, T, [&](uint64_t tb, uint64_t te, int) {
        for (uint64_t tile = tb; tile < te; tile++) {
            for (uint32_t q = 0; q < (uint32_t)kTileRows; q++) {
                uint64_t row = tile * kTileRows + q;
                if (row >= c.n) break;
                uint64_t code = get(row);
                uint64_t aligned = code << (8 * S - k);
                for (int s = 1; s <= S; s++)
                    c.h_dense[(uint64_t)(s - 1) * sb + tile * kTileRows + tile_byte_pos(q)] =
                        (uint8_t)(aligned >> (8 * (S - s)));
            }
        }
    }, 64);
    c.len_hist[S] = c.n;
}

template <class Get>
static void emit_bitpacked(Column &c, Get get, int T) {
    const int k = c.k;
    c.h_packed.assign(c.packed_words(), 0);
    // 32 consecutive codes fill exactly k words: chunk q owns words [q*k, q*k + k)
    uint64_t nchunks = (uint64_t)c.n_tiles * kTileWords;
    parallel_for(nchunks, T, [&](uint64_t qb, uint64_t qe, int) {
        for (uint64_t q = qb; q < qe; q++) {
            uint32_t *w = &c.h_packed[q * (uint64_t)k];
            for (uint32_t r = 0; r < 32; r++) {
                uint64_t row = q * 32 + r;
                if (row >= c.n) break;
                uint64_t code = get(row);
                uint64_t bit = (uint64_t)r * (uint64_t)k;
                uint64_t wi = bit >> 5;
                uint32_t sh = (uint32_t)(bit & 31);
                w[wi] |= (uint32_t)(code << sh);
                if (sh + (uint32_t)k > 32) w[wi + 1] |= (uint32_t)(code >> (32 - sh));
            }
        }
    }, 1024);
    c.len_hist[(k + 7) / 8] = c.n;
}

// Declared dictionary with counts: A sorted, Q permuted alongside, and every
// row's index in A (INVALID_ARG for an undeclared value or a repeated one).
static int declared_dictionary(const int32_t *v, uint64_t n, int T, const bs_encode_opts &o,
                               std::vector<int32_t> &A, std::vector<uint64_t> &Q, std::vector<uint32_t> &ridx) {
    if (!o.domain_values || o.n_domain == 0 || o.n_domain > (1ull << 32)) return BS_ERR_INVALID_ARG;
    std::vector<uint32_t> order(o.n_domain);
    for (uint64_t i = 0; i < o.n_domain; i++) order[i] = (uint32_t)i;
    std::sort(order.begin(), order.end(),
              [&](uint32_t a, uint32_t b) { return o.domain_values[a] < o.domain_values[b]; });
    A.resize(o.n_domain);
    Q.resize(o.n_domain);
    for (uint64_t i = 0; i < o.n_domain; i++) {
        A[i] = o.domain_values[order[i]];
        Q[i] = o.domain_counts[order[i]];
        if (i && A[i] == A[i - 1]) return BS_ERR_INVALID_ARG;
    }
    ridx.assign(n, 0);
    std::atomic<bool> bad{false};
    parallel_for(n, T, [&](uint64_t b, uint64_t e, int) {
        for (uint64_t i = b; i < e; i++) {
            auto it = std::lower_bound(A.begin(), A.end(), v[i]);
            if (it == A.end() || *it != v[i]) { bad = true; return; }
            ridx[i] = (uint32_t)(it - A.begin());
        }
    });
    return bad ? BS_ERR_INVALID_ARG : BS_OK;
}

// Q[i] = rows of this column whose value is A[i].
static void count_rows(const std::vector<uint32_t> &ridx, size_t nd, int T, std::vector<uint64_t> &Q) {
    Q.assign(nd, 0);
    const uint64_t n = ridx.size();
    const uint64_t tt = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)T, (n >> 16) + 1));
    if (tt == 1 || (uint64_t)nd * tt * 8 > (1ull << 30)) {
        for (uint32_t i : ridx) Q[i]++;
        return;
    }
    std::vector<std::vector<uint64_t>> part(tt);
    parallel_for(n, (int)tt, [&](uint64_t b, uint64_t e, int t) {
        part[t].assign(nd, 0);
        for (uint64_t i = b; i < e; i++) part[t][ridx[i]]++;
    }, 1);
    for (auto &h : part)
        for (size_t i = 0; i < h.size(); i++) Q[i] += h[i];
}

static int code_bits_for(uint64_t count) {  // max(1, ceil(log2(count)))
    int k = 0;
    while (k < 63 && (1ull << k) < count) k++;
    return std::max(1, k);
}

// ---------------------------------------------------------------- entry
int encode_values(const int32_t *values, uint64_t n, bs_layout layout, const bs_encode_opts &o, Column &c) {
    if (n >= (1ull << 32)) return BS_ERR_INVALID_ARG;
    if (n && !values) return BS_ERR_INVALID_ARG;
    const int T = resolve_threads(o.threads);
    c.layout = layout;
    c.n = n;
    c.n_tiles = (uint32_t)((n + kTileRows - 1) / kTileRows);
    c.raw = false;
    try {
        if (layout == BS_PPVBS) {
            std::vector<uint64_t> Q;
            std::vector<uint32_t> ridx;
            if (o.domain_counts) {
                // codes from the declared dictionary's counts (a row shard of a
                // larger column); Q below is then recounted over this column's rows
                int rc = declared_dictionary(values, n, T, o, c.dict, Q, ridx);
                if (rc) return rc;
            } else {
                int rc = build_dictionary(values, n, T, c.dict, Q, ridx);
                if (rc) return rc;
            }
            if (o.categorical) ppe_categorical(c.dict, Q, c);
            else ppe_numerical(Q, c.dcode, c.dlen, T);
            if (o.domain_counts) count_rows(ridx, c.dict.size(), T, Q);
            c.dcount = Q;
            c.dcum.assign(Q.size() + 1, 0);
            for (size_t i = 0; i < Q.size(); i++) c.dcum[i + 1] = c.dcum[i] + Q[i];
            build_decode_tables(c);
            c.first_byte_rows.assign(256, 0);
            for (size_t i = 0; i < Q.size(); i++)
                c.first_byte_rows[(size_t)((c.dcode[i] >> (8 * (c.dlen[i] - 1))) & 0xFF)] += Q[i];
            c.K = 1;
            for (uint8_t l : c.dlen) c.K = std::max<int>(c.K, l);
            const uint64_t *dc = c.dcode.data();
            const uint8_t *dl = c.dlen.data();
            const uint32_t *ri = ridx.data();
            emit_vbs(c, [=](uint64_t row, uint64_t &code, uint32_t &len) {
                uint32_t i = ri[row];
                code = dc[i];
                len = dl[i];
            }, T);
            return BS_OK;
        }
        if (layout != BS_BYTESLICE && layout != BS_BITPACKED) return BS_ERR_INVALID_ARG;
        std::vector<uint32_t> ridx;
        const uint32_t *ri = nullptr;
        if (o.domain_bits > 0) {
            if (o.domain_bits > 32) return BS_ERR_INVALID_ARG;
            c.identity = true;
            c.k = o.domain_bits;
            c.domain_min = o.domain_min;
            const int64_t lim = (int64_t)(1ull << c.k);
            std::atomic<bool> bad{false};
            parallel_for(n, T, [&](uint64_t b, uint64_t e, int) {
                for (uint64_t i = b; i < e; i++) {
                    int64_t d = (int64_t)values[i] - c.domain_min;
                    if (d < 0 || d >= lim) { bad = true; return; }
                }
            });
            if (bad) return BS_ERR_INVALID_ARG;
        } else {
            c.identity = false;
            if (o.domain_values && o.n_domain) {
                c.dict.assign(o.domain_values, o.domain_values + o.n_domain);
                std::sort(c.dict.begin(), c.dict.end());
                c.dict.erase(std::unique(c.dict.begin(), c.dict.end()), c.dict.end());
                ridx.assign(n, 0);
                std::atomic<bool> bad{false};
                parallel_for(n, T, [&](uint64_t b, uint64_t e, int) {
                    for (uint64_t i = b; i < e; i++) {
                        auto it = std::lower_bound(c.dict.begin(), c.dict.end(), values[i]);
                        if (it == c.dict.end() || *it != values[i]) { bad = true; return; }
                        ridx[i] = (uint32_t)(it - c.dict.begin());
                    }
                });
                if (bad) return BS_ERR_INVALID_ARG;
            } else {
                std::vector<uint64_t> Q;
                int rc = build_dictionary(values, n, T, c.dict, Q, ridx);
                if (rc) return rc;
                c.dcount = Q;
                c.dcum.assign(Q.size() + 1, 0);
                for (size_t i = 0; i < Q.size(); i++) c.dcum[i + 1] = c.dcum[i] + Q[i];
            }
            c.k = code_bits_for(c.dict.size());
            ri = ridx.data();
        }
        c.S = (c.k + 7) / 8;
        c.K = c.S;
        const bool idn = c.identity;
        const int64_t dmin = c.domain_min;
        auto get = [=](uint64_t row) -> uint64_t {
            return idn ? (uint64_t)((int64_t)values[row] - dmin) : (uint64_t)ri[row];
        };
        if (layout == BS_BYTESLICE) emit_byteslice(c, get, T);
        else emit_bitpacked(c, get, T);
        return BS_OK;
    } catch (const std::bad_alloc &) {
        return BS_ERR_OOM;
    }
}

int encode_raw(const uint64_t *codes, const uint8_t *lens, uint64_t n, bs_layout layout, int code_bits,
               const bs_encode_opts &o, Column &c) {
    if (n >= (1ull << 32) || (n && !codes)) return BS_ERR_INVALID_ARG;
    const int T = resolve_threads(o.threads);
    c.layout = layout;
    c.n = n;
    c.n_tiles = (uint32_t)((n + kTileRows - 1) / kTileRows);
    c.raw = true;
    try {
        if (layout == BS_PPVBS) {
            if (n && !lens) return BS_ERR_INVALID_ARG;
            c.K = 1;
            for (uint64_t i = 0; i < n; i++) {
                if (lens[i] < 1 || lens[i] > kMaxCodeBytes) return BS_ERR_INVALID_ARG;
                if (lens[i] < 8 && (codes[i] >> (8 * lens[i]))) return BS_ERR_INVALID_ARG;
                c.K = std::max<int>(c.K, lens[i]);
            }
            emit_vbs(c, [=](uint64_t row, uint64_t &code, uint32_t &len) {
                code = codes[row];
                len = lens[row];
            }, T);
            return BS_OK;
        }
        if (layout != BS_BYTESLICE && layout != BS_BITPACKED) return BS_ERR_INVALID_ARG;
        if (code_bits < 1 || code_bits > 32) return BS_ERR_INVALID_ARG;
        for (uint64_t i = 0; i < n; i++)
            if (code_bits < 64 && (codes[i] >> code_bits)) return BS_ERR_INVALID_ARG;
        c.k = code_bits;
        c.S = (c.k + 7) / 8;
        c.K = c.S;
        c.identity = true;
        auto get = [=](uint64_t row) -> uint64_t { return codes[row]; };
        if (layout == BS_BYTESLICE) emit_byteslice(c, get, T);
        else emit_bitpacked(c, get, T);
        return BS_OK;
    } catch (const std::bad_alloc &) {
        return BS_ERR_OOM;
    }
}

// ------------------------------------------------------- literal rewrite
// The code space is order-isomorphic to the sorted value list (dictionary or
// declared range), so every predicate on a value literal becomes a predicate on
// a present code (or a constant result). u = first position whose value >= x.
namespace {
struct CodeSpace {
    const Column &c;
    uint64_t size() const {
        if (c.identity) return 1ull << c.k;
        return c.dict.size();
    }
    uint64_t lower_bound(int64_t x) const {
        if (c.identity) {
            int64_t d = x - c.domain_min;
            if (d < 0) return 0;
            return std::min<uint64_t>((uint64_t)d, size());
        }
        return (uint64_t)(std::lower_bound(c.dict.begin(), c.dict.end(), (int32_t)x) - c.dict.begin());
    }
    int64_t value(uint64_t u) const { return c.identity ? (int64_t)u + c.domain_min : (int64_t)c.dict[u]; }
    LitCode code(uint64_t u) const {
        LitCode l{};
        if (c.layout == BS_PPVBS) {
            l.code = c.dcode[u];
            l.len = c.dlen[u];
        } else {
            l.code = u;
            l.len = (uint32_t)c.S;
        }
        return l;
    }
};
}  // namespace

int rewrite_literal(const Column &c, int op, int32_t lit, int32_t lit2, KPred &out) {
    out = KPred{};
    out.mode = Pred::kNormal;
    if (c.raw) return BS_ERR_UNSUPPORTED;
    // Algorithm 2's codes do not follow value order: equality predicates only
    if (c.categorical && op != BS_EQ && op != BS_NE) return BS_ERR_UNSUPPORTED;
    CodeSpace cs{c};
    const uint64_t N = cs.size();
    auto set = [&](int kop, uint64_t u) { out.op = kop; out.lit[0] = cs.code(u); };
    if (op == BS_BETWEEN) {
        if (lit > lit2 || N == 0) { out.mode = Pred::kNone; return BS_OK; }
        uint64_t lo = cs.lower_bound(lit);
        uint64_t hi_ex = cs.lower_bound((int64_t)lit2 + 1);  // first value > lit2
        if (lo >= N || hi_ex == 0 || lo >= hi_ex) { out.mode = Pred::kNone; return BS_OK; }
        out.op = BS_BETWEEN;
        out.lit[0] = cs.code(lo);
        out.lit[1] = cs.code(hi_ex - 1);
        return BS_OK;
    }
    if (N == 0) { out.mode = (op == BS_NE || op == BS_LT || op == BS_LE) ? Pred::kAll : Pred::kNone;
                  if (c.n == 0) out.mode = Pred::kNone; return BS_OK; }
    uint64_t u = cs.lower_bound(lit);
    bool exact = u < N && cs.value(u) == (int64_t)lit;
    switch (op) {
    case BS_LT:
        if (u >= N) out.mode = Pred::kAll; else set(BS_LT, u);
        break;
    case BS_LE:
        if (exact) set(BS_LE, u);
        else if (u >= N) out.mode = Pred::kAll;
        else set(BS_LT, u);
        break;
    case BS_GT:
        if (exact) set(BS_GT, u);
        else if (u >= N) out.mode = Pred::kNone;
        else set(BS_GE, u);
        break;
    case BS_GE:
        if (u >= N) out.mode = Pred::kNone; else set(BS_GE, u);
        break;
    case BS_EQ:
        if (exact) set(BS_EQ, u); else out.mode = Pred::kNone;
        break;
    case BS_NE:
        if (exact) set(BS_NE, u); else out.mode = Pred::kAll;
        break;
    default:
        return BS_ERR_INVALID_ARG;
    }
    return BS_OK;
}

int make_code_pred(const Column &c, int op, uint64_t code, int len, uint64_t code2, int len2, KPred &out) {
    out = KPred{};
    out.mode = Pred::kNormal;
    if (op < BS_LT || op > BS_BETWEEN) return BS_ERR_INVALID_ARG;
    out.op = op;
    auto mk = [&](uint64_t cd, int ln, LitCode &l) -> int {
        if (c.layout == BS_PPVBS) {
            if (ln < 1 || ln > kMaxCodeBytes) return BS_ERR_INVALID_ARG;
            if (ln < 8 && (cd >> (8 * ln))) return BS_ERR_INVALID_ARG;
            l.code = cd;
            l.len = (uint32_t)ln;
        } else {
            if (c.k < 64 && (cd >> c.k)) return BS_ERR_INVALID_ARG;
            l.code = cd;
            l.len = (uint32_t)c.S;
        }
        return BS_OK;
    };
    int rc = mk(code, len, out.lit[0]);
    if (rc) return rc;
    if (op == BS_BETWEEN) {
        rc = mk(code2, len2, out.lit[1]);
        if (rc) return rc;
    }
    return BS_OK;
}

}  // namespace bs

namespace bs {

// Rows whose value satisfies (op, lit, lit2), from the dictionary counts when
// the column has them (else every row).
uint64_t estimate_rows(const Column &c, int op, int32_t lit, int32_t lit2) {
    if (c.dcum.size() != c.dict.size() + 1 || c.dict.empty()) return c.n;
    auto below = [&](int64_t x) -> uint64_t {  // rows with value < x
        if (x > INT32_MAX) return c.n;
        if (x <= INT32_MIN) return 0;
        const size_t u = (size_t)(std::lower_bound(c.dict.begin(), c.dict.end(), (int32_t)x) - c.dict.begin());
        return c.dcum[u];
    };
    const int64_t x = lit, y = lit2;
    switch (op) {
    case BS_LT: return below(x);
    case BS_LE: return below(x + 1);
    case BS_GT: return c.n - below(x + 1);
    case BS_GE: return c.n - below(x);
    case BS_EQ: return below(x + 1) - below(x);
    case BS_NE: return c.n - (below(x + 1) - below(x));
    default: return x > y ? 0 : below(y + 1) - below(x);
    }
}

}  // namespace bs
