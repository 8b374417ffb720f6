// Effective-bytes counter: the bytes a scan or lookup must move, replayed on
// the host from the column's host copy at the granularity the kernels read
// (32-byte DRAM sectors, 256-row mask groups, 1024-row tiles). It is the
// numerator of the roofline fraction and the cost of the layout advisor's
// deterministic mode.
//
// Scan (per tile, in the kernel's order): every lane with a valid (seeded) row
// reads its 32 bytes of the dense slice; for PP-VBS, a row still equal to the
// literal after byte j-1 makes its 256-row group read the M_j sector, and a row
// that has byte j with j <= l makes its group read its off_j entry and the
// BS_j sector holding that byte; ByteSlice lanes with pending rows read their
// 32 bytes of the next slice. Results are written as 4-byte words; seeds are
// read as 4-byte words. Distinct sectors are counted once.
#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "bs_internal.h"

namespace bs {
namespace {

struct SectorRun {  // distinct 32-byte sectors of a non-decreasing address stream
    uint64_t count = 0, first = ~0ull, last = ~0ull;
    void add(uint64_t byte_addr) {
        const uint64_t s = byte_addr >> 5;
        if (s == last) return;
        if (first == ~0ull) first = s;
        last = s;
        count++;
    }
};

// merge per-chunk runs in chunk order (a sector may straddle two chunks)
uint64_t merge_runs(const std::vector<SectorRun> &runs) {
    uint64_t total = 0, prev_last = ~0ull;
    for (const auto &r : runs) {
        if (!r.count) continue;
        total += r.count;
        if (r.first == prev_last) total--;
        prev_last = r.last;
    }
    return total;
}

struct Lit {
    int len = 0;
    uint8_t b[kMaxCodeBytes + 1] = {0};  // 1-based
};

Lit to_lit(const LitCode &l) {
    Lit o;
    o.len = (int)l.len;
    for (int j = 1; j <= o.len; j++) o.b[j] = (uint8_t)(l.code >> (8 * (o.len - j)));
    return o;
}

struct Acc {
    uint64_t dense = 0, mask = 0, deep = 0, off = 0, paper = 0;
    uint64_t pending[kMaxCodeBytes + 2] = {0};
    SectorRun deep_run[kMaxCodeBytes + 1], off_run[kMaxCodeBytes + 1];
};

// Resolve one row against one literal: the deepest level that still needs the
// row's mask bit (pend_to) and the deepest level whose byte is read (byte_to).
// Levels are 1-based; 1 means only BS_1 was needed.
// need_eq: the predicate distinguishes "equal" from "larger" for this literal
// (otherwise rows equal after the literal's last byte are never read again).
void replay_row(const uint8_t *code, int L, const Lit &lit, int K, bool need_eq, int &pend_to, int &byte_to) {
    pend_to = 1;
    byte_to = 1;
    if (code[1] != lit.b[1]) return;
    const int jend = need_eq ? std::min(lit.len + 1, K) : std::min(lit.len, K);
    for (int j = 2; j <= jend; j++) {
        pend_to = j;                       // mask M_j consulted
        if (L < j) return;                 // row ended: decided
        if (j > lit.len) return;           // literal ended, row continues: decided
        byte_to = j;                       // byte j compared
        if (code[j] != lit.b[j]) return;
    }
}

}  // namespace

// sel (fused scan + lookup on the same column): the predicate's result; the
// rows it selects also have every byte of their code read, with the M_j sector
// and off_j entry of each level they reach (as the lookup reads them), and 4
// output bytes each; write_bits: the result bit vector is written (else it is
// not counted).
int scan_bytes_impl(const Column &c, const KPred &p, const uint32_t *seed, uint64_t tile_stride, const uint32_t *sel,
                    bool write_bits, bs_scan_bytes_t *out) {
    std::memset(out, 0, sizeof *out);
    const uint64_t n = c.n;
    const uint64_t nwords = (n + 31) / 32;
    if (n == 0) return BS_OK;
    if (!c.has_host) return BS_ERR_UNSUPPORTED;
    if (tile_stride == 0) tile_stride = 1;
    const uint64_t nt = c.n_tiles;
    const uint64_t sampled = (nt + tile_stride - 1) / tile_stride;
    const double scale = (double)nt / (double)sampled;
    uint64_t selected = 0;
    if (sel)
        for (uint64_t w = 0; w < nwords; w++) {
            const uint32_t v = (w == nwords - 1 && (n & 31)) ? ((1u << (n & 31)) - 1u) : 0xFFFFFFFFu;
            selected += (uint64_t)__builtin_popcount(sel[w] & v);
        }
    out->result_bytes = (write_bits ? 4 * nwords : 0) + (seed ? 4 * nwords : 0) + 4 * selected;
    if (p.mode != Pred::kNormal) {
        if (sel && selected) return BS_ERR_UNSUPPORTED;  // constant predicates: not replayed for lookups
        out->bytes = out->result_bytes;
        out->paper_model_bytes = out->result_bytes;
        return BS_OK;
    }
    if (c.layout == BS_BITPACKED) {
        // no early stop: every round with a seeded row reads its k words
        uint64_t words = 0;
        for (uint64_t w = 0; w < nwords; w++) {
            uint32_t v = (w == nwords - 1 && (n & 31)) ? ((1u << (n & 31)) - 1u) : 0xFFFFFFFFu;
            if (seed) v &= seed[w];
            if (v) words += (uint64_t)c.k;
        }
        out->dense_bytes = 4 * words;
        out->bytes = out->dense_bytes + out->result_bytes;
        out->paper_model_bytes = (n * (uint64_t)c.k + 7) / 8 + (n + 7) / 8;
        return BS_OK;
    }
    const int nlit = p.op == BS_BETWEEN ? 2 : 1;
    Lit lits[2];
    for (int i = 0; i < nlit; i++) {
        LitCode l = p.lit[i];
        if (c.layout == BS_BYTESLICE) {
            l.code <<= (8 * c.S - c.k);
            l.len = (uint32_t)c.S;
        }
        lits[i] = to_lit(l);
    }
    const int K = c.layout == BS_PPVBS ? c.K : c.S;
    const uint64_t slice = c.dense_slice_bytes();
    int T = resolve_threads(0);
    T = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)T, sampled / 64 + 1));
    std::vector<Acc> acc(T);
    auto work = [&](int ti) {
        Acc &A = acc[ti];
        const uint64_t sb = sampled * (uint64_t)ti / T, se = sampled * (uint64_t)(ti + 1) / T;
        uint8_t code[kMaxCodeBytes + 2];
        for (uint64_t si = sb; si < se; si++) {
            const uint64_t t = si * tile_stride;
            bool lane_active[32] = {false};
            bool lane_pend[kMaxCodeBytes + 2][32];
            bool grp_pend[kMaxCodeBytes + 2][4], grp_byte[kMaxCodeBytes + 2][4];
            std::memset(lane_pend, 0, sizeof lane_pend);
            std::memset(grp_pend, 0, sizeof grp_pend);
            std::memset(grp_byte, 0, sizeof grp_byte);
            // cursors into BS_j for the first row of the tile
            uint64_t cur[kMaxCodeBytes + 1] = {0};
            if (c.layout == BS_PPVBS)
                for (int j = 2; j <= K; j++) cur[j] = c.h_off[j][t * kGroupsPerTile];
            int block_stop[32] = {0};
            for (uint32_t q = 0; q < (uint32_t)kTileRows; q++) {
                const uint64_t row = t * kTileRows + q;
                if (row >= n) break;
                const uint32_t lane = q >> 5, g = q >> 8;
                const uint64_t w = row >> 5;
                const bool on = !seed || ((seed[w] >> (row & 31)) & 1u);
                // the row's code (the cursors advance whether or not it is scanned)
                int L = 1;
                const uint64_t pos1 = t * kTileRows + tile_byte_pos(q);
                code[1] = c.h_dense[pos1];
                uint64_t byte_addr[kMaxCodeBytes + 1] = {0};
                if (c.layout == BS_PPVBS) {
                    for (int j = 2; j <= K; j++) {
                        if (!((c.h_mask[j][w] >> (row & 31)) & 1u)) break;
                        byte_addr[j] = cur[j];
                        code[j] = c.h_deep[j][cur[j]++];
                        L = j;
                    }
                } else {
                    for (int s = 2; s <= K; s++) code[s] = c.h_dense[(uint64_t)(s - 1) * slice + pos1];
                    L = K;
                }
                if (!on) continue;
                lane_active[lane] = true;
                const bool picked = sel && ((sel[w] >> (row & 31)) & 1u);
                int pend_to = 1, byte_to = 1;
                for (int i = 0; i < nlit; i++) {
                    int pt, bt;
                    if (c.layout == BS_PPVBS) {
                        const bool need_eq = i == 1 || !(p.op == BS_LT || p.op == BS_GE || p.op == BS_BETWEEN);
                        replay_row(code, L, lits[i], K, need_eq, pt, bt);
                    } else {
                        pt = 1;
                        for (int s = 1; s <= K; s++) {
                            pt = s;
                            if (code[s] != lits[i].b[s]) break;
                        }
                        bt = pt;
                    }
                    pend_to = std::max(pend_to, pt);
                    byte_to = std::max(byte_to, bt);
                }
                for (int j = 2; j <= pend_to; j++) {
                    A.pending[j]++;
                    lane_pend[j][lane] = true;
                    grp_pend[j][g] = true;
                }
                block_stop[lane] = std::max(block_stop[lane], pend_to);
                if (picked) {
                    // the lookup of a selected row: every byte of its code
                    for (int j = 2; j <= std::min(L + 1, K); j++) {
                        grp_pend[j][g] = true;
                        grp_byte[j][g] = true;
                    }
                }
                if (c.layout == BS_PPVBS) {
                    const int read_to = picked ? std::max(byte_to, L) : byte_to;
                    for (int j = 2; j <= read_to; j++) {
                        grp_byte[j][g] = true;
                        A.deep_run[j].add(byte_addr[j]);
                    }
                }
            }
            // dense slice 1: lanes (2m, 2m+1) share sectors m and 16 + m of the tile
            for (int m = 0; m < 16; m++)
                if (lane_active[2 * m] || lane_active[2 * m + 1]) A.dense += 64;
            if (c.layout == BS_BYTESLICE) {
                for (int s = 2; s <= K; s++)
                    for (int m = 0; m < 16; m++)
                        if (lane_pend[s][2 * m] || lane_pend[s][2 * m + 1]) A.dense += 64;
            } else {
                for (int j = 2; j <= K; j++) {
                    for (int g = 0; g < 4; g++) {
                        if (grp_pend[j][g]) A.mask += 32;
                        if (grp_byte[j][g]) A.off_run[j].add((t * kGroupsPerTile + g) * 4);
                    }
                }
                // Algorithm 3 as printed: masks of levels 2..min(l+1,K) for every block,
                // a 32-byte SIMD load of BS_j for every block that reaches level j
                const int lmax = std::max(lits[0].len, nlit == 2 ? lits[1].len : 0);
                const int eager = std::max(0, std::min(lmax + 1, K) - 1);
                for (int lane = 0; lane < 32; lane++) {
                    if (t * kTileRows + (uint64_t)lane * 32 >= n) break;
                    A.paper += 32 + 4 + 4 * (uint64_t)eager;
                    for (int j = 2; j <= std::min(block_stop[lane], lmax); j++) A.paper += 32;
                }
            }
        }
    };
    std::vector<std::thread> th;
    for (int i = 1; i < T; i++) th.emplace_back(work, i);
    work(0);
    for (auto &x : th) x.join();
    uint64_t dense = 0, mask = 0, paper = 0;
    for (auto &A : acc) {
        dense += A.dense;
        mask += A.mask;
        paper += A.paper;
        for (int j = 0; j <= kMaxCodeBytes + 1 && j < 9; j++) out->pending_rows[j] += A.pending[j];
    }
    uint64_t deep = 0, off = 0;
    for (int j = 2; j <= kMaxCodeBytes; j++) {
        std::vector<SectorRun> dr, orr;
        for (auto &A : acc) { dr.push_back(A.deep_run[j]); orr.push_back(A.off_run[j]); }
        deep += merge_runs(dr) * 32;
        off += merge_runs(orr) * 32;
    }
    out->dense_bytes = (uint64_t)(dense * scale);
    out->mask_bytes = (uint64_t)(mask * scale);
    out->deep_bytes = (uint64_t)(deep * scale);
    out->offset_bytes = (uint64_t)(off * scale);
    for (int j = 0; j < 9; j++) out->pending_rows[j] = (uint64_t)(out->pending_rows[j] * scale);
    out->bytes = out->dense_bytes + out->mask_bytes + out->deep_bytes + out->offset_bytes + out->result_bytes;
    out->paper_model_bytes = c.layout == BS_PPVBS ? (uint64_t)(paper * scale) + 4 * nwords : out->bytes;
    out->sampled_tiles = sampled;
    return BS_OK;
}

int scan_bytes(const Column &c, const KPred &p, const uint32_t *seed, uint64_t tile_stride, bs_scan_bytes_t *out) {
    return scan_bytes_impl(c, p, seed, tile_stride, nullptr, true, out);
}

int scan_lookup_bytes(const Column &c, const KPred &p, const uint32_t *sel, bool write_bits, bs_scan_bytes_t *out) {
    if (!sel && c.n) return BS_ERR_INVALID_ARG;
    // ByteSlice lookups read single sectors of the deeper slices, which the
    // scan's lane-pair accounting does not express: not counted here
    if (c.layout == BS_BYTESLICE) return BS_ERR_UNSUPPORTED;
    return scan_bytes_impl(c, p, nullptr, 1, sel, write_bits, out);
}

// Lookup: the bit vector once, the output values, and the distinct sectors of
// every byte gathered (dense slice, mask groups reached, offsets, BS_j bytes).
int lookup_bytes(const Column &c, const uint32_t *bits, bs_lookup_bytes_t *out) {
    std::memset(out, 0, sizeof *out);
    const uint64_t n = c.n, nwords = (n + 31) / 32;
    if (!c.has_host) return BS_ERR_UNSUPPORTED;
    SectorRun dense[kMaxCodeBytes + 1], deep[kMaxCodeBytes + 1], off[kMaxCodeBytes + 1];
    uint64_t m = 0, mask = 0;
    const uint64_t slice = c.dense_slice_bytes();
    std::vector<uint64_t> dense_sectors;
    for (uint64_t t = 0; t < c.n_tiles; t++) {
        uint64_t cur[kMaxCodeBytes + 1] = {0};
        if (c.layout == BS_PPVBS)
            for (int j = 2; j <= c.K; j++) cur[j] = c.h_off[j][t * kGroupsPerTile];
        bool grp[kMaxCodeBytes + 1][4] = {{false}};
        std::vector<uint64_t> tile_dense;
        for (uint32_t q = 0; q < (uint32_t)kTileRows; q++) {
            const uint64_t row = t * kTileRows + q;
            if (row >= n) break;
            const uint64_t w = row >> 5;
            const bool sel = (bits[w] >> (row & 31)) & 1u;
            const uint64_t pos1 = t * kTileRows + tile_byte_pos(q);
            if (c.layout == BS_PPVBS) {
                int L = 1;
                uint64_t addr[kMaxCodeBytes + 1];
                for (int j = 2; j <= c.K; j++) {
                    if (!((c.h_mask[j][w] >> (row & 31)) & 1u)) break;
                    addr[j] = cur[j]++;
                    L = j;
                }
                if (!sel) continue;
                m++;
                tile_dense.push_back(pos1 >> 5);
                for (int j = 2; j <= std::min(L + 1, c.K); j++) grp[j][q >> 8] = true;
                for (int j = 2; j <= L; j++) deep[j].add(addr[j]);
            } else if (c.layout == BS_BYTESLICE) {
                if (!sel) continue;
                m++;
                for (int s = 0; s < c.S; s++) tile_dense.push_back(((uint64_t)s * slice + pos1) >> 5);
            } else {
                if (!sel) continue;
                m++;
                const uint64_t b0 = row * (uint64_t)c.k, b1 = b0 + (uint64_t)c.k - 1;
                dense[0].add(b0 >> 3);
                dense[0].add(b1 >> 3);
            }
        }
        std::sort(tile_dense.begin(), tile_dense.end());
        tile_dense.erase(std::unique(tile_dense.begin(), tile_dense.end()), tile_dense.end());
        out->dense_bytes += 32 * (uint64_t)tile_dense.size();
        if (c.layout == BS_PPVBS)
            for (int j = 2; j <= c.K; j++)
                for (int g = 0; g < 4; g++)
                    if (grp[j][g]) {
                        mask += 32;
                        off[j].add((t * kGroupsPerTile + g) * 4);
                    }
    }
    out->dense_bytes += 32 * dense[0].count;
    uint64_t d = 0, o = 0;
    for (int j = 2; j <= kMaxCodeBytes; j++) {
        d += 32 * deep[j].count;
        o += 32 * off[j].count;
    }
    out->selected = m;
    out->bits_bytes = 4 * nwords;
    out->out_bytes = 4 * m;
    out->mask_bytes = mask;
    out->deep_bytes = d;
    out->offset_bytes = o;
    out->bytes = out->bits_bytes + out->out_bytes + out->dense_bytes + mask + d + o;
    return BS_OK;
}

}  // namespace bs
