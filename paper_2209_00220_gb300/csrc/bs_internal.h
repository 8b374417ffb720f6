// Internal definitions of libbytestore (not part of the C ABI).
//
// Device layout of a column (all sub-buffers of one cudaMalloc arena):
//   * Rows are processed in tiles of 1024 rows (one warp per tile). Every dense
//     byte slice -- BS_1 of PP-VBS and each ByteSlice slice -- is stored tile by
//     tile with a fixed permutation inside the tile: lane L of the warp owns rows
//     32L..32L+31 of the tile and reads them as two 16-byte loads at tile offsets
//     16L and 512 + 16L, so both loads of the warp are fully coalesced. Inside the
//     lane's 32 bytes, 32-bit word w (0..7) byte b holds row 8b + w, so the most-
//     significant bits of a per-byte SWAR compare mask gather into a row-ordered
//     32-bit result word with shifts alone (word w shifted right by 7 - w).
//   * PP-VBS bitmasks M_j (j >= 2) are plain row-ordered uint32 words (bit i of
//     word w = row 32w + i), as in Section 3.2.
//   * PP-VBS deeper slices BS_j (j >= 2) are packed in row order exactly as in
//     Section 3.2. Algorithm 3 tracks its position in BS_j with a running index
//     I_j; on the GPU every 256-row group (8 mask words, one 32-byte sector)
//     instead stores off_j[g] = number of BS_j bytes before the group, so any
//     tile finds its bytes without a sequential pass.
//   * Bit-Packed is the plain little-endian bit stream of Section 2.3 in uint32
//     words, padded with zero words.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bytestore.h"

namespace bs {

constexpr int kTileRows = 1024;
constexpr int kTileWords = 32;
constexpr int kGroupRows = 256;
constexpr int kGroupWords = 8;
constexpr int kGroupsPerTile = 4;
constexpr int kMaxCodeBytes = 8;     // raw-code columns; Algorithm 1 yields <= 6

// Byte offset, inside its tile, of the byte of tile-local row q (0..1023).
inline uint32_t tile_byte_pos(uint32_t q) {
    uint32_t lane = q >> 5, r = q & 31u, b = r >> 3, w = r & 7u;
    return (w >> 2) * 512u + lane * 16u + (w & 3u) * 4u + b;
}

enum class Pred : int32_t { kNormal = 0, kAll = 1, kNone = 2 };

// A literal code as the kernels see it.
struct LitCode {
    uint32_t len;       // bytes (PP-VBS: 1..8; ByteSlice: S)
    uint32_t pad_;
    uint64_t code;      // unpadded code, first byte most significant
};

// A predicate after literal rewriting: mode kAll/kNone short-circuit.
struct KPred {
    Pred mode;
    int32_t op;         // bs_op on codes
    LitCode lit[2];
};

struct Column {
    bs_layout layout = BS_PPVBS;
    uint64_t n = 0;
    uint32_t n_tiles = 0;
    int device = 0;
    bool raw = false;           // built from raw codes, no dictionary

    // code mapping
    bool identity = false;      // code = value - domain_min over [0, 2^k)
    int64_t domain_min = 0;
    int k = 0;                  // ByteSlice / Bit-Packed code bits
    int S = 0;                  // ByteSlice slices
    int K = 1;                  // PP-VBS longest code in bytes
    bool categorical = false;   // PP-VBS codes by Algorithm 2 (= and != only)
    int cat_B = 0;              // Algorithm 2: levels of the balanced tree
    std::vector<int32_t> rank_dict;  // Algorithm 2: values in code-assignment (frequency) order
    std::vector<int32_t> dict;  // sorted distinct values (dictionary)
    std::vector<uint64_t> dcode;  // PP-VBS: code of dict[i] (unpadded)
    std::vector<uint8_t> dlen;    // PP-VBS: its length in bytes
    std::vector<uint64_t> dcount; // rows holding dict[i] (observed dictionaries)
    std::vector<uint64_t> dcum;   // prefix sums of dcount (dict.size() + 1 entries)
    std::vector<uint64_t> first_byte_rows;  // PP-VBS: rows whose code starts with byte b
    std::vector<int32_t> val2;    // PP-VBS decode: value of codes <= 2 bytes, by first two bytes
    std::vector<uint32_t> leaf2;  // PP-VBS decode: first dictionary index of a level-2 leaf
    std::vector<int32_t> val1;    // PP-VBS decode: value of each one-byte code

    // host copy of the device layout (kept for host_only / keep_host)
    bool has_host = false;
    std::vector<uint8_t> h_dense;                  // PP-VBS BS_1 / ByteSlice slices (S * n_tiles * 1024)
    std::vector<uint32_t> h_mask[kMaxCodeBytes + 1];  // [j] for j = 2..K
    std::vector<uint32_t> h_off[kMaxCodeBytes + 1];
    std::vector<uint8_t> h_deep[kMaxCodeBytes + 1];
    uint64_t deep_len[kMaxCodeBytes + 1] = {0};
    std::vector<uint32_t> h_packed;                // Bit-Packed stream
    uint64_t len_hist[kMaxCodeBytes + 1] = {0};

    // device arena
    void *d_arena = nullptr;
    size_t d_bytes = 0;
    const uint8_t *d_dense = nullptr;
    const uint32_t *d_mask[kMaxCodeBytes + 1] = {nullptr};
    const uint32_t *d_off[kMaxCodeBytes + 1] = {nullptr};
    const uint8_t *d_deep[kMaxCodeBytes + 1] = {nullptr};
    const uint32_t *d_packed = nullptr;
    const int32_t *d_val2 = nullptr;
    const int32_t *d_val1 = nullptr;  // PP-VBS: value of each one-byte code (256 entries)
    const uint32_t *d_leaf2 = nullptr;
    const int32_t *d_dict = nullptr;
    uint64_t dict_size() const { return dict.size(); }
    uint64_t dense_slice_bytes() const { return (uint64_t)n_tiles * kTileRows; }
    uint64_t packed_words() const { return (uint64_t)n_tiles * kTileWords * (uint64_t)k + 2; }
};

// host encoder (encode.cpp)
int encode_values(const int32_t *values, uint64_t n, bs_layout layout, const bs_encode_opts &o, Column &c);
int encode_raw(const uint64_t *codes, const uint8_t *lens, uint64_t n, bs_layout layout, int code_bits,
               const bs_encode_opts &o, Column &c);
int rewrite_literal(const Column &c, int op, int32_t lit, int32_t lit2, KPred &out);
int make_code_pred(const Column &c, int op, uint64_t code, int len, uint64_t code2, int len2, KPred &out);
int resolve_threads(int requested);
uint64_t estimate_rows(const Column &c, int op, int32_t lit, int32_t lit2);

// effective-bytes counter (bytes_model.cpp); tile_stride > 1 samples every
// tile_stride-th tile and scales up
int scan_bytes(const Column &c, const KPred &p, const uint32_t *seed, uint64_t tile_stride, bs_scan_bytes_t *out);
int lookup_bytes(const Column &c, const uint32_t *bits, bs_lookup_bytes_t *out);
int scan_lookup_bytes(const Column &c, const KPred &p, const uint32_t *sel, bool write_bits, bs_scan_bytes_t *out);

// device side (column.cu)
int upload_column(Column &c);
void free_device(Column &c);

}  // namespace bs

struct bs_column {
    bs::Column c;
};
