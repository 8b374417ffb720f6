/*
 * CPU ORACLE for ByteStore scan and lookup -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library. The product path (the CUDA library and its Python
 * binding) never calls it, and it shares no code, header, table or helper with
 * that path.
 *
 * It is plain, slow and sequential on purpose:
 *   - the dictionary (sorted distinct values and counts, Section 2.2);
 *   - prefix-preserving encoding of numerical columns, Algorithm 1, in the
 *     paper's order (recursive, 256-way, top-255 frequencies per node, leaf when
 *     e - s < 256 or b >= 2);
 *   - prefix-preserving encoding of categorical columns, Algorithm 2;
 *   - the three physical layouts in their plain definitions: VBS (Section 3.2:
 *     BS_1 dense, BS_j packed in row order with bitmask M_j), ByteSlice
 *     (Section 2.5: byte j of every code in slice j) and Bit-Packed (Section 2.3:
 *     codes back to back across byte boundaries);
 *   - sequential decoders for each layout (a running cursor per VBS slice);
 *   - code -> value by binary search in the sorted (zero-padded code, value)
 *     table, which is valid because the code order is the value order;
 *   - the scan by its plain definition (Section 2.2: bit i of the result bit
 *     vector is pred(v_i)), on values or on zero-padded codes (Section 3.1.1:
 *     a shorter code compares as if padded with zero bytes);
 *   - the lookup by its plain definition (values of the set rows, ascending).
 *
 * Readings taken where the paper is silent (each one also listed in the
 * repository's design notes):
 *   - ties among equal frequencies in Algorithm 1 go to the smaller index;
 *   - beta-leaf codes (b >= 2) are the beta-byte integers 1..e-s and may end in a
 *     zero byte; no trailing byte is ever stripped;
 *   - ByteSlice codes of k bits are left-aligned in ceil(k/8) bytes, slice 1
 *     holding the most significant byte;
 *   - Bit-Packed is a little-endian bit stream: code i occupies stream bits
 *     [i*k, (i+1)*k), least significant bit first;
 *   - result bit i of word w is row 32*w + i; bits at or past n are zero.
 *
 * Parity pins for every function live in the repository's CPU tests.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_LT = 0, ORC_LE, ORC_GT, ORC_GE, ORC_EQ, ORC_NE, ORC_BETWEEN };

/* ------------------------------------------------------------ dictionary */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Sorted distinct values A and their counts Q. A and Q need room for n entries.
 * Returns the number of distinct values. */
uint64_t orc_dictionary(const int32_t *values, uint64_t n, int32_t *A, uint64_t *Q) {
    if (n == 0) return 0;
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!tmp) return 0;
    memcpy(tmp, values, sizeof(int32_t) * n);
    qsort(tmp, n, sizeof(int32_t), cmp_i32);
    uint64_t nd = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (nd > 0 && A[nd - 1] == tmp[i]) {
            Q[nd - 1]++;
        } else {
            A[nd] = tmp[i];
            Q[nd] = 1;
            nd++;
        }
    }
    free(tmp);
    return nd;
}

/* ---------------------------------------------------------- Algorithm 1 */
typedef struct { uint64_t q; uint64_t idx; } freq_item;

static int cmp_freq_desc(const void *a, const void *b) {
    const freq_item *x = (const freq_item *)a, *y = (const freq_item *)b;
    if (x->q != y->q) return x->q > y->q ? -1 : 1;      /* larger frequency first */
    return (x->idx > y->idx) - (x->idx < y->idx);       /* tie: smaller index first */
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* beta = ceil(log_256(x)) for x >= 1: the smallest beta with 256^beta >= x */
static int ceil_log256(uint64_t x) {
    int beta = 0;
    unsigned __int128 p = 1;
    while (p < x) { p *= 256; beta++; }
    return beta;
}

/* PPE_NUMERICAL(C, L, b, s, e): encode values s..e-1 in a sub-tree whose parent
 * node is at level b. Returns 0, or -1 when memory runs out. */
static int ppe_numerical(uint64_t *C, uint8_t *L, const uint64_t *Q, int b, uint64_t s, uint64_t e) {
    if (e - s < 256 || b >= 2) {
        /* leaf: slot sub-codes 1..e-s, each beta bytes wide */
        int beta = ceil_log256(e - s + 1);
        for (uint64_t i = s; i < e; i++) {
            C[i] = (C[i] << (8 * beta)) + 1 + (i - s);
            L[i] = (uint8_t)(b + beta);
        }
        return 0;
    }
    /* the 255 largest frequencies in Q_s..Q_{e-1}, their indices ascending */
    uint64_t m = e - s;
    freq_item *items = (freq_item *)malloc(sizeof(freq_item) * m);
    uint64_t I[255];
    if (!items) return -1;
    for (uint64_t i = 0; i < m; i++) { items[i].q = Q[s + i]; items[i].idx = s + i; }
    qsort(items, m, sizeof(freq_item), cmp_freq_desc);
    for (int t = 0; t < 255; t++) I[t] = items[t].idx;
    free(items);
    qsort(I, 255, sizeof(uint64_t), cmp_u64);

    /* the 255 slots of this node: slot sub-codes 1..255, length b + 1 */
    for (int t = 0; t < 255; t++) {
        L[I[t]] = (uint8_t)(b + 1);
        C[I[t]] = (C[I[t]] << 8) + (uint64_t)t + 1;
    }
    /* sub-trees between adjacent slots: pointer sub-code t + 1 */
    for (int t = 0; t < 254; t++) {
        for (uint64_t i = I[t] + 1; i < I[t + 1]; i++) C[i] = (C[i] << 8) + (uint64_t)t + 1;
        if (ppe_numerical(C, L, Q, b + 1, I[t] + 1, I[t + 1])) return -1;
    }
    /* leftmost sub-tree: pointer sub-code 0 */
    for (uint64_t i = s; i < I[0]; i++) C[i] = C[i] << 8;
    if (ppe_numerical(C, L, Q, b + 1, s, I[0])) return -1;
    /* rightmost sub-tree: pointer sub-code 255 */
    for (uint64_t i = I[254] + 1; i < e; i++) C[i] = (C[i] << 8) + 255;
    if (ppe_numerical(C, L, Q, b + 1, I[254] + 1, e)) return -1;
    return 0;
}

/* Algorithm 1 over nd distinct values (ascending) with weights Q.
 * C receives the codes as integers (first byte most significant, unpadded),
 * L the lengths in bytes. Returns 0 on success. */
int orc_ppe_numerical(const uint64_t *Q, uint64_t nd, uint64_t *C, uint8_t *L) {
    for (uint64_t i = 0; i < nd; i++) C[i] = 0;
    for (uint64_t i = 0; i < nd; i++) L[i] = 0;
    return ppe_numerical(C, L, Q, 0, 0, nd);
}

/* ---------------------------------------------------------- Algorithm 2 */
/* Categorical PPE. The nd values are given in descending frequency order; the
 * tree is filled level by level (levels 1..B-1 full), and the remaining values
 * are spread over the last level slot-major so every last-level node gets a
 * share. Returns 0, or -1 for nd == 0. */
int orc_ppe_categorical(uint64_t nd, uint64_t *C, uint8_t *L) {
    if (nd == 0) return -1;
    int B = ceil_log256(nd + 1);
    uint64_t alpha = 0;
    for (int b = 1; b <= B - 1; b++) {
        uint64_t nodes = 1;
        for (int t = 0; t < b - 1; t++) nodes *= 256;
        for (uint64_t c = 0; c < nodes; c++) {
            for (uint64_t i = 1; i <= 255; i++) {
                C[alpha] = (c << 8) + i;
                L[alpha] = (uint8_t)b;
                alpha++;
            }
        }
    }
    uint64_t last_nodes = 1;
    for (int t = 0; t < B - 1; t++) last_nodes *= 256;
    for (uint64_t i = 1; i <= 255 && alpha < nd; i++) {
        for (uint64_t j = 0; j < last_nodes && alpha < nd; j++) {
            C[alpha] = (j << 8) + i;
            L[alpha] = (uint8_t)B;
            alpha++;
        }
    }
    return 0;
}

/* ------------------------------------------------------------ VBS layout */
static uint8_t code_byte(uint64_t code, int len, int j) { /* j = 1..len */
    return (uint8_t)((code >> (8 * (len - j))) & 0xFF);
}

/* Byte counts of the VBS layout: out_len[j-2] = |BS_j| for j = 2..K. */
void orc_vbs_slice_lengths(const uint8_t *lens, uint64_t n, int K, uint64_t *out_len) {
    for (int j = 2; j <= K; j++) {
        uint64_t c = 0;
        for (uint64_t i = 0; i < n; i++)
            if (lens[i] >= j) c++;
        out_len[j - 2] = c;
    }
}

/* Build the VBS layout in its plain form.
 *   bs1   : n bytes, the first byte of every code
 *   masks : (K-1) * ceil(n/32) words; bit i%32 of word i/32 of mask j is (L_i >= j)
 *   deep  : BS_2 .. BS_K concatenated, each holding byte j of the codes that have
 *           one, in row order (lengths from orc_vbs_slice_lengths). */
int orc_vbs_build(const uint64_t *codes, const uint8_t *lens, uint64_t n, int K,
                  uint8_t *bs1, uint32_t *masks, uint8_t *deep) {
    uint64_t nw = (n + 31) / 32;
    for (uint64_t i = 0; i < n; i++) {
        if (lens[i] < 1 || lens[i] > K) return -1;
        bs1[i] = code_byte(codes[i], lens[i], 1);
    }
    memset(masks, 0, sizeof(uint32_t) * nw * (uint64_t)(K > 1 ? K - 1 : 0));
    uint64_t pos = 0;
    for (int j = 2; j <= K; j++) {
        uint32_t *M = masks + (uint64_t)(j - 2) * nw;
        for (uint64_t i = 0; i < n; i++) {
            if (lens[i] >= j) {
                M[i / 32] |= 1u << (i % 32);
                deep[pos++] = code_byte(codes[i], lens[i], j);
            }
        }
    }
    return 0;
}

/* Where the sequential decoder's cursors stand at row `row`: cursor[j-2] =
 * the number of rows before `row` whose mask-j bit is set (whole words
 * popcounted, then the partial word), j = 2..K. */
void orc_vbs_cursors_at(const uint32_t *masks, uint64_t n, int K, uint64_t row, uint64_t *cursor) {
    uint64_t nw = (n + 31) / 32;
    for (int j = 2; j <= K; j++) {
        const uint32_t *M = masks + (uint64_t)(j - 2) * nw;
        uint64_t c = 0;
        for (uint64_t w = 0; w < row / 32; w++) c += (uint64_t)__builtin_popcount(M[w]);
        if (row % 32) c += (uint64_t)__builtin_popcount(M[row / 32] & ((1u << (row % 32)) - 1u));
        cursor[j - 2] = c;
    }
}

/* Sequential decoder over rows [r0, r1): one cursor per slice, starting at
 * cursor0[j-2] (orc_vbs_cursors_at(r0)) and advanced whenever a row's mask
 * bit is set. Writes the zero-padded K-byte codes (as integers) and lengths
 * of rows r0.. at padded[0..], lens[0..]. Disjoint ranges decoded separately
 * give the same codes as one pass over all rows. */
int orc_vbs_decode_range(const uint8_t *bs1, const uint32_t *masks, const uint8_t *deep,
                         const uint64_t *slice_len, uint64_t n, int K, uint64_t r0, uint64_t r1,
                         const uint64_t *cursor0, uint64_t *padded, uint8_t *lens) {
    uint64_t nw = (n + 31) / 32;
    uint64_t start[8], cursor[8];
    uint64_t acc = 0;
    if (K < 1 || K > 8 || r1 > n || r0 > r1) return -1;
    for (int j = 2; j <= K; j++) {
        start[j] = acc;
        cursor[j] = cursor0 ? cursor0[j - 2] : 0;
        acc += slice_len[j - 2];
    }
    for (uint64_t i = r0; i < r1; i++) {
        uint64_t code = bs1[i];
        int len = 1;
        for (int j = 2; j <= K; j++) {
            const uint32_t *M = masks + (uint64_t)(j - 2) * nw;
            if ((M[i / 32] >> (i % 32)) & 1u) {
                if (cursor[j] >= slice_len[j - 2]) return -2;
                code = (code << 8) | deep[start[j] + cursor[j]];
                cursor[j]++;
                len = j;
            }
        }
        padded[i - r0] = code << (8 * (K - len));
        lens[i - r0] = (uint8_t)len;
    }
    return 0;
}

/* Sequential decoder over all rows. Returns the zero-padded K-byte codes (as
 * integers) and lengths. */
int orc_vbs_decode(const uint8_t *bs1, const uint32_t *masks, const uint8_t *deep,
                   const uint64_t *slice_len, uint64_t n, int K, uint64_t *padded, uint8_t *lens) {
    return orc_vbs_decode_range(bs1, masks, deep, slice_len, n, K, 0, n, NULL, padded, lens);
}

/* ------------------------------------------------------ ByteSlice layout */
static int slices_for_bits(int k) { return (k + 7) / 8; }

/* slices: S * n bytes, slice s (1-based) at offset (s-1)*n. */
int orc_byteslice_build(const uint64_t *codes, uint64_t n, int k, uint8_t *slices) {
    int S = slices_for_bits(k);
    if (k < 1 || k > 32) return -1;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t aligned = codes[i] << (8 * S - k);
        for (int s = 1; s <= S; s++)
            slices[(uint64_t)(s - 1) * n + i] = (uint8_t)((aligned >> (8 * (S - s))) & 0xFF);
    }
    return 0;
}

int orc_byteslice_decode(const uint8_t *slices, uint64_t n, int k, uint64_t *codes) {
    int S = slices_for_bits(k);
    if (k < 1 || k > 32) return -1;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t aligned = 0;
        for (int s = 1; s <= S; s++) aligned = (aligned << 8) | slices[(uint64_t)(s - 1) * n + i];
        codes[i] = aligned >> (8 * S - k);
    }
    return 0;
}

/* ----------------------------------------------------- Bit-Packed layout */
/* stream: ceil(n*k/8) bytes; bit p of the stream is bit p%8 of byte p/8. */
int orc_bitpacked_build(const uint64_t *codes, uint64_t n, int k, uint8_t *stream) {
    if (k < 1 || k > 32) return -1;
    uint64_t nbytes = (n * (uint64_t)k + 7) / 8;
    memset(stream, 0, nbytes);
    for (uint64_t i = 0; i < n; i++) {
        for (int t = 0; t < k; t++) {
            if ((codes[i] >> t) & 1u) {
                uint64_t p = i * (uint64_t)k + (uint64_t)t;
                stream[p / 8] |= (uint8_t)(1u << (p % 8));
            }
        }
    }
    return 0;
}

int orc_bitpacked_decode(const uint8_t *stream, uint64_t n, int k, uint64_t *codes) {
    if (k < 1 || k > 32) return -1;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t c = 0;
        for (int t = 0; t < k; t++) {
            uint64_t p = i * (uint64_t)k + (uint64_t)t;
            if ((stream[p / 8] >> (p % 8)) & 1u) c |= (uint64_t)1 << t;
        }
        codes[i] = c;
    }
    return 0;
}

/* -------------------------------------------------------- code -> value */
/* sorted_codes: the dictionary's zero-padded codes in ascending order, aligned
 * with the values in A. Each code is found by binary search. Returns 0, or -1
 * if a code is not in the dictionary. */
int orc_codes_to_values(const uint64_t *codes, uint64_t n, const uint64_t *sorted_codes,
                        const int32_t *A, uint64_t nd, int32_t *values) {
    for (uint64_t i = 0; i < n; i++) {
        uint64_t lo = 0, hi = nd;
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (sorted_codes[mid] < codes[i]) lo = mid + 1; else hi = mid;
        }
        if (lo >= nd || sorted_codes[lo] != codes[i]) return -1;
        values[i] = A[lo];
    }
    return 0;
}

/* ------------------------------------------------------------ predicates */
static int pred_i64(int op, int64_t v, int64_t c, int64_t c2) {
    switch (op) {
    case ORC_LT: return v < c;
    case ORC_LE: return v <= c;
    case ORC_GT: return v > c;
    case ORC_GE: return v >= c;
    case ORC_EQ: return v == c;
    case ORC_NE: return v != c;
    case ORC_BETWEEN: return c <= v && v <= c2;
    default: return 0;
    }
}

static int pred_u64(int op, uint64_t v, uint64_t c, uint64_t c2) {
    switch (op) {
    case ORC_LT: return v < c;
    case ORC_LE: return v <= c;
    case ORC_GT: return v > c;
    case ORC_GE: return v >= c;
    case ORC_EQ: return v == c;
    case ORC_NE: return v != c;
    case ORC_BETWEEN: return c <= v && v <= c2;
    default: return 0;
    }
}

/* bits: ceil(n/32) words, fully written (bits >= n are zero). */
void orc_scan_values(const int32_t *v, uint64_t n, int op, int32_t lit, int32_t lit2, uint32_t *bits) {
    uint64_t nw = (n + 31) / 32;
    memset(bits, 0, sizeof(uint32_t) * nw);
    for (uint64_t i = 0; i < n; i++)
        if (pred_i64(op, v[i], lit, lit2)) bits[i / 32] |= 1u << (i % 32);
}

/* Scan on zero-padded codes (all codes and literals padded to the same width). */
void orc_scan_codes(const uint64_t *padded, uint64_t n, int op, uint64_t lit, uint64_t lit2, uint32_t *bits) {
    uint64_t nw = (n + 31) / 32;
    memset(bits, 0, sizeof(uint32_t) * nw);
    for (uint64_t i = 0; i < n; i++)
        if (pred_u64(op, padded[i], lit, lit2)) bits[i / 32] |= 1u << (i % 32);
}

/* out receives v_i for every set bit i < n, in ascending i. Returns the count. */
uint64_t orc_lookup(const int32_t *v, uint64_t n, const uint32_t *bits, int32_t *out) {
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; i++)
        if ((bits[i / 32] >> (i % 32)) & 1u) out[m++] = v[i];
    return m;
}

/* out[t] = v[rowids[t]]. Returns -1 if a row id is out of range. */
int orc_lookup_rowids(const int32_t *v, uint64_t n, const uint32_t *rowids, uint64_t m, int32_t *out) {
    for (uint64_t t = 0; t < m; t++) {
        if (rowids[t] >= n) return -1;
        out[t] = v[rowids[t]];
    }
    return 0;
}

/* ------------------------------------------------ layout byte accounting */
/* Bytes taken by one block of `rows` codes with the given lengths: VBS counts
 * the BS_1 bytes, the materialised deeper bytes and one 32-bit mask word per
 * slice j >= 2 for every 32 rows; ByteSlice counts K dense slices. */
uint64_t orc_vbs_block_bytes(const uint8_t *lens, uint64_t rows, int K) {
    uint64_t bytes = rows;
    for (int j = 2; j <= K; j++) {
        bytes += 4 * ((rows + 31) / 32);
        for (uint64_t i = 0; i < rows; i++)
            if (lens[i] >= j) bytes++;
    }
    return bytes;
}

uint64_t orc_byteslice_block_bytes(uint64_t rows, int K) { return rows * (uint64_t)K; }
