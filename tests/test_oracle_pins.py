"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: values printed in the
paper's worked examples (tests/golden), closed forms derived by hand from
Algorithm 1 / Algorithm 2, library routines (numpy searchsorted / packbits /
byte views) for the plain scan and lookup definitions and for the layouts, and
invariants the paper states (order preservation, Lemma 1, Property 1, mask
nesting). None of these tests needs a GPU.
"""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth


# ------------------------------------------------------------------ fixtures
def _read_golden(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _hex_code(h):
    return int(h, 16), len(h) // 2


# --------------------------------------------------- worked scan example
def test_worked_scan_example(golden_dir):
    rows = _read_golden(os.path.join(golden_dir, "scan_worked_example.txt"))
    codes = [(r[1], _hex_code(r[2])) for r in rows if r[0] == "code"]
    lits = {r[1]: _hex_code(r[2]) for r in rows if r[0] == "literal"}
    K = max(l for _, (_, l) in codes)
    C = np.array([c for _, (c, _) in codes], np.uint64)
    L = np.array([l for _, (_, l) in codes], np.uint8)
    padded = orc.pad(C, L, K)
    for r in rows:
        if r[0] != "expect":
            continue
        op, lit = r[1], lits[r[2]]
        want = [int(x) for x in r[3:]]
        lit_pad = lit[0] << (8 * (K - lit[1]))
        bits = orc.scan_codes(padded, op, lit_pad)
        got = [(int(bits[0]) >> i) & 1 for i in range(len(want))]
        assert got == want, (r, got)
    # the plain VBS layout of the same four rows
    bs1, masks, slices = orc.vbs_build(C, L, K)
    lay = {r[1]: r[2:] for r in rows if r[0] == "layout"}
    assert list(bs1) == [int(x, 16) for x in lay["bs1"]]
    assert [(int(masks[0][0]) >> i) & 1 for i in range(4)] == [int(x) for x in lay["m2_bits"]]
    assert list(slices[0]) == [int(x, 16) for x in lay["bs2"]]
    # and the sequential decoder inverts it
    dp, dl = orc.vbs_decode(bs1, masks, slices, len(C), K)
    assert list(dp) == list(padded) and list(dl) == list(L)


def test_vbs_block_accounting(golden_dir):
    g = {r[0]: int(r[1]) for r in _read_golden(os.path.join(golden_dir, "vbs_block_example.txt"))}
    lens = np.ones(g["rows"], np.uint8)
    lens[: g["with_second_byte"]] = 2
    lens[: g["with_third_byte"]] = 3
    assert orc.vbs_block_bytes(lens, g["max_len"]) == g["vbs_bytes"]
    assert orc.byteslice_block_bytes(g["rows"], g["max_len"]) == g["byteslice_bytes"]


# --------------------------------------------------- Algorithm 1 closed forms
@pytest.mark.parametrize("n", [1, 2, 17, 200, 255])
def test_ppe_small_dictionary_is_one_leaf(n):
    # e - s < 256 at the root: slot sub-codes 1..n, one byte each
    C, L = orc.ppe_numerical(np.arange(n, 0, -1))
    assert list(C) == list(range(1, n + 1))
    assert set(L.tolist()) == {1}


def test_ppe_equal_weights_300():
    # ties go to the smaller index: indices 0..254 fill the root's slots, the
    # 45 values after them form the rightmost sub-tree (pointer 255), one leaf
    C, L = orc.ppe_numerical(np.ones(300, np.uint64))
    for i in range(300):
        if i < 255:
            assert (C[i], L[i]) == (i + 1, 1)
        else:
            assert (C[i], L[i]) == ((255 << 8) | (i - 255 + 1), 2)


def test_ppe_increasing_weights_300():
    # the 255 heaviest are indices 45..299; indices 0..44 form the leftmost
    # sub-tree (pointer sub-code 0)
    C, L = orc.ppe_numerical(np.arange(1, 301, dtype=np.uint64))
    for i in range(300):
        if i >= 45:
            assert (C[i], L[i]) == (i - 45 + 1, 1)
        else:
            assert (C[i], L[i]) == ((0 << 8) | (i + 1), 2)


def test_ppe_interleaved_slots_and_pointers():
    # even indices are heavy: slot t holds index 2t; the single odd value
    # between slots t and t+1 sits under pointer t+1; index 509 under 255
    Q = np.where(np.arange(510) % 2 == 0, 2, 1).astype(np.uint64)
    C, L = orc.ppe_numerical(Q)
    for i in range(510):
        if i % 2 == 0:
            assert (C[i], L[i]) == (i // 2 + 1, 1)
        elif i < 509:
            assert (C[i], L[i]) == (((i // 2 + 1) << 8) | 1, 2)
        else:
            assert (C[i], L[i]) == ((255 << 8) | 1, 2)


def test_ppe_beta_leaf_codes_may_end_in_zero():
    # root: indices 0..254 (heavy). Rightmost sub-tree [255, 855) at level 1 is
    # internal: its slots are 255..509 (ties -> smaller index). Its rightmost
    # sub-tree [510, 855) has 345 values at b = 2: a leaf with beta = 2 whose
    # codes are the 2-byte integers 1..345 under the pointer path 255.255.
    Q = np.ones(855, np.uint64)
    Q[:255] = 1000
    C, L = orc.ppe_numerical(Q)
    for i in range(855):
        if i < 255:
            want = (i + 1, 1)
        elif i < 510:
            want = ((255 << 8) | (i - 255 + 1), 2)
        else:
            want = ((255 << 24) | (255 << 16) | (i - 510 + 1), 4)
        assert (int(C[i]), int(L[i])) == want
    # the 256th leaf value has code ...0x01 0x00: a trailing zero byte that must
    # not be stripped
    assert int(C[510 + 255]) & 0xFF == 0 and int(L[510 + 255]) == 4


# ------------------------------------------------------ Algorithm 2 pins
def test_ppe_categorical_levels():
    C, L = orc.ppe_categorical(255)
    assert list(C) == list(range(1, 256)) and set(L.tolist()) == {1}
    C, L = orc.ppe_categorical(300)
    assert list(C[:255]) == list(range(1, 256))
    # the last level is filled slot-major: slot 1 under pointers 0, 1, ..., 44
    assert [int(c) for c in C[255:]] == [(j << 8) | 1 for j in range(45)]
    assert set(L[255:].tolist()) == {2}
    # balanced (Property 2): only the last two levels occur
    C, L = orc.ppe_categorical(70000)
    assert set(L.tolist()) == {1, 2, 3}
    assert len(set(zip(C.tolist(), L.tolist()))) == 70000


# ------------------------------------------------------ invariants
def _dict_from(values):
    A, Q = orc.dictionary(values)
    C, L = orc.ppe_numerical(Q)
    return A, Q, C, L


def _zipf_values(n, N, s, seed, monotone=False):
    return synth.zipf_column(n, N, s, seed, mapping="identity" if monotone else "feistel",
                             d=int(np.log2(N)))


DICT_CASES = [
    (20000, 1 << 12, 1.0, 1, False),
    (20000, 1 << 12, 0.0, 2, False),
    (50000, 1 << 16, 1.5, 3, False),
    (60000, 1 << 16, 1.0, 4, True),    # monotone: frequent = small, forces beta leaves
    (200000, 1 << 20, 0.5, 5, True),
]


@pytest.mark.parametrize("n,N,s,seed,mono", DICT_CASES)
def test_order_preservation_and_prefix_tails(n, N, s, seed, mono):
    A, Q, C, L = _dict_from(_zipf_values(n, N, s, seed, mono))
    K = int(L.max())
    padded = orc.pad(C, L, K)
    # in-order traversal = value order: padded codes strictly increase with A
    assert np.all(padded[1:] > padded[:-1])
    if mono and A.size > 766:
        assert K >= 4  # the level-2 leaf of the heavy right spine holds >= 256 values
    # every code that extends another code has a positive tail (Lemma 1's premise)
    codeset = set(zip(C.tolist(), L.tolist()))
    for c, l in zip(C.tolist(), L.tolist()):
        for p in range(1, l):
            pre = c >> (8 * (l - p))
            if (pre, p) in codeset:
                assert c & ((1 << (8 * (l - p))) - 1) > 0
    # slot sub-codes are never zero outside beta >= 2 leaves (length <= 3)
    short = L <= 3
    assert np.all((C[short] & np.uint64(0xFF)) != 0)
    assert K <= 6


@pytest.mark.parametrize("n,N,s,seed,mono", DICT_CASES)
def test_property1_internal_nodes_full(n, N, s, seed, mono):
    A, Q, C, L = _dict_from(_zipf_values(n, N, s, seed, mono))
    # internal nodes exist only at levels 0 and 1 (recursion stops at b >= 2,
    # where a leaf may extend its path by beta >= 2 bytes); at those levels a
    # leaf has beta = 1, so a path P of length p <= 1 leads to an internal node
    # iff some code extends P by two or more bytes. Such a node must hold all
    # 255 slot sub-codes.
    paths = set()
    for c, l in zip(C.tolist(), L.tolist()):
        for p in range(0, min(l - 1, 2)):
            paths.add((c >> (8 * (l - p)), p))
    for (P, p) in paths:
        sel = (L == p + 1) & ((C >> np.uint64(8)) == np.uint64(P))
        slots = np.sort(C[sel] & np.uint64(0xFF))
        assert slots.tolist() == list(range(1, 256)), (hex(P), p)


def _lemma1_sign(cu, lu, cv, lv):
    m = min(lu, lv)
    pu, pv = cu >> (8 * (lu - m)), cv >> (8 * (lv - m))
    if pu != pv:
        return -1 if pu < pv else 1
    if lu == lv:
        return 0
    return -1 if lu < lv else 1


def test_lemma1_pairwise():
    # Lemma 1: comparing the first min(l1, l2) bytes plus the length rule gives
    # the same answer as comparing zero-padded codes, for every pair
    for seed, mono in ((11, True), (12, False)):
        A, Q, C, L = _dict_from(_zipf_values(40000, 1 << 14, 1.0, seed, mono))
        idx = np.linspace(0, C.size - 1, min(C.size, 1500)).astype(int)
        K = int(L.max())
        cu, lu = C[idx][:, None], L[idx].astype(np.int64)[:, None]
        cv, lv = C[idx][None, :], L[idx].astype(np.int64)[None, :]
        P = orc.pad(C[idx], L[idx], K)
        want = np.sign(P[:, None].astype(np.float64) - P[None, :].astype(np.float64))
        want = np.where(P[:, None] > P[None, :], 1, np.where(P[:, None] < P[None, :], -1, 0))
        m = np.minimum(lu, lv)
        pu = cu >> (8 * (lu - m)).astype(np.uint64)
        pv = cv >> (8 * (lv - m)).astype(np.uint64)
        lemma = np.where(pu != pv, np.where(pu < pv, -1, 1),
                         np.where(lu == lv, 0, np.where(lu < lv, -1, 1)))
        assert np.array_equal(lemma, want)
        # spot-check the scalar statement of the rule on a few pairs
        for i in range(0, idx.size, 97):
            j = (i * 7) % idx.size
            assert _lemma1_sign(int(C[idx[i]]), int(L[idx[i]]), int(C[idx[j]]), int(L[idx[j]])) == want[i, j]


@pytest.mark.parametrize("n,N,s,seed,mono", DICT_CASES)
def test_vbs_mask_nesting_and_decode_roundtrip(n, N, s, seed, mono):
    values = _zipf_values(n, N, s, seed, mono)
    col = orc.OracleColumn(values, "ppvbs")
    K = col.K
    for j in range(K - 2):  # M_{j+1} is a subset of M_j
        assert np.all((col.masks[j + 1] & ~col.masks[j]) == 0)
    for j in range(K - 1):  # |BS_j| = popcount(M_j)
        pc = int(np.unpackbits(col.masks[j].view(np.uint8)).sum())
        assert col.slices[j].size == pc
    assert np.array_equal(col.decode_values(), values)


@pytest.mark.parametrize("layout", ["byteslice", "bitpacked"])
def test_fixed_width_decode_roundtrip(layout):
    values = _zipf_values(30001, 1 << 12, 1.0, 21)
    col = orc.OracleColumn(values, layout)
    assert np.array_equal(col.decode_values(), values)
    col = orc.OracleColumn(values, layout, domain_bits=12, domain_min=0)
    assert np.array_equal(col.decode_values(), values)
    v32 = synth.config_sweep_column(5000, 32, 1.0, 3)
    col = orc.OracleColumn(v32, layout, domain_bits=32, domain_min=-(1 << 31))
    assert np.array_equal(col.decode_values(), v32)


# ---------------------------------------------- layouts vs library byte views
def test_bitpacked_k32_is_plain_int32():
    codes = synth.u64(1, 2, 1000).astype(np.uint32)
    stream = orc.bitpacked_build(codes, 32)
    assert stream.tobytes() == codes.astype("<u4").tobytes()


@pytest.mark.parametrize("k", [1, 3, 7, 8, 11, 12, 17, 24, 31])
def test_bitpacked_matches_numpy_packbits(k):
    n = 777
    codes = (synth.u64(3, k, n) & np.uint64((1 << k) - 1)).astype(np.uint64)
    bitmat = ((codes[:, None] >> np.arange(k, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.uint8)
    want = np.packbits(bitmat.reshape(-1), bitorder="little")
    assert np.array_equal(orc.bitpacked_build(codes, k), want)
    assert np.array_equal(orc.bitpacked_decode(want, n, k), codes)


def test_byteslice_16_and_12_match_big_endian_bytes():
    codes = (synth.u64(4, 0, 500) & np.uint64(0xFFFF)).astype(np.uint64)
    sl = orc.byteslice_build(codes, 16)
    be = codes.astype(">u2").view(np.uint8).reshape(-1, 2).T
    assert np.array_equal(sl, be)
    c12 = codes & np.uint64(0xFFF)
    sl12 = orc.byteslice_build(c12, 12)
    be12 = (c12 << np.uint64(4)).astype(">u2").view(np.uint8).reshape(-1, 2).T
    assert np.array_equal(sl12, be12)


# -------------------------------------------- scan and lookup definitions
def _bits_to_bool(bits, n):
    return np.unpackbits(bits.view(np.uint8), bitorder="little")[:n].astype(bool)


def test_scan_counts_match_searchsorted():
    v = synth.zipf_column(10007, 1 << 10, 1.0, 31, mapping="feistel", d=10) - 300
    sv = np.sort(v)
    n = v.size
    lits = [int(sv[0]) - 1, int(sv[0]), int(sv[-1]), int(sv[-1]) + 1, -(1 << 31), (1 << 31) - 1, 5, 0, 333]
    for x in lits:
        lo, hi = np.searchsorted(sv, x, "left"), np.searchsorted(sv, x, "right")
        want = {"lt": lo, "le": hi, "gt": n - hi, "ge": n - lo, "eq": hi - lo, "ne": n - (hi - lo)}
        for op, w in want.items():
            bits = orc.scan_values(v, op, x)
            assert int(_bits_to_bool(bits, n).sum()) == w, (op, x)
            assert np.all((_bits_to_bool(bits, bits.size * 32))[n:] == 0)
    for a, b in [(0, 100), (100, 0), (int(sv[0]), int(sv[-1])), (-5, -5)]:
        bits = orc.scan_values(v, "between", a, b)
        w = max(0, np.searchsorted(sv, b, "right") - np.searchsorted(sv, a, "left")) if a <= b else 0
        assert int(_bits_to_bool(bits, n).sum()) == w


def test_scan_bit_order_is_little_endian_words():
    v = synth.zipf_column(1000, 64, 0.0, 5, mapping="identity")
    mask = v < 20
    want = np.packbits(mask, bitorder="little")
    want = np.concatenate([want, np.zeros((-want.size) % 4, np.uint8)]).view("<u4")
    assert np.array_equal(orc.scan_values(v, "lt", 20), want)


def test_lookup_matches_flatnonzero():
    v = synth.zipf_column(5003, 1 << 12, 1.0, 8, mapping="feistel", d=12)
    bits = orc.scan_values(v, "ge", 2000)
    want = v[np.flatnonzero(_bits_to_bool(bits, v.size))]
    assert np.array_equal(orc.lookup(v, bits), want)
    rid = (synth.u64(2, 2, 100) % np.uint64(v.size)).astype(np.uint32)
    assert np.array_equal(orc.lookup_rowids(v, rid), v[rid.astype(np.int64)])


@pytest.mark.parametrize("nd", [1, 2, 255, 256, 257, 511, 800])
def test_brute_force_tiny_columns(nd):
    # every op and every literal between min-1 and max+1, on the decode path
    # every value once plus Zipf draws that favour the smallest values, so the
    # observed dictionary has exactly nd entries (nd = 800 forces beta leaves)
    rng_vals = synth.distinct_values(nd, seed=nd)
    r = synth.zipf_ranks(max(64, 2 * nd), nd, 1.0, seed=nd)
    v = np.concatenate([rng_vals[synth.permutation(nd, nd)], rng_vals[r]])
    for layout in ("ppvbs", "byteslice", "bitpacked"):
        col = orc.OracleColumn(v, layout)
        dec = col.decode_values()
        assert np.array_equal(dec, v)
    sv = np.sort(np.unique(v))
    lits = sorted(set([int(sv[0]) - 1, int(sv[-1]) + 1] + [int(x) for x in sv[:: max(1, sv.size // 40)]]))
    col = orc.OracleColumn(v, "ppvbs")
    for op in ("lt", "le", "gt", "ge", "eq", "ne"):
        for x in lits:
            got = _bits_to_bool(col.scan(op, x), v.size)
            want = {"lt": v < x, "le": v <= x, "gt": v > x, "ge": v >= x, "eq": v == x, "ne": v != x}[op]
            assert np.array_equal(got, want)


def test_code_scan_equals_value_scan_under_order_preservation():
    # order preservation (Section 3.1.1) makes the padded-code compare agree with
    # the value compare for every literal taken from the dictionary
    v = _zipf_values(30000, 1 << 16, 1.0, 17, monotone=True)
    col = orc.OracleColumn(v, "ppvbs")
    padded, _ = col.decode_codes()
    dict_pad = orc.pad(col.C, col.L, col.K)
    for t in np.linspace(0, col.A.size - 1, 25).astype(int):
        for op in ("lt", "le", "gt", "ge", "eq", "ne"):
            assert np.array_equal(orc.scan_codes(padded, op, int(dict_pad[t])),
                                  orc.scan_values(v, op, int(col.A[t])))


# ------------------------------------------ Algorithm 2 inside a column
def test_categorical_column_hands_out_codes_by_frequency():
    # counts: 3 and 7 five times (tie: the smaller value first), 9 twice, 1 once
    v = np.array([7] * 5 + [3] * 5 + [9] * 2 + [1], np.int32)
    oc = orc.OracleColumn(v, "ppvbs", categorical=True)
    code = {int(a): (int(c), int(l)) for a, c, l in zip(oc.A, oc.C, oc.L)}
    assert code == {3: (1, 1), 7: (2, 1), 9: (3, 1), 1: (4, 1)}
    assert np.array_equal(oc.decode_values(), v)


def test_categorical_column_second_level_and_roundtrip():
    # 300 values with distinct counts 300, 299, ..., 1 (value i has count 300 - i)
    vals = np.repeat(np.arange(300, dtype=np.int32), np.arange(300, 0, -1))
    oc = orc.OracleColumn(vals, "ppvbs", categorical=True)
    assert oc.K == 2
    # ranks 0..254 take the one-byte codes 1..255; rank 255 + j takes (j, 1)
    assert [int(c) for c in oc.C[:255]] == list(range(1, 256))
    assert [int(c) for c in oc.C[255:]] == [(j << 8) | 1 for j in range(45)]
    assert np.array_equal(oc.decode_values(), vals)
    # three levels once more than 255 + 256 * 255 values exist
    big = np.arange(70000, dtype=np.int32)
    ob = orc.OracleColumn(big, "ppvbs", categorical=True)
    assert ob.K == 3 and np.array_equal(ob.decode_values(), big)


@pytest.mark.parametrize("n,d,s,mono,step", [(100003, 24, 0.7, True, 32 * 311), (50000, 12, 1.0, False, 777),
                                             (4097, 16, 1.2, True, 1)])
def test_vbs_range_decode_equals_one_pass(n, d, s, mono, step):
    """The range decoder (cursors started where a full pass has them) gives
    every row's value, for ranges that start at any row, including mid-word."""
    v = synth.config_sweep_column(n, d, s, 5 + d, monotone=mono)
    o = orc.OracleColumn(v, "ppvbs")
    parts = [o.decode_values_range(a, min(a + step, n)) for a in range(0, n, step)] if step > 1 else \
        [o.decode_values_range(a, a + 1) for a in range(0, n, 97)]
    got = np.concatenate(parts)
    if step > 1:
        assert np.array_equal(got, v)
    else:
        assert np.array_equal(got, v[::97])
