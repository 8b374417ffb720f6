"""The effective-bytes counter (bs_scan_bytes, bs_lookup_bytes,
bs_scan_lookup_bytes) against a brute-force replay written here from the
kernels' documented access rules, on small host-only columns. These counts
are the numerators of every roofline fraction the bench reports and the cost
of the advisor's deterministic mode.

Access rules restated (one warp per 1024-row tile; lane L owns rows
32L..32L+31):
  * dense slice (PP-VBS BS_1, ByteSlice slices): lane L's 32 bytes sit at tile
    offsets 16L.. and 512 + 16L.. (word w byte b of the lane's bytes is row
    8b + w), so a lane that scans reads 32-byte sectors L // 2 and 16 + L // 2
    of its tile;
  * scan, PP-VBS (Algorithm 3 with Lemma 1's early stop): a row is pending at
    level j >= 2 while its bytes 1..j-1 exist and equal the literal's (j-1 <=
    the literal's length) and j does not pass the deepest level the predicate
    needs (the literal's length, or one more when "equal" must be told from
    "larger", capped at K); a pending row makes its 256-row group read the
    group's M_j sector; a pending row that has byte j with j <= the literal's
    length makes the group read its off_j entry (4 bytes) and the BS_j sector
    of that byte;
  * scan, ByteSlice: a lane with a row whose bytes 1..s-1 equal the literal's
    reads its 32 bytes of slice s;
  * scan, Bit-Packed: a 32-row word with a valid row reads k stream words;
  * lookup of a selected PP-VBS row: its BS_1 byte, every BS_j byte of its
    code, and the M_j sector and off_j entry of its group for j up to one past
    its length; ByteSlice: its byte in every slice; Bit-Packed: the bytes of
    its k-bit field;
  * distinct sectors are counted once; the result is ceil(n/32) 4-byte words.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth

TILE = 1024


@pytest.fixture(scope="module")
def B():
    from paper_2209_00220_gb300 import build_lib
    build_lib.build()
    from paper_2209_00220_gb300 import bytestore
    return bytestore


def tile_pos(q):
    """Position of tile-local row q inside its tile's 1024 dense bytes."""
    q = np.asarray(q, dtype=np.int64)
    lane, r = q >> 5, q & 31
    w, b = r & 7, r >> 3
    return np.where(w < 4, 16 * lane + 4 * w, 512 + 16 * lane + 4 * (w - 4)) + b


def code_bytes(codes, lens, K):
    """n x (K + 1) array: column j = byte j (1-based) of each code, 0 past its length."""
    codes = np.asarray(codes, dtype=np.uint64)
    lens = np.asarray(lens, dtype=np.int64)
    out = np.zeros((codes.size, K + 1), dtype=np.int64)
    for j in range(1, K + 1):
        sh = np.clip(lens - j, 0, None).astype(np.uint64) * np.uint64(8)
        out[:, j] = np.where(lens >= j, ((codes >> sh) & np.uint64(0xFF)).astype(np.int64), 0)
    return out


def deep_positions(masks_j, n):
    """Index into BS_j of each row's byte j (-1 for rows without one), from the
    row-ordered mask words: rank of the row among the rows whose bit is set."""
    bits = np.unpackbits(np.asarray(masks_j, dtype=np.uint32).view(np.uint8), bitorder="little")[:n].astype(bool)
    pos = np.cumsum(bits) - 1
    return np.where(bits, pos, -1)


def sectors(addrs):
    return int(np.unique(np.asarray(addrs, dtype=np.int64) >> 5).size)


def pending_levels(cb, lens, lit_b, l, K, need_eq):
    """(pend, read): n x (K + 1) booleans, row pending at level j / byte j read."""
    n = cb.shape[0]
    jend = min(l + 1, K) if need_eq else min(l, K)
    pend = np.zeros((n, K + 1), dtype=bool)
    read = np.zeros((n, K + 1), dtype=bool)
    ok = np.ones(n, dtype=bool)
    for j in range(2, jend + 1):
        ok = ok & (cb[:, j - 1] == lit_b[j - 1]) & (lens >= j - 1) & (l >= j - 1)
        pend[:, j] = ok
        read[:, j] = ok & (lens >= j) & (j <= l)
    return pend, read


def ppvbs_replay(ocol, lits, need_eqs, sel=None, seed=None):
    """Brute-force sector counts of a PP-VBS scan (plus the lookup of `sel`)."""
    n, K = ocol.n, ocol.K
    lens = ocol.row_lens.astype(np.int64)
    cb = code_bytes(ocol.row_codes, lens, K)
    rows = np.arange(n)
    on = np.ones(n, dtype=bool) if seed is None else \
        np.unpackbits(seed.view(np.uint8), bitorder="little")[:n].astype(bool)
    pend = np.zeros((n, K + 1), dtype=bool)
    read = np.zeros((n, K + 1), dtype=bool)
    for (lc, ll), ne in zip(lits, need_eqs):
        lb = code_bytes(np.array([lc]), np.array([ll]), max(K, ll))[0]
        p, r = pending_levels(cb, lens, lb, ll, K, ne)
        pend |= p
        read |= r
    pend &= on[:, None]
    read &= on[:, None]
    picked = np.zeros(n, dtype=bool) if sel is None else \
        np.unpackbits(sel.view(np.uint8), bitorder="little")[:n].astype(bool)
    for j in range(2, K + 1):
        reach = picked & (lens >= j - 1)       # M_j / off_j of the group: up to one past the length
        pend[:, j] |= reach
        read[:, j] |= picked & (lens >= j)     # every byte of a selected code
    tile, q = rows // TILE, rows % TILE
    lane_key = tile * 32 + (q >> 5)
    dense = 0
    for half in (0, 16):  # sectors L // 2 and 16 + L // 2 of a scanning lane
        dense += 32 * np.unique((tile * 32 + half + ((q >> 5) >> 1))[on]).size
    del lane_key
    group = rows >> 8
    mask = off = deep = 0
    for j in range(2, K + 1):
        mask += 32 * np.unique(group[pend[:, j]]).size
        # off_j entries: groups with a byte read at level j, or reached by a selected row
        og = np.unique(group[read[:, j] | (picked & (lens >= j - 1))])
        off += 32 * sectors(og * 4)
        pos = deep_positions(ocol.masks[j - 2], n)
        deep += 32 * sectors(pos[read[:, j]])
    return {"dense_bytes": dense, "mask_bytes": mask, "offset_bytes": off, "deep_bytes": deep}


def _lit_code(ocol, x):
    i = int(np.searchsorted(ocol.A, x))
    assert ocol.A[i] == x
    return int(ocol.C[i]), int(ocol.L[i])


PP_CASES = [
    (20_000, 16, 1.2, True),    # K >= 3, beta leaves
    (30_001, 12, 1.0, False),   # the bench's distribution, ragged tail
    (12_345, 24, 0.7, True),    # up to five-byte codes
]


@pytest.mark.parametrize("n,d,s,mono", PP_CASES)
def test_ppvbs_scan_bytes_brute_force(B, n, d, s, mono):
    v = synth.config_sweep_column(n, d, s, 100 + d, monotone=mono)
    ocol = orc.OracleColumn(v, "ppvbs")
    col = B.bs_encode_column(v, "ppvbs", host_only=True)
    nwords = (n + 31) // 32
    picks = [int(v[7]), int(v[n // 2]), int(ocol.A[0]), int(ocol.A[-1]), int(ocol.A[ocol.A.size // 3])]
    for x in picks:
        lc = _lit_code(ocol, x)
        for op in ("lt", "le", "gt", "ge", "eq", "ne"):
            need_eq = op not in ("lt", "ge")
            want = ppvbs_replay(ocol, [lc], [need_eq])
            got = B.bs_scan_bytes(col, op, x)
            for k, w in want.items():
                assert got[k] == w, (x, op, k, got[k], w)
            assert got["result_bytes"] == 4 * nwords
            assert got["bytes"] == sum(want.values()) + 4 * nwords
    # BETWEEN: the lower end never needs "equal", the upper end does
    for a, b in ((picks[2], picks[1]), (picks[0], picks[3])):
        lo, hi = min(a, b), max(a, b)
        want = ppvbs_replay(ocol, [_lit_code(ocol, lo), _lit_code(ocol, hi)], [False, True])
        got = B.bs_scan_bytes(col, "between", lo, hi)
        for k, w in want.items():
            assert got[k] == w, ("between", lo, hi, k)
    # seeded: rows outside the seed are not scanned
    seed = orc.scan_values(v, "lt", int(np.median(v)))
    seed[: seed.size // 3] = 0
    lc = _lit_code(ocol, picks[1])
    want = ppvbs_replay(ocol, [lc], [True], seed=seed)
    got = B.bs_scan_bytes(col, "eq", picks[1], seed=seed)
    for k, w in want.items():
        assert got[k] == w, ("seeded", k)
    assert got["result_bytes"] == 8 * nwords


@pytest.mark.parametrize("n,d,s,mono", PP_CASES)
def test_ppvbs_lookup_and_fused_bytes_brute_force(B, n, d, s, mono):
    v = synth.config_sweep_column(n, d, s, 200 + d, monotone=mono)
    ocol = orc.OracleColumn(v, "ppvbs")
    col = B.bs_encode_column(v, "ppvbs", host_only=True)
    n, K = ocol.n, ocol.K
    lens = ocol.row_lens.astype(np.int64)
    rows = np.arange(n)
    nwords = (n + 31) // 32
    for op, t in (("lt", 0.1), ("ge", 0.6), ("eq", 0.02)):
        x, _ = synth.pick_literals(v, op, t, 3)
        x = int(ocol.A[min(int(np.searchsorted(ocol.A, x)), ocol.A.size - 1)])
        sel = orc.scan_values(v, op, x)
        picked = np.unpackbits(sel.view(np.uint8), bitorder="little")[:n].astype(bool)
        m = int(picked.sum())
        # lookup alone
        got = B.bs_lookup_bytes(col, sel)
        tile, q = rows // TILE, rows % TILE
        dense = 32 * sectors((tile * TILE + tile_pos(q))[picked])
        group = rows >> 8
        mask = off = deep = 0
        for j in range(2, K + 1):
            g = np.unique(group[picked & (lens >= j - 1)])
            mask += 32 * g.size
            off += 32 * sectors(g * 4)
            deep += 32 * sectors(deep_positions(ocol.masks[j - 2], n)[picked & (lens >= j)])
        assert got["selected"] == m and got["out_bytes"] == 4 * m and got["bits_bytes"] == 4 * nwords
        assert (got["dense_bytes"], got["mask_bytes"], got["offset_bytes"], got["deep_bytes"]) == \
            (dense, mask, off, deep), (op, x)
        # fused: the scan's sectors and the lookup's, each once
        want = ppvbs_replay(ocol, [_lit_code(ocol, x)], [op not in ("lt", "ge")], sel=sel)
        for wb in (True, False):
            f = B.bs_scan_lookup_bytes(col, op, x, 0, sel, write_bits=wb)
            for k, w in want.items():
                assert f[k] == w, (op, x, k, f[k], w)
            assert f["result_bytes"] == 4 * m + (4 * nwords if wb else 0)
            assert f["bytes"] == sum(want.values()) + f["result_bytes"]


@pytest.mark.parametrize("d", [9, 16, 20])
def test_byteslice_scan_and_lookup_bytes_brute_force(B, d):
    n = 25_003
    v = synth.config_sweep_column(n, d, 1.0, 300 + d)
    ocol = orc.OracleColumn(v, "byteslice")
    col = B.bs_encode_column(v, "byteslice", host_only=True)
    k = ocol.k
    S = (k + 7) // 8
    lb_codes = ocol.row_codes.astype(np.uint64) << np.uint64(8 * S - k)
    cb = code_bytes(lb_codes, np.full(n, S), S)
    rows = np.arange(n)
    tile, q = rows // TILE, rows % TILE
    lane = tile * 32 + (q >> 5)
    nwords = (n + 31) // 32
    for x in (int(v[5]), int(v[n // 3]), int(ocol.A[0]), int(ocol.A[-1])):
        rank = int(np.searchsorted(ocol.A, x))
        lit = code_bytes(np.array([rank << (8 * S - k)], dtype=np.uint64), np.array([S]), S)[0]
        got = B.bs_scan_bytes(col, "eq", x)
        # slice 1 by every lane; slice s by lanes with a row equal over bytes 1..s-1
        dense = 0
        eq = np.ones(n, dtype=bool)
        for s in range(1, S + 1):
            if s > 1:
                eq &= cb[:, s - 1] == lit[s - 1]
            act = lane[eq] if s > 1 else lane
            pairs = np.unique(act >> 1)
            dense += 64 * pairs.size
        assert got["dense_bytes"] == dense, (d, x)
        assert got["bytes"] == dense + 4 * nwords
    sel = orc.scan_values(v, "lt", int(np.median(v)))
    picked = np.unpackbits(sel.view(np.uint8), bitorder="little")[:n].astype(bool)
    got = B.bs_lookup_bytes(col, sel)
    slice_bytes = ((n + TILE - 1) // TILE) * TILE
    want = 0
    for s in range(S):
        want += 32 * sectors((s * slice_bytes + tile * TILE + tile_pos(q))[picked])
    assert got["dense_bytes"] == want


@pytest.mark.parametrize("k", [5, 13, 27])
def test_bitpacked_lookup_bytes_brute_force(B, k):
    n = 20_011
    v = (synth.u64(k, 4, n) % np.uint64(1 << k)).astype(np.int32)
    col = B.bs_encode_column(v, "bitpacked", domain_bits=k, host_only=True)
    sel = orc.scan_values(v, "lt", int(np.median(v)))
    picked = np.flatnonzero(np.unpackbits(sel.view(np.uint8), bitorder="little")[:n])
    first = (picked * k) >> 3
    last = (picked * k + k - 1) >> 3
    got = B.bs_lookup_bytes(col, sel)
    assert got["dense_bytes"] == 32 * sectors(np.concatenate([first, last]))
    f = B.bs_scan_lookup_bytes(col, "lt", int(np.median(v)), 0, sel, write_bits=True)
    s = B.bs_scan_bytes(col, "lt", int(np.median(v)))
    assert f["dense_bytes"] == s["dense_bytes"] == 4 * k * ((n + 31) // 32)
    assert f["result_bytes"] == 4 * picked.size + 4 * ((n + 31) // 32)
