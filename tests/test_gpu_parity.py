"""GPU parity: every bit vector and lookup of the CUDA path equals the CPU
oracle's, bit for bit, on seeded inputs (several tiles plus a ragged tail),
the paper's worked example, an exhaustive small-alphabet code set, edge cases
and the full 2^30-row workload. All calls go through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth

pytestmark = pytest.mark.gpu

OPS = ("lt", "le", "gt", "ge", "eq", "ne")


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00220_gb300 import build_lib
    build_lib.build()
    from paper_2209_00220_gb300 import bytestore
    return bytestore


def _bits(t, n):
    w = t.cpu().numpy().view(np.uint32)[: (n + 31) // 32]
    return w


def _check_clean(B):
    assert B.bs_last_device_error() == 0


# ------------------------------------------------------------ code level
def test_worked_example_on_gpu(B):
    codes = np.array([0x81, 0xC0, 0x77A9, 0x8189], np.uint64)
    lens = np.array([1, 1, 2, 2], np.uint8)
    col = B.bs_column_from_codes(codes, lens, "ppvbs")
    got = _bits(B.bs_scan_code(col, "gt", 0x81, 1), 4)
    assert [(int(got[0]) >> i) & 1 for i in range(4)] == [0, 1, 0, 1]
    got = _bits(B.bs_scan_code(col, "gt", 0x8050, 2), 4)
    assert [(int(got[0]) >> i) & 1 for i in range(4)] == [1, 1, 0, 1]
    _check_clean(B)


def _alphabet_codes(max_len=3, alpha=(0, 1, 2, 0x7F, 0x80, 0xFE, 0xFF)):
    codes, lens = [], []
    for l in range(1, max_len + 1):
        for t in np.ndindex(*([len(alpha)] * l)):
            bs_ = [alpha[i] for i in t]
            if bs_[-1] == 0:
                continue
            c = 0
            for b in bs_:
                c = (c << 8) | b
            codes.append(c)
            lens.append(l)
    return np.array(codes, np.uint64), np.array(lens, np.uint8)


def test_exhaustive_small_alphabet(B):
    import torch
    codes, lens = _alphabet_codes()
    n = 5000  # five tiles and a ragged tail
    idx = (synth.u64(5, 1, n) % np.uint64(codes.size)).astype(np.int64)
    col = B.bs_column_from_codes(codes[idx], lens[idx], "ppvbs")
    K = 4  # literals may be one byte longer than any stored code
    padded = orc.pad(codes[idx], lens[idx], K)
    lit_codes, lit_lens = _alphabet_codes(4)
    pick = np.concatenate([np.arange(codes.size), codes.size + (synth.u64(6, 2, 60) %
                                                                np.uint64(lit_codes.size - codes.size)).astype(np.int64)])
    out = torch.empty(col.n_words, dtype=torch.int32, device="cuda")
    for i in pick:
        lc, ll = int(lit_codes[i]), int(lit_lens[i])
        lp = lc << (8 * (K - ll))
        for op in OPS:
            got = _bits(B.bs_scan_code(col, op, lc, ll, out=out), n)
            want = orc.scan_codes(padded, op, lp)
            assert np.array_equal(got, want), (hex(lc), ll, op)
    # BETWEEN on a sample of literal pairs
    pairs = (synth.u64(7, 3, 400) % np.uint64(lit_codes.size)).astype(np.int64).reshape(-1, 2)
    for a, b in pairs:
        la, lb = int(lit_lens[a]), int(lit_lens[b])
        got = _bits(B.bs_scan_code(col, "between", int(lit_codes[a]), la, int(lit_codes[b]), lb, out=out), n)
        want = orc.scan_codes(padded, "between", int(lit_codes[a]) << (8 * (K - la)),
                              int(lit_codes[b]) << (8 * (K - lb)))
        assert np.array_equal(got, want)
    # zero-padded codes read back by the lookup (Algorithm 4's output)
    allbits = B.bs_scan_code(col, "ge", 0, 1, out=out)
    vals, cnt = B.bs_lookup_codes(col, allbits)
    assert int(cnt.item()) == n
    assert np.array_equal(vals[:n].cpu().numpy().view(np.uint64), orc.pad(codes[idx], lens[idx], 3))
    _check_clean(B)


# ----------------------------------------------------------- value level
def _value_cases():
    v1, dom = synth.config_single_column(seed=0, n=150000)
    yield "single_column_zipf1", v1, {"byteslice": {"domain_values": dom}, "bitpacked": {"domain_values": dom}}
    yield "d12_zipf1", synth.config_sweep_column(70001, 12, 1.0, 11), {}
    yield "d16_uniform", synth.config_sweep_column(50007, 16, 0.0, 12), {}
    yield "d20_zipf15", synth.config_sweep_column(80000, 20, 1.5, 13), {}
    yield "monotone_d16_beta", synth.config_sweep_column(90000, 16, 1.0, 14, monotone=True), {}
    yield "monotone_d24_K5", synth.config_sweep_column(400000, 24, 0.7, 15, monotone=True), {}
    yield "d32_zipf05", synth.config_sweep_column(60000, 32, 0.5, 16), {
        "byteslice": {"domain_bits": 32, "domain_min": -(1 << 31)},
        "bitpacked": {"domain_bits": 32, "domain_min": -(1 << 31)}}
    yield "d8_declared", synth.config_sweep_column(33000, 8, 1.0, 17), {
        "byteslice": {"domain_bits": 8}, "bitpacked": {"domain_bits": 8}}
    # Gaussian data (Section 6's additional experiments): narrow and wide
    yield "gauss_d16_narrow", synth.gaussian_column(120000, 16, 0.01, 18), {}
    yield "gauss_d20_wide", synth.gaussian_column(90000, 20, 0.2, 19), {}


def _literals(v, seed):
    u = np.unique(v)
    picks = [int(u[0]) - 1, int(u[0]), int(u[-1]), int(u[-1]) + 1, -(1 << 31), (1 << 31) - 1]
    picks += [int(x) for x in u[(synth.u64(seed, 4, 12) % np.uint64(u.size)).astype(np.int64)]]
    picks += [int(x) + 1 for x in u[(synth.u64(seed, 5, 6) % np.uint64(u.size)).astype(np.int64)]]  # often absent
    for op in ("lt", "eq", "between"):
        for t in (0.001, 0.1, 0.5, 0.9):
            a, b = synth.pick_literals(v, op, t, seed)
            picks += [a, b]
    return sorted(set(max(-(1 << 31), min((1 << 31) - 1, p)) for p in picks))


CASES = list(_value_cases())


@pytest.mark.parametrize("layout", ["ppvbs", "byteslice", "bitpacked"])
@pytest.mark.parametrize("name,values,extra", CASES, ids=[c[0] for c in CASES])
def test_scan_and_lookup_match_oracle(B, layout, name, values, extra):
    import torch
    opts = extra.get(layout, {})
    col = B.bs_encode_column(values, layout, **opts)
    ocol = orc.OracleColumn(values, layout, **({"domain": opts["domain_values"]} if "domain_values" in opts else
                                                {k: v for k, v in opts.items()}))
    dec = ocol.decode_values()
    assert np.array_equal(dec, values)
    n = values.size
    out = torch.empty(col.n_words, dtype=torch.int32, device="cuda")
    lits = _literals(values, n)
    for x in lits:
        for op in OPS:
            got = _bits(B.bs_scan(col, op, x, out=out), n)
            want = orc.scan_values(dec, op, x)
            assert np.array_equal(got, want), (name, layout, op, x)
    pairs = list(zip(lits[::2], lits[1::2])) + [(lits[-1], lits[0]), (lits[3], lits[3])]
    for a, b in pairs:
        got = _bits(B.bs_scan(col, "between", a, b, out=out), n)
        assert np.array_equal(got, orc.scan_values(dec, "between", a, b)), (name, layout, a, b)
    # lookup of a few results, and the row-id lookup
    for op, t in (("lt", 0.1), ("ge", 0.5), ("eq", 0.01)):
        a, _ = synth.pick_literals(values, op, t, 3)
        bits = B.bs_scan(col, op, a)
        vals, cnt = B.bs_lookup(col, bits)
        want = orc.lookup(dec, _bits(bits, n))
        assert int(cnt.item()) == want.size
        assert np.array_equal(vals[: want.size].cpu().numpy(), want), (name, layout, op)
    rid = torch.from_numpy((synth.u64(n, 9, 3000) % np.uint64(n)).astype(np.int32)).cuda()
    got = B.bs_lookup_rowids(col, rid).cpu().numpy()
    assert np.array_equal(got, orc.lookup_rowids(dec, rid.cpu().numpy().view(np.uint32)))
    _check_clean(B)


LONG_CODE_CASES = [
    # (rows, code width d, Zipf s, monotone): K = 4 with every length 1..4 present
    (300000, 24, 0.0, False),
    (200000, 20, 1.0, True),
    # K = 3, nearly all codes two bytes long
    (250007, 16, 0.0, False),
]


@pytest.mark.parametrize("n,d,s,mono", LONG_CODE_CASES)
def test_lookup_dense_tiles_long_codes(B, n, d, s, mono):
    """Lookups of columns whose codes reach three or four bytes, at
    selectivities that make every tile dense (the staged path) and sparse ones,
    plus a capacity smaller than the count; the values equal the oracle's."""
    import torch
    v = synth.config_sweep_column(n, d, s, 40 + d, monotone=mono)
    col = B.bs_encode_column(v, "ppvbs")
    assert col.info()["max_code_bytes"] in (3, 4)
    dec = orc.OracleColumn(v, "ppvbs").decode_values()
    for op, t in (("lt", 0.05), ("lt", 0.5), ("ge", 0.2), ("gt", 0.9), ("ne", 0.01), ("eq", 0.01)):
        a, _ = synth.pick_literals(v, op, t, 5)
        bits = B.bs_scan(col, op, a)
        sel = _bits(bits, n)
        want = orc.lookup(dec, sel)
        vals, cnt = B.bs_lookup(col, bits)
        assert int(cnt.item()) == want.size
        assert np.array_equal(vals[: want.size].cpu().numpy(), want), (op, t)
        if want.size > 10:
            cap = want.size // 3 + 1
            out = torch.full((cap + 8,), -7, dtype=torch.int32, device="cuda")
            vals, cnt = B.bs_lookup(col, bits, out=out, out_cap=cap)
            got = out.cpu().numpy()
            assert int(cnt.item()) == want.size
            assert np.array_equal(got[:cap], want[:cap]) and np.all(got[cap:] == -7), (op, t)
    _check_clean(B)


@pytest.mark.parametrize("layout", ["ppvbs", "byteslice", "bitpacked"])
def test_seeded_scans_and_conjunction(B, layout):
    import torch
    n = 123457
    cols_v = [synth.config_sweep_column(n, d, s, 20 + d) for d, s in ((12, 1.0), (16, 0.5), (10, 1.5), (20, 0.0))]
    cols = [B.bs_encode_column(v, layout) for v in cols_v]
    preds = []
    for i, v in enumerate(cols_v):
        op = ("lt", "ge", "between", "ne")[i]
        a, b = synth.pick_literals(v, op, (0.3, 0.6, 0.5, 0.9)[i], i)
        preds.append((cols[i], op, a, b))
    want = None
    for (c, op, a, b), v in zip(preds, cols_v):
        w = orc.scan_values(v, op, a, b)
        want = w if want is None else (want & w)
        got = _bits(B.bs_scan_conj(preds[: preds.index((c, op, a, b)) + 1]), n)
        assert np.array_equal(got, want)
    # an explicit seed that is zero on whole tiles
    seed_np = orc.scan_values(cols_v[0], "lt", int(np.quantile(cols_v[0], 0.05)))
    seed_np[: len(seed_np) // 2] = 0
    seed = torch.from_numpy(seed_np.view(np.int32).copy()).cuda()
    got = _bits(B.bs_scan_seeded(cols[1], "ge", preds[1][2], 0, seed), n)
    assert np.array_equal(got, seed_np & orc.scan_values(cols_v[1], "ge", preds[1][2]))
    _check_clean(B)


# ------------------------------------------------------------- edge cases
@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1023, 1024, 1025, 16385])
@pytest.mark.parametrize("layout", ["ppvbs", "byteslice", "bitpacked"])
def test_sizes_and_ragged_tails(B, n, layout):
    import torch
    v = synth.config_sweep_column(max(n, 1), 9, 1.0, n)[:n]
    col = B.bs_encode_column(v, layout)
    x = int(np.median(v)) if n else 0
    out = torch.full((max(1, (n + 31) // 32) + 1,), -1, dtype=torch.int32, device="cuda")
    B.bs_scan(col, "le", x, out=out)
    got = out.cpu().numpy().view(np.uint32)
    nw = (n + 31) // 32
    if n:
        assert np.array_equal(got[:nw], orc.scan_values(v, "le", x))
    assert got[nw] == 0xFFFFFFFF  # nothing written past ceil(n/32) words
    vals, cnt = B.bs_lookup(col, out)
    want = v[v <= x] if n else v[:0]
    assert int(cnt.item()) == want.size
    assert np.array_equal(vals[: want.size].cpu().numpy(), want)
    _check_clean(B)


def test_constant_column_and_capacity(B):
    import torch
    v = np.full(5000, 42, np.int32)
    for layout in ("ppvbs", "byteslice", "bitpacked"):
        col = B.bs_encode_column(v, layout)
        for op, x, cnt_want in (("eq", 42, 5000), ("lt", 42, 0), ("gt", 41, 5000), ("ne", 42, 0), ("eq", 43, 0)):
            bits = B.bs_scan(col, op, x)
            got = np.unpackbits(_bits(bits, 5000).view(np.uint8), bitorder="little")[:5000]
            assert int(got.sum()) == cnt_want, (layout, op, x)
        bits = B.bs_scan(col, "eq", 42)
        out = torch.full((1000,), -7, dtype=torch.int32, device="cuda")
        _, cnt = B.bs_lookup(col, bits, out=out, out_cap=100)
        assert int(cnt.item()) == 5000
        o = out.cpu().numpy()
        assert np.all(o[:100] == 42) and np.all(o[100:] == -7)
    _check_clean(B)


# ------------------------------------------------------- full-size workload
@pytest.mark.slow
def test_full_size_sweep_column(B):
    """2^30 rows, d = 12, Zipf 1.0, PP-VBS, as bench.py times it: the whole bit
    vector and every looked-up value of bs_scan + bs_lookup and of the fused
    bs_scan_lookup against the oracle, which decodes every row from its own
    layout of the column (about a minute of host time)."""
    import torch
    n = 1 << 30
    v = synth.config_sweep_column(n, 12, 1.0, 0)
    col = B.bs_encode_column(v, "ppvbs")
    lit, _ = synth.pick_literals(v, "lt", 0.10, 0)
    bits = B.bs_scan(col, "lt", lit)
    vals, cnt = B.bs_lookup(col, bits)
    torch.cuda.synchronize()
    got_bits = _bits(bits, n)
    got_vals = vals[: int(cnt.item())].cpu().numpy()
    # the fused scan + lookup on the same column, bit vector included
    fbits = torch.empty_like(bits)
    fvals, fcnt = B.bs_scan_lookup([(col, "lt", lit)], out=vals, bits=fbits)
    torch.cuda.synchronize()
    assert int(fcnt.item()) == got_vals.size
    assert torch.equal(fbits, bits)
    fused_vals = fvals[: int(fcnt.item())].cpu().numpy()
    del vals, bits, fbits, fvals, col
    ocol = orc.OracleColumn(v, "ppvbs")
    dec = ocol.decode_values()
    del ocol
    want = orc.scan_values(dec, "lt", lit)
    assert np.array_equal(got_bits, want)
    want_vals = orc.lookup(dec, want)
    assert got_vals.size == want_vals.size
    assert np.array_equal(got_vals, want_vals)
    assert np.array_equal(fused_vals, want_vals)
    _check_clean(B)
