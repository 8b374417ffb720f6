"""GPU parity of the lookup on columns whose dictionary is a run of
consecutive integers, the shape of many real columns (ids, day numbers, small
counters, any domain whose every value occurs).

Algorithm 1 gives the values of one leaf consecutive codes 1, 2, ... after
their first byte, in dictionary order, and the lookup decodes a code of three
or more bytes as dictionary entry leaf2[first two bytes] + rest - 1. On a
dictionary of consecutive integers that entry is the run's first value plus
the index, so the lookup computes it instead of reading it (as it does for
ByteSlice and Bit-Packed codes, which index the sorted dictionary directly),
and a decode that is off by one code shows up as a value off by one. Each
case takes a Zipf column, maps its distinct values onto a run of consecutive
integers (or onto a run with one hole, which must read the dictionary), and
compares bs_lookup and bs_scan_lookup with the oracle's decode at several
predicates and selectivities, for codes of two to five bytes and runs that
end at the int32 limits; the ByteSlice and Bit-Packed cases do the same for
dictionary-coded columns."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth

pytestmark = pytest.mark.gpu

INT32_MIN, INT32_MAX = -(1 << 31), (1 << 31) - 1


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
    return t.cpu().numpy().view(np.uint32)[: (n + 31) // 32]


def _run(v, base, gap_at=None):
    """v's distinct values mapped, in order, onto base, base + 1, ...; with
    gap_at, the values from that rank on move up by one (a run with a hole)."""
    u, inv = np.unique(v, return_inverse=True)
    r = inv.astype(np.int64) + base
    if gap_at is not None:
        r += inv >= gap_at
    assert r.min() >= INT32_MIN and r.max() <= INT32_MAX
    return r.astype(np.int32)


def _cases():
    n = (1 << 20) + 12345  # 64 chunks of 16 tiles and a ragged last tile
    z1 = synth.config_sweep_column(n, 12, 1.0, 71)
    z15 = synth.config_sweep_column(n, 11, 1.5, 72)
    uni = synth.config_sweep_column(n, 10, 0.0, 73)
    mono = synth.config_sweep_column(n, 12, 1.0, 73, monotone=True)
    nd1 = np.unique(z1).size
    yield "d12_zipf1_from0", _run(z1, 0), True, 2
    yield "d12_zipf1_negative", _run(z1, -1234567), True, 2
    yield "d12_zipf1_to_int32_max", _run(z1, INT32_MAX - nd1 + 1), True, 2
    yield "d12_zipf1_from_int32_min", _run(z1, INT32_MIN), True, 2
    yield "d11_zipf15_skewed", _run(z15, 1000), True, 2
    yield "d10_uniform", _run(uni, -5), True, 2
    yield "d12_zipf1_one_gap", _run(z1, 0, gap_at=nd1 // 2), False, 2
    yield "d12_zipf1_gap_first", _run(z1, 0, gap_at=1), False, 2
    yield "d12_monotone_k4", _run(mono, -5), True, 4
    # codes of three to five bytes: the value of a long code is entry
    # leaf2[first two bytes] + rest - 1 of the dictionary, which for a run of
    # consecutive integers is that run's first value plus the index
    u16 = synth.config_sweep_column(n, 16, 0.0, 81)
    z16 = synth.config_sweep_column(n, 16, 1.0, 82)
    z20 = synth.config_sweep_column(n, 20, 0.5, 83)
    u24 = synth.config_sweep_column(n, 24, 0.0, 84)
    m24 = synth.config_sweep_column(n, 24, 0.7, 85, monotone=True)
    m20 = synth.config_sweep_column(n, 20, 1.0, 86, monotone=True)
    nd24 = np.unique(u24).size
    yield "d16_uniform_k3", _run(u16, 0), True, 3
    yield "d16_zipf1_k3_one_gap", _run(z16, -40, gap_at=777), False, 3
    yield "d20_zipf05_k4", _run(z20, -300), True, 4
    yield "d24_uniform_k4_to_int32_max", _run(u24, INT32_MAX - nd24 + 1), True, 4
    yield "d24_uniform_k4_one_gap", _run(u24, 5, gap_at=nd24 - 2), False, 4
    yield "monotone_d24_k5_from_int32_min", _run(m24, INT32_MIN), True, 5
    yield "monotone_d20_k5_one_gap", _run(m20, 0, gap_at=1000), False, 5


CASES = list(_cases())


def _checks(v):
    out = []
    for op, t in (("lt", 0.001), ("lt", 0.137), ("ge", 0.5), ("eq", 0.01), ("between", 0.3), ("ne", 0.9)):
        a, b = synth.pick_literals(v, op, t, 3)
        out.append((op, a, b))
    return out


@pytest.mark.parametrize("name,values,dense,K", CASES, ids=[c[0] for c in CASES])
def test_dense_dictionary_lookup_matches_oracle(B, name, values, dense, K):
    import torch
    u = np.unique(values)
    assert (int(u[-1]) - int(u[0]) + 1 == u.size) == dense
    col = B.bs_encode_column(values, "ppvbs")
    assert col.info()["max_code_bytes"] == K
    hist = col.info()["len_hist"]
    assert hist[1] > 0 and hist[2] > 0  # one- and two-byte codes both occur
    dec = orc.OracleColumn(values, "ppvbs").decode_values()
    assert np.array_equal(dec, values)
    n = values.size
    out = torch.full((n + 64,), -7, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.bs_scan_lookup_workspace_bytes(col) // 4 + 1, dtype=torch.int32, device="cuda")
    fbits = torch.empty(col.n_words, dtype=torch.int32, device="cuda")
    for op, a, b in _checks(values):
        want_bits = orc.scan_values(dec, op, a, b)
        want = orc.lookup(dec, want_bits)
        bits = B.bs_scan(col, op, a, b)
        assert np.array_equal(_bits(bits, n), want_bits), (name, op, a, b)
        got, cnt = B.bs_lookup(col, bits, out=out)
        assert int(cnt.item()) == want.size, (name, op, a, b)
        g = got.cpu().numpy()
        assert np.array_equal(g[: want.size], want), (name, op, a, b)
        assert np.all(g[want.size:] == -7), (name, op, a, b)
        out.fill_(-7)
        got, cnt = B.bs_scan_lookup([(col, op, a, b)], out=out, bits=fbits, workspace=ws)
        assert int(cnt.item()) == want.size, (name, "fused", op, a, b)
        g = got.cpu().numpy()
        assert np.array_equal(g[: want.size], want), (name, "fused", op, a, b)
        assert np.all(g[want.size:] == -7), (name, "fused", op, a, b)
        assert np.array_equal(_bits(fbits, n), want_bits), (name, "fused", op, a, b)
        out.fill_(-7)
    assert B.bs_last_device_error() == 0


def test_dense_dictionary_projection_of_other_column(B):
    """A predicate on one column projected onto a dense-dictionary column:
    the values come from the projected column's own decode tables."""
    import torch
    n = 300007
    pv = _run(synth.config_sweep_column(n, 12, 1.0, 74), -77)
    fv = synth.config_sweep_column(n, 16, 0.5, 75)
    proj = B.bs_encode_column(pv, "ppvbs")
    filt = B.bs_encode_column(fv, "byteslice")
    assert proj.info()["max_code_bytes"] == 2
    dec = orc.OracleColumn(pv, "ppvbs").decode_values()
    a, _ = synth.pick_literals(fv, "lt", 0.4, 1)
    want = orc.lookup(dec, orc.scan_values(fv, "lt", a, 0))
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    got, cnt = B.bs_scan_lookup([(filt, "lt", a)], proj=proj, out=out)
    m = int(cnt.item())
    assert m == want.size
    assert np.array_equal(got[:m].cpu().numpy(), want)
    bits = B.bs_scan(filt, "lt", a)
    out.fill_(-7)
    got, cnt = B.bs_lookup(proj, bits, out=out)
    assert int(cnt.item()) == want.size
    assert np.array_equal(got[: want.size].cpu().numpy(), want)
    assert B.bs_last_device_error() == 0


@pytest.mark.parametrize("layout", ["byteslice", "bitpacked"])
def test_dense_dictionary_fixed_width_layouts(B, layout):
    """Dictionary-coded ByteSlice and Bit-Packed columns (no declared domain:
    the code is the value's index in the sorted dictionary)."""
    import torch
    n = (1 << 20) + 999
    z = synth.config_sweep_column(n, 12, 1.0, 87)
    u = synth.config_sweep_column(n, 20, 0.0, 88)
    cases = (("d12_run", _run(z, -9)), ("d12_one_gap", _run(z, -9, gap_at=100)),
             ("d20_run_to_int32_max", _run(u, INT32_MAX - np.unique(u).size + 1)),
             ("d20_run_from_int32_min", _run(u, INT32_MIN)))
    out = torch.full((n + 64,), -7, dtype=torch.int32, device="cuda")
    for name, values in cases:
        col = B.bs_encode_column(values, layout)
        assert col.info()["n_dict"] == np.unique(values).size, name
        dec = orc.OracleColumn(values, layout).decode_values()
        assert np.array_equal(dec, values), name
        for op, a, b in _checks(values):
            want = orc.lookup(values, orc.scan_values(values, op, a, b))
            bits = B.bs_scan(col, op, a, b)
            got, cnt = B.bs_lookup(col, bits, out=out)
            assert int(cnt.item()) == want.size, (name, op, a, b)
            g = got.cpu().numpy()
            assert np.array_equal(g[: want.size], want), (name, op, a, b)
            assert np.all(g[want.size:] == -7), (name, op, a, b)
            out.fill_(-7)
            got, cnt = B.bs_scan_lookup([(col, op, a, b)], out=out)
            assert int(cnt.item()) == want.size, (name, "fused", op, a, b)
            assert np.array_equal(got[: want.size].cpu().numpy(), want), (name, "fused", op, a, b)
            out.fill_(-7)
    assert B.bs_last_device_error() == 0
