"""GPU parity of the lookup on PP-VBS columns whose dictionary is a run of
consecutive integers, the shape of many real columns (ids, day numbers,
small counters).

Algorithm 1 gives the values of one leaf consecutive codes 1, 2, ... after
their first byte, in dictionary order; on such columns a neighbouring value
differs from its code's neighbour by one, so a decode that is off by one code
(a wrong BS_2 rank, a wrong leaf) shows up here as a value off by one. Each
case takes a Zipf column, maps its distinct values onto a run of consecutive
integers (or onto a run with one hole), and compares bs_lookup and
bs_scan_lookup with the oracle's decode at several predicates and
selectivities, including runs that end at the int32 limits."""
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
    # a run of consecutive integers with codes of up to four bytes: the table path
    yield "d12_monotone_k4", _run(mono, -5), True, 4


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
