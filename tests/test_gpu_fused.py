"""GPU parity of the fused scan + lookup (bs_scan_lookup): for every value
case, layout, predicate and selectivity from 0.01 % to 90 %, the values and
count equal the oracle's plain definition (Section 2.2: the values of the
projected column at the rows where every predicate holds, ascending), and the
optional bit vector equals the oracle's scan; also conjunctions of up to four
predicates over columns of different layouts projected onto another column,
ragged lengths around the two-tile work unit, and output capacities below the
count. All calls go through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth

pytestmark = pytest.mark.gpu

OPS = ("lt", "le", "gt", "ge", "eq", "ne")
TARGETS = (0.0001, 0.001, 0.01, 0.1, 0.5, 0.9)


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


def _cases():
    v1, dom = synth.config_single_column(seed=0, n=150001)
    yield "single_column_zipf1", v1, {"byteslice": {"domain_values": dom}, "bitpacked": {"domain_values": dom}}
    yield "d12_zipf1", synth.config_sweep_column(100003, 12, 1.0, 61), {}
    yield "d16_uniform", synth.config_sweep_column(70001, 16, 0.0, 62), {}
    yield "d20_zipf15", synth.config_sweep_column(80000, 20, 1.5, 63), {}
    yield "monotone_d16_beta", synth.config_sweep_column(90000, 16, 1.0, 64, monotone=True), {}
    yield "monotone_d24_K5", synth.config_sweep_column(400000, 24, 0.7, 65, monotone=True), {}
    yield "d32_zipf05", synth.config_sweep_column(60000, 32, 0.5, 66), {
        "byteslice": {"domain_bits": 32, "domain_min": -(1 << 31)},
        "bitpacked": {"domain_bits": 32, "domain_min": -(1 << 31)}}
    yield "gauss_d16_narrow", synth.gaussian_column(120000, 16, 0.01, 67), {}


def _oracle_col(values, layout, opts):
    return orc.OracleColumn(values, layout, **({"domain": opts["domain_values"]} if "domain_values" in opts else
                                               dict(opts)))


def _literals(v, seed):
    u = np.unique(v)
    picks = {int(u[0]) - 1, int(u[0]), int(u[-1]), int(u[-1]) + 1, -(1 << 31), (1 << 31) - 1}
    for op in ("lt", "eq", "between"):
        for t in TARGETS:
            a, b = synth.pick_literals(v, op, t, seed)
            picks.update((a, b))
    picks.update(int(x) for x in u[(synth.u64(seed, 4, 8) % np.uint64(u.size)).astype(np.int64)])
    return sorted(max(-(1 << 31), min((1 << 31) - 1, p)) for p in picks)


CASES = list(_cases())


@pytest.mark.parametrize("layout", ["ppvbs", "byteslice", "bitpacked"])
@pytest.mark.parametrize("name,values,extra", CASES, ids=[c[0] for c in CASES])
def test_fused_single_predicate_matches_oracle(B, layout, name, values, extra):
    import torch
    opts = extra.get(layout, {})
    col = B.bs_encode_column(values, layout, **opts)
    dec = _oracle_col(values, layout, opts).decode_values()
    assert np.array_equal(dec, values)
    n = values.size
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    bits = torch.empty(col.n_words, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(B.bs_scan_lookup_workspace_bytes(col) // 4 + 1, dtype=torch.int32, device="cuda")
    lits = _literals(values, 5)
    checks = [(op, x, 0) for x in lits for op in OPS]
    checks += [("between", a, b) for a, b in zip(lits[::2], lits[1::2])] + [("between", lits[-1], lits[0])]
    for op, a, b in checks:
        B.bs_scan_lookup([(col, op, a, b)], out=out, count=cnt, bits=bits, workspace=ws)
        want_bits = orc.scan_values(dec, op, a, b)
        want = orc.lookup(dec, want_bits)
        assert np.array_equal(_bits(bits, n), want_bits), (name, layout, op, a, b)
        m = int(cnt.item())
        assert m == want.size, (name, layout, op, a, b)
        assert np.array_equal(out[:m].cpu().numpy(), want), (name, layout, op, a, b)
    assert B.bs_last_device_error() == 0


@pytest.mark.parametrize("proj_layout", ["ppvbs", "byteslice", "bitpacked"])
def test_fused_conjunction_and_projection(B, proj_layout):
    """1..4 predicates over columns of mixed layouts, values of a fifth column."""
    import torch
    n = 200003
    specs = [(12, 1.0, "ppvbs"), (16, 0.5, "byteslice"), (10, 1.5, "bitpacked"), (20, 0.0, "ppvbs")]
    vals = [synth.config_sweep_column(n, d, s, 70 + d) for d, s, _ in specs]
    cols = [B.bs_encode_column(v, lay) for v, (_, _, lay) in zip(vals, specs)]
    pv = synth.config_sweep_column(n, 24, 0.8, 77, monotone=True)  # up to five-byte PP-VBS codes
    proj = B.bs_encode_column(pv, proj_layout)
    pdec = orc.OracleColumn(pv, proj_layout).decode_values()
    assert np.array_equal(pdec, pv)
    ops = ("lt", "ge", "between", "ne")
    for k in range(1, 5):
        for t in (0.001, 0.05, 0.6, 0.97):
            preds, mask = [], None
            for i in range(k):
                a, b = synth.pick_literals(vals[i], ops[i], t ** (1.0 / k), 11 * i + k)
                preds.append((cols[i], ops[i], a, b))
                w = orc.scan_values(vals[i], ops[i], a, b)
                mask = w if mask is None else (mask & w)
            bits = torch.empty(cols[0].n_words, dtype=torch.int32, device="cuda")
            got, cnt = B.bs_scan_lookup(preds, proj=proj, bits=bits)
            want = orc.lookup(pdec, mask)
            assert np.array_equal(_bits(bits, n), mask), (k, t)
            assert int(cnt.item()) == want.size, (k, t)
            assert np.array_equal(got[: want.size].cpu().numpy(), want), (k, t)
            # the same as the unfused calls
            b2 = B.bs_scan_conj(preds)
            v2, c2 = B.bs_lookup(proj, b2)
            assert int(c2.item()) == want.size
            assert np.array_equal(v2[: want.size].cpu().numpy(), want)
    assert B.bs_last_device_error() == 0


@pytest.mark.parametrize("n", [0, 1, 31, 1023, 1024, 1025, 2047, 2048, 2049, 4097, 16385, 65536 * 3 + 5])
@pytest.mark.parametrize("layout", ["ppvbs", "byteslice", "bitpacked"])
def test_fused_ragged_lengths(B, n, layout):
    import torch
    v = synth.config_sweep_column(max(n, 1), 11, 1.0, n + 3)[:n]
    col = B.bs_encode_column(v, layout)
    x = int(np.median(v)) if n else 0
    bits = torch.full((max(1, (n + 31) // 32) + 1,), -1, dtype=torch.int32, device="cuda")
    got, cnt = B.bs_scan_lookup([(col, "le", x)], bits=bits)
    want = v[v <= x] if n else v[:0]
    assert int(cnt.item()) == want.size
    assert np.array_equal(got[: want.size].cpu().numpy(), want)
    nw = (n + 31) // 32
    b = bits.cpu().numpy().view(np.uint32)
    if n:
        assert np.array_equal(b[:nw], orc.scan_values(v, "le", x))
    assert b[nw] == 0xFFFFFFFF  # nothing written past ceil(n/32) words
    assert B.bs_last_device_error() == 0


def test_fused_capacity_and_workspace(B):
    import torch
    n = 300001
    v = synth.config_sweep_column(n, 12, 1.0, 99)
    col = B.bs_encode_column(v, "ppvbs")
    a, _ = synth.pick_literals(v, "lt", 0.3, 1)
    want = v[v < a]
    cap = want.size // 3 + 1
    out = torch.full((cap + 100,), -7, dtype=torch.int32, device="cuda")
    got, cnt = B.bs_scan_lookup([(col, "lt", a)], out=out, out_cap=cap)
    o = out.cpu().numpy()
    assert int(cnt.item()) == want.size
    assert np.array_equal(o[:cap], want[:cap]) and np.all(o[cap:] == -7)
    # a workspace that is too small is refused before any launch
    small = torch.empty(8, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BsError):
        B.bs_scan_lookup([(col, "lt", a)], workspace=small)
    # the same workspace reused across calls (it is cleared by each call)
    ws = torch.empty(B.bs_scan_lookup_workspace_bytes(col) // 4 + 1, dtype=torch.int32, device="cuda")
    for op, t in (("lt", 0.1), ("ge", 0.7), ("eq", 0.01)):
        x, _ = synth.pick_literals(v, op, t, 2)
        got, cnt = B.bs_scan_lookup([(col, op, x)], workspace=ws)
        w = orc.lookup(v, orc.scan_values(v, op, x))
        assert int(cnt.item()) == w.size and np.array_equal(got[: w.size].cpu().numpy(), w)
    assert B.bs_last_device_error() == 0
