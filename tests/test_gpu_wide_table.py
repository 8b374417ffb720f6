"""Synthetic denormalised wide table: 20 int32 columns (categorical, date-like
day counts, a monotone id, heavy-tailed amounts, mixed uniform / Zipf; see
synth.WIDE_TABLE), each stored in the layout the advisor (Algorithm 5,
deterministic mode) picks for it; seeded conjunctive queries of 1-4 predicates
(Section 3.3.1) followed by lookups of 2-4 projected columns. Every bit vector
and every looked-up value equals the plain evaluation on the plain values."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth

pytestmark = pytest.mark.gpu

NAMES = [w[0] for w in synth.WIDE_TABLE]


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00220_gb300 import build_lib
    build_lib.build()
    from paper_2209_00220_gb300 import bytestore
    return bytestore


def _table(B, n, seed, advise_rows):
    vals, cols, layouts = [], [], []
    for nm in NAMES:
        v = synth.wide_table_column(nm, n, seed)
        lay = B.bs_advise_layout(v[:advise_rows], B.ADVISE_BYTES_MODEL, host_only=True)["layout"]
        vals.append(v)
        cols.append(B.bs_encode_column(v, lay))
        layouts.append(lay)
    return vals, cols, layouts


def _queries(count, seed):
    r = synth.u64(seed, 77, 16 * count)
    out = []
    for i in range(count):
        order = synth.permutation(len(NAMES), seed * 1000 + i)
        npred = 1 + int(r[i] % np.uint64(4))
        nproj = 2 + int(r[count + i] % np.uint64(3))
        preds = []
        for j in range(npred):
            op = ("lt", "eq", "between")[int(r[(2 + j) * count + i] % np.uint64(3))]
            tgt = 10 ** (-2 + 1.8 * float(r[(6 + j) * count + i] >> np.uint64(11)) / float(1 << 53))
            preds.append((int(order[j]), op, tgt))
        proj = [int(x) for x in order[len(NAMES) - nproj:]]
        out.append((preds, proj))
    return out


def _run(B, vals, cols, queries, seed):
    import torch
    n = vals[0].size
    bits = torch.empty((n + 31) // 32, dtype=torch.int32, device="cuda")
    for qi, (preds, proj) in enumerate(queries):
        ps, want = [], None
        for j, (ci, op, tgt) in enumerate(preds):
            a, b = synth.pick_literals(vals[ci], op, tgt, seed + qi * 4 + j)
            ps.append((cols[ci], op, a, b))
            w = orc.scan_values(vals[ci], op, a, b)
            want = w if want is None else (want & w)
        B.bs_scan_conj(ps, out=bits)
        got = bits[: want.size].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), (qi, [(NAMES[p[0]], p[1]) for p in preds])
        for pj in proj:
            out, cnt = B.bs_lookup(cols[pj], bits)
            wv = orc.lookup(vals[pj], want)
            assert int(cnt.item()) == wv.size, (qi, NAMES[pj])
            assert np.array_equal(out[: wv.size].cpu().numpy(), wv), (qi, NAMES[pj])


def test_wide_table_small(B):
    n = (1 << 20) + 333  # ragged last tile
    vals, cols, layouts = _table(B, n, 0, n)
    assert {"byteslice", "ppvbs"} <= set(layouts)
    _run(B, vals, cols, _queries(100, 5), 5)
    assert B.bs_last_device_error() == 0


@pytest.mark.slow
def test_wide_table_full_size(B):
    # 2^26 rows x 20 columns; the advisor profiles each column's first 2^22 rows
    n = 1 << 26
    vals, cols, layouts = _table(B, n, 1, 1 << 22)
    _run(B, vals, cols, _queries(40, 6), 6)
    assert B.bs_last_device_error() == 0
