"""Categorical PP-VBS (Algorithm 2): equality scans, conjunctions, lookups by
bit vector and by row id, and the batched form, against the oracle's plain
evaluation -- one-, two- and three-level trees."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00220_gb300 import build_lib
    build_lib.build()
    from paper_2209_00220_gb300 import bytestore
    return bytestore


CASES = [  # (rows, code width d, Zipf s, seed): trees of 1, 2 and 3 levels
    (300007, 8, 1.0, 1),
    ((1 << 20) + 77, 12, 1.2, 2),
    (1 << 21, 20, 0.3, 3),
]


def _literals(v):
    a, q = np.unique(v, return_counts=True)
    order = np.lexsort((a, -q))
    absent = int(a.max()) + 1 if a.max() < np.iinfo(np.int32).max else int(a.min()) - 1
    return [int(a[order[0]]), int(a[order[len(order) // 2]]), int(a[order[-1]]), absent]


@pytest.mark.parametrize("n,d,s,seed", CASES)
def test_equality_scans_and_lookups(B, n, d, s, seed):
    import torch
    v = synth.config_sweep_column(n, d, s, seed)
    col = B.bs_encode_column(v, "ppvbs", categorical=True)
    ocol = orc.OracleColumn(v, "ppvbs", categorical=True)
    assert np.array_equal(ocol.decode_values(), v)
    for lit in _literals(v):
        for op in ("eq", "ne"):
            want = orc.scan_values(v, op, lit)
            bits = B.bs_scan(col, op, lit)
            assert np.array_equal(bits[: want.size].cpu().numpy().view(np.uint32), want), (op, lit)
            vals, cnt = B.bs_lookup(col, bits)
            wv = orc.lookup(v, want)
            assert int(cnt.item()) == wv.size
            assert np.array_equal(vals[: wv.size].cpu().numpy(), wv), (op, lit)
    rows = (synth.u64(seed, 3, 5000) % np.uint64(n)).astype(np.uint32)
    got = B.bs_lookup_rowids(col, torch.from_numpy(rows.view(np.int32)).cuda())
    assert np.array_equal(got.cpu().numpy(), v[rows.astype(np.int64)])
    with pytest.raises(B.BsError):
        B.bs_scan(col, "lt", int(v[0]))
    assert B.bs_last_device_error() == 0


def test_conjunction_and_batch_with_numerical_column(B):
    import torch
    n = (1 << 20) + 5
    vc = synth.config_sweep_column(n, 16, 1.1, 11)
    vn = synth.config_sweep_column(n, 12, 1.0, 12)
    cc = B.bs_encode_column(vc, "ppvbs", categorical=True)
    cn = B.bs_encode_column(vn, "ppvbs")
    lit = _literals(vc)[1]
    a, _ = synth.pick_literals(vn, "lt", 0.4, 1)
    want = orc.scan_values(vc, "ne", lit) & orc.scan_values(vn, "lt", a)
    bits = B.bs_scan_conj([(cc, "ne", lit), (cn, "lt", a)])
    assert np.array_equal(bits[: want.size].cpu().numpy().view(np.uint32), want)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    batch = B.bs_batch_create([{"preds": [(cn, "lt", a), (cc, "ne", lit)], "proj": cc, "out": out, "count": cnt}])
    batch.launch()
    torch.cuda.synchronize()
    wv = orc.lookup(vc, want)
    assert int(cnt.item()) == wv.size and np.array_equal(out[: wv.size].cpu().numpy(), wv)
    assert B.bs_last_device_error() == 0


def test_advisor_categorical_timed(B):
    v = synth.config_sweep_column(1 << 21, 14, 1.0, 21)
    t = B.bs_advise_layout(v, B.ADVISE_TIMED, categorical=True)
    m = B.bs_advise_layout(v, B.ADVISE_BYTES_MODEL, categorical=True, host_only=True)
    assert t["layout"] in ("byteslice", "ppvbs") and t["selectivity"] == m["selectivity"]
    assert min(t["cost_ppvbs"]) > 0
    assert B.bs_last_device_error() == 0
