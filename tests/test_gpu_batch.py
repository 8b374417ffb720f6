"""Batched form: every request of a mixed batch (three layouts, uneven column
lengths, conjunctions of 1-4 predicates, projections onto another column)
gives exactly the bit vector, count and values of the plain per-query calls and
of the oracle -- alone and in the mix, graph-captured or launched directly."""
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


def _pool(B, seed=0):
    """Columns of uneven length, three layouts, several widths and skews."""
    pool = []
    specs = [(70001, 12, 1.0, "ppvbs"), (300000, 16, 0.5, "byteslice"), (40000, 9, 1.5, "bitpacked"),
             (1 << 20, 20, 1.0, "ppvbs"), (123457, 24, 0.0, "bitpacked"), (5000, 8, 1.2, "byteslice"),
             (250000, 32, 0.8, "ppvbs"), (1025, 10, 1.0, "ppvbs")]
    for i, (n, d, s, lay) in enumerate(specs):
        v = synth.config_sweep_column(n, d, s, seed + i)
        opts = {} if lay == "ppvbs" or i % 2 else {"domain_bits": d, "domain_min": synth.domain_min_for_bits(d)}
        pool.append((v, B.bs_encode_column(v, lay, **opts)))
    # a second column of the same length as pool[3] for conjunctions / projection
    v2 = synth.config_sweep_column(1 << 20, 14, 1.3, 99)
    pool.append((v2, B.bs_encode_column(v2, "byteslice")))
    return pool


def _mask(v, op, a, b):
    return {"lt": v < a, "le": v <= a, "gt": v > a, "ge": v >= a, "eq": v == a, "ne": v != a,
            "between": (v >= a) & (v <= b)}[op]


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_matches_plain_and_oracle(B, use_graph):
    import torch
    pool = _pool(B)
    reqs, expect = [], []
    rng = synth.u64(7, 1, 4000)
    ops = ("lt", "le", "gt", "ge", "eq", "ne", "between")
    for i in range(60):
        ci = int(rng[i] % np.uint64(len(pool) - 1))
        v, col = pool[ci]
        op = ops[int(rng[100 + i] % np.uint64(len(ops)))]
        tgt = float(10 ** (-3.5 + 3.2 * (int(rng[200 + i] % np.uint64(1000)) / 1000.0)))
        a, b = synth.pick_literals(v, op, tgt, i)
        preds = [(col, op, a, b)]
        mask = _mask(v, op, a, b)
        proj_v, proj = v, None
        if ci == 3 and i % 2 == 0:  # conjunction with a second column, projected on it
            v2, c2 = pool[-1]
            a2, _ = synth.pick_literals(v2, "lt", 0.6, i)
            preds.append((c2, "lt", a2))
            mask = mask & (v2 < a2)
            proj_v, proj = v2, c2
        n = v.size
        out = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        bits = torch.zeros((n + 31) // 32 + 1, dtype=torch.int32, device="cuda")
        reqs.append({"preds": preds, "out": out, "out_cap": n, "count": cnt, "bits": bits, "proj": proj})
        expect.append((mask, proj_v, preds, proj))
    batch = B.bs_batch_create(reqs, use_graph=use_graph)
    for _ in range(2):  # the second launch must reproduce the first
        batch.launch()
        torch.cuda.synchronize()
        for q, (mask, proj_v, preds, proj) in zip(reqs, expect):
            m = int(mask.sum())
            assert int(q["count"].item()) == m
            got = q["out"][:m].cpu().numpy()
            assert np.array_equal(got, proj_v[mask])
            assert int(q["out"][m].item()) == -7 or m == q["out_cap"]
            n = proj_v.size
            gbits = q["bits"].cpu().numpy().view(np.uint32)[: (n + 31) // 32]
            want = np.packbits(mask, bitorder="little")
            want = np.concatenate([want, np.zeros((-want.size) % 4, np.uint8)]).view("<u4")
            assert np.array_equal(gbits, want)
    # alone: the plain calls give the same values
    for q, (mask, proj_v, preds, proj) in list(zip(reqs, expect))[:12]:
        bits = B.bs_scan_conj([p for p in preds])
        col = proj if proj is not None else preds[0][0]
        vals, cnt = B.bs_lookup(col, bits)
        m = int(cnt.item())
        assert np.array_equal(vals[:m].cpu().numpy(), q["out"][:m].cpu().numpy())
    info = batch.info()
    assert info["ctas"] > 0 and info["threads"] in (128, 256, 512)
    if use_graph:
        print("batch shape", info)
    assert B.bs_last_device_error() == 0


def test_batch_capacity_and_autotune(B, tmp_path):
    import torch
    v = synth.config_sweep_column(200000, 12, 1.0, 5)
    col = B.bs_encode_column(v, "ppvbs")
    a, _ = synth.pick_literals(v, "lt", 0.3, 0)
    m = int((v < a).sum())
    out = torch.full((100,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    cache = str(tmp_path / "tune.jsonl")
    batch = B.bs_batch_create([{"preds": [(col, "lt", a)], "out": out, "out_cap": 50, "count": cnt}],
                              autotune=True, tune_cache=cache)
    batch.launch()
    torch.cuda.synchronize()
    assert int(cnt.item()) == m
    assert np.array_equal(out[:50].cpu().numpy(), v[v < a][:50]) and np.all(out[50:].cpu().numpy() == -1)
    text = open(cache).read()
    for key in ('"threads"', '"blocks_per_sm"', '"stages"', '"unit_chunks"', '"stop_rows"'):
        assert key in text
    sh = batch.shape()
    assert sh["stages"] in (2, 3, 4) and sh["unit_chunks"] in (1, 2, 4) and sh["stop_rows"] in (256, 1024)
    assert sh["persistent_requests"] == 1 and sh["single_query_requests"] == 0
    # a second batch with the same signature reuses the cached shape
    b2 = B.bs_batch_create([{"preds": [(col, "lt", a)], "out": out, "out_cap": 50, "count": cnt}],
                           tune_cache=cache)
    sh2 = b2.shape()
    for key in ("threads", "blocks_per_sm", "stages", "unit_chunks", "stop_rows"):
        assert sh2[key] == sh[key], key
    b2.launch()
    torch.cuda.synchronize()
    assert int(cnt.item()) == m
    assert B.bs_last_device_error() == 0


def test_long_columns_take_single_query_kernels_in_batch_and_server(B):
    # columns of 2^28 rows or more run the specialised single-query kernels
    # inside the batch (and the server's batches); a mix of long and short
    # requests must still give the oracle's results for every request
    import torch
    n = 1 << 28
    v1 = synth.config_sweep_column(n, 12, 1.0, 41)
    v2 = synth.config_sweep_column(n, 18, 0.6, 42)
    c1, c2 = B.bs_encode_column(v1, "ppvbs"), B.bs_encode_column(v2, "byteslice")
    vs = synth.config_sweep_column(70001, 12, 1.0, 43)
    cs = B.bs_encode_column(vs, "ppvbs")
    a1, _ = synth.pick_literals(v1, "lt", 0.05, 1)
    a2, b2 = synth.pick_literals(v2, "between", 0.3, 2)
    a3, _ = synth.pick_literals(vs, "lt", 0.2, 3)
    m1 = v1 < a1
    want_long = v1[m1]
    want_conj = v2[m1 & (v2 >= a2) & (v2 <= b2)]
    want_short = vs[vs < a3]
    cases = [([(c1, "lt", a1)], None, want_long), ([(c1, "lt", a1), (c2, "between", a2, b2)], c2, want_conj),
             ([(cs, "lt", a3)], None, want_short)]
    outs = [torch.empty(w.size + 7, dtype=torch.int32, device="cuda") for _, _, w in cases]
    cnts = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in cases]
    reqs = [{"preds": p, "proj": pj, "out": o, "count": c} for (p, pj, _), o, c in zip(cases, outs, cnts)]
    for use_graph in (True, False):
        batch = B.bs_batch_create(reqs, use_graph=use_graph)
        for o in outs:
            o.fill_(-1)
        batch.launch()
        torch.cuda.synchronize()
        for (p, pj, w), o, c in zip(cases, outs, cnts):
            assert int(c.item()) == w.size
            assert np.array_equal(o[: w.size].cpu().numpy(), w)
        batch.free()
    srv = B.bs_server_create(max_batch=8, slots=2, result_bytes=1 << 30, scratch_bytes=2 << 30)
    tickets = [srv.submit(p, pj) for p, pj, _ in cases for _ in range(2)]
    for t, (p, pj, w) in zip(tickets, [c for c in cases for _ in range(2)]):
        r = srv.wait(t, 60000)
        assert r["status"] == 0 and r["count"] == w.size
        assert np.array_equal(srv.values(t, r["count"]).cpu().numpy(), w)
        srv.release(t)
    srv.destroy()
    assert B.bs_last_device_error() == 0


@pytest.mark.parametrize("shape", [{"stages": 2}, {"stages": 4}, {"unit_chunks": 2}, {"unit_chunks": 4},
                                   {"stop_rows": 1024}, {"threads": 128, "blocks_per_sm": 1},
                                   {"threads": 512, "stages": 4, "unit_chunks": 4, "stop_rows": 1024}])
def test_every_tunable_shape_matches_oracle(B, shape):
    """Each value the autotuner can pick for ring stages, chunks per claim and
    early-stop granularity (and the CTA shapes), forced once: every request's
    count, values and bit vector equal the oracle's."""
    import torch
    pool = _pool(B, seed=3)
    rng = synth.u64(11, 2, 400)
    ops = ("lt", "ge", "eq", "between", "ne")
    reqs, expect = [], []
    for i in range(24):
        ci = int(rng[i] % np.uint64(len(pool) - 1))
        v, col = pool[ci]
        op = ops[i % len(ops)]
        a, b = synth.pick_literals(v, op, float(10 ** (-3 + 2.5 * (int(rng[50 + i] % np.uint64(100)) / 100.0))), i)
        mask = _mask(v, op, a, b)
        n = v.size
        out = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        bits = torch.zeros((n + 31) // 32, dtype=torch.int32, device="cuda")
        reqs.append({"preds": [(col, op, a, b)], "out": out, "out_cap": n, "count": cnt, "bits": bits})
        expect.append((mask, v))
    batch = B.bs_batch_create(reqs, **shape)
    got_shape = batch.shape()
    for k, val in shape.items():
        assert got_shape[k] == val, (k, got_shape)
    batch.launch()
    torch.cuda.synchronize()
    for q, (mask, v) in zip(reqs, expect):
        m = int(mask.sum())
        assert int(q["count"].item()) == m
        assert np.array_equal(q["out"][:m].cpu().numpy(), v[mask])
        assert int(q["out"][m].item()) == -7 or m == q["out_cap"]
        want = np.packbits(mask, bitorder="little")
        want = np.concatenate([want, np.zeros((-want.size) % 4, np.uint8)]).view("<u4")
        assert np.array_equal(q["bits"].cpu().numpy().view(np.uint32), want)
    assert B.bs_last_device_error() == 0
