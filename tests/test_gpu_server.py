"""Serving loop: queries submitted while others run are batched continuously,
and each one's result is exactly what it gives alone (plain calls) and what the
oracle gives -- in any mix, with admission limited by result memory."""
import time

import numpy as np
import pytest

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


def _table(B, n, seed, k=3):
    vals = [synth.config_sweep_column(n, d, s, seed + i) for i, (d, s) in enumerate(((12, 1.0), (16, 0.7), (10, 1.4))[:k])]
    return vals, [B.bs_encode_column(v, "ppvbs") for v in vals]


def _queries(tables, count, seed):
    rng = synth.u64(seed, 5, 10 * count)
    out = []
    for i in range(count):
        ti = int(rng[i] % np.uint64(len(tables)))
        vals, cols = tables[ti]
        npred = 1 + int(rng[count + i] % np.uint64(3))
        preds, mask = [], None
        for j in range(npred):
            op = ("lt", "eq", "between")[int(rng[2 * count + 3 * i + j] % np.uint64(3))]
            tgt = (10 ** (-4 + 3 * (int(rng[5 * count + 3 * i + j] % np.uint64(1000)) / 1000.0))) ** (1.0 / npred)
            a, b = synth.pick_literals(vals[j], op, tgt, i * 7 + j)
            preds.append((cols[j], op, a, b))
            m = {"lt": vals[j] < a, "eq": vals[j] == a, "between": (vals[j] >= a) & (vals[j] <= b)}[op]
            mask = m if mask is None else (mask & m)
        pj = int(rng[8 * count + i] % np.uint64(len(cols)))
        out.append((preds, cols[pj], vals[pj][mask]))
    return out


def test_server_results_match_alone_and_oracle(B):
    import torch
    tables = [_table(B, 300007, 1), _table(B, 1 << 20, 11), _table(B, 65537, 21)]
    qs = _queries(tables, 120, 3)
    srv = B.bs_server_create(max_batch=16, slots=2, result_bytes=64 << 20, scratch_bytes=512 << 20)
    tickets = []
    for preds, proj, want in qs:  # bursts: later queries arrive while earlier batches run
        tickets.append(srv.submit(preds, proj))
        if len(tickets) % 10 == 0:
            time.sleep(0.0005)
    for t, (preds, proj, want) in zip(tickets, qs):
        r = srv.wait(t, 60000)
        assert r["status"] == 0 and r["count"] == want.size
        got = srv.values(t, r["count"])
        assert np.array_equal(got.cpu().numpy(), want)
        assert r["latency_us"] >= r["queue_us"] >= 0
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == len(qs) and st["batches"] >= 2 and st["mean_batch"] > 1
    assert st["result_bytes_in_use"] == 0 and st["scratch_bytes_in_use"] == 0
    # alone: the plain calls agree with the served results
    for preds, proj, want in qs[:10]:
        bits = B.bs_scan_conj(list(preds))
        vals, cnt = B.bs_lookup(proj, bits)
        assert np.array_equal(vals[: int(cnt.item())].cpu().numpy(), want)
    srv.destroy()
    assert B.bs_last_device_error() == 0


def test_server_admission_by_memory(B):
    vals, cols = _table(B, 1 << 20, 31, k=1)
    v = vals[0]
    a, _ = synth.pick_literals(v, "lt", 0.4, 0)
    want = v[v < a]
    need = want.size * 4
    # room for one result at a time: the second query waits for the first release
    srv = B.bs_server_create(max_batch=4, slots=2, result_bytes=need + 4096, scratch_bytes=256 << 20)
    t1 = srv.submit([(cols[0], "lt", a)])
    t2 = srv.submit([(cols[0], "lt", a)])
    r1 = srv.wait(t1, 60000)
    time.sleep(0.05)
    assert srv.poll(t2) is None and srv.stats()["queued"] == 1
    srv.release(t1)
    r2 = srv.wait(t2, 60000)
    assert r1["count"] == r2["count"] == want.size
    assert np.array_equal(srv.values(t2, r2["count"]).cpu().numpy(), want)
    srv.release(t2)
    # a query that can never fit is rejected at submission
    with pytest.raises(B.BsError):
        B.bs_server_create(max_batch=4, result_bytes=1024).submit([(cols[0], "lt", a)])
    srv.destroy()
    assert B.bs_last_device_error() == 0


def test_server_reports_failed_launch_per_query(B):
    """A batch whose launch fails (faked on the host, before anything is
    enqueued) completes its queries with that error as their own status, no
    count and no values, and frees their memory; the next queries run normally."""
    vals, cols = _table(B, 300007, 41, k=1)
    v = vals[0]
    a, _ = synth.pick_literals(v, "lt", 0.2, 0)
    want = v[v < a]
    srv = B.bs_server_create(max_batch=4, slots=1, result_bytes=64 << 20, scratch_bytes=256 << 20)
    srv.fail_next_launches(1)
    t_bad = srv.submit([(cols[0], "lt", a)])
    r = srv.wait(t_bad, 60000)
    assert r["status"] == B.BS_ERR_CUDA and r["count"] == 0 and not r["d_values"]
    with pytest.raises(B.BsError):
        srv.values(t_bad, 1)
    st = srv.stats()
    assert st["failed"] == 1 and st["result_bytes_in_use"] == 0 and st["scratch_bytes_in_use"] == 0
    srv.release(t_bad)
    t_ok = srv.submit([(cols[0], "lt", a)])
    r = srv.wait(t_ok, 60000)
    assert r["status"] == 0 and r["count"] == want.size
    assert np.array_equal(srv.values(t_ok, r["count"]).cpu().numpy(), want)
    srv.release(t_ok)
    assert srv.stats()["failed"] == 1
    srv.destroy()
    assert B.bs_last_device_error() == 0


def test_serial_single_query_server_matches_batched(B):
    """Serial plain execution through the same dispatcher (one query per launch,
    one slot, single-query kernels only) gives the batched server's results;
    the per-path counters show which kernels served the queries."""
    tables = [_table(B, 300007, 51), _table(B, 1 << 20, 61)]
    qs = _queries(tables, 40, 9)
    batched = B.bs_server_create(max_batch=16, slots=2, result_bytes=64 << 20, scratch_bytes=512 << 20)
    serial = B.bs_server_create(max_batch=1, slots=1, result_bytes=64 << 20, scratch_bytes=512 << 20,
                                single_query_kernels=True)
    for srv in (batched, serial):
        tickets = [srv.submit(p, pj) for p, pj, _ in qs]
        for t, (p, pj, want) in zip(tickets, qs):
            r = srv.wait(t, 60000)
            assert r["status"] == 0 and r["count"] == want.size
            assert np.array_equal(srv.values(t, r["count"]).cpu().numpy(), want)
            srv.release(t)
    sb, ss = batched.stats(), serial.stats()
    assert sb["persistent_queries"] == len(qs) and sb["single_query_queries"] == 0
    assert ss["single_query_queries"] == len(qs) and ss["persistent_queries"] == 0
    assert ss["batches"] == len(qs) and ss["mean_batch"] == 1.0
    batched.destroy()
    serial.destroy()
    assert B.bs_last_device_error() == 0
