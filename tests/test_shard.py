"""Row-range sharding of a column over ranks. CPU: shard ranges, dictionary
merge, shards encoded against the whole column's dictionary give the whole
column's codes, and a world-size-2 gloo run exchanges dictionaries and output
offsets; the ranks' oracle results, placed at their offsets, are the whole
column's. GPU: shards of one column scanned and looked up separately
concatenate to the whole column's results and the oracle's."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import shard, synth


@pytest.fixture(scope="module")
def B():
    from paper_2209_00220_gb300 import build_lib
    build_lib.build()
    from paper_2209_00220_gb300 import bytestore
    return bytestore


@pytest.mark.parametrize("n", [0, 1, 1023, 1024, 1025, 5 * 1024 + 7, 1 << 20])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_ranges_tile_the_column(n, world):
    prev = 0
    sizes = []
    for r in range(world):
        lo, hi = shard.shard_range(n, world, r)
        assert lo == prev and lo <= hi and (lo % 1024 == 0 or lo == n)
        prev = hi
        sizes.append((hi - lo + 1023) // 1024)
    assert prev == n
    assert max(sizes) - min(sizes) <= 1


def test_merge_dictionaries():
    v = synth.config_sweep_column(100_000, 12, 1.0, 4)
    parts = [shard.local_dictionary(v[a:b]) for a, b in ((0, 3000), (3000, 3000), (3000, 77_777), (77_777, 100_000))]
    a, q = shard.merge_dictionaries(parts)
    wa, wq = np.unique(v, return_counts=True)
    assert np.array_equal(a, wa) and np.array_equal(q, wq.astype(np.uint64))


@pytest.mark.parametrize("layout", ["ppvbs", "byteslice", "bitpacked"])
def test_shard_codes_equal_whole_column_codes(B, layout):
    v = synth.config_sweep_column(3 * 1024 * 7 + 555, 16, 1.2, 9, monotone=True)
    whole = B.bs_encode_column(v, layout, host_only=True)
    wc, wl = B.bs_column_row_codes(whole)
    d = shard.local_dictionary(v)
    for r in range(3):
        lo, hi = shard.shard_range(v.size, 3, r)
        col = shard.encode_shard(B, v[lo:hi], layout, d, host_only=True)
        c, ln = B.bs_column_row_codes(col)
        assert np.array_equal(c, wc[lo:hi]) and np.array_equal(ln, wl[lo:hi]), (layout, r)


def test_declared_counts_reject_undeclared_values(B):
    v = np.array([1, 2, 3, 4], np.int32)
    with pytest.raises(B.BsError):
        B.bs_encode_column(v, "ppvbs", domain_values=np.array([1, 2, 3], np.int32),
                           domain_counts=np.array([1, 1, 1], np.uint64), host_only=True)
    with pytest.raises(B.BsError):
        B.bs_encode_column(v, "ppvbs", domain_values=np.array([1, 2, 2, 3, 4], np.int32),
                           domain_counts=np.ones(5, np.uint64), host_only=True)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    try:
        import torch.distributed as dist
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=rank, world_size=world)
        from paper_2209_00220_gb300 import bytestore as B
        v = synth.config_sweep_column(9 * 1024 + 300, 14, 1.1, 21)
        lo, hi = shard.shard_range(v.size, world, rank)
        mine = v[lo:hi]
        d = shard.global_dictionary(mine)
        col = shard.encode_shard(B, mine, "ppvbs", d, host_only=True)
        codes, _ = B.bs_column_row_codes(col)
        lit, _ = synth.pick_literals(v, "lt", 0.3, 1)
        vals = orc.lookup(mine, orc.scan_values(mine, "lt", lit))
        off, total = shard.output_offset(vals.size)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, lo, hi, d[0], d[1], codes, off, total, vals))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, "error", repr(e)))


def test_two_gloo_ranks_exchange_dictionary_and_offsets(B):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    errs = [g for g in got if g[1] == "error"]
    assert not errs, errs
    v = synth.config_sweep_column(9 * 1024 + 300, 14, 1.1, 21)
    wa, wq = np.unique(v, return_counts=True)
    whole = B.bs_encode_column(v, "ppvbs", host_only=True)
    wc, _ = B.bs_column_row_codes(whole)
    lit, _ = synth.pick_literals(v, "lt", 0.3, 1)
    want = orc.lookup(v, orc.scan_values(v, "lt", lit))
    out = np.full(want.size, -1, np.int64)
    for rank, lo, hi, a, qq, codes, off, total, vals in sorted(got, key=lambda g: g[0]):
        assert np.array_equal(a, wa) and np.array_equal(qq, wq.astype(np.uint64))
        assert np.array_equal(codes, wc[lo:hi])
        assert total == want.size
        out[off:off + vals.size] = vals
    assert np.array_equal(out, want.astype(np.int64))


@pytest.mark.gpu
@pytest.mark.parametrize("layout", ["ppvbs", "byteslice", "bitpacked"])
def test_gpu_shards_concatenate_to_whole_column(B, layout):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    v = synth.config_sweep_column(5 * 1024 * 11 + 77, 20, 1.0, 31)
    world = 3
    d = shard.local_dictionary(v)
    whole = B.bs_encode_column(v, layout, **({} if layout == "ppvbs" else {"domain_values": d[0]}))
    for op, target in (("lt", 0.2), ("eq", 0.01), ("between", 0.05)):
        a, b = synth.pick_literals(v, op, target, 3)
        want_bits = orc.scan_values(v, op, a, b)
        want_vals = orc.lookup(v, want_bits)
        whole_bits = B.bs_scan(whole, op, a, b)
        assert np.array_equal(whole_bits[: want_bits.size].cpu().numpy().view(np.uint32), want_bits)
        words, vals = [], []
        for r in range(world):
            lo, hi = shard.shard_range(v.size, world, r)
            col = shard.encode_shard(B, v[lo:hi], layout, d)
            bits = B.bs_scan(col, op, a, b)
            words.append(bits[: (hi - lo + 31) // 32].cpu().numpy().view(np.uint32))
            out, cnt = B.bs_lookup(col, bits)
            vals.append(out[: int(cnt.item())].cpu().numpy())
        assert np.array_equal(np.concatenate(words), want_bits), (layout, op)
        assert np.array_equal(np.concatenate(vals), want_vals), (layout, op)
    assert B.bs_last_device_error() == 0


def _bench_rank(rank, world, port, q):
    try:
        import sys
        import torch.distributed as dist
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=rank, world_size=world)
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        sys.path.insert(0, root)
        import bench
        from paper_2209_00220_gb300 import bytestore as B
        n = 3 * 1024 + 100
        values, lo, hi, d, lit = bench.shard_column(n, world, rank)
        col = shard.encode_shard(B, values, "ppvbs", d, host_only=True)
        codes, _ = B.bs_column_row_codes(col)
        vals = orc.lookup(values, orc.scan_values(values, "lt", lit))
        off, total = shard.output_offset(vals.size)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, lo, hi, lit, codes, off, total, vals))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, "error", repr(e)))


def test_bench_row_shards_on_two_gloo_ranks(B):
    """The multi-rank bench's setup on CPU ranks with host-only columns: the
    ranks' row ranges are pieces of one column (the one-rank bench column
    extended), their codes are the whole column's, the literal is shared,
    and the values placed at the exchanged offsets are the whole column's."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    ps = [ctx.Process(target=_bench_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    got = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    errs = [g for g in got if g[1] == "error"]
    assert not errs, errs
    n = 3 * 1024 + 100
    v = synth.config_sweep_column(n * world, 12, 1.0, 0)
    one, _ = bench.make_column(n, 0)
    assert np.array_equal(v[:n], one)  # the one-rank column is this column's first rows
    whole = B.bs_encode_column(v, "ppvbs", host_only=True)
    wc, _ = B.bs_column_row_codes(whole)
    lits = {g[3] for g in got}
    assert len(lits) == 1
    lit = lits.pop()
    want = orc.lookup(v, orc.scan_values(v, "lt", lit))
    out = np.full(want.size, -1, np.int64)
    for rank, lo, hi, _, codes, off, total, vals in sorted(got, key=lambda g: g[0]):
        assert np.array_equal(codes, wc[lo:hi])
        assert total == want.size
        out[off:off + vals.size] = vals
    assert np.array_equal(out, want.astype(np.int64))
