"""GPU parity of bs_lookup on columns long enough that the gather gives every
16-tile chunk its own warp (the bench's shape: one warp resolves a chunk's
tiles at the output offset the count and offset kernels gave it, Algorithm
4's dense output).

Every value and the count are compared with the oracle's decode for each
layout and code length (two-, four- and five-byte PP-VBS codes, ByteSlice,
Bit-Packed) at such lengths with a ragged last tile, with empty, sparse,
dense and full selections, output capacities below the count, a caller's
workspace full of garbage (the count kernel overwrites every word the later
kernels read), and a column with more chunks than resident warps (each warp
takes several chunks in turn)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth

pytestmark = pytest.mark.gpu

CHUNK_ROWS = 16 * 1024
WARPS_PER_CTA = 8


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


def _dev_bits(words):
    import torch
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint32).view(np.int32)).cuda()


# (label, d, Zipf s, monotone, layout, longest code): two-, four- and
# five-byte PP-VBS codes, ByteSlice and Bit-Packed
COLUMNS = [
    ("ppvbs_k2", 12, 1.0, False, "ppvbs", 2),
    ("ppvbs_k4", 24, 0.0, False, "ppvbs", 4),
    ("ppvbs_k5", 24, 0.7, True, "ppvbs", 5),
    ("byteslice_d16", 16, 0.5, False, "byteslice", 2),
    ("bitpacked_d13", 13, 1.0, False, "bitpacked", 2),
]


def _resident_warps(B, d, s, mono, layout):
    """Resident warps of the gather kernel for this column's longest code class
    (read from a smaller column of the same class)."""
    probe = B.bs_encode_column(synth.config_sweep_column(1 << 22, d, s, 90 + d, monotone=mono), layout)
    warps = B.bs_lookup_shape(probe)["resident_ctas"] * WARPS_PER_CTA
    del probe
    return warps


def _one_part_rows(warps):
    """Rows giving the gather one warp per chunk: more chunks than half the
    resident warps (it splits chunks while chunks * 2 <= warps); the last
    chunk 777 rows short."""
    return (warps // 2 + 1) * CHUNK_ROWS - 777


@pytest.fixture(scope="module")
def columns(B):
    out = {}
    for label, d, s, mono, layout, K in COLUMNS:
        n = _one_part_rows(_resident_warps(B, d, s, mono, layout))
        v = synth.config_sweep_column(n, d, s, 90 + d, monotone=mono)
        col = B.bs_encode_column(v, layout)
        if layout == "ppvbs":
            assert col.info()["max_code_bytes"] == K, label
        assert B.bs_lookup_shape(col)["parts"] == 1, label
        dec = orc.OracleColumn(v, layout).decode_values()
        assert np.array_equal(dec, v)
        out[label] = (v, col)
    return out


def _selections(v, n):
    """(name, bit vector words) from the oracle: none, sparse, the bench's
    13.7 %, half, and every row."""
    nw = (n + 31) // 32
    yield "none", np.zeros(nw, np.uint32)
    for op, t in (("lt", 0.0001), ("lt", 0.137), ("ge", 0.5)):
        lit, _ = synth.pick_literals(v, op, t, 5)
        yield "%s_%g" % (op, t), orc.scan_values(v, op, lit, 0)
    yield "all", orc.scan_values(v, "ge", -(1 << 31), 0)


@pytest.mark.parametrize("label", [c[0] for c in COLUMNS])
def test_long_column_lookup_matches_oracle(B, columns, label):
    import torch
    v, col = columns[label]
    n = v.size
    out = torch.full((n + 64,), -7, dtype=torch.int32, device="cuda")
    for name, words in _selections(v, n):
        want = orc.lookup(v, words)
        got, cnt = B.bs_lookup(col, _dev_bits(words), out=out)
        assert int(cnt.item()) == want.size, (label, name)
        g = got.cpu().numpy()
        assert np.array_equal(g[: want.size], want), (label, name)
        assert np.all(g[want.size:] == -7), (label, name)  # nothing past the count
        out.fill_(-7)
    assert B.bs_last_device_error() == 0


@pytest.mark.parametrize("label", ["ppvbs_k2", "ppvbs_k4", "bitpacked_d13"])
def test_long_column_capacity_below_count(B, columns, label):
    import torch
    v, col = columns[label]
    lit, _ = synth.pick_literals(v, "lt", 0.3, 2)
    words = orc.scan_values(v, "lt", lit, 0)
    want = orc.lookup(v, words)
    bits = _dev_bits(words)
    for cap in (0, 1, want.size // 3, want.size - 1):
        out = torch.full((want.size + 64,), -7, dtype=torch.int32, device="cuda")
        got, cnt = B.bs_lookup(col, bits, out=out, out_cap=cap)
        assert int(cnt.item()) == want.size, (label, cap)  # the full count, whatever the capacity
        g = got.cpu().numpy()
        assert np.array_equal(g[:cap], want[:cap]), (label, cap)
        assert np.all(g[cap:] == -7), (label, cap)  # nothing at or past the capacity
    assert B.bs_last_device_error() == 0


def test_long_column_workspace_garbage_and_reuse(B, columns):
    """The caller's workspace holds anything on entry (here 0xFF bytes, then
    the previous call's counts and offsets): the count kernel overwrites every
    word the offset and gather kernels read."""
    import torch
    v, col = columns["ppvbs_k2"]
    n = v.size
    ws_bytes = B.bs_lookup_workspace_bytes(col)
    assert ws_bytes >= 4 * ((n + CHUNK_ROWS - 1) // CHUNK_ROWS)
    ws = torch.full((ws_bytes // 4 + 1,), -1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for op, t in (("lt", 0.137), ("ge", 0.9), ("lt", 0.01)):
        lit, _ = synth.pick_literals(v, op, t, 3)
        words = orc.scan_values(v, op, lit, 0)
        want = orc.lookup(v, words)
        B.bs_lookup(col, _dev_bits(words), out=out, count=cnt, workspace=ws)
        assert int(cnt.item()) == want.size, (op, t)
        assert np.array_equal(out[: want.size].cpu().numpy(), want), (op, t)
    assert B.bs_last_device_error() == 0


def test_long_column_more_chunks_than_warps(B):
    """Twice as many chunks as resident warps plus a few: most warps claim
    several chunks in turn."""
    warps = _resident_warps(B, 12, 1.0, False, "ppvbs")
    n = (2 * warps + 37) * CHUNK_ROWS - 321
    v = synth.config_sweep_column(n, 12, 1.0, 93)
    col = B.bs_encode_column(v, "ppvbs")
    assert B.bs_lookup_shape(col)["parts"] == 1
    lit, _ = synth.pick_literals(v, "lt", 0.137, 4)
    words = orc.scan_values(v, "lt", lit, 0)
    want = orc.lookup(v, words)
    got, cnt = B.bs_lookup(col, _dev_bits(words))
    assert int(cnt.item()) == want.size
    assert np.array_equal(got[: want.size].cpu().numpy(), want)
    assert B.bs_last_device_error() == 0


def test_long_column_scan_then_lookup_all_layouts(B, columns):
    """bs_scan's own bit vector into the lookup, for every column."""
    for label, (v, col) in columns.items():
        lit, hi = synth.pick_literals(v, "between", 0.2, 6)
        bits = B.bs_scan(col, "between", lit, hi)
        words = orc.scan_values(v, "between", lit, hi)
        assert np.array_equal(_bits(bits, v.size), words), label
        want = orc.lookup(v, words)
        got, cnt = B.bs_lookup(col, bits)
        assert int(cnt.item()) == want.size, label
        assert np.array_equal(got[: want.size].cpu().numpy(), want), label
    assert B.bs_last_device_error() == 0
