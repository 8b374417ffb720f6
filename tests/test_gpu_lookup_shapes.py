"""GPU parity of the lookup's gather at every launch shape it can take.

bs_lookup's gather splits each chunk of 16 tiles over 1, 2, 4, 8 or 16 warps,
depending on how many chunks the column has against the warps resident on the
GPU (Algorithm 4 restated for the GPU: a unit's first output slot is its
chunk's offset plus the counts of the tiles before it). Each case below sizes
a column so that the gather takes one given split (asserted through
bs_lookup_shape), then compares the count and every value with the oracle's
decode of the same column, for two- and four-byte PP-VBS codes, ByteSlice and
Bit-Packed, at sparse and dense selectivities, with a ragged last tile."""
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


def _rows_for_parts(resident_ctas, parts):
    """A row count whose chunk count c makes the gather pick `parts` warps per
    chunk. The gather doubles the split while c * split * 2 <= resident warps
    (up to 16), so it stops at `parts` exactly when warps / (2 parts) < c <=
    warps / parts; take the smallest such c, and leave a ragged tail of 777
    rows missing from the last chunk."""
    warps = resident_ctas * WARPS_PER_CTA
    chunks = warps // (2 * parts) + 1
    assert chunks * parts <= warps
    return chunks * CHUNK_ROWS - 777


# (label, d, Zipf s, monotone, layout): two-byte PP-VBS codes (the bench's
# d = 12 column), three/four-byte PP-VBS codes, and the homogeneous layouts
COLUMNS = [
    ("ppvbs_k2", 12, 1.0, False, "ppvbs"),
    ("ppvbs_k4", 24, 0.0, False, "ppvbs"),
    ("byteslice_d16", 16, 0.5, False, "byteslice"),
    ("bitpacked_d13", 13, 1.0, False, "bitpacked"),
]


@pytest.mark.parametrize("parts", [8, 4, 2, 1])
@pytest.mark.parametrize("label,d,s,mono,layout", COLUMNS, ids=[c[0] for c in COLUMNS])
def test_lookup_split_shapes_match_oracle(B, parts, label, d, s, mono, layout):
    import torch
    # the resident CTAs of this column's gather kernel, read from a smaller
    # column with the same longest code class (the kernel variant depends only
    # on it: up to two, three or four bytes)
    probe_v = synth.config_sweep_column(1 << 22, d, s, 90 + d, monotone=mono)
    probe = B.bs_encode_column(probe_v, layout)
    resident = B.bs_lookup_shape(probe)["resident_ctas"]
    del probe
    n = _rows_for_parts(resident, parts)
    v = synth.config_sweep_column(n, d, s, 90 + d, monotone=mono)
    col = B.bs_encode_column(v, layout)
    shape = B.bs_lookup_shape(col)
    assert shape["parts"] == parts, (n, shape)
    dec = orc.OracleColumn(v, layout).decode_values()
    assert np.array_equal(dec, v)
    out = torch.full((n + 64,), -7, dtype=torch.int32, device="cuda")
    for op, t in (("lt", 0.01), ("lt", 0.137), ("ge", 0.5)):
        lit, _ = synth.pick_literals(v, op, t, parts)
        bits = B.bs_scan(col, op, lit)
        sel = _bits(bits, n)
        want = orc.lookup(dec, sel)
        got, cnt = B.bs_lookup(col, bits, out=out)
        assert int(cnt.item()) == want.size, (label, parts, op, t)
        g = got.cpu().numpy()
        assert np.array_equal(g[: want.size], want), (label, parts, op, t)
        assert np.all(g[want.size:] == -7), (label, parts, op, t)  # nothing past the count
        out.fill_(-7)
    assert B.bs_last_device_error() == 0
