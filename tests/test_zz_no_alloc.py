"""The allocation-free lookup (bs_lookup_noalloc) against bs_lookup.

Callers that cannot allocate device memory while they look up use
bs_lookup_noalloc, whose scratch is a fixed array inside the library. This
file is collected last so that a failure here comes after every other test;
it also passes on its own in a fresh process. Two calls in a row on different
bit vectors must each match bs_lookup exactly (the shared scratch keeps the
previous call's contents)."""
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


@pytest.mark.parametrize("layout", ["ppvbs", "byteslice", "bitpacked"])
def test_noalloc_lookup_matches_lookup_twice(B, layout):
    import torch
    n = 3 * 16384 + 777  # several scratch chunks and a ragged tail
    v = synth.config_sweep_column(n, 14, 1.0, 42)
    col = B.bs_encode_column(v, layout)
    for op, target in (("lt", 0.3), ("ge", 0.05)):  # two calls in a row
        lit, _ = synth.pick_literals(v, op, target, 1)
        bits = B.bs_scan(col, op, lit)
        want, want_cnt = B.bs_lookup(col, bits)
        got = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        got, cnt = B.bs_lookup_noalloc(col, bits, out=got)
        torch.cuda.synchronize()
        m = int(want_cnt.item())
        assert int(cnt.item()) == m
        assert torch.equal(got[:m], want[:m])
        assert np.array_equal(got[:m].cpu().numpy(), v[(v < lit) if op == "lt" else (v >= lit)])
    assert B.bs_last_device_error() == 0


def test_noalloc_lookup_long_and_short_columns_alternating(B):
    """A long column (the gather gives each 16,384-row chunk one warp, and
    the scratch holds thousands of chunk counts) alternating with a short one
    (each chunk split over several warps, a few counts): the array keeps the
    longer call's counts past the shorter one's end, and each call must still
    match bs_lookup."""
    import torch
    probe = B.bs_encode_column(synth.config_sweep_column(1 << 22, 12, 1.0, 43), "ppvbs")
    warps = B.bs_lookup_shape(probe)["resident_ctas"] * 8
    del probe
    n_long = (warps // 2 + 5) * 16384 - 555
    cols = []
    for n, seed in ((n_long, 44), (5 * 16384 + 3, 45)):
        v = synth.config_sweep_column(n, 12, 1.0, seed)
        cols.append((v, B.bs_encode_column(v, "ppvbs")))
    assert B.bs_lookup_shape(cols[0][1])["parts"] == 1
    assert B.bs_lookup_shape(cols[1][1])["parts"] > 1
    for k in range(4):
        v, col = cols[k % 2]
        lit, _ = synth.pick_literals(v, "lt", 0.137 + 0.2 * (k // 2), 1)
        bits = B.bs_scan(col, "lt", lit)
        want, want_cnt = B.bs_lookup(col, bits)
        got = torch.full((v.size,), -1, dtype=torch.int32, device="cuda")
        got, cnt = B.bs_lookup_noalloc(col, bits, out=got)
        torch.cuda.synchronize()
        m = int(want_cnt.item())
        assert int(cnt.item()) == m, k
        assert torch.equal(got[:m], want[:m]), k
        assert np.array_equal(got[:m].cpu().numpy(), v[v < lit]), k
    assert B.bs_last_device_error() == 0
