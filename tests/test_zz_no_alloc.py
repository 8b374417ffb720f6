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


def test_noalloc_lookup_leaves_free_device_memory_unchanged(B):
    """The point of the entry point: a caller running under a fixed device
    memory budget (or in a section where no allocator may be touched) can
    look up without the device's free memory moving. After one warm-up call
    (the first call looks up the scratch array's address and loads the
    kernels), a call on a new bit vector must leave cudaMemGetInfo's free
    bytes exactly where they were, and still match bs_lookup."""
    import torch
    n = 9 * 16384 + 101
    v = synth.config_sweep_column(n, 16, 0.5, 46)
    col = B.bs_encode_column(v, "ppvbs")
    lit0, _ = synth.pick_literals(v, "lt", 0.2, 1)
    lit1, _ = synth.pick_literals(v, "ge", 0.4, 2)
    bits0 = B.bs_scan(col, "lt", lit0)
    bits1 = B.bs_scan(col, "ge", lit1)
    want, want_cnt = B.bs_lookup(col, bits1)
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.bs_lookup_noalloc(col, bits0, out=out, count=cnt)  # warm-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    B.bs_lookup_noalloc(col, bits1, out=out, count=cnt)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    m = int(want_cnt.item())
    assert int(cnt.item()) == m
    assert torch.equal(out[:m], want[:m])
    assert B.bs_last_device_error() == 0
