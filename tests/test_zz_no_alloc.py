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
