"""Encoded columns written to a file and read back: the loaded column carries
the same codes, dictionary and layout bytes (CPU), and on the GPU scans and
looks up exactly like the column it was saved from; damaged files are refused."""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth


@pytest.fixture(scope="module")
def B():
    from paper_2209_00220_gb300 import build_lib
    build_lib.build()
    from paper_2209_00220_gb300 import bytestore
    return bytestore


LAYOUTS = [("ppvbs", {}), ("ppvbs", {"categorical": True}), ("byteslice", {}),
           ("bitpacked", {"domain_bits": 16})]


@pytest.mark.parametrize("layout,extra", LAYOUTS)
def test_save_load_host(B, tmp_path, layout, extra):
    v = synth.config_sweep_column(70001, 16, 1.1, 3, monotone=True)
    col = B.bs_encode_column(v, layout, host_only=True, **extra)
    path = str(tmp_path / "col.bs")
    B.bs_column_save(col, path)
    back = B.bs_column_load(path, host_only=True)
    assert back.n == v.size
    c0, l0 = B.bs_column_row_codes(col)
    c1, l1 = B.bs_column_row_codes(back)
    assert np.array_equal(c0, c1) and np.array_equal(l0, l1)
    i0, i1 = col.info(), back.info()
    assert {k: i0[k] for k in ("layout", "max_code_bytes", "code_bits", "n_dict", "layout_bytes")} == \
           {k: i1[k] for k in ("layout", "max_code_bytes", "code_bits", "n_dict", "layout_bytes")}
    lit = int(v[17])
    op = "eq" if extra.get("categorical") else "lt"
    assert B.bs_scan_bytes(col, op, lit) == B.bs_scan_bytes(back, op, lit)


def test_damaged_files_are_refused(B, tmp_path):
    v = synth.config_sweep_column(5000, 12, 1.0, 4)
    col = B.bs_encode_column(v, "ppvbs", host_only=True)
    path = str(tmp_path / "col.bs")
    B.bs_column_save(col, path)
    raw = open(path, "rb").read()
    for bad in (raw[:100], b"XXXXXXXX" + raw[8:], raw[:-9]):
        p = str(tmp_path / "bad.bs")
        open(p, "wb").write(bad)
        with pytest.raises(B.BsError):
            B.bs_column_load(p, host_only=True)
    with pytest.raises(B.BsError):
        B.bs_column_load(str(tmp_path / "missing.bs"), host_only=True)


@pytest.mark.gpu
@pytest.mark.parametrize("layout,extra", LAYOUTS)
def test_save_from_device_load_to_device(B, tmp_path, layout, extra):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    v = synth.config_sweep_column((1 << 20) + 3, 16, 0.9, 5)
    col = B.bs_encode_column(v, layout, **extra)  # device only: save reads the arena back
    path = str(tmp_path / "col.bs")
    B.bs_column_save(col, path)
    back = B.bs_column_load(path)
    op = "eq" if extra.get("categorical") else "lt"
    lit = int(np.median(v))
    want = orc.scan_values(v, op, lit)
    for c in (col, back):
        bits = B.bs_scan(c, op, lit)
        assert np.array_equal(bits[: want.size].cpu().numpy().view(np.uint32), want)
        vals, cnt = B.bs_lookup(c, bits)
        assert np.array_equal(vals[: int(cnt.item())].cpu().numpy(), orc.lookup(v, want))
    assert B.bs_last_device_error() == 0
