"""CPU checks of the product library (no GPU): every symbol the header declares
is exported, and the host encoder's dictionary, Algorithm 1 codes and per-row
layout contents equal the oracle's, bit for bit."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2209_00220_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2209_00220_gb300 import build_lib
    build_lib.build()
    from paper_2209_00220_gb300 import bytestore
    return bytestore


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(bs_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(B):
    names = _declared_functions()
    assert {"bs_encode_column", "bs_scan", "bs_scan_conj", "bs_lookup", "bs_advise_layout"} <= names
    L = B.lib()
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def _columns():
    yield "zipf1_d12", synth.config_sweep_column(40000, 12, 1.0, 1)
    yield "uniform_d16", synth.config_sweep_column(40000, 16, 0.0, 2)
    yield "zipf15_d20", synth.config_sweep_column(60000, 20, 1.5, 3)
    yield "monotone_d16", synth.config_sweep_column(70000, 16, 1.0, 4, monotone=True)   # beta leaves
    yield "monotone_d24", synth.config_sweep_column(300000, 24, 0.7, 5, monotone=True)  # K = 5
    yield "small", synth.config_sweep_column(1000, 7, 1.0, 6)                            # root leaf
    v = synth.distinct_values(256, 9)
    yield "exactly256", np.concatenate([v, v[:10]])
    yield "negative", (synth.config_sweep_column(30000, 14, 1.0, 7) - 9000).astype(np.int32)
    yield "single_value", np.full(777, -5, np.int32)
    yield "tail_1025", synth.config_sweep_column(1025, 10, 1.0, 8)


@pytest.mark.parametrize("name,values", list(_columns()), ids=[n for n, _ in _columns()])
def test_ppvbs_encoder_matches_oracle(B, name, values):
    col = B.bs_encode_column(values, "ppvbs", host_only=True)
    ocol = orc.OracleColumn(values, "ppvbs")
    A, C, L = B.bs_column_dictionary(col)
    assert np.array_equal(A, ocol.A)
    assert np.array_equal(C, ocol.C)
    assert np.array_equal(L, ocol.L)
    codes, lens = B.bs_column_row_codes(col)
    assert np.array_equal(codes, ocol.row_codes)
    assert np.array_equal(lens, ocol.row_lens)
    info = col.info()
    assert info["max_code_bytes"] == ocol.K and info["n_rows"] == values.size and not info["on_device"]
    hist = np.bincount(ocol.row_lens, minlength=9)
    assert info["len_hist"][1:9] == hist[1:9].tolist()
    want_bytes = values.size + sum(4 * ((values.size + 31) // 32) + s.size for s in ocol.slices)
    assert info["layout_bytes"] == want_bytes


@pytest.mark.parametrize("layout", ["byteslice", "bitpacked"])
def test_fixed_width_encoders_match_oracle(B, layout):
    for name, values in _columns():
        col = B.bs_encode_column(values, layout, host_only=True)
        ocol = orc.OracleColumn(values, layout)
        codes, lens = B.bs_column_row_codes(col)
        assert np.array_equal(codes, ocol.row_codes), name
        assert col.info()["code_bits"] == ocol.k
    # declared value ranges, including the full int32 range
    for d in (8, 12, 17, 24, 32):
        v = synth.config_sweep_column(20000, d, 1.0, d)
        dmin = synth.domain_min_for_bits(d)
        col = B.bs_encode_column(v, layout, host_only=True, domain_bits=d, domain_min=dmin)
        ocol = orc.OracleColumn(v, layout, domain_bits=d, domain_min=dmin)
        codes, _ = B.bs_column_row_codes(col)
        assert np.array_equal(codes, ocol.row_codes), d
    # a declared dictionary (the single-column workload's 65,536 values)
    v, dom = synth.config_single_column(seed=0, n=50000)
    col = B.bs_encode_column(v, layout, host_only=True, domain_values=dom)
    ocol = orc.OracleColumn(v, layout, domain=dom)
    assert np.array_equal(B.bs_column_row_codes(col)[0], ocol.row_codes)
    assert col.info()["code_bits"] == 16


def test_raw_code_columns_roundtrip(B):
    # the exhaustive small-alphabet code set: every code of <= 3 bytes over a
    # 7-letter byte alphabet whose last byte is non-zero
    alpha = [0, 1, 2, 0x7F, 0x80, 0xFE, 0xFF]
    codes, lens = [], []
    for l in (1, 2, 3):
        for t in np.ndindex(*([len(alpha)] * l)):
            bs_ = [alpha[i] for i in t]
            if bs_[-1] == 0:
                continue
            c = 0
            for b in bs_:
                c = (c << 8) | b
            codes.append(c)
            lens.append(l)
    codes = np.array(codes, np.uint64)
    lens = np.array(lens, np.uint8)
    perm = synth.permutation(codes.size, 3)
    codes, lens = codes[perm], lens[perm]
    col = B.bs_column_from_codes(codes, lens, "ppvbs", host_only=True)
    c2, l2 = B.bs_column_row_codes(col)
    assert np.array_equal(c2, codes) and np.array_equal(l2, lens)
    bs1, masks, slices = orc.vbs_build(codes, lens, 3)
    assert col.info()["layout_bytes"] == codes.size + sum(4 * masks.shape[1] + s.size for s in slices)


def test_encoder_rejects_bad_input(B):
    v = np.arange(100, dtype=np.int32)
    with pytest.raises(B.BsError):
        B.bs_encode_column(v, "byteslice", host_only=True, domain_bits=4)  # values outside 0..15
    with pytest.raises(B.BsError):
        B.bs_column_from_codes(np.array([0x1FF], np.uint64), np.array([1], np.uint8), "ppvbs", host_only=True)


@pytest.mark.parametrize("n,d,s,seed", [(50000, 8, 1.0, 1), (120000, 12, 0.7, 2), (300000, 17, 0.3, 3),
                                        (200000, 20, 1.4, 4)])
def test_categorical_codes_match_oracle(B, n, d, s, seed):
    v = synth.config_sweep_column(n, d, s, seed)
    ocol = orc.OracleColumn(v, "ppvbs", categorical=True)
    col = B.bs_encode_column(v, "ppvbs", categorical=True, host_only=True)
    codes, lens = B.bs_column_row_codes(col)
    assert np.array_equal(codes, ocol.row_codes) and np.array_equal(lens, ocol.row_lens)
    dv, dc, dl = B.bs_column_dictionary(col)
    assert np.array_equal(dv, ocol.A) and np.array_equal(dc, ocol.C) and np.array_equal(dl, ocol.L)


def test_categorical_columns_take_only_equality(B):
    v = synth.config_sweep_column(5000, 10, 1.0, 9)
    col = B.bs_encode_column(v, "ppvbs", categorical=True, host_only=True)
    for op in ("lt", "le", "gt", "ge", "between"):
        with pytest.raises(B.BsError):
            B.bs_scan_bytes(col, op, int(v[0]), int(v[0]))
    assert B.bs_scan_bytes(col, "eq", int(v[0]))["bytes"] > 0
