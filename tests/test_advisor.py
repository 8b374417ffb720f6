"""Layout advisor (Algorithm 5) and the effective-bytes counter it uses in its
deterministic mode. The CPU checks pin what does not need a device: the 100
profiling literals (row quantiles of the value distribution, recomputed here
from numpy's own unique/count), the trapezoid areas and the ByteSlice-on-ties
decision (recomputed from the returned profiles), closed forms of the byte
counter where nothing stops early, and its pending-row counts against brute
force over the oracle's codes. The GPU check runs the timed mode."""
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


def _quantile_selectivities(values):
    """Algorithm 5's literal choice as read here: for target share (i+0.5)/100
    the smallest dictionary value u with share(v < u) >= target (the largest
    value when none reaches it); its selectivity is share(v < u)."""
    A, Q = np.unique(values, return_counts=True)
    cum = np.concatenate([[0], np.cumsum(Q)])
    n = values.size
    out = []
    for i in range(100):
        u = int(np.searchsorted(cum, (i + 0.5) / 100 * n, side="left"))
        u = min(u, A.size - 1)
        out.append(cum[u] / n)
    return np.array(out)


def _trapezoid(sel, cost):
    order = np.argsort(sel, kind="stable")
    x, y = np.asarray(sel)[order], np.asarray(cost)[order]
    if x[-1] - x[0] <= 0:
        return float(np.mean(y))
    return float(np.sum((x[1:] - x[:-1]) * 0.5 * (y[1:] + y[:-1])))


def _advise(B, values, **kw):
    return B.bs_advise_layout(values, B.ADVISE_BYTES_MODEL, host_only=True, **kw)


@pytest.mark.parametrize("d,s", [(12, 1.0), (16, 0.0), (10, 1.5), (20, 0.5)])
def test_profile_literals_areas_and_decision(B, d, s):
    v = synth.config_sweep_column(1 << 18, d, s, 17 + d)
    a = _advise(B, v)
    sel = np.array(a["selectivity"])
    assert len(sel) == 100
    assert np.array_equal(sel, _quantile_selectivities(v))
    assert a["auc_byteslice"] == pytest.approx(_trapezoid(sel, a["cost_byteslice"]), rel=1e-12)
    assert a["auc_ppvbs"] == pytest.approx(_trapezoid(sel, a["cost_ppvbs"]), rel=1e-12)
    want = "byteslice" if a["auc_byteslice"] <= a["auc_ppvbs"] else "ppvbs"
    assert a["layout"] == want


def test_one_byte_codes_cost_the_same_and_tie_to_byteslice(B):
    # at most 255 distinct values: every PP-VBS code is one byte (a leaf at the
    # root) and ByteSlice has one slice, so every scan reads the n bytes of the
    # slice plus the n/8-byte result and nothing else, on both layouts
    n = 1 << 20
    v = synth.config_sweep_column(n, 7, 1.0, 5)
    a = _advise(B, v)
    assert set(a["cost_ppvbs"]) == {float(n + n // 8)}
    assert set(a["cost_byteslice"]) == {float(n + n // 8)}
    assert a["layout"] == "byteslice"


def test_skewed_wide_codes_favour_ppvbs(B):
    # Section 6: on skewed data most rows get one-byte PP-VBS codes and stop
    # after BS_1, while two-slice ByteSlice keeps rows pending wherever a
    # frequent value shares the literal's first byte
    v = synth.config_single_column(0, 1 << 20, 65536, 1.0)[0]
    a = _advise(B, v)
    assert a["auc_ppvbs"] < a["auc_byteslice"]
    assert a["layout"] == "ppvbs"


@pytest.mark.parametrize("k", [3, 8, 13, 32])
def test_bitpacked_bytes_closed_form(B, k):
    n = 10 * 1024  # whole tiles: no early stop, every 32-row round reads k words
    v = (synth.u64(k, 1, n) % np.uint64(1 << min(k, 31))).astype(np.int64)
    v = (v + synth.domain_min_for_bits(k)).astype(np.int32)
    col = B.bs_encode_column(v, "bitpacked", domain_bits=k, domain_min=synth.domain_min_for_bits(k),
                             host_only=True)
    r = B.bs_scan_bytes(col, "lt", int(np.median(v)))
    assert r["dense_bytes"] == n * k // 8
    assert r["result_bytes"] == n // 8
    assert r["bytes"] == n * k // 8 + n // 8


def test_ppvbs_pending_rows_by_brute_force(B):
    # rows pending entering byte j = rows whose code bytes 1..j-1 equal the
    # literal's (for "=", which needs the byte after the literal's last one)
    v = synth.config_sweep_column(50_000, 16, 1.2, 23, monotone=True)
    ocol = orc.OracleColumn(v, "ppvbs")
    K = ocol.K
    assert K >= 3
    col = B.bs_encode_column(v, "ppvbs", host_only=True)
    padded = orc.pad(ocol.row_codes, ocol.row_lens, K)
    byte = lambda c, j: (np.asarray(c, dtype=np.uint64) >> np.uint64(8 * (K - j))) & np.uint64(0xFF)
    for lit in (int(v[7]), int(v[123]), int(np.max(v))):
        i = int(np.searchsorted(ocol.A, lit))
        lc, ll = int(ocol.C[i]), int(ocol.L[i])
        lpad = lc << (8 * (K - ll))
        r = B.bs_scan_bytes(col, "eq", lit)
        same = np.ones(v.size, dtype=bool)
        for j in range(2, min(ll + 1, K) + 1):
            same &= byte(padded, j - 1) == np.uint64((lpad >> (8 * (K - j + 1))) & 0xFF)
            # a row shorter than j - 1 bytes was decided before byte j
            same &= ocol.row_lens >= j - 1
            assert r["pending_rows"][j] == int(np.count_nonzero(same)), (lit, j)


@pytest.mark.gpu
def test_timed_mode_on_gpu(B):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    v = synth.config_sweep_column(1 << 22, 12, 1.0, 3)
    t = B.bs_advise_layout(v, B.ADVISE_TIMED)
    m = _advise(B, v)
    assert t["layout"] in ("byteslice", "ppvbs")
    assert t["selectivity"] == m["selectivity"]
    assert min(t["cost_byteslice"]) > 0 and min(t["cost_ppvbs"]) > 0
    assert t["auc_ppvbs"] == pytest.approx(_trapezoid(t["selectivity"], t["cost_ppvbs"]), rel=1e-12)
    assert B.bs_last_device_error() == 0


def test_categorical_profile_uses_equality_at_frequency_ranks(B):
    v = synth.config_sweep_column(1 << 18, 12, 1.2, 5)
    a = _advise(B, v, categorical=True)
    vals, counts = np.unique(v, return_counts=True)
    order = np.lexsort((vals, -counts))
    ranks = [int(i * (order.size - 1) / 99 + 0.5) for i in range(100)]
    assert np.allclose(a["selectivity"], counts[order[ranks]] / v.size, rtol=0, atol=0)
    assert a["auc_byteslice"] == pytest.approx(_trapezoid(np.array(a["selectivity"]), a["cost_byteslice"]), rel=1e-12)


def test_known_selectivity_range_restricts_the_profile(B):
    # Section 5: with a known selectivity range the advisor profiles only it
    v = synth.config_sweep_column(1 << 18, 12, 1.0, 8)
    a = _advise(B, v, sel_range=(0.2, 0.4))
    sel = np.array(a["selectivity"])
    vals, counts = np.unique(v, return_counts=True)
    cum = np.concatenate([[0], np.cumsum(counts)])
    want = []
    for i in range(100):
        u = min(int(np.searchsorted(cum, (0.2 + (i + 0.5) / 100 * 0.2) * v.size, side="left")), vals.size - 1)
        want.append(cum[u] / v.size)
    assert np.array_equal(sel, np.array(want))
    assert sel.min() >= 0.2 - 0.05 and sel.max() <= 0.4 + 0.05
    c = _advise(B, v, categorical=True, sel_range=(0.0, 0.01))
    assert max(c["selectivity"]) <= 0.01
    with pytest.raises(B.BsError):
        _advise(B, v, sel_range=(0.5, 0.2))
