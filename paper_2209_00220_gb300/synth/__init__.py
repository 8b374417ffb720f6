"""Seeded synthetic inputs for ByteStore workloads (shared by the oracle's tests,
the GPU parity tests and ``bench.py``).

This module only draws random numbers and maps them to plain int32 column
values and predicate literals. It contains none of the storage method's
arithmetic: no dictionary, no prefix-preserving code, no layout and no scan.

Workload recipes (Section 6.1 of the paper generates a column of 10^9 values in
[0, 2^d) drawn from a Zipf distribution; the paper does not say which value gets
which Zipf rank, so a seeded bijection decides it):

* ``zipf_column(n, N, s, seed, mapping)``: rank r ~ Zipf(s) over N ranks
  (s = 0 is uniform), value = mapping(r).
* ``config_single_column``: 2^20 rows, Zipf s = 1.0 over a seeded set of 65,536
  distinct signed int32 values (seeded shuffle decides which value is frequent).
* ``config_sweep_column``: values in [0, 2^d) (d = 32: the whole int32 range) via
  a seeded Feistel bijection of the rank, or the identity ("monotone").
* ``pick_literals``: literals that reach a target selectivity on a bounded
  seeded sample of the column (the achieved selectivity is always measured on
  the result, never assumed).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libbssynth.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libbssynth.so`` beside it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            u64, i32, dbl, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.synth_u64.argtypes = [u64, u64, u64, u64, vp, i32]
            lib.synth_u64.restype = None
            lib.synth_zipf.argtypes = [u64, u64, u64, u64, dbl, vp, i32]
            lib.synth_zipf.restype = i32
            lib.synth_zipf_at.argtypes = [u64, u64, u64, u64, u64, dbl, vp, i32]
            lib.synth_zipf_at.restype = i32
            lib.synth_feistel.argtypes = [vp, u64, i32, u64, vp, i32]
            lib.synth_feistel.restype = i32
            lib.synth_gather.argtypes = [vp, u64, vp, vp, i32]
            lib.synth_gather.restype = None
            _lib = lib
    return _lib


def _threads() -> int:
    try:
        return max(1, min(64, len(os.sched_getaffinity(0))))
    except AttributeError:  # pragma: no cover
        return max(1, min(64, os.cpu_count() or 1))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ----------------------------------------------------------------- primitives
def u64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n counter-based 64-bit draws of (seed, stream), indices start..start+n-1."""
    out = np.empty(n, dtype=np.uint64)
    _load().synth_u64(seed, stream, start, n, _ptr(out), _threads())
    return out


def zipf_ranks(n: int, N: int, s: float, seed: int, stream: int = 0, start: int = 0) -> np.ndarray:
    """n ranks in [0, N) with P(rank r) proportional to (r + 1)^-s: rows
    start..start+n-1 of the stream (each row depends on its index alone)."""
    out = np.empty(n, dtype=np.uint32)
    rc = _load().synth_zipf_at(seed, stream, start, n, N, float(s), _ptr(out), _threads())
    if rc != 0:
        raise ValueError("synth_zipf failed (%d) for N=%d s=%g" % (rc, N, s))
    return out


def feistel(x: np.ndarray, d: int, seed: int) -> np.ndarray:
    """Seeded bijection of [0, 2^d) applied to every element of x (uint32)."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    out = np.empty_like(x)
    rc = _load().synth_feistel(_ptr(x), x.size, d, seed, _ptr(out), _threads())
    if rc != 0:
        raise ValueError("bad d=%d" % d)
    return out


def gather(idx: np.ndarray, table: np.ndarray) -> np.ndarray:
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    table = np.ascontiguousarray(table, dtype=np.int32)
    if idx.size and int(idx.max()) >= table.size:
        raise IndexError("gather index out of range")
    out = np.empty(idx.size, dtype=np.int32)
    _load().synth_gather(_ptr(idx), idx.size, _ptr(table), _ptr(out), _threads())
    return out


def distinct_values(count: int, seed: int, stream: int = 7) -> np.ndarray:
    """A seeded set of ``count`` distinct signed int32 values, sorted ascending."""
    have = np.empty(0, dtype=np.int32)
    start = 0
    while have.size < count:
        need = (count - have.size) * 2 + 64
        cand = u64(seed, stream, need, start).astype(np.uint32).view(np.int32)
        start += need
        allv = np.concatenate([have, cand])
        _, first = np.unique(allv, return_index=True)
        have = allv[np.sort(first)][:count]
    return np.sort(have)


def permutation(count: int, seed: int, stream: int = 11) -> np.ndarray:
    """Seeded permutation of range(count) (argsort of counter-based keys)."""
    keys = u64(seed, stream, count)
    return np.argsort(keys, kind="stable")


# -------------------------------------------------------------------- columns
def zipf_column(n: int, N: int, s: float, seed: int, mapping="feistel", d: int | None = None,
                stream: int = 0) -> np.ndarray:
    """n int32 values: rank ~ Zipf(s) over N ranks, value = mapping(rank).

    mapping: "identity" (value = rank, the monotone variant), "feistel" (seeded
    bijection of [0, 2^d), N must be 2^d), or an int32 table of N values.
    """
    r = zipf_ranks(n, N, s, seed, stream)
    if isinstance(mapping, str):
        if mapping == "identity":
            return r.view(np.int32) if N > (1 << 31) else r.astype(np.int32)
        if mapping == "feistel":
            if d is None or N != (1 << d):
                raise ValueError("feistel mapping needs N == 2^d")
            return feistel(r, d, seed ^ 0x5A5A).view(np.int32)
        raise ValueError(mapping)
    return gather(r, np.asarray(mapping, dtype=np.int32))


def config_single_column(seed: int = 0, n: int = 1 << 20, distinct: int = 65536, s: float = 1.0):
    """Zipf(s) over a seeded set of ``distinct`` signed int32 values.

    Returns (values, domain) where domain is the sorted value set (the declared
    dictionary of the fixed-width layouts)."""
    domain = distinct_values(distinct, seed)
    table = domain[permutation(distinct, seed)]
    return zipf_column(n, distinct, s, seed, mapping=table), domain


def config_sweep_column(n: int, d: int, s: float, seed: int, monotone: bool = False, start: int = 0) -> np.ndarray:
    """Values in [0, 2^d) for d < 32 (whole int32 range for d = 32), rank ~ Zipf(s);
    rows start..start+n-1 of the column (a row range of a longer column)."""
    N = 1 << d
    r = zipf_ranks(n, N, s, seed, start=start)
    if not monotone:
        r = feistel(r, d, seed ^ 0x5A5A)
    return r.view(np.int32)


def _uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of the counter generator."""
    return (u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def lognormal_amounts(n: int, mu: float, sigma: float, cap_bits: int, seed: int) -> np.ndarray:
    """Heavy-tailed non-negative amounts: floor(exp(mu + sigma z)) with z standard
    normal (Box-Muller over two counter streams), capped at 2^cap_bits - 1."""
    u1 = _uniform01(seed, 31, n)
    u2 = _uniform01(seed, 32, n)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    a = np.floor(np.exp(mu + sigma * z))
    return np.minimum(a, float((1 << cap_bits) - 1)).astype(np.int32)


def gaussian_column(n: int, d: int, sigma: float, seed: int) -> np.ndarray:
    """Values in [0, 2^d): round(2^(d-1) + sigma * 2^d * z) clipped, z standard
    normal (the Gaussian data of Section 6's extra experiments; sigma is the
    standard deviation as a fraction of the domain)."""
    u1 = _uniform01(seed, 41, n)
    u2 = _uniform01(seed, 42, n)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    x = np.rint(float(1 << (d - 1)) + sigma * float(1 << d) * z)
    return np.clip(x, 0, (1 << d) - 1).astype(np.int64).astype(np.int32)


# (name, kind, parameters) of the 20 columns of the synthetic denormalised wide
# table: 5 categorical, 4 date-like day counts, 1 monotone id, 4 heavy-tailed
# amounts, 6 mixed uniform / Zipf columns.
WIDE_TABLE = (
    ("cat_2", "categorical", (2, 0.0)), ("cat_16", "categorical", (16, 0.5)),
    ("cat_256", "categorical", (256, 1.0)), ("cat_4k", "categorical", (4096, 1.5)),
    ("cat_64k", "categorical", (65536, 0.8)),
    ("day_a", "date", (0.0,)), ("day_b", "date", (0.0,)), ("day_c", "date", (0.7,)), ("day_d", "date", (1.2,)),
    ("id", "monotone", (1000,)),
    ("amt_a", "amount", (4.0, 1.0, 20)), ("amt_b", "amount", (6.0, 1.5, 24)),
    ("amt_c", "amount", (8.0, 2.0, 24)), ("amt_d", "amount", (3.0, 0.5, 16)),
    ("mix_10", "mixed", (10, 0.0)), ("mix_13", "mixed", (13, 1.2)), ("mix_16", "mixed", (16, 0.0)),
    ("mix_19", "mixed", (19, 0.7)), ("mix_22", "mixed", (22, 0.0)), ("mix_24", "mixed", (24, 1.5)),
)


def wide_table_column(name: str, n: int, seed: int = 0) -> np.ndarray:
    """One column of the wide table (see WIDE_TABLE), n rows."""
    i = [w[0] for w in WIDE_TABLE].index(name)
    _, kind, p = WIDE_TABLE[i]
    cs = seed * 100 + i
    if kind == "categorical":
        card, s = p
        table = distinct_values(card, cs)[permutation(card, cs)]
        return zipf_column(n, card, s, cs, mapping=table)
    if kind == "date":
        # day counts 0..3650; s > 0: a seeded order of the days is Zipf-weighted
        (s,) = p
        days = permutation(3651, cs).astype(np.int32)
        return zipf_column(n, 3651, s, cs, mapping=days)
    if kind == "monotone":
        (off,) = p
        return (np.arange(n, dtype=np.int64) + off).astype(np.int32)
    if kind == "amount":
        mu, sigma, cap = p
        return lognormal_amounts(n, mu, sigma, cap, cs)
    d, s = p
    return config_sweep_column(n, d, s, cs)


def domain_min_for_bits(d: int) -> int:
    return -(1 << 31) if d == 32 else 0


# ------------------------------------------------------------------- literals
OPS = ("lt", "le", "gt", "ge", "eq", "ne", "between")


def _sample(values: np.ndarray, seed: int, k: int = 1 << 20) -> np.ndarray:
    if values.size <= k:
        return np.sort(values.astype(np.int64))
    idx = (u64(seed, 99, k) % np.uint64(values.size)).astype(np.int64)
    return np.sort(values[idx].astype(np.int64))


def pick_literals(values: np.ndarray, op: str, target: float, seed: int = 0):
    """Literals (lit, lit2) aiming at selectivity ``target`` for ``op``, read off
    a bounded seeded sample (exact targets are impossible on discrete data):

    lt: the smallest value c with share(v < c) >= target; le: the smallest c with
    share(v <= c) >= target; ge / gt: the largest c with share(v >= c) resp.
    share(v > c) >= target; eq: the value whose share is closest to target;
    ne: closest to 1 - target; between: lo at a seeded quantile, hi the smallest
    value with share(lo <= v <= hi) >= target. lit2 is 0 unless between.
    """
    smp = _sample(values, seed)
    m = smp.size
    u, cnt = np.unique(smp, return_counts=True)
    below = np.concatenate([[0], np.cumsum(cnt)[:-1]])  # rows < u[i]
    upto = below + cnt                                  # rows <= u[i]
    want = target * m
    clip = lambda x: int(np.clip(x, -(1 << 31), (1 << 31) - 1))
    if op == "lt":
        i = np.flatnonzero(below >= want)
        return (clip(u[i[0]]) if i.size else clip(u[-1] + 1)), 0
    if op == "le":
        i = np.flatnonzero(upto >= want)
        return (clip(u[i[0]]) if i.size else clip(u[-1])), 0
    if op == "ge":
        i = np.flatnonzero(m - below >= want)
        return (clip(u[i[-1]]) if i.size else clip(u[0])), 0
    if op == "gt":
        i = np.flatnonzero(m - upto >= want)
        return (clip(u[i[-1]]) if i.size else clip(u[-1])), 0
    if op in ("eq", "ne"):
        f = cnt / m
        w = target if op == "eq" else 1.0 - target
        return clip(u[int(np.argmin(np.abs(f - w)))]), 0
    if op == "between":
        q0 = float(u64(seed, 123, 1)[0] >> np.uint64(11)) / float(1 << 53) * max(0.0, 1.0 - target)
        lo_i = int(np.searchsorted(below, q0 * m, side="right")) - 1
        lo_i = max(0, min(lo_i, u.size - 1))
        got = upto - below[lo_i]
        j = np.flatnonzero((np.arange(u.size) >= lo_i) & (got >= want))
        hi_i = int(j[0]) if j.size else u.size - 1
        return clip(u[lo_i]), clip(u[hi_i])
    raise ValueError(op)
