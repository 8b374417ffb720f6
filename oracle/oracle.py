"""CPU oracle for ByteStore scan + lookup -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline and
reference arms import this module. It wraps ``bs_oracle.c`` (plain, sequential C)
and shares no code with the CUDA product path.

``OracleColumn`` follows the pipeline the paper describes for one column:
dictionary (Section 2.2) -> codes (Algorithm 1 for PP-VBS; the dictionary rank or
a declared value range for ByteSlice and Bit-Packed) -> plain physical layout
(Sections 2.3, 2.5, 3.2) -> sequential decode of every row back to its value ->
predicate on the plain value (scan) or gather of plain values (lookup).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5, "between": 6}
LAYOUTS = ("bitpacked", "byteslice", "ppvbs")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2) into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            u64, i32, vp = ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p
            sig = {
                "orc_dictionary": ([vp, u64, vp, vp], u64),
                "orc_ppe_numerical": ([vp, u64, vp, vp], ctypes.c_int),
                "orc_ppe_categorical": ([u64, vp, vp], ctypes.c_int),
                "orc_vbs_slice_lengths": ([vp, u64, ctypes.c_int, vp], None),
                "orc_vbs_build": ([vp, vp, u64, ctypes.c_int, vp, vp, vp], ctypes.c_int),
                "orc_vbs_decode": ([vp, vp, vp, vp, u64, ctypes.c_int, vp, vp], ctypes.c_int),
                "orc_vbs_cursors_at": ([vp, u64, ctypes.c_int, u64, vp], None),
                "orc_vbs_decode_range": ([vp, vp, vp, vp, u64, ctypes.c_int, u64, u64, vp, vp, vp], ctypes.c_int),
                "orc_byteslice_build": ([vp, u64, ctypes.c_int, vp], ctypes.c_int),
                "orc_byteslice_decode": ([vp, u64, ctypes.c_int, vp], ctypes.c_int),
                "orc_bitpacked_build": ([vp, u64, ctypes.c_int, vp], ctypes.c_int),
                "orc_bitpacked_decode": ([vp, u64, ctypes.c_int, vp], ctypes.c_int),
                "orc_codes_to_values": ([vp, u64, vp, vp, u64, vp], ctypes.c_int),
                "orc_scan_values": ([vp, u64, ctypes.c_int, i32, i32, vp], None),
                "orc_scan_codes": ([vp, u64, ctypes.c_int, u64, u64, vp], None),
                "orc_lookup": ([vp, u64, vp, vp], u64),
                "orc_lookup_rowids": ([vp, u64, vp, u64, vp], ctypes.c_int),
                "orc_vbs_block_bytes": ([vp, u64, ctypes.c_int], u64),
                "orc_byteslice_block_bytes": ([u64, ctypes.c_int], u64),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ functions
def dictionary(values) -> tuple[np.ndarray, np.ndarray]:
    """Sorted distinct values A and their counts Q."""
    v = _c(values, np.int32)
    A = np.empty(max(1, v.size), np.int32)
    Q = np.empty(max(1, v.size), np.uint64)
    nd = lib().orc_dictionary(_p(v), v.size, _p(A), _p(Q))
    return A[:nd].copy(), Q[:nd].copy()


def ppe_numerical(Q) -> tuple[np.ndarray, np.ndarray]:
    """Algorithm 1: (codes C as unpadded integers, lengths L in bytes)."""
    Q = _c(Q, np.uint64)
    C = np.zeros(max(1, Q.size), np.uint64)
    L = np.zeros(max(1, Q.size), np.uint8)
    if Q.size and lib().orc_ppe_numerical(_p(Q), Q.size, _p(C), _p(L)) != 0:
        raise MemoryError("orc_ppe_numerical")
    return C[:Q.size].copy(), L[:Q.size].copy()


def ppe_categorical(nd: int) -> tuple[np.ndarray, np.ndarray]:
    """Algorithm 2 for nd values given in descending frequency order."""
    C = np.zeros(max(1, nd), np.uint64)
    L = np.zeros(max(1, nd), np.uint8)
    if lib().orc_ppe_categorical(nd, _p(C), _p(L)) != 0:
        raise ValueError("nd must be positive")
    return C[:nd].copy(), L[:nd].copy()


def frequency_order(A, Q) -> np.ndarray:
    """Dictionary positions by descending count, equal counts by smaller value
    (Algorithm 2's input order; the reading of its unstated tie rule)."""
    A = np.asarray(A)
    Q = np.asarray(Q, dtype=np.int64)
    return np.lexsort((A, -Q))


def pad(codes, lens, K: int) -> np.ndarray:
    """Zero-pad each code to K bytes (the comparison of Section 3.1.1)."""
    codes = _c(codes, np.uint64)
    shift = (8 * (K - _c(lens, np.int64))).astype(np.uint64)
    return codes << shift


def vbs_build(codes, lens, K: int):
    """Plain VBS layout: (bs1, masks[(K-1), nw], [BS_2, .., BS_K])."""
    codes, lens = _c(codes, np.uint64), _c(lens, np.uint8)
    n = codes.size
    nw = (n + 31) // 32
    sl = np.zeros(max(1, K - 1), np.uint64)
    lib().orc_vbs_slice_lengths(_p(lens), n, K, _p(sl))
    bs1 = np.zeros(max(1, n), np.uint8)
    masks = np.zeros(max(1, (K - 1) * nw), np.uint32)
    deep = np.zeros(max(1, int(sl[:K - 1].sum())), np.uint8)
    if lib().orc_vbs_build(_p(codes), _p(lens), n, K, _p(bs1), _p(masks), _p(deep)) != 0:
        raise ValueError("code length outside 1..K")
    slices, off = [], 0
    for j in range(K - 1):
        slices.append(deep[off:off + int(sl[j])].copy())
        off += int(sl[j])
    return bs1[:n].copy(), masks[:(K - 1) * nw].reshape(K - 1, nw).copy(), slices


def vbs_decode(bs1, masks, slices, n: int, K: int):
    """Sequential decode: (zero-padded codes, lengths)."""
    bs1 = _c(bs1, np.uint8)
    masks = _c(masks, np.uint32).reshape(-1)
    sl = np.array([s.size for s in slices] + [0], np.uint64)
    deep = _c(np.concatenate(slices) if slices else np.zeros(1, np.uint8), np.uint8)
    if deep.size == 0:
        deep = np.zeros(1, np.uint8)
    padded = np.zeros(max(1, n), np.uint64)
    lens = np.zeros(max(1, n), np.uint8)
    masks_buf = masks if masks.size else np.zeros(1, np.uint32)
    rc = lib().orc_vbs_decode(_p(bs1), _p(masks_buf), _p(deep), _p(sl), n, K, _p(padded), _p(lens))
    if rc != 0:
        raise ValueError("orc_vbs_decode failed (%d)" % rc)
    return padded[:n].copy(), lens[:n].copy()


def byteslice_build(codes, k: int) -> np.ndarray:
    codes = _c(codes, np.uint64)
    S = (k + 7) // 8
    out = np.zeros(max(1, S * codes.size), np.uint8)
    if lib().orc_byteslice_build(_p(codes), codes.size, k, _p(out)) != 0:
        raise ValueError("k")
    return out[:S * codes.size].reshape(S, codes.size).copy()


def byteslice_decode(slices, n: int, k: int) -> np.ndarray:
    slices = _c(slices, np.uint8)
    out = np.zeros(max(1, n), np.uint64)
    if lib().orc_byteslice_decode(_p(slices), n, k, _p(out)) != 0:
        raise ValueError("k")
    return out[:n].copy()


def bitpacked_build(codes, k: int) -> np.ndarray:
    codes = _c(codes, np.uint64)
    nb = (codes.size * k + 7) // 8
    out = np.zeros(max(1, nb), np.uint8)
    if lib().orc_bitpacked_build(_p(codes), codes.size, k, _p(out)) != 0:
        raise ValueError("k")
    return out[:nb].copy()


def bitpacked_decode(stream, n: int, k: int) -> np.ndarray:
    stream = _c(stream, np.uint8)
    if stream.size == 0:
        stream = np.zeros(1, np.uint8)
    out = np.zeros(max(1, n), np.uint64)
    if lib().orc_bitpacked_decode(_p(stream), n, k, _p(out)) != 0:
        raise ValueError("k")
    return out[:n].copy()


def scan_values(values, op: str, lit: int, lit2: int = 0) -> np.ndarray:
    """Result bit vector (uint32 words) of pred(v_i) on plain values."""
    v = _c(values, np.int32)
    nw = (v.size + 31) // 32
    bits = np.zeros(max(1, nw), np.uint32)
    lib().orc_scan_values(_p(v), v.size, OPS[op], int(lit), int(lit2), _p(bits))
    return bits[:nw].copy()


def scan_codes(padded, op: str, lit: int, lit2: int = 0) -> np.ndarray:
    """Result bit vector of pred on zero-padded codes (all padded to one width)."""
    p = _c(padded, np.uint64)
    nw = (p.size + 31) // 32
    bits = np.zeros(max(1, nw), np.uint32)
    lib().orc_scan_codes(_p(p), p.size, OPS[op], int(lit), int(lit2), _p(bits))
    return bits[:nw].copy()


def lookup(values, bits) -> np.ndarray:
    v = _c(values, np.int32)
    b = _c(bits, np.uint32)
    out = np.empty(max(1, v.size), np.int32)
    m = lib().orc_lookup(_p(v), v.size, _p(b if b.size else np.zeros(1, np.uint32)), _p(out))
    return out[:m].copy()


def lookup_rowids(values, rowids) -> np.ndarray:
    v = _c(values, np.int32)
    r = _c(rowids, np.uint32)
    out = np.empty(max(1, r.size), np.int32)
    if lib().orc_lookup_rowids(_p(v), v.size, _p(r if r.size else np.zeros(1, np.uint32)), r.size, _p(out)):
        raise IndexError("row id out of range")
    return out[:r.size].copy()


def vbs_block_bytes(lens, K: int) -> int:
    lens = _c(lens, np.uint8)
    return int(lib().orc_vbs_block_bytes(_p(lens), lens.size, K))


def byteslice_block_bytes(rows: int, K: int) -> int:
    return int(lib().orc_byteslice_block_bytes(rows, K))


# ------------------------------------------------------------------- a column
class OracleColumn:
    """One column encoded the paper's way, decoded row by row for every query.

    layout: "ppvbs" (Algorithm 1 over the observed dictionary, or Algorithm 2
    with ``categorical=True``), "byteslice" or "bitpacked" (code = rank in
    ``domain`` if given, else in the observed dictionary; or code = value -
    domain_min over a declared 2^domain_bits range).
    """

    def __init__(self, values, layout: str, domain=None, domain_bits: int | None = None,
                 domain_min: int = 0, categorical: bool = False):
        self.values = _c(values, np.int32)
        self.n = self.values.size
        self.layout = layout
        if layout == "ppvbs":
            A, Q = dictionary(self.values)
            if categorical:
                # Algorithm 2 takes the values in descending frequency (ties:
                # smaller value first) and hands out its codes in that order
                rank = frequency_order(A, Q)
                Cr, Lr = ppe_categorical(A.size)
                C = np.zeros(A.size, np.uint64)
                L = np.zeros(A.size, np.uint8)
                C[rank], L[rank] = Cr, Lr
            else:
                C, L = ppe_numerical(Q)
            self.A, self.Q, self.C, self.L = A, Q, C, L
            self.K = int(L.max()) if L.size else 1
            idx = np.searchsorted(A, self.values)
            self.row_codes, self.row_lens = C[idx], L[idx]
            self.bs1, self.masks, self.slices = vbs_build(self.row_codes, self.row_lens, self.K)
            dict_padded = pad(C, L, self.K)
            order = np.argsort(dict_padded, kind="stable")
            self._sorted_codes = dict_padded[order]
            self._sorted_vals = A[order]
        elif layout in ("byteslice", "bitpacked"):
            self.identity = domain_bits is not None
            if self.identity:
                self.k = int(domain_bits)
                self.domain_min = int(domain_min)
                codes = (self.values.astype(np.int64) - self.domain_min)
                if codes.size and (codes.min() < 0 or codes.max() >= (1 << self.k)):
                    raise ValueError("value outside the declared range")
                self.row_codes = codes.astype(np.uint64)
            else:
                A = np.unique(self.values) if domain is None else _c(np.unique(domain), np.int32)
                self.A = A
                self.k = max(1, int(np.ceil(np.log2(A.size)))) if A.size > 1 else 1
                idx = np.searchsorted(A, self.values)
                if self.n and (idx.max() >= A.size or np.any(A[np.minimum(idx, A.size - 1)] != self.values)):
                    raise ValueError("value outside the declared domain")
                self.row_codes = idx.astype(np.uint64)
            if layout == "byteslice":
                self.slices = byteslice_build(self.row_codes, self.k)
            else:
                self.stream = bitpacked_build(self.row_codes, self.k)
        else:
            raise ValueError(layout)

    def decode_codes(self):
        if self.layout == "ppvbs":
            return vbs_decode(self.bs1, self.masks, self.slices, self.n, self.K)
        if self.layout == "byteslice":
            return byteslice_decode(self.slices, self.n, self.k), None
        return bitpacked_decode(self.stream, self.n, self.k), None

    def decode_values(self) -> np.ndarray:
        """Every row decoded from the layout back to its int32 value."""
        codes, _ = self.decode_codes()
        if self.layout == "ppvbs":
            out = np.empty(max(1, self.n), np.int32)
            sc = _c(self._sorted_codes, np.uint64)
            sv = _c(self._sorted_vals, np.int32)
            if lib().orc_codes_to_values(_p(codes), self.n, _p(sc), _p(sv), sc.size, _p(out)) != 0:
                raise ValueError("decoded code missing from the dictionary")
            return out[:self.n].copy()
        if self.identity:
            return (codes.astype(np.int64) + self.domain_min).astype(np.int32)
        return self.A[codes.astype(np.int64)]

    def decode_values_range(self, r0: int, r1: int) -> np.ndarray:
        """Rows [r0, r1) decoded from the layout to their values: the same
        sequential decoder, its cursors started where a full pass would have
        them at r0 (PP-VBS only). Disjoint ranges may run on several threads."""
        if self.layout != "ppvbs":
            raise ValueError("ranges are decoded for PP-VBS columns")
        if not hasattr(self, "_flat"):
            sl = np.array([s.size for s in self.slices] + [0], np.uint64)
            deep = np.concatenate(self.slices) if self.slices else np.zeros(1, np.uint8)
            masks = _c(self.masks, np.uint32).reshape(-1)
            self._flat = (_c(self.bs1, np.uint8), masks if masks.size else np.zeros(1, np.uint32),
                          _c(deep if deep.size else np.zeros(1, np.uint8), np.uint8), sl)
        bs1, masks, deep, sl = self._flat
        cur = np.zeros(8, np.uint64)
        lib().orc_vbs_cursors_at(_p(masks), self.n, self.K, r0, _p(cur))
        m = r1 - r0
        padded = np.zeros(max(1, m), np.uint64)
        lens = np.zeros(max(1, m), np.uint8)
        rc = lib().orc_vbs_decode_range(_p(bs1), _p(masks), _p(deep), _p(sl), self.n, self.K, r0, r1, _p(cur),
                                        _p(padded), _p(lens))
        if rc != 0:
            raise ValueError("orc_vbs_decode_range failed (%d)" % rc)
        out = np.empty(max(1, m), np.int32)
        sc = _c(self._sorted_codes, np.uint64)
        sv = _c(self._sorted_vals, np.int32)
        if lib().orc_codes_to_values(_p(padded), m, _p(sc), _p(sv), sc.size, _p(out)) != 0:
            raise ValueError("decoded code missing from the dictionary")
        return out[:m]

    def scan(self, op: str, lit: int, lit2: int = 0) -> np.ndarray:
        return scan_values(self.decode_values(), op, lit, lit2)

    def lookup(self, bits) -> np.ndarray:
        return lookup(self.decode_values(), bits)
