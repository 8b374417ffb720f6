"""ByteStore on GB300: predicate scan and row lookup over PP-VBS, ByteSlice and
Bit-Packed column layouts (Zhang, Feng, Lo, Qin, "ByteStore: Hybrid Layouts for
Main-Memory Column Stores").

The compute path is the CUDA library ``libbytestore.so`` (hand-written sm_103a
kernels behind a C ABI, declared in ``include/bytestore.h``). This package is a
thin ctypes binding with the same names; it loads the library on first use and
raises ``ImportError`` if it is missing -- there is no CPU fallback.
"""

_BINDING_NAMES = None


def __getattr__(name):
    # the binding is imported lazily so that ``paper_2209_00220_gb300.synth``
    # (input generation) stays usable on machines without the CUDA library
    if name.startswith("bs_") or name in ("Column", "LAYOUTS", "OPS", "BsError", "lib", "build_library"):
        from . import bytestore as _b
        return getattr(_b, name)
    raise AttributeError(name)
