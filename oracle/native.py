"""Builds the plain-C part of the oracle (rows.c) into oracle/_rows.so.

Test infrastructure only (see the package docstring)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rows.c")
LIB = os.path.join(HERE, "_rows.so")


def build():
    if not os.path.exists(SRC):
        return None
    tmp = LIB + ".tmp"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        import ctypes
        if not os.path.exists(LIB):
            build()
        _lib = ctypes.CDLL(LIB)
        D = ctypes.POINTER(ctypes.c_double)
        I64 = ctypes.POINTER(ctypes.c_int64)
        _lib.ncs_oracle_rows.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, D, D, D,
                                         ctypes.c_double, ctypes.c_int64, I64, D, D, D]
        _lib.ncs_oracle_rows.restype = ctypes.c_int
    return _lib


def rows(pre, centres, x, patches, nodes):
    """z at (patch, node) targets by the compressed sums (Section 7.1), FP64 in C.
    pre: oracle Precompute; patches, nodes: equal-length index arrays."""
    import ctypes
    import numpy as np
    lib = _load()
    D = ctypes.POINTER(ctypes.c_double)
    c = np.ascontiguousarray(centres, dtype=np.float64)
    T = np.ascontiguousarray(pre.idr.T, dtype=np.float64)
    st = np.ascontiguousarray(pre.idr.t_skel, dtype=np.float64)
    sth = np.ascontiguousarray(pre.idr.th_skel, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    pi = np.ascontiguousarray(patches, dtype=np.int64)
    nr = np.ascontiguousarray(pre.r_z[np.asarray(nodes)], dtype=np.float64)
    nth = np.ascontiguousarray(pre.th_z[np.asarray(nodes)], dtype=np.float64)
    out = np.zeros(pi.size)
    rc = lib.ncs_oracle_rows(c.shape[0], pre.K, T.shape[0], pre.mode, c.ctypes.data_as(D), T.ctypes.data_as(D),
                             st.ctypes.data_as(D), sth.ctypes.data_as(D), xx.ctypes.data_as(D), pre.eps, pi.size,
                             pi.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), nr.ctypes.data_as(D),
                             nth.ctypes.data_as(D), out.ctypes.data_as(D))
    if rc != 0:
        raise MemoryError("oracle rows: allocation failed")
    return out
