"""CPU oracle for binary tensor contractions -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library
(``paper_1307_2100_gb300``) never imports it and shares no code with it.

* :func:`contract` -- the FP64 loop-nest contraction (``tco.c``): the
  definition of Sec. 2.1/2.3 and the Appendix written out.  Parity: pinned.
* :mod:`oracle.classify` -- the paper's classification, requirements and
  recipes (Sec. 3.1, 3.2).  Parity: pinned.
* :mod:`oracle.precision` -- reduced-precision forms: BF16 rounding and
  split terms, FP8-E4M3 block quantisation.  Parity: pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tco.c")
_LIB = os.path.join(_HERE, "libtco.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                                  os.path.getmtime(os.path.join(_HERE, "tco.h")))):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, _LIB)
        return _LIB


class _Desc(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32),
                ("labels", ctypes.POINTER(ctypes.c_int32)),
                ("extents", ctypes.POINTER(ctypes.c_int64)),
                ("strides", ctypes.POINTER(ctypes.c_int64))]


def _configure(lib):
    lib.tco_contract_f64.restype = ctypes.c_int
    lib.tco_contract_f64.argtypes = [
        ctypes.POINTER(_Desc), ctypes.c_void_p, ctypes.POINTER(_Desc), ctypes.c_void_p,
        ctypes.POINTER(_Desc), ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
        ctypes.c_int]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


def _desc(labels, extents, strides, keep):
    n = len(labels)
    la = (ctypes.c_int32 * max(n, 1))(*[int(x) for x in labels])
    ex = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in extents])
    st = None
    if strides is not None:
        st = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in strides])
    keep += [la, ex, st]
    d = _Desc(n, la, ex, st if st is not None else ctypes.POINTER(ctypes.c_int64)())
    return d


class OracleError(RuntimeError):
    pass


def contract_raw(la, ea, sa, a, lb, eb, sb, b, lc, ec, sc, c, alpha=1.0, beta=0.0,
                 nthreads: int = 0) -> np.ndarray:
    """Contract flat float64 buffers described by (labels, extents, strides).

    `c` is updated in place (it must be a contiguous float64 array) and
    returned.  `sa/sb/sc` may be None for column-major storage.
    """
    lib = _load()
    keep = []
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if not (isinstance(c, np.ndarray) and c.dtype == np.float64 and c.flags.c_contiguous):
        raise TypeError("c must be a contiguous float64 array")
    dA = _desc(la, ea, sa, keep)
    dB = _desc(lb, eb, sb, keep)
    dC = _desc(lc, ec, sc, keep)
    st = lib.tco_contract_f64(ctypes.byref(dA), a.ctypes.data if a.size else None,
                              ctypes.byref(dB), b.ctypes.data if b.size else None,
                              ctypes.byref(dC), c.ctypes.data if c.size else None,
                              float(alpha), float(beta), int(nthreads))
    if st != 0:
        raise OracleError(f"tco_contract_f64 status {st}")
    return c


def contract(A, B, C, alpha=1.0, beta=0.0, c_init=None, nthreads: int = 0) -> np.ndarray:
    """Contract tensors given as objects with labels/extents/strides/data.

    Inputs of any float dtype are widened to float64 (exact).  Returns a new
    float64 buffer laid out like C (C.data is used as the initial C when
    beta != 0, unless `c_init` is given)."""
    if c_init is None:
        c_init = C.data
    c = np.array(c_init, dtype=np.float64, copy=True)
    return contract_raw(A.labels, A.extents, A.strides, np.asarray(A.data, np.float64),
                        B.labels, B.extents, B.strides, np.asarray(B.data, np.float64),
                        C.labels, C.extents, C.strides, c, alpha, beta, nthreads)


def contract_problem(p, nthreads: int = 0, A_data=None, B_data=None) -> np.ndarray:
    """Oracle result (float64, laid out like p.C) of a tcsynth.Problem."""
    import copy
    A = copy.copy(p.A)
    B = copy.copy(p.B)
    if A_data is not None:
        A.data = A_data
    if B_data is not None:
        B.data = B_data
    return contract(A, B, p.C, p.alpha, p.beta, nthreads=nthreads)


def rel_fro(x, ref) -> float:
    """Relative Frobenius error ||x - ref||_F / ||ref||_F (absolute if ref is 0)."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.linalg.norm((x - ref).ravel())
    n = np.linalg.norm(ref.ravel())
    return float(d / n) if n > 0 else float(d)
