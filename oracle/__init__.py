"""Plain CPU oracle for the Faugere-Lachartre reduction over GF(p).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA product path never imports, links or executes it, and it
shares no code with that path: the only module both sides use is the seeded
input generator ``paper_1602_06097_gb300.synth``, which holds none of the
method's arithmetic.

``oracle.c`` holds the arithmetic (exact uint64 with ``%``); this module only
compiles it with gcc and marshals numpy arrays through ctypes.  Passages
followed (GBLA paper, arXiv 1602.06097):

* :func:`rref`     -- textbook Gauss-Jordan on the whole matrix: FL steps 4-5
  and the reduced-echelon pass (Sec. 4.1), Alg. 3's normalise/reduce rule.
* :func:`rref32`, :func:`echelon32` -- :func:`rref` and :func:`echelon` for
  primes p < 2^31 with uint32 values (the paper's 32-bit coefficient type,
  Sec. 2), every addition reduced.
* :func:`echelon`  -- the new order of operations (Alg. 2, Sec. 4.3) in plain
  row form, then Gauss-Jordan of the Schur complement.
* :func:`row_counts` -- the work counts of Alg. 2's row reduction alone.
* :func:`pivots`   -- the FL step-1 pivot choice (Sec. 3.1, Sec. 4.1 step 1).
* :func:`multiline` -- the 2-multiline vector of Definition 1 (Sec. 4.2).
* :mod:`oracle.formats` -- readers of the two binary matrix files of Sec. 3.2
  (Table 2) into the reduction's CSR input.

Every function is pinned by ``tests/test_oracle.py`` against results fixed by
the mathematics (brute-force row spaces, determinant ranks, closed forms,
invariants) and, for :func:`multiline`, by the paper's Example 1; the file
readers by ``tests/test_formats.py`` (files assembled by hand from Table 2);
:func:`rref32` and :func:`echelon32` by ``tests/test_oracle32.py`` (sympy's
RREF over GF(p) of the matrix and of its Schur complement, closed forms,
invariants, agreement with the 16-bit functions below 2^16).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LOCK = threading.Lock()
_LIBS: dict = {}


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_HERE, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP for the row-parallel forward pass)."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           f"-DORACLE_MUTANT={int(mutant)}", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(mutant: int = 0):
    with _LOCK:
        if mutant in _LIBS:
            return _LIBS[mutant]
        lib = ctypes.CDLL(build(mutant))
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u16p = ctypes.POINTER(ctypes.c_uint16)
        vp = ctypes.c_void_p
        lib.oracle_rref.restype = ctypes.c_int
        lib.oracle_rref.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32, vp, vp, vp,
                                    i64p, ctypes.POINTER(i64p), ctypes.POINTER(i32p),
                                    ctypes.POINTER(u16p)]
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_rref32.restype = ctypes.c_int
        lib.oracle_rref32.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32, vp, vp, vp,
                                      i64p, ctypes.POINTER(i64p), ctypes.POINTER(i32p),
                                      ctypes.POINTER(u32p)]
        lib.oracle_echelon32.restype = ctypes.c_int
        lib.oracle_echelon32.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32, vp, vp, vp,
                                         i64p, ctypes.POINTER(i64p), ctypes.POINTER(i32p),
                                         ctypes.POINTER(u32p), i64p]
        lib.oracle_echelon.restype = ctypes.c_int
        lib.oracle_echelon.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32, vp, vp, vp,
                                       i64p, ctypes.POINTER(i64p), ctypes.POINTER(i32p),
                                       ctypes.POINTER(u16p), i64p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
        lib.oracle_row_counts.restype = ctypes.c_int
        lib.oracle_row_counts.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32, vp, vp, vp,
                                          ctypes.POINTER(ctypes.c_double), i64p, ctypes.POINTER(ctypes.c_double)]
        lib.oracle_pivots.restype = ctypes.c_int64
        lib.oracle_pivots.argtypes = [ctypes.c_int64, ctypes.c_int64, vp, vp, vp]
        lib.oracle_free.restype = None
        lib.oracle_free.argtypes = [vp]
        _LIBS[mutant] = lib
        return lib


def _csr_args(row_ptr, col, val):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.uint16)
    return row_ptr, col, val


def _take(lib, rank, rp, cl, vl):
    r = int(rank.value)
    row_ptr = np.ctypeslib.as_array(rp, shape=(r + 1,)).copy()
    nnz = int(row_ptr[-1])
    col = np.ctypeslib.as_array(cl, shape=(max(nnz, 1),))[:nnz].copy()
    val = np.ctypeslib.as_array(vl, shape=(max(nnz, 1),))[:nnz].copy()
    for ptr in (rp, cl, vl):
        lib.oracle_free(ctypes.cast(ptr, ctypes.c_void_p))
    return r, row_ptr, col, val


class OracleError(RuntimeError):
    pass


def rref(m, n, p, row_ptr, col, val, mutant: int = 0):
    """RREF(M) over GF(p): returns (rank, row_ptr, col, val), rows by pivot column."""
    lib = _lib(mutant)
    row_ptr, col, val = _csr_args(row_ptr, col, val)
    rank = ctypes.c_int64(0)
    rp = ctypes.POINTER(ctypes.c_int64)()
    cl = ctypes.POINTER(ctypes.c_int32)()
    vl = ctypes.POINTER(ctypes.c_uint16)()
    rc = lib.oracle_rref(m, n, p, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                         ctypes.byref(rank), ctypes.byref(rp), ctypes.byref(cl), ctypes.byref(vl))
    if rc != 0:
        raise OracleError(f"oracle_rref failed with code {rc}")
    return _take(lib, rank, rp, cl, vl)


def rref32(m, n, p, row_ptr, col, val, mutant: int = 0):
    """RREF(M) over GF(p) for a prime p < 2^31 with uint32 values (the
    paper's 32-bit coefficient type): returns (rank, row_ptr, col, val)."""
    lib = _lib(mutant)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.uint32)
    rank = ctypes.c_int64(0)
    rp = ctypes.POINTER(ctypes.c_int64)()
    cl = ctypes.POINTER(ctypes.c_int32)()
    vl = ctypes.POINTER(ctypes.c_uint32)()
    rc = lib.oracle_rref32(m, n, p, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                           ctypes.byref(rank), ctypes.byref(rp), ctypes.byref(cl), ctypes.byref(vl))
    if rc != 0:
        raise OracleError(f"oracle_rref32 failed with code {rc}")
    return _take(lib, rank, rp, cl, vl)


def echelon32(m, n, p, row_ptr, col, val, mutant: int = 0):
    """The new-order echelon form for a prime p < 2^31 with uint32 values:
    returns (rank, row_ptr, col, val, npiv)."""
    lib = _lib(mutant)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.uint32)
    rank = ctypes.c_int64(0)
    npiv = ctypes.c_int64(0)
    rp = ctypes.POINTER(ctypes.c_int64)()
    cl = ctypes.POINTER(ctypes.c_int32)()
    vl = ctypes.POINTER(ctypes.c_uint32)()
    rc = lib.oracle_echelon32(m, n, p, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data, ctypes.byref(rank),
                              ctypes.byref(rp), ctypes.byref(cl), ctypes.byref(vl), ctypes.byref(npiv))
    if rc != 0:
        raise OracleError(f"oracle_echelon32 failed with code {rc}")
    return _take(lib, rank, rp, cl, vl) + (int(npiv.value),)


def echelon(m, n, p, row_ptr, col, val, mutant: int = 0, phase_seconds=None, ops=None):
    """Canonical echelon form (normalised pivot rows + RREF of the Schur
    complement): returns (rank, row_ptr, col, val, npiv).  If
    ``phase_seconds`` is a list it receives the wall times of the row
    reduction by the pivot rows and of the Gauss-Jordan pass.  If ``ops`` is
    a list it receives the work counts [ops_b, ops_c, ops_d, ops_e] in
    modular multiply-adds with a nonzero operand entry: the sparse C*A^-1
    (Alg. 2), the Schur update, the Gauss-Jordan pass on the Schur
    complement, and the back-substitution of the top block (0 in this
    form)."""
    lib = _lib(mutant)
    row_ptr, col, val = _csr_args(row_ptr, col, val)
    rank = ctypes.c_int64(0)
    npiv = ctypes.c_int64(0)
    rp = ctypes.POINTER(ctypes.c_int64)()
    cl = ctypes.POINTER(ctypes.c_int32)()
    vl = ctypes.POINTER(ctypes.c_uint16)()
    secs = (ctypes.c_double * 2)()
    counts = (ctypes.c_double * 4)()
    rc = lib.oracle_echelon(m, n, p, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                            ctypes.byref(rank), ctypes.byref(rp), ctypes.byref(cl),
                            ctypes.byref(vl), ctypes.byref(npiv), secs, counts)
    if phase_seconds is not None:
        phase_seconds[:] = [secs[0], secs[1]]
    if ops is not None:
        ops[:] = [counts[i] for i in range(4)]
    if rc != 0:
        raise OracleError(f"oracle_echelon failed with code {rc}")
    return _take(lib, rank, rp, cl, vl) + (int(npiv.value),)


def row_counts(m, n, p, row_ptr, col, val, mutant: int = 0):
    """Work counts of Alg. 2's row reduction alone: returns (ops_b, ops_c,
    npiv, seconds), the first two exactly as :func:`echelon` counts them,
    without the Gauss-Jordan pass (for matrices whose Schur complement is too
    large for it)."""
    lib = _lib(mutant)
    row_ptr, col, val = _csr_args(row_ptr, col, val)
    ops = (ctypes.c_double * 2)()
    npiv = ctypes.c_int64(0)
    secs = ctypes.c_double(0)
    rc = lib.oracle_row_counts(m, n, p, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data, ops,
                               ctypes.byref(npiv), ctypes.byref(secs))
    if rc != 0:
        raise OracleError(f"oracle_row_counts failed with code {rc}")
    return float(ops[0]), float(ops[1]), int(npiv.value), float(secs.value)


def pivots(m, n, row_ptr, col, mutant: int = 0):
    """FL step-1 pivot choice: array piv_row[c] (-1 where no row leads at c)."""
    lib = _lib(mutant)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    out = np.empty(max(n, 1), dtype=np.int64)
    lib.oracle_pivots(m, n, row_ptr.ctypes.data, col.ctypes.data, out.ctypes.data)
    return out[:n]


def multiline(cols1, vals1, cols2, vals2):
    """2-multiline vector of two sparse rows (Definition 1, Sec. 4.2).

    ``pos`` lists, ascending, every column where at least one of the two rows
    is nonzero; ``val`` stores the two rows' entries at ``pos[i]`` next to each
    other (row 1 first), with explicit zeros where only one row is nonzero.
    """
    a = dict(zip((int(c) for c in cols1), (int(v) for v in vals1)))
    b = dict(zip((int(c) for c in cols2), (int(v) for v in vals2)))
    pos = sorted(set(a) | set(b))
    val = []
    for c in pos:
        val.append(a.get(c, 0))
        val.append(b.get(c, 0))
    return np.array(pos, dtype=np.int64), np.array(val, dtype=np.int64)
