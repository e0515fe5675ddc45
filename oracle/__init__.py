"""CPU oracle for the Gustavson SpGEMM path -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
and its Python binding) never does; the two share no code.

The arithmetic lives in ``spgemm_oracle.c`` (plain single-threaded C,
compiled with ``-O2 -ffp-contract=off``); this module only builds it and
marshals numpy arrays through ctypes.  Each function cites the passage of the
paper it follows (Sec. 2.2 row-wise Gustavson and the sorted merge of sparse
rows; Table 1 for the per-nonzero product count).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(dense brute force, identity/permutation/diagonal products, stencil closed
forms, the (A*B)*x = A*(B*x) invariant, finite differences for the
gradient, a hand-worked example, triangle counts of graphs with known
counts for the masked product); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# The benchmark's CPU leg and the tests read the generators' CSR class.
_REPO = os.path.dirname(_HERE)
if _REPO not in sys.path:
    sys.path.insert(0, _REPO)
from paper_2112_10037_gb300.gen import CSR  # noqa: E402  (inputs only, no arithmetic)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no vector extensions)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_spgemm_rowptr.argtypes = [I64, I64, P, P, P, P, P]
        lib.oracle_spgemm_rowptr.restype = ctypes.c_int
        lib.oracle_spgemm.argtypes = [I64, I64, P, P, P, P, P, P, P, P, P]
        lib.oracle_spgemm.restype = ctypes.c_int
        lib.oracle_spgemm_backward.argtypes = [I64, I64, P, P, P, P, P, P, I64, P, P, P, P, P]
        lib.oracle_spgemm_backward.restype = ctypes.c_int
        lib.oracle_transpose.argtypes = [I64, I64, P, P, P, P, P, P]
        lib.oracle_transpose.restype = ctypes.c_int
        lib.oracle_spmv.argtypes = [I64, P, P, P, P, P]
        lib.oracle_spmv.restype = None
        lib.oracle_row_products.argtypes = [I64, P, P, P, P]
        lib.oracle_row_products.restype = None
        lib.oracle_masked.argtypes = [I64, I64, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_masked.restype = ctypes.c_int
        lib.oracle_masked_semiring.argtypes = [I64, I64, ctypes.c_int32, P, P, P, P, P, P, P, P, P]
        lib.oracle_masked_semiring.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def spgemm(A: CSR, B: CSR) -> CSR:
    """C = A*B by row-wise Gustavson (Sec. 2.2): per row, a dense accumulator
    with a marker array, products in stored order, touched columns sorted
    ascending.  Values are float64; row_ptr is int64 (the oracle does not
    assume nnz(C) < 2^31)."""
    if A.ncols != B.nrows:
        raise ValueError("A.ncols != B.nrows")
    lib = _load()
    arp, aci, av = _c(A.row_ptr, np.int32), _c(A.col_idx, np.int32), _c(A.vals, np.float64)
    brp, bci, bv = _c(B.row_ptr, np.int32), _c(B.col_idx, np.int32), _c(B.vals, np.float64)
    crp = np.zeros(A.nrows + 1, np.int64)
    if lib.oracle_spgemm_rowptr(A.nrows, B.ncols, _p(arp), _p(aci), _p(brp), _p(bci), _p(crp)):
        raise MemoryError("oracle allocation failed")
    nnz = int(crp[-1])
    cci = np.empty(nnz, np.int32)
    cv = np.empty(nnz, np.float64)
    if lib.oracle_spgemm(A.nrows, B.ncols, _p(arp), _p(aci), _p(av), _p(brp), _p(bci), _p(bv),
                         _p(crp), _p(cci), _p(cv)):
        raise MemoryError("oracle allocation failed")
    return CSR(A.nrows, B.ncols, crp, cci, cv)


def spgemm_rowptr(A: CSR, B: CSR) -> np.ndarray:
    """Row pointer of C = A*B (int64), from the same marker loop."""
    lib = _load()
    arp, aci = _c(A.row_ptr, np.int32), _c(A.col_idx, np.int32)
    brp, bci = _c(B.row_ptr, np.int32), _c(B.col_idx, np.int32)
    crp = np.zeros(A.nrows + 1, np.int64)
    if lib.oracle_spgemm_rowptr(A.nrows, B.ncols, _p(arp), _p(aci), _p(brp), _p(bci), _p(crp)):
        raise MemoryError("oracle allocation failed")
    return crp


def backward(A: CSR, B: CSR, C_row_ptr, C_col_idx, dC_vals):
    """(dA, dB) of L = sum W*C on C's pattern, dC = W: dA = (dC B^T) on
    pattern(A), dB = (A^T dC) on pattern(B).  Returns two float64 arrays
    aligned with A.vals and B.vals."""
    lib = _load()
    arp, aci, av = _c(A.row_ptr, np.int32), _c(A.col_idx, np.int32), _c(A.vals, np.float64)
    brp, bci, bv = _c(B.row_ptr, np.int32), _c(B.col_idx, np.int32), _c(B.vals, np.float64)
    crp, cci = _c(C_row_ptr, np.int64), _c(C_col_idx, np.int32)
    dc = _c(dC_vals, np.float64)
    da = np.empty(A.nnz, np.float64)
    db = np.empty(B.nnz, np.float64)
    if lib.oracle_spgemm_backward(A.nrows, B.ncols, _p(arp), _p(aci), _p(av), _p(brp), _p(bci),
                                  _p(bv), B.nnz, _p(crp), _p(cci), _p(dc), _p(da), _p(db)):
        raise MemoryError("oracle allocation failed")
    return da, db


def transpose(A: CSR) -> CSR:
    """A^T as CSR (the CSC form of Sec. 2.1), rows of A^T in source-row order."""
    lib = _load()
    rp, ci, v = _c(A.row_ptr, np.int32), _c(A.col_idx, np.int32), _c(A.vals, np.float64)
    trp = np.zeros(A.ncols + 1, np.int64)
    tci = np.empty(A.nnz, np.int32)
    tv = np.empty(A.nnz, np.float64)
    if lib.oracle_transpose(A.nrows, A.ncols, _p(rp), _p(ci), _p(v), _p(trp), _p(tci), _p(tv)):
        raise MemoryError("oracle allocation failed")
    return CSR(A.ncols, A.nrows, trp, tci, tv)


def spmv(A: CSR, x) -> np.ndarray:
    lib = _load()
    rp, ci, v = _c(A.row_ptr, np.int32), _c(A.col_idx, np.int32), _c(A.vals, np.float64)
    x = _c(x, np.float64)
    y = np.empty(A.nrows, np.float64)
    lib.oracle_spmv(A.nrows, _p(rp), _p(ci), _p(v), _p(x), _p(y))
    return y


def row_products(A: CSR, B: CSR) -> np.ndarray:
    """prod[i] = sum over A(i,k) of nnz(B(k,:)) (the per-nonzero B_NUM_VEC
    count of Table 1, summed over the row)."""
    lib = _load()
    arp, aci, brp = _c(A.row_ptr, np.int32), _c(A.col_idx, np.int32), _c(B.row_ptr, np.int32)
    out = np.empty(A.nrows, np.int64)
    lib.oracle_row_products(A.nrows, _p(arp), _p(aci), _p(brp), _p(out))
    return out


def masked(A: CSR, B: CSR, M: CSR, use_mask_values: bool = True) -> np.ndarray:
    """C<M> = (A*B) .* M on M's pattern: for entry p = (i,j) of M,
    M(i,j) * sum_k A(i,k) B(k,j) over the k with both entries stored (0 if
    none), accumulated in the Gustavson product order of Sec. 2.2.  Without
    ``use_mask_values`` M is a pure pattern (factor 1).  Returns nnz(M)
    float64 values aligned with M's entries."""
    lib = _load()
    arp, aci, av = _c(A.row_ptr, np.int32), _c(A.col_idx, np.int32), _c(A.vals, np.float64)
    brp, bci, bv = _c(B.row_ptr, np.int32), _c(B.col_idx, np.int32), _c(B.vals, np.float64)
    mrp, mci = _c(M.row_ptr, np.int32), _c(M.col_idx, np.int32)
    mv = _c(M.vals, np.float64) if use_mask_values else None
    out = np.empty(M.nnz, np.float64)
    if lib.oracle_masked(A.nrows, B.ncols, _p(arp), _p(aci), _p(av), _p(brp), _p(bci), _p(bv),
                         _p(mrp), _p(mci), _p(mv) if mv is not None else None, _p(out)):
        raise MemoryError("oracle allocation failed")
    return out


SEMIRINGS = {"plus_times": 0, "min_plus": 1, "max_plus": 2, "or_and": 3}


def masked_semiring(A: CSR, B: CSR, M: CSR, semiring: str) -> np.ndarray:
    """Masked product over a semiring on M's pattern (M's values unused):
    min-plus (min of a + b, +inf where no product reaches), max-plus (max of
    a + b, -inf), or-and (1.0 where some product has both factors nonzero,
    else 0.0), plus-times (the sum of a * b).  The products run in the
    row-wise Gustavson order of Sec. 2.2."""
    lib = _load()
    arp, aci, av = _c(A.row_ptr, np.int32), _c(A.col_idx, np.int32), _c(A.vals, np.float64)
    brp, bci, bv = _c(B.row_ptr, np.int32), _c(B.col_idx, np.int32), _c(B.vals, np.float64)
    mrp, mci = _c(M.row_ptr, np.int32), _c(M.col_idx, np.int32)
    out = np.empty(M.nnz, np.float64)
    r = lib.oracle_masked_semiring(A.nrows, B.ncols, SEMIRINGS[semiring], _p(arp), _p(aci), _p(av), _p(brp),
                                   _p(bci), _p(bv), _p(mrp), _p(mci), _p(out))
    if r:
        raise MemoryError("oracle allocation failed") if r == -1 else ValueError(semiring)
    return out


def omar(A: CSR, pes: int) -> float:
    """Off-chip memory access reduction (Eq. 1) of the buffering scheme of
    Sec. 3: rows are taken pes at a time (one per computing unit), and one
    CSV vector is the group's nonzeros in one column, so all of them share
    one read of that row of B.  OMAR(%) = sum over the nonzero vectors v of
    (nnz(v) - 1), divided by nnz(A), times 100.  Counted vector by vector:
    for each group of rows, the nonzeros per column (np.unique with counts)."""
    rp = np.asarray(A.row_ptr, np.int64)
    total = 0
    for g0 in range(0, A.nrows, pes):
        cols = np.asarray(A.col_idx[rp[g0]:rp[min(g0 + pes, A.nrows)]])
        if len(cols):
            _, counts = np.unique(cols, return_counts=True)
            total += int((counts - 1).sum())
    return 100.0 * total / A.nnz if A.nnz else 0.0


def select_rows(A: CSR, rows) -> CSR:
    """The sub-matrix of the given rows of A (input slicing, no arithmetic)."""
    rows = np.asarray(rows, np.int64)
    rp = A.row_ptr.astype(np.int64)
    lens = rp[rows + 1] - rp[rows]
    new_rp = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(lens, out=new_rp[1:])
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if len(rows) else np.zeros(0, np.int64)
    idx = idx.astype(np.int64)
    return CSR(len(rows), A.ncols, new_rp.astype(np.int32), A.col_idx[idx], A.vals[idx])
