"""Whole-product comparison of a device result with the oracle, range by range.

The device's C (row pointer, columns, values) is copied once into
memory-mapped host files together with the inputs; a pool of spawned host processes
(spawn, never fork, because the parent already holds a CUDA context) then
runs the oracle on contiguous row ranges of A -- each call an ordinary
single-threaded oracle product of those rows with B -- and compares its
rows with the same rows of the device result:

* the row sizes (row pointer differences) and every column index exactly;
* every value within the FP64 criterion of the parity helpers,
  |c - c*| <= rtol * max(|c*|, sum_k |A(i,k) B(k,j)|), or bit-exactly with
  ``exact=True`` (integer-valued inputs).

When every stored value of A and B is positive, all terms of every sum share
one sign, so the magnitude sum equals |c*| and the second oracle product on
|A|, |B| is skipped.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile

import numpy as np

_SH = {}


class Store:
    """A directory of raw array files shared with the worker processes
    (memory-mapped; on /dev/shm when it has room, else the temp directory)."""

    def __init__(self, need_bytes):
        base = "/dev/shm"
        try:
            room = shutil.disk_usage(base).free if os.path.isdir(base) else 0
        except OSError:
            room = 0
        self.dir = tempfile.mkdtemp(prefix="spgemm_cmp_", dir=base if room > 1.2 * need_bytes else None)
        self.specs = {}

    def empty(self, name, shape, dtype):
        dtype = np.dtype(dtype)
        path = os.path.join(self.dir, name)
        n = int(np.prod(shape))
        arr = np.memmap(path, dtype=dtype, mode="w+", shape=(max(n, 1),))[:n].reshape(shape)
        self.specs[name] = (path, tuple(shape), dtype.str)
        return arr

    def put(self, name, a):
        a = np.ascontiguousarray(a)
        self.empty(name, a.shape, a.dtype)[...] = a

    def close(self):
        shutil.rmtree(self.dir, ignore_errors=True)


def _init(specs):
    for name, (path, shape, dt) in specs.items():
        n = int(np.prod(shape))
        _SH[name] = np.memmap(path, dtype=np.dtype(dt), mode="r", shape=(max(n, 1),))[:n].reshape(shape)


def _get(name):
    return _SH[name]


def _rows(prefix, r0, r1, ncols):
    from paper_2112_10037_gb300.gen import CSR
    rp = _get(prefix + "rp").astype(np.int64)
    lo, hi = int(rp[r0]), int(rp[r1])
    return CSR(r1 - r0, ncols, (rp[r0:r1 + 1] - lo).astype(np.int32), _get(prefix + "ci")[lo:hi],
               np.asarray(_get(prefix + "v")[lo:hi], np.float64))


def _check_range(task):
    px, r0, r1, a_ncols, b_ncols, rtol, exact, positive = task
    import oracle
    from paper_2112_10037_gb300.gen import CSR
    A = _rows(px + "a_", r0, r1, a_ncols)
    brp = _get(px + "b_rp")
    B = CSR(len(brp) - 1, b_ncols, brp, _get(px + "b_ci"), np.asarray(_get(px + "b_v"), np.float64))
    R = oracle.spgemm(A, B)
    crp = _get(px + "c_rp").astype(np.int64)
    lo, hi = int(crp[r0]), int(crp[r1])
    out = {"item": px, "r0": r0, "r1": r1, "nnz": hi - lo, "rp_ok": True, "ci_ok": True, "max_err": 0.0,
           "bad": 0}
    if not np.array_equal(crp[r0:r1 + 1] - lo, np.asarray(R.row_ptr, np.int64)):
        out["rp_ok"] = False
        return out
    ci = _get(px + "c_ci")[lo:hi]
    if not np.array_equal(ci, R.col_idx):
        out["ci_ok"] = False
        out["first_ci"] = int(np.flatnonzero(ci != R.col_idx)[0]) + lo
        return out
    got = np.asarray(_get(px + "c_v")[lo:hi], np.float64)
    ref = np.asarray(R.vals, np.float64)
    if exact:
        bad = got != ref
        out["bad"] = int(bad.sum())
        out["max_err"] = float(np.max(np.abs(got - ref))) if len(ref) else 0.0
        return out
    if positive:
        scale = np.abs(ref)
    else:
        absA = CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx, np.abs(A.vals))
        absB = CSR(B.nrows, B.ncols, B.row_ptr, B.col_idx, np.abs(B.vals))
        scale = oracle.spgemm(absA, absB).vals
    den = np.maximum(np.abs(ref), scale)
    den = np.where(den == 0, 1.0, den)
    rel = np.abs(got - ref) / den
    out["max_err"] = float(rel.max()) if len(rel) else 0.0
    out["bad"] = int((rel > rtol).sum())
    return out


def balanced_ranges(prod, nranges):
    """Row boundaries cutting rows into about nranges ranges of equal
    product count (a single heavy row may form a range alone)."""
    cs = np.concatenate([[0], np.cumsum(np.asarray(prod, np.int64))])
    cuts = np.searchsorted(cs, cs[-1] * np.arange(1, nranges) / nranges)
    b = np.unique(np.concatenate([[0], cuts, [len(prod)]]))
    return [(int(x), int(y)) for x, y in zip(b[:-1], b[1:]) if y > x]


def _tasks(A, B, prod, prefix, rtol, exact, nranges):
    positive = bool(len(A.vals) == 0 or np.min(A.vals) > 0) and bool(len(B.vals) == 0 or np.min(B.vals) > 0)
    return [(prefix, r0, r1, A.ncols, B.ncols, rtol, exact, positive) for r0, r1 in balanced_ranges(prod, nranges)]


def put_inputs(store, A, B, prefix=""):
    for name, arr in (("a_rp", A.row_ptr), ("a_ci", A.col_idx), ("a_v", np.asarray(A.vals, np.float64)),
                      ("b_rp", B.row_ptr), ("b_ci", B.col_idx), ("b_v", np.asarray(B.vals, np.float64))):
        store.put(prefix + name, arr)


def compare_product(A, B, store, prod, rtol=1e-12, exact=False, processes=None, ranges_per_process=6):
    """Compares the whole product with the oracle.  ``store`` holds the
    device result as "c_rp" (int64), "c_ci" and "c_v" (see ``Store``).
    Returns the list of per-range results."""
    processes = processes or os.cpu_count() or 4
    put_inputs(store, A, B)
    tasks = _tasks(A, B, prod, "", rtol, exact, processes * ranges_per_process)
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes, initializer=_init, initargs=(store.specs,)) as pool:
        return pool.map(_check_range, tasks, chunksize=1)


def compare_many(items, store, processes=None, ranges_per_item=4):
    """Several products compared in one pool: ``items`` is a list of
    (prefix, A, B, prod, rtol, exact) whose device results the caller put in
    ``store`` as prefix + "c_rp" / "c_ci" / "c_v"; the inputs are stored
    here.  Returns the per-range results of all items (each tagged with its
    prefix as "item")."""
    processes = processes or os.cpu_count() or 4
    tasks = []
    for prefix, A, B, prod, rtol, exact in items:
        put_inputs(store, A, B, prefix)
        tasks += _tasks(A, B, prod, prefix, rtol, exact, ranges_per_item)
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes, initializer=_init, initargs=(store.specs,)) as pool:
        return pool.map(_check_range, tasks, chunksize=1)


def summarise(res):
    """(all_ok, max_err, entries, message) of compare_product's results."""
    max_err = max((r["max_err"] for r in res), default=0.0)
    entries = sum(r["nnz"] for r in res)
    for r in res:
        where = "%srows [%d, %d)" % (r["item"] + " " if r.get("item") else "", r["r0"], r["r1"])
        if not r["rp_ok"]:
            return False, max_err, entries, "row sizes differ in " + where
        if not r["ci_ok"]:
            return False, max_err, entries, "columns differ in %s at entry %d" % (where, r["first_ci"])
        if r["bad"]:
            return False, max_err, entries, "%d values outside the bound in %s" % (r["bad"], where)
    return True, max_err, entries, "ok"
