"""Seeded synthetic sparse matrices for the workloads of the Gustavson SpGEMM path.

This module only *builds inputs*: CSR patterns and values from seeded numpy
generators.  It contains no part of the product arithmetic (no row products,
no accumulation, no sorting of partial products), so the CPU oracle and the
CUDA path can both consume its output without sharing any of the method.

All matrices are returned as :class:`CSR` with int32 ``row_ptr`` / ``col_idx``
(column indices strictly ascending inside each row) and float64 values.

Workload recipes (the paper evaluates on SuiteSparse matrices, Sec. 5.1 /
Table 4, which are not available; these synthetic stand-ins have the shapes
and structure of the paper's PDE-type and power-law-graph inputs):

* ``laplacian_2d(64)``     2D 5-point operator, diagonal 4, off-diagonal -1.
* ``rmat(18, 16)``         R-MAT power-law adjacency, (a,b,c,d) =
                           (0.57, 0.19, 0.19, 0.05), self-loops dropped,
                           duplicates merged, values U(0.5, 1.5).
* ``laplacian_3d(96)`` and ``aggregation_3d(96)``  the Galerkin triple
                           product operands (7-point operator, 2x2x2
                           piecewise-constant aggregation).
* ``batched_instances``    512 uneven independent products.
* ``random_rows``          uniformly random distinct columns per row.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSR", "laplacian_2d", "laplacian_3d", "aggregation_3d", "rmat",
    "random_rows", "random_csr", "identity", "permutation", "diagonal",
    "batched_instances", "BatchInstance", "instance_seeds", "from_dense",
    "to_dense",
]


@dataclasses.dataclass
class CSR:
    """Compressed sparse row matrix (Sec. 2.1: V, COL_INDEX, ROW_PTR)."""

    nrows: int
    ncols: int
    row_ptr: np.ndarray  # int32, nrows + 1
    col_idx: np.ndarray  # int32, nnz
    vals: np.ndarray     # float64 (or float32), nnz

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.nrows > 0 else 0

    def check(self) -> "CSR":
        """Validate the CSR invariants this library assumes; returns self."""
        rp, ci = self.row_ptr, self.col_idx
        assert rp.dtype == np.int32 and ci.dtype == np.int32
        assert rp.shape == (self.nrows + 1,)
        assert rp[0] == 0 and np.all(np.diff(rp.astype(np.int64)) >= 0)
        assert ci.shape == (self.nnz,) and self.vals.shape == (self.nnz,)
        if self.nnz:
            assert ci.min() >= 0 and ci.max() < self.ncols
            rows = np.repeat(np.arange(self.nrows), np.diff(rp))
            same = rows[1:] == rows[:-1]
            assert np.all(ci[1:][same] > ci[:-1][same]), "columns must ascend"
        return self

    def astype(self, dtype) -> "CSR":
        return CSR(self.nrows, self.ncols, self.row_ptr, self.col_idx,
                   self.vals.astype(dtype))


def _csr_from_sorted_coo(nrows, ncols, rows, cols, vals) -> CSR:
    """Build CSR from COO triples already ordered by (row, col), no repeats."""
    counts = np.bincount(rows, minlength=nrows) if len(rows) else np.zeros(nrows, np.int64)
    rp = np.zeros(nrows + 1, np.int64)
    np.cumsum(counts, out=rp[1:])
    if rp[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return CSR(nrows, ncols, rp.astype(np.int32), np.asarray(cols, np.int32),
               np.asarray(vals, np.float64))


def _stencil(dims, offsets_and_vals):
    """Constant-coefficient stencil on a grid with Dirichlet truncation.

    ``dims`` = (nx, ny, nz...) with x fastest; ``offsets_and_vals`` is a list
    of ((dx, dy, ...), value) sorted so that the flattened column offsets
    ascend (which keeps every row's columns sorted).
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    coords = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]  # x fastest
    strides = np.cumprod((1,) + dims[:-1])
    offs = []
    for delta, _ in offsets_and_vals:
        offs.append(sum(int(d) * int(s) for d, s in zip(delta, strides)))
    order = np.argsort(offs, kind="stable")
    cols_l, valid_l, vals_l = [], [], []
    base = np.arange(n, dtype=np.int64)
    for o in order:
        delta, v = offsets_and_vals[o]
        ok = np.ones(n, bool)
        for ax, d in enumerate(delta):
            c = coords[ax] + d
            ok &= (c >= 0) & (c < dims[ax])
        cols_l.append(base + offs[o])
        valid_l.append(ok)
        vals_l.append(np.full(n, float(v)))
    cols = np.stack(cols_l, 1)
    valid = np.stack(valid_l, 1)
    vals = np.stack(vals_l, 1)
    rows = np.broadcast_to(base[:, None], cols.shape)
    return _csr_from_sorted_coo(n, n, rows[valid], cols[valid], vals[valid])


def laplacian_2d(nx: int, ny: int | None = None) -> CSR:
    """2D 5-point Poisson operator: 4 on the diagonal, -1 to each grid
    neighbour, Dirichlet boundary (neighbours outside the grid are dropped)."""
    ny = nx if ny is None else ny
    st = [((0, -1), -1.0), ((-1, 0), -1.0), ((0, 0), 4.0), ((1, 0), -1.0), ((0, 1), -1.0)]
    return _stencil((nx, ny), st)


def laplacian_3d(n: int) -> CSR:
    """3D 7-point Poisson operator on an n^3 grid: 6 on the diagonal, -1 to
    each face neighbour, Dirichlet boundary."""
    st = [((0, 0, -1), -1.0), ((0, -1, 0), -1.0), ((-1, 0, 0), -1.0), ((0, 0, 0), 6.0),
          ((1, 0, 0), -1.0), ((0, 1, 0), -1.0), ((0, 0, 1), -1.0)]
    return _stencil((n, n, n), st)


def aggregation_3d(n: int, agg: int = 2) -> CSR:
    """Piecewise-constant aggregation P (n^3 x (n/agg)^3): fine node (x,y,z)
    carries a single 1.0 in the column of its agg^3 coarse aggregate."""
    assert n % agg == 0
    nc = n // agg
    idx = np.arange(n ** 3, dtype=np.int64)
    x, y, z = idx % n, (idx // n) % n, idx // (n * n)
    col = ((z // agg) * nc + (y // agg)) * nc + (x // agg)
    return _csr_from_sorted_coo(n ** 3, nc ** 3, idx, col, np.ones(n ** 3))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, lo: float = 0.5, hi: float = 1.5) -> CSR:
    """R-MAT adjacency (Chakrabarti et al.): 2^scale vertices and
    edge_factor * 2^scale drawn edges.

    Each edge draws one uniform number per level, most significant bit
    first; it falls in quadrant a (row bit 0, col bit 0), b (0, 1), c (1, 0)
    or d (1, 1).  No noise and no vertex permutation, so hubs sit at low
    ids.  The graph stays directed; self-loops are dropped and repeated
    edges merged into one entry.  Values U(lo, hi) are drawn after merging,
    in (row, col) order.  Generator: numpy PCG64(seed).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 1 << scale
    e = edge_factor * n
    row = np.zeros(e, np.int64)
    col = np.zeros(e, np.int64)
    for _ in range(scale):
        u = rng.random(e)
        rbit = u >= (a + b)
        cbit = ((u >= a) & (u < a + b)) | (u >= (a + b + c))
        row = (row << 1) | rbit
        col = (col << 1) | cbit
    keep = row != col
    key = np.unique(row[keep] * n + col[keep])
    rows, cols = key // n, key % n
    vals = rng.uniform(lo, hi, size=len(key))
    return _csr_from_sorted_coo(n, n, rows, cols, vals)


def random_rows(nrows: int, ncols: int, counts, rng: np.random.Generator,
                values: str = "normal") -> CSR:
    """Rows with ``counts[i]`` distinct uniformly random columns each.

    Columns are drawn with replacement, then repeats inside a row are redrawn
    until every row is duplicate-free.  Values are drawn afterwards in
    (row, col) order: N(0,1) for ``values="normal"``, U(0.5,1.5) for
    ``"uniform"``, small integers in [-3, 3] for ``"int"``.
    """
    counts = np.asarray(counts, np.int64)
    assert counts.shape == (nrows,)
    if nrows and counts.max(initial=0) > ncols:
        raise ValueError("row count exceeds ncols")
    total = int(counts.sum())
    rows = np.repeat(np.arange(nrows, dtype=np.int64), counts)
    cols = rng.integers(0, max(ncols, 1), size=total, dtype=np.int64)
    while total:
        key = rows * ncols + cols
        key.sort()
        dup = np.flatnonzero(key[1:] == key[:-1]) + 1
        rows, cols = key // ncols, key % ncols
        if len(dup) == 0:
            break
        cols[dup] = rng.integers(0, ncols, size=len(dup), dtype=np.int64)
    if values == "normal":
        vals = rng.standard_normal(total)
    elif values == "uniform":
        vals = rng.uniform(0.5, 1.5, total)
    elif values == "int":
        vals = rng.integers(-3, 4, total).astype(np.float64)
    else:
        raise ValueError(values)
    return _csr_from_sorted_coo(nrows, ncols, rows, cols, vals)


def random_csr(nrows: int, ncols: int, density: float, seed: int,
               values: str = "normal", empty_rows: float = 0.0) -> CSR:
    """Small random matrix: each row has Binomial(ncols, density) distinct
    columns; a fraction ``empty_rows`` of rows is forced empty."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.binomial(ncols, density, size=nrows) if ncols else np.zeros(nrows, np.int64)
    if empty_rows > 0 and nrows:
        counts[rng.random(nrows) < empty_rows] = 0
    return random_rows(nrows, ncols, counts, rng, values)


def identity(n: int) -> CSR:
    i = np.arange(n, dtype=np.int64)
    return _csr_from_sorted_coo(n, n, i, i, np.ones(n))


def diagonal(d) -> CSR:
    d = np.asarray(d, np.float64)
    i = np.arange(len(d), dtype=np.int64)
    return _csr_from_sorted_coo(len(d), len(d), i, i, d)


def permutation(perm) -> CSR:
    """P with P[i, perm[i]] = 1, so (P @ A) row i = A row perm[i]."""
    perm = np.asarray(perm, np.int64)
    i = np.arange(len(perm), dtype=np.int64)
    return _csr_from_sorted_coo(len(perm), len(perm), i, perm, np.ones(len(perm)))


def lower_triangle_undirected(G: CSR) -> CSR:
    """Strictly lower triangle L of the simple undirected graph on G's
    pattern (G square; edges (i,j) and (j,i) are one edge, self-loops are
    dropped), every stored value 1.0.  Triangle counting takes it as all three
    operands of the masked product: sum((L*L) .* L) counts each triangle
    i > k > j once."""
    assert G.nrows == G.ncols
    rows = np.repeat(np.arange(G.nrows, dtype=np.int64), np.diff(np.asarray(G.row_ptr, np.int64)))
    cols = np.asarray(G.col_idx, np.int64)
    hi, lo = np.maximum(rows, cols), np.minimum(rows, cols)
    keep = hi != lo
    key = np.unique(hi[keep] * G.ncols + lo[keep])
    r, c = key // G.ncols, key % G.ncols
    return _csr_from_sorted_coo(G.nrows, G.ncols, r, c, np.ones(len(key)))


def from_dense(d: np.ndarray) -> CSR:
    """Pattern = nonzero entries of ``d`` (explicit zeros are not stored)."""
    d = np.asarray(d, np.float64)
    r, c = np.nonzero(d)
    return _csr_from_sorted_coo(d.shape[0], d.shape[1], r, c, d[r, c])


def to_dense(m: CSR) -> np.ndarray:
    out = np.zeros((m.nrows, m.ncols), np.float64)
    rows = np.repeat(np.arange(m.nrows), np.diff(m.row_ptr))
    out[rows, m.col_idx] = m.vals
    return out


# ---------------------------------------------------------------------------
# Batched workload: many independent products of uneven size.
# ---------------------------------------------------------------------------

BATCH_SEED = 2112_10037


@dataclasses.dataclass
class BatchInstance:
    kind: str          # "stencil2d", "stencil3d" or "random"
    rows: int
    A: CSR
    B: CSR             # for stencil instances B is A (C = A*A)


def instance_seeds(count: int, seed: int = BATCH_SEED):
    return np.random.SeedSequence(seed).spawn(count)


def batched_instance(i: int, count: int = 512, rows_lo: int = 1024, rows_hi: int = 200_000,
                     seed: int = BATCH_SEED, scale_rows: float = 1.0, seeds=None) -> BatchInstance:
    """Instance ``i`` of the batch of ``count`` (see ``batched_instances``),
    built from its own spawned seed alone, so instances can be generated
    independently (in parallel processes) and still match the sequence."""
    if seeds is None:
        seeds = instance_seeds(count, seed)
    rng = np.random.Generator(np.random.PCG64(seeds[i]))
    r = int(round(math.exp(rng.uniform(math.log(rows_lo), math.log(rows_hi))) * scale_rows))
    r = max(r, 1)
    if i < count // 2:
        if i % 2 == 0:
            side = max(1, int(round(math.sqrt(r))))
            A = laplacian_2d(side)
            return BatchInstance("stencil2d", A.nrows, A, A)
        side = max(1, int(round(r ** (1.0 / 3.0))))
        A = laplacian_3d(side)
        return BatchInstance("stencil3d", A.nrows, A, A)
    hi = min(64, r)
    lo = min(2, hi)
    A = random_rows(r, r, rng.integers(lo, hi + 1, size=r), rng)
    B = random_rows(r, r, rng.integers(lo, hi + 1, size=r), rng)
    return BatchInstance("random", r, A, B)


def batched_instances(count: int = 512, rows_lo: int = 1024, rows_hi: int = 200_000,
                      seed: int = BATCH_SEED, scale_rows: float = 1.0):
    """Yield ``count`` independent instances (lazily, one at a time).

    Instance i draws its row count log-uniformly in [rows_lo, rows_hi] from
    its own spawned seed.  The first half are stencil squares (2D 5-point
    with side round(sqrt(r)) for even i, 3D 7-point with side round(cbrt(r))
    for odd i; C = A*A with the operator's integer values).  The second half
    are A*B with independent square r x r operands whose rows hold
    U{2..64} distinct uniform columns and N(0,1) values.  ``scale_rows``
    shrinks every instance (used for small test batches).
    """
    seeds = instance_seeds(count, seed)
    for i in range(count):
        yield batched_instance(i, count, rows_lo, rows_hi, seed, scale_rows, seeds)


def _instance_task(args):
    i, count, scale_rows = args
    return batched_instance(i, count, scale_rows=scale_rows)


def batched_instances_parallel(count: int = 512, scale_rows: float = 1.0, processes=None):
    """The list ``list(batched_instances(count, scale_rows=scale_rows))``,
    generated by a pool of spawned host processes (each instance comes from
    its own seed, so the result is the same)."""
    import multiprocessing as mp
    import os
    procs = max(1, min(count, processes or os.cpu_count() or 1))
    if procs == 1:
        return list(batched_instances(count, scale_rows=scale_rows))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_instance_task, [(i, count, scale_rows) for i in range(count)], chunksize=1)
