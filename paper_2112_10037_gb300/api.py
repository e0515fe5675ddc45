"""Torch-facing helpers over the C ABI: device CSR containers, plans, and the
one-call product.  PyTorch supplies device memory (its caching allocator)
and the current CUDA stream; every step of the product runs in the CUDA
library through ``_native``.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from typing import Optional

import numpy as np
import torch

from . import _native as nat

_DT = {torch.float64: nat.SPGEMM_F64, torch.float32: nat.SPGEMM_F32}
_DT_INV = {v: k for k, v in _DT.items()}


@dataclasses.dataclass
class DeviceCSR:
    """CSR matrix held in device tensors (int32 row_ptr / col_idx)."""

    nrows: int
    ncols: int
    row_ptr: torch.Tensor
    col_idx: torch.Tensor
    vals: Optional[torch.Tensor]

    @property
    def nnz(self) -> int:
        return int(self.col_idx.numel())

    @staticmethod
    def from_host(m, device="cuda", dtype=torch.float64) -> "DeviceCSR":
        """From a host CSR (``gen.CSR`` or any object with nrows, ncols,
        row_ptr, col_idx, vals as numpy arrays)."""
        rp = torch.from_numpy(np.ascontiguousarray(m.row_ptr, np.int32)).to(device)
        ci = torch.from_numpy(np.ascontiguousarray(m.col_idx, np.int32)).to(device)
        v = None
        if m.vals is not None:
            v = torch.from_numpy(np.ascontiguousarray(m.vals)).to(device=device, dtype=dtype)
        return DeviceCSR(int(m.nrows), int(m.ncols), rp, ci, v)

    def to_host(self):
        from .gen import CSR
        vals = self.vals.double().cpu().numpy() if self.vals is not None else np.zeros(self.nnz)
        return CSR(self.nrows, self.ncols, self.row_ptr.cpu().numpy().astype(np.int32),
                   self.col_idx.cpu().numpy(), vals)

    @staticmethod
    def from_torch(t: torch.Tensor) -> "DeviceCSR":
        """From a ``torch.sparse_csr_tensor`` (its index tensors converted to
        int32; the values are used as they are)."""
        if not isinstance(t, torch.Tensor) or t.layout != torch.sparse_csr:
            raise TypeError("expected a torch.sparse_csr_tensor")
        if t.dim() != 2:
            raise ValueError("expected a 2-D sparse CSR tensor")
        rp = t.crow_indices().to(torch.int32).contiguous()
        ci = t.col_indices().to(torch.int32).contiguous()
        return DeviceCSR(int(t.shape[0]), int(t.shape[1]), rp, ci, t.values().contiguous())

    @staticmethod
    def from_tuple(parts) -> "DeviceCSR":
        """From (indptr, indices, values, (nrows, ncols)) tensors."""
        indptr, indices, values, shape = parts
        return DeviceCSR(int(shape[0]), int(shape[1]), indptr.to(torch.int32).contiguous(),
                         indices.to(torch.int32).contiguous(), values.contiguous() if values is not None else None)

    def to_torch(self) -> torch.Tensor:
        """As a ``torch.sparse_csr_tensor`` sharing this matrix's tensors."""
        vals = self.vals if self.vals is not None else torch.ones(self.nnz, dtype=torch.float64,
                                                                  device=self.row_ptr.device)
        return torch.sparse_csr_tensor(self.row_ptr, self.col_idx, vals, size=(self.nrows, self.ncols))

    def to_tuple(self):
        """(indptr, indices, values, (nrows, ncols))."""
        return self.row_ptr, self.col_idx, self.vals, (self.nrows, self.ncols)

    def c_struct(self) -> nat.spgemm_csr:
        s = nat.spgemm_csr()
        s.nrows, s.ncols, s.nnz = self.nrows, self.ncols, self.nnz
        s.row_ptr = self.row_ptr.data_ptr()
        s.col_idx = self.col_idx.data_ptr() if self.nnz else 0
        s.vals = self.vals.data_ptr() if (self.vals is not None and self.nnz) else 0
        return s


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def make_opts(dtype=torch.float64, validate=False, row_range=None, force_path=-1, warp_max=0,
              window_warp=0, window_block=0, split_min=0, backward=False, num_block_min=0,
              block_warps=0, sort_max=0, hash_max=0, rank_min=0, rank_accum=0,
              semiring="plus_times") -> nat.spgemm_opts:
    o = nat.spgemm_opts_default()
    o.dtype = _DT[dtype]
    o.validate = 1 if validate else 0
    if row_range is not None:
        o.row_begin, o.row_end = int(row_range[0]), int(row_range[1])
    o.force_path = int(force_path)
    o.warp_max = int(warp_max)
    o.window_warp = int(window_warp)
    o.window_block = int(window_block)
    o.split_min = int(split_min)
    o.backward = 1 if backward else 0
    o.num_block_min = int(num_block_min)
    o.block_warps = int(block_warps)
    o.sort_max = int(sort_max)
    o.hash_max = int(hash_max)
    o.rank_min = int(rank_min)
    o.rank_accum = int(rank_accum)
    o.semiring = SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)
    return o


class Plan:
    """An analysed product C = A*B (``spgemm_analyse``) with its workspace.

    ``symbolic()`` sizes C (``spgemm_symbolic``, blocks once for nnz(C));
    ``numeric(a_vals, b_vals)`` fills C's columns and values
    (``spgemm_numeric``) and can be repeated for new values.  A's and B's
    structure tensors must stay alive and unchanged while the plan lives.
    """

    def __init__(self, A: DeviceCSR, B: DeviceCSR, dtype=torch.float64, stream=None, **opt_kw):
        self.A, self.B = A, B
        self.dtype = dtype
        self.opts = make_opts(dtype=dtype, **opt_kw)
        self._a, self._b = A.c_struct(), B.c_struct()
        nbytes = nat.spgemm_workspace_size(self._a, self._b, self.opts)
        self.workspace = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=A.row_ptr.device)
        self.stream = _stream_handle(stream)
        self.handle = nat.spgemm_analyse(self._a, self._b, self.opts, self.workspace.data_ptr(), nbytes,
                                         self.stream)
        self.nrows = (self.opts.row_end if self.opts.row_end >= 0 else A.nrows) - self.opts.row_begin
        self.row_ptr: Optional[torch.Tensor] = None
        self.col_idx: Optional[torch.Tensor] = None
        self.nnz: Optional[int] = None

    def rows(self, row_begin: int, row_end: int, stream=None) -> "Plan":
        """Plan for rows [row_begin, row_end) of this product that reads this
        plan's preprocessing of B (``spgemm_analyse_rows``), issuing on
        ``stream`` (default: the current stream), which must be ordered after
        this plan's analysis; this plan must outlive it."""
        p = object.__new__(Plan)
        p.A, p.B, p.dtype, p.stream = self.A, self.B, self.dtype, _stream_handle(stream)
        p.opts = make_opts(dtype=self.dtype)
        p._a, p._b = self._a, self._b
        nbytes = nat.spgemm_rows_workspace_size(self.handle, row_begin, row_end)
        p.workspace = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=self.workspace.device)
        p.handle = nat.spgemm_analyse_rows(self.handle, row_begin, row_end, p.workspace.data_ptr(), nbytes,
                                           p.stream)
        p.nrows = row_end - row_begin
        p.row_ptr, p.col_idx, p.nnz = None, None, None
        p._base = self  # keeps the base plan alive
        return p

    def adopt(self, row_ptr: torch.Tensor, nnz: int):
        """Size this plan from row offsets computed elsewhere
        (``spgemm_plan_adopt_row_ptr``): ``row_ptr`` (device int32, nrows + 1)
        holds where each row's entries go in the C arrays later given to
        ``numeric``; ``nnz`` entries in all.  Blocks on the plan's stream."""
        nat.spgemm_plan_adopt_row_ptr(self.handle, int(nnz), self.stream)
        self.row_ptr = row_ptr
        self.nnz = int(nnz)

    def symbolic(self):
        self.row_ptr = torch.empty(self.nrows + 1, dtype=torch.int32, device=self.workspace.device)
        self.nnz = nat.spgemm_symbolic(self.handle, self.row_ptr.data_ptr(), self.stream)
        return self.row_ptr, self.nnz

    def numeric(self, a_vals: torch.Tensor, b_vals: torch.Tensor, col_idx=None, vals=None):
        if self.row_ptr is None:
            self.symbolic()
        dev = self.workspace.device
        if col_idx is None:
            col_idx = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        if vals is None:
            vals = torch.empty(self.nnz, dtype=self.dtype, device=dev)
        assert a_vals.dtype == self.dtype and b_vals.dtype == self.dtype
        self.col_idx = col_idx
        nat.spgemm_numeric(self.handle, a_vals.data_ptr() if a_vals.numel() else 0,
                           b_vals.data_ptr() if b_vals.numel() else 0, self.row_ptr.data_ptr(),
                           col_idx.data_ptr() if self.nnz else 0, vals.data_ptr() if self.nnz else 0,
                           self.stream)
        return col_idx, vals

    def stats(self):
        """(total products, largest row's products, rows per path
        [register-sort, hash, warp, block] of the symbolic pass)."""
        return nat.spgemm_plan_stats(self.handle, self.stream)

    def check(self):
        nat.spgemm_plan_check(self.handle, self.stream)

    def close(self):
        if getattr(self, "handle", None):
            nat.spgemm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _as_csr(M):
    """(DeviceCSR, kind) for a DeviceCSR, a torch.sparse_csr_tensor or an
    (indptr, indices, values, shape) tuple."""
    if isinstance(M, DeviceCSR):
        return M, "csr"
    if isinstance(M, torch.Tensor):
        return DeviceCSR.from_torch(M), "torch"
    if isinstance(M, (tuple, list)) and len(M) == 4:
        return DeviceCSR.from_tuple(M), "tuple"
    raise TypeError("expected DeviceCSR, torch.sparse_csr_tensor or (indptr, indices, values, shape)")


def _as_kind(C: DeviceCSR, kind):
    return C.to_torch() if kind == "torch" else (C.to_tuple() if kind == "tuple" else C)


def spgemm(A, B, dtype=None, **opt_kw):
    """C = A*B on the device (analyse, symbolic, numeric).  A and B are
    DeviceCSR, ``torch.sparse_csr_tensor`` (indices converted to int32) or
    (indptr, indices, values, shape) tuples on the device; C comes back in
    A's form."""
    A, kind = _as_csr(A)
    B, _ = _as_csr(B)
    dtype = dtype or (A.vals.dtype if A.vals is not None else torch.float64)
    plan = Plan(A, B, dtype=dtype, **opt_kw)
    rp, nnz = plan.symbolic()
    ci, v = plan.numeric(A.vals, B.vals)
    plan.close()
    return _as_kind(DeviceCSR(plan.nrows, B.ncols, rp, ci, v), kind)


def batched(pairs, dtype=torch.float64, **opt_kw):
    """C_i = A_i * B_i for every pair through one ``Batch`` (stacked
    launches, waves as needed); returns the list of C_i as DeviceCSR."""
    b = Batch([(_as_csr(a)[0], _as_csr(bb)[0]) for a, bb in pairs], dtype=dtype, **opt_kw)
    b.symbolic()
    b.numeric()
    return b.results()


def galerkin(P, A, dtype=torch.float64, **opt_kw):
    """The coarse operator P^T (A P) (``Galerkin``, one call); returned in
    A's form."""
    P_, _ = _as_csr(P)
    A_, kind = _as_csr(A)
    return _as_kind(Galerkin(P_, A_, dtype=dtype, **opt_kw).Ac, kind)


def spgemm_colwise(A: DeviceCSR, B: DeviceCSR, dtype=None, **opt_kw) -> DeviceCSR:
    """C = A*B by the column-wise Gustavson method (Sec. 2.2: the row-wise
    method with rows and columns switched, column j of C the sum of the
    columns A(:,k) scaled by B(k,j)): C^T = B^T A^T computed row by row on
    the transposes, then transposed back.  Same C as ``spgemm``; the sums
    run in B's column order instead of A's row order."""
    dtype = dtype or (A.vals.dtype if A.vals is not None else torch.float64)
    Ct = spgemm(transpose(B, dtype=dtype), transpose(A, dtype=dtype), dtype=dtype, **opt_kw)
    return transpose(Ct, dtype=dtype)


def omar(A: DeviceCSR, pes: int, stream=None) -> float:
    """Off-chip memory access reduction (Eq. 1) of the buffering scheme of
    Sec. 3 for ``pes`` computing units: rows are taken ``pes`` at a time and
    the group's nonzeros in one column (one CSV vector) share one read of
    that row of B.  The number of such vectors is nnz(G*A) for the 0/1
    matrix G that sums each group of rows, so the symbolic pass of this
    library counts them; OMAR(%) = 100 * (nnz(A) - nnz(G*A)) / nnz(A)."""
    if pes < 1:
        raise ValueError("pes must be at least 1")
    if A.nnz == 0:
        return 0.0
    dev = A.row_ptr.device
    groups = (A.nrows + pes - 1) // pes
    g_rp = torch.clamp(torch.arange(groups + 1, device=dev, dtype=torch.int64) * pes, max=A.nrows).to(torch.int32)
    g_ci = torch.arange(A.nrows, device=dev, dtype=torch.int32)
    G = DeviceCSR(groups, A.nrows, g_rp, g_ci, None)
    plan = Plan(G, A, stream=stream)
    _, vectors = plan.symbolic()
    plan.close()
    return 100.0 * (A.nnz - vectors) / A.nnz


_streams = {}
_staging = {}
_staging_lock = threading.Lock()


def release_staging():
    """Free the device staging buffers that spgemm_to_host keeps between calls."""
    with _staging_lock:
        _staging.clear()


def _stream_pool(dev, name, n):
    key = (dev.index, name)
    pool = _streams.get(key)
    if pool is None or len(pool) < n:
        pool = _streams[key] = [torch.cuda.Stream(device=dev) for _ in range(n)]
    return pool[:n]


def spgemm_to_host(A: DeviceCSR, B: DeviceCSR, dtype=torch.float64, chunks: int = 4, streams: int = 1, out=None,
                   order: str = "rows", trace=None, **opt_kw):
    """See _spgemm_to_host; calls on one process are serialised, since they
    share the device staging buffers (``release_staging`` frees them)."""
    with _staging_lock:
        return _spgemm_to_host(A, B, dtype, chunks, streams, out, order, trace, **opt_kw)


class _Trace:
    """Timeline of one spgemm_to_host call: host clock marks and CUDA events
    on the streams that did the work, read after the call's final sync."""

    def __init__(self, comp):
        self.t0 = time.perf_counter()
        self.start = torch.cuda.Event(enable_timing=True)
        self.start.record(comp)
        self.host = {}
        self.events = []  # (name, index, event)

    def mark(self, name):
        self.host[name] = round(1e3 * (time.perf_counter() - self.t0), 3)

    def event(self, name, idx, stream):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        self.events.append((name, idx, e))

    def result(self):
        dev = {}
        for name, idx, e in self.events:
            dev.setdefault(name, {})[idx] = round(self.start.elapsed_time(e), 3)
        return {"host_ms": self.host, "device_ms": {k: [v[i] for i in sorted(v)] for k, v in dev.items()}}


def _spgemm_to_host(A: DeviceCSR, B: DeviceCSR, dtype=torch.float64, chunks: int = 4, streams: int = 1, out=None,
                    order: str = "rows", trace=None, **opt_kw):
    """C = A*B with C delivered in pinned host memory.

    One plan over all rows analyses the product and sizes C (one symbolic
    pass).  Rows of C are independent (Sec. 2.2), so the numeric pass then
    runs in ``chunks`` row ranges of about equal output, each a plan sharing
    the whole plan's preprocessing of B (``spgemm_analyse_rows``) and sized
    from the whole row pointer (``spgemm_plan_adopt_row_ptr``), so it writes
    its rows in place; a copy stream brings each finished range to the host
    while later ranges compute on ``streams`` compute streams.  Only the first
    range's computation and the last range's copy are not hidden.
    ``order="products"`` computes the lightest range first, the second
    lightest last and the others heaviest first (``"rows"``: row order).
    ``out`` = (row_ptr, col_idx, vals) pinned CPU tensors to fill, reused when
    large enough.  Returns CPU tensors (row_ptr, col_idx, vals); blocks until
    they are complete.  ``trace``: a dict that receives the call's timeline
    (host milliseconds at each phase; per range, the device milliseconds at
    which its numeric pass and its copy started and ended)."""
    dev = A.row_ptr.device
    comp = torch.cuda.current_stream(dev)
    copy = _stream_pool(dev, "copy", 1)[0]
    work = _stream_pool(dev, "compute", max(1, int(streams)))
    tr = _Trace(comp) if trace is not None else None
    m = A.nrows
    base = Plan(A, B, dtype=dtype, **opt_kw)
    rp, total = base.symbolic()
    if tr:
        tr.mark("symbolic")
    if total >= 2**31:
        raise nat.SpgemmError("nnz(C) does not fit int32")
    if out is None or out[0].numel() < m + 1 or out[1].numel() < total or out[2].numel() < total:
        out = (torch.empty(m + 1, dtype=torch.int32).pin_memory(),
               torch.empty(max(total, 1), dtype=torch.int32).pin_memory(),
               torch.empty(max(total, 1), dtype=dtype).pin_memory())
    h_rp, h_ci, h_v = out
    # ranges of about equal output
    k = max(1, min(int(chunks), m))
    if k > 1:
        targets = (torch.arange(1, k, device=dev, dtype=torch.int64) * total // k).to(torch.int32)
        cuts = torch.searchsorted(rp, targets).cpu().tolist()
    else:
        cuts = []
    bounds = sorted(set([0, m] + [min(max(int(c), 0), m) for c in cuts]))
    offs = rp[torch.tensor(bounds, device=dev)].cpu().tolist()
    if tr:
        tr.mark("ranges")
    ranges = [(bounds[i], bounds[i + 1], offs[i], offs[i + 1] - offs[i]) for i in range(len(bounds) - 1)
              if bounds[i + 1] > bounds[i]]
    # device staging for C, kept between calls (repeated products of one
    # shape reuse it instead of allocating 12 bytes per entry each time)
    key = (dev.index, dtype)
    ci, v = _staging.get(key, (None, None))
    if ci is None or ci.numel() < max(total, 1):
        _staging.pop(key, None)
        ci = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        v = torch.empty(max(total, 1), dtype=dtype, device=dev)
        _staging[key] = (ci, v)
    a_vals = A.vals.to(dtype)
    b_vals = B.vals.to(dtype)
    ready = torch.cuda.Event()
    ready.record(comp)  # inputs, their values in dtype, B's run lists, C's row pointer
    copy.wait_event(ready)
    with torch.cuda.stream(copy):
        h_rp[:m + 1].copy_(rp, non_blocking=True)
    for s in work:
        s.wait_event(ready)
    plans = []
    for i, (rb, re, o, n) in enumerate(ranges):
        with torch.cuda.stream(work[i % len(work)]):  # the plan's workspace lives there
            pl = base.rows(rb, re)
            pl.adopt(rp[rb:re + 1], n)
            plans.append(pl)
    if order == "products" and len(plans) > 2:
        # the range computed first and the range copied last are not hidden:
        # make them the two lightest, heavy ranges in between
        prods = [pl.stats()[0] for pl in plans]
        by = sorted(range(len(plans)), key=lambda i: prods[i])
        seq = [by[0]] + sorted(by[2:], key=lambda i: -prods[i]) + [by[1]]
    else:
        seq = list(range(len(plans)))
    if tr:
        tr.mark("plans")
    for idx in seq:
        pl, (rb, re, o, n) = plans[idx], ranges[idx]
        ws = work[idx % len(work)]
        if tr:
            tr.event("numeric_start", idx, ws)
        with torch.cuda.stream(ws):
            pl.numeric(a_vals, b_vals, col_idx=ci, vals=v)
        done = torch.cuda.Event()
        done.record(ws)
        if tr:
            tr.event("numeric_end", idx, ws)
        copy.wait_event(done)
        if tr:
            tr.event("copy_start", idx, copy)
        if n:
            with torch.cuda.stream(copy):
                h_ci[o:o + n].copy_(ci[o:o + n], non_blocking=True)
                h_v[o:o + n].copy_(v[o:o + n], non_blocking=True)
        if tr:
            tr.event("copy_end", idx, copy)
    if tr:
        tr.mark("issued")
    rp.record_stream(copy)
    copy.synchronize()
    for s in work:  # the staging buffers are reused by the next call
        s.synchronize()
    for pl in plans:
        pl.close()
    base.close()
    if tr:
        tr.mark("done")
        trace.update(tr.result())
    return h_rp[:m + 1], h_ci[:total], h_v[:total]


_host_buffers = {}


def _host_array(x, np_dtype):
    """A contiguous host array of np_dtype for x (numpy array or CPU tensor;
    converted only when needed, pinned tensors pass through)."""
    if isinstance(x, torch.Tensor):
        assert x.device.type == "cpu"
        t = x if x.dtype == torch.from_numpy(np.zeros(0, np_dtype)).dtype else x.to(
            torch.from_numpy(np.zeros(0, np_dtype)).dtype)
        return t.contiguous()
    return np.ascontiguousarray(x, dtype=np_dtype)


def _host_struct(M, dtype):
    """(spgemm_csr of a host CSR, the arrays it points into, to keep alive)."""
    vt = np.float64 if dtype == torch.float64 else np.float32
    rp, ci, v = _host_array(M.row_ptr, np.int32), _host_array(M.col_idx, np.int32), _host_array(M.vals, vt)
    ptr = lambda a: a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data
    s = nat.spgemm_csr()
    s.nrows, s.ncols = int(M.nrows), int(M.ncols)
    s.nnz = int(rp[-1]) if int(M.nrows) > 0 else 0
    s.row_ptr = ptr(rp)
    s.col_idx = ptr(ci) if s.nnz else 0
    s.vals = ptr(v) if s.nnz else 0
    return s, (rp, ci, v)


def _device_buffer(dev, name, nbytes):
    key = (dev.index, name)
    buf = _host_buffers.get(key)
    if buf is None or buf.numel() < max(nbytes, 16):
        _host_buffers.pop(key, None)
        buf = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=dev)
        _host_buffers[key] = buf
    return buf


def spgemm_host(A, B=None, dtype=torch.float64, chunks: int = 4, out=None, trace=None, device=None, **opt_kw):
    """C = A*B from host memory to host memory through the C ABI's
    host-buffer product (``spgemm_host_product_begin`` / ``_finish``): the
    inputs are copied to the device, one symbolic pass sizes C, and the
    numeric pass runs in ``chunks`` row ranges cut by output (a small range
    of the last rows, computed first so the copies start early, then equal
    ones from the bottom up), each copied back while the next ones compute.  A, B: host CSR (``gen.CSR``
    or objects with nrows / ncols / row_ptr / col_idx / vals as numpy arrays
    or CPU tensors -- pinned memory for overlapped copies -- values already
    of ``dtype``); B defaults to A (copied once).  ``out`` = (row_ptr,
    col_idx, vals) pinned CPU tensors to fill, reused when large enough.
    ``trace``: a dict that receives host marks (ms after the call's start
    when begin -- copies in, analysis, symbolic pass -- and finish returned)
    and the per-range device timeline.  Returns
    CPU tensors (row_ptr, col_idx, vals).  Calls on one device share the
    device buffers, so they are serialised."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    with _staging_lock:
        sa, keep_a = _host_struct(A, dtype)
        sb, keep_b = (sa, keep_a) if B is None or B is A else _host_struct(B, dtype)
        opts = make_opts(dtype=dtype, **opt_kw)
        nbytes = nat.spgemm_host_product_workspace_size(sa, sb, opts)
        ws = _device_buffer(dev, "workspace", nbytes)
        stream = torch.cuda.current_stream(dev)
        copy = _stream_pool(dev, "copy", 1)[0]
        h, nnz = nat.spgemm_host_product_begin(sa, sb, opts, int(chunks), ws.data_ptr(), nbytes,
                                               int(stream.cuda_stream))
        t_begin = time.perf_counter()
        try:
            st_bytes = nat.spgemm_host_product_staging_size(h)
            stg = _device_buffer(dev, "staging", st_bytes)
            m = int(A.nrows)
            if out is None or out[0].numel() < m + 1 or out[1].numel() < nnz or out[2].numel() < nnz:
                out = (torch.empty(m + 1, dtype=torch.int32).pin_memory(),
                       torch.empty(max(nnz, 1), dtype=torch.int32).pin_memory(),
                       torch.empty(max(nnz, 1), dtype=dtype).pin_memory())
            h_rp, h_ci, h_v = out
            nat.spgemm_host_product_finish(h, h_rp.data_ptr(), h_ci.data_ptr(), h_v.data_ptr(), stg.data_ptr(),
                                           st_bytes, int(stream.cuda_stream), int(copy.cuda_stream))
            if trace is not None:
                nr = nat.spgemm_host_product_ranges(h)
                tl = nat.spgemm_host_product_timeline(h, 4 * nr)
                ms = lambda t: round((t - t0) * 1e3, 3)
                trace.update({"host_ms": {"begin_returned": ms(t_begin), "finish_returned": ms(time.perf_counter())},
                              "device_ms": {"numeric_start": tl[0::4], "numeric_end": tl[1::4],
                                            "copy_start": tl[2::4], "copy_end": tl[3::4]}})
        finally:
            nat.spgemm_host_product_destroy(h)
    return h_rp[:m + 1], h_ci[:nnz], h_v[:nnz]


def transpose(M: DeviceCSR, want_src: bool = False, dtype=None, stream=None):
    """M^T as a DeviceCSR (``spgemm_transpose``); with ``want_src`` also the
    int32 source positions (t_vals[q] = M.vals[src[q]])."""
    dev = M.row_ptr.device
    dtype = dtype or (M.vals.dtype if M.vals is not None else torch.float64)
    nbytes = nat.spgemm_transpose_workspace_size(M.nrows, M.ncols, M.nnz)
    ws = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=dev)
    t_rp = torch.empty(M.ncols + 1, dtype=torch.int32, device=dev)
    t_ci = torch.empty(M.nnz, dtype=torch.int32, device=dev)
    t_v = torch.empty(M.nnz, dtype=dtype, device=dev) if M.vals is not None else None
    src = torch.empty(M.nnz, dtype=torch.int32, device=dev) if want_src else None
    s = M.c_struct()
    nat.spgemm_transpose(s, _DT[dtype], t_rp.data_ptr(), t_ci.data_ptr() if M.nnz else 0,
                         t_v.data_ptr() if (t_v is not None and M.nnz) else 0,
                         src.data_ptr() if (src is not None and M.nnz) else 0,
                         ws.data_ptr(), nbytes, _stream_handle(stream))
    nat.spgemm_transpose_check(ws.data_ptr(), _stream_handle(stream))
    T = DeviceCSR(M.ncols, M.nrows, t_rp, t_ci, t_v)
    return (T, src) if want_src else T


def masked_spgemm(A: DeviceCSR, B: DeviceCSR, M: DeviceCSR, use_mask_values: bool = True, dtype=None,
                  stream=None) -> torch.Tensor:
    """C<M> = (A*B) .* M on M's pattern (``spgemm_masked``): a tensor of
    nnz(M) values aligned with M's col_idx, entry (i,j) holding
    M(i,j) * sum_k A(i,k) B(k,j) (0 where no product reaches it); without
    ``use_mask_values`` M is a pure pattern.  Asynchronous on ``stream``."""
    dtype = dtype or A.vals.dtype
    out = torch.empty(M.nnz, dtype=dtype, device=M.row_ptr.device)
    if use_mask_values and M.vals is not None and M.vals.dtype != dtype:
        raise TypeError("mask values must have the product's dtype")
    nat.spgemm_masked(A.c_struct(), B.c_struct(), M.c_struct(), _DT[dtype], bool(use_mask_values),
                      out.data_ptr() if M.nnz else 0, _stream_handle(stream))
    return out


SEMIRINGS = {"plus_times": nat.SPGEMM_PLUS_TIMES, "min_plus": nat.SPGEMM_MIN_PLUS, "max_plus": nat.SPGEMM_MAX_PLUS,
             "or_and": nat.SPGEMM_OR_AND}


def masked_semiring(A: DeviceCSR, B: DeviceCSR, M: DeviceCSR, semiring: str = "min_plus", dtype=None,
                    stream=None) -> torch.Tensor:
    """The masked product over a semiring on M's pattern
    (``spgemm_semiring``): nnz(M) values aligned with M's col_idx, entry
    (i,j) the semiring sum over k of product(A(i,k), B(k,j)) -- min of a + b
    ("min_plus", +inf where no product reaches), max of a + b ("max_plus",
    -inf), 1/0 for some product with both factors nonzero ("or_and"), or the
    ordinary sum of a * b ("plus_times").  M's values are not read."""
    dtype = dtype or A.vals.dtype
    out = torch.empty(M.nnz, dtype=dtype, device=M.row_ptr.device)
    nat.spgemm_semiring(A.c_struct(), B.c_struct(), M.c_struct(), _DT[dtype], SEMIRINGS[semiring],
                        out.data_ptr() if M.nnz else 0, _stream_handle(stream))
    return out


def spgemm_semiring(A: DeviceCSR, B: DeviceCSR, semiring: str = "min_plus", dtype=None, **opt_kw) -> DeviceCSR:
    """C = A (x) B over a semiring on the full pattern of A*B: one symbolic
    pass and one numeric pass whose accumulators use the semiring's sum and
    product (the plan option ``semiring``)."""
    dtype = dtype or A.vals.dtype
    plan = Plan(A, B, dtype=dtype, semiring=semiring, **opt_kw)
    rp, _ = plan.symbolic()
    ci, v = plan.numeric(A.vals, B.vals)
    plan.close()
    return DeviceCSR(plan.nrows, B.ncols, rp, ci, v)


def _plan_backward(self, a_vals, b_vals, dc_vals, need_a=True, need_b=True):
    """(dA, dB) for dC on this plan's C pattern (``spgemm_backward``)."""
    dev = self.workspace.device
    da = torch.empty(self.A.nnz, dtype=self.dtype, device=dev) if need_a else None
    db = torch.empty(self.B.nnz, dtype=self.dtype, device=dev) if need_b else None
    nat.spgemm_backward(self.handle, a_vals.data_ptr() if a_vals.numel() else 0,
                        b_vals.data_ptr() if b_vals.numel() else 0, self.row_ptr.data_ptr(),
                        self.col_idx.data_ptr() if self.nnz else 0,
                        dc_vals.data_ptr() if self.nnz else 0,
                        da.data_ptr() if (da is not None and da.numel()) else 0,
                        db.data_ptr() if (db is not None and db.numel()) else 0, self.stream)
    return da, db


Plan.backward = _plan_backward


class SparseMatmul:
    """Differentiable C = A*B for fixed patterns of A and B.

    ``op = SparseMatmul(A, B)`` analyses the product once (with the
    transpose of A's structure kept for the adjoint) and fixes C's pattern
    (``op.row_ptr``, ``op.col_idx``).  ``op(a_vals, b_vals)`` returns C's
    values and is differentiable in both arguments through
    :class:`SpGEMMFn`, whose backward is ``spgemm_backward``.
    """

    def __init__(self, A: DeviceCSR, B: DeviceCSR, dtype=torch.float64, **opt_kw):
        self.plan = Plan(A, B, dtype=dtype, backward=True, **opt_kw)
        self.row_ptr, self.nnz = self.plan.symbolic()
        dev = A.row_ptr.device
        # one numeric pass on zero values fixes C's column indices
        za = torch.zeros(A.nnz, dtype=dtype, device=dev)
        zb = torch.zeros(B.nnz, dtype=dtype, device=dev)
        self.col_idx, _ = self.plan.numeric(za, zb)
        self.dtype = dtype

    def __call__(self, a_vals, b_vals):
        return SpGEMMFn.apply(a_vals, b_vals, self)


class SpGEMMFn(torch.autograd.Function):
    """Values of C = A*B on the fixed pattern; backward gives
    dA = (dC B^T) on pattern(A) and dB = (A^T dC) on pattern(B)."""

    @staticmethod
    def forward(ctx, a_vals, b_vals, op):
        p = op.plan
        vals = torch.empty(op.nnz, dtype=op.dtype, device=a_vals.device)
        nat.spgemm_numeric(p.handle, a_vals.data_ptr() if a_vals.numel() else 0,
                           b_vals.data_ptr() if b_vals.numel() else 0, op.row_ptr.data_ptr(),
                           op.col_idx.data_ptr() if op.nnz else 0, vals.data_ptr() if op.nnz else 0, p.stream)
        ctx.save_for_backward(a_vals, b_vals)
        ctx.op = op
        return vals

    @staticmethod
    def backward(ctx, dc):
        a_vals, b_vals = ctx.saved_tensors
        op = ctx.op
        dc = dc.contiguous().to(op.dtype)
        da, db = op.plan.backward(a_vals, b_vals, dc, need_a=ctx.needs_input_grad[0],
                                  need_b=ctx.needs_input_grad[1])
        return da, db, None


class _Wave:
    """One ``spgemm_batched`` call: a run of consecutive instances stacked
    into one block-diagonal product with its own C."""

    def __init__(self, pairs, opts, dev, stream):
        self.pairs = pairs
        self.dtype = _DT_INV[opts.dtype]
        self._as = [a.c_struct() for a, _ in pairs]
        self._bs = [b.c_struct() for _, b in pairs]
        for s_, (a, b) in zip(self._as, pairs):
            s_.vals = a.vals.data_ptr() if a.nnz else 0
        for s_, (a, b) in zip(self._bs, pairs):
            s_.vals = b.vals.data_ptr() if b.nnz else 0
        nbytes = nat.spgemm_batch_workspace_size(self._as, self._bs, opts)
        self.workspace = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=dev)
        self.stream = stream
        self.handle = nat.spgemm_batched(self._as, self._bs, opts, self.workspace.data_ptr(), nbytes, stream)
        self.rows = nat.spgemm_batch_rows(self.handle)
        self.device = dev
        self.row_ptr = self.col_idx = self.vals = None
        self.nnz = None
        self.graph = None

    def symbolic(self):
        self.row_ptr = torch.empty(self.rows + 1, dtype=torch.int32, device=self.device)
        self.nnz = nat.spgemm_batch_symbolic(self.handle, len(self.pairs), self.row_ptr.data_ptr(), self.stream)
        total = self.nnz[-1]
        self.col_idx = torch.empty(total, dtype=torch.int32, device=self.device)
        self.vals = torch.empty(total, dtype=self.dtype, device=self.device)
        return self.nnz

    def numeric(self):
        nat.spgemm_batch_numeric(self.handle, self.row_ptr.data_ptr(),
                                 self.col_idx.data_ptr() if self.nnz[-1] else 0,
                                 self.vals.data_ptr() if self.nnz[-1] else 0, self.stream)

    def capture(self, stream):
        self.drop_graph()
        g = nat.spgemm_batch_capture(self.handle, self.row_ptr.data_ptr(),
                                     self.col_idx.data_ptr() if self.nnz[-1] else 0,
                                     self.vals.data_ptr() if self.nnz[-1] else 0, int(stream.cuda_stream))
        self.graph = (g, nat.spgemm_graph_instantiate(g))

    def drop_graph(self):
        if getattr(self, "graph", None):
            nat.spgemm_graph_destroy(*self.graph)
            self.graph = None

    def results(self):
        out, r0, e0 = [], 0, 0
        for (a, b), n in zip(self.pairs, self.nnz[:-1]):
            rp = self.row_ptr[r0:r0 + a.nrows + 1] - e0
            out.append(DeviceCSR(a.nrows, b.ncols, rp, self.col_idx[e0:e0 + n], self.vals[e0:e0 + n]))
            r0 += a.nrows
            e0 += n
        return out

    def close(self):
        self.drop_graph()
        if getattr(self, "handle", None):
            nat.spgemm_batch_destroy(self.handle)
            self.handle = None


class Batch:
    """Independent products C_i = A_i * B_i computed together
    (``spgemm_batched``): one analysis and one persistent launch per pass
    over all instances' rows.

    One stacked product must keep its counts (rows, nnz of A, B and C) inside
    int32, so the instances are cut into waves of consecutive instances
    (``spgemm_batch_products`` counts each instance's scalar products on the
    device, an upper bound of its nnz(C); ``spgemm_batch_waves`` cuts the list
    so that no wave holds more than ``max_products`` of them, 2^31 - 1 by
    default, and, with ``max_b_nnz``, no more B entries than that).  Each wave
    is one ``spgemm_batched`` call with its own stacked C; a batch that fits
    one wave is a single call.

    ``symbolic()`` sizes every C_i; ``numeric()`` fills the stacked C of every
    wave from the current values of every A_i / B_i (update ``A_i.vals`` in
    place for new values); ``results()`` returns per-instance DeviceCSR views.
    ``capture()`` records each wave's numeric pass in a CUDA graph
    (``spgemm_batch_capture``); ``replay()`` launches them in order.
    """

    def __init__(self, pairs, dtype=torch.float64, stream=None, max_products: int = 0, max_b_nnz: int = 0,
                 **opt_kw):
        self.pairs = list(pairs)
        self.dtype = dtype
        self.opts = make_opts(dtype=dtype, **opt_kw)
        dev = self.pairs[0][0].row_ptr.device if self.pairs else torch.device("cuda")
        self.device = dev
        self.stream = _stream_handle(stream)
        As = [a.c_struct() for a, _ in self.pairs]
        Bs = [b.c_struct() for _, b in self.pairs]
        n = len(self.pairs)
        self.products = [0] * n
        if n:
            wsb = nat.spgemm_batch_products_workspace_size(n)
            ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=dev)
            prod = torch.empty(n, dtype=torch.int64, device=dev)
            nat.spgemm_batch_products(As, Bs, prod.data_ptr(), ws.data_ptr(), wsb, self.stream)
            host = torch.empty(n, dtype=torch.int64, pin_memory=True)
            host.copy_(prod, non_blocking=True)
            (stream if stream is not None else torch.cuda.current_stream(dev)).synchronize()
            self.products = [int(x) for x in host.tolist()]
        self.wave_first = nat.spgemm_batch_waves(As, Bs, self.products, int(max_products), int(max_b_nnz))
        self.waves = [_Wave(self.pairs[a:b], self.opts, dev, self.stream)
                      for a, b in zip(self.wave_first[:-1], self.wave_first[1:])]
        self.rows = sum(w.rows for w in self.waves)
        self.nnz = None

    def symbolic(self):
        nnz = []
        for w in self.waves:
            nnz.extend(w.symbolic()[:-1])
        self.nnz = nnz + [sum(nnz)]
        return self.nnz

    def numeric(self):
        if self.nnz is None:
            self.symbolic()
        for w in self.waves:
            w.numeric()

    def capture(self):
        """Record each wave's numeric pass in a CUDA graph through
        ``spgemm_batch_capture`` (after symbolic()); ``replay()`` launches
        them on the current stream."""
        if self.nnz is None:
            self.symbolic()
        s = torch.cuda.Stream(device=self.device)
        for w in self.waves:
            w.capture(s)
        return [w.graph for w in self.waves]

    def replay(self, stream=None):
        h = _stream_handle(stream)
        for w in self.waves:
            nat.spgemm_graph_launch(w.graph[1], h)

    def results(self):
        out = []
        for w in self.waves:
            out.extend(w.results())
        return out

    def plan_handles(self):
        return [nat.spgemm_batch_plan(w.handle) for w in self.waves]

    def plan_handle(self):
        return self.plan_handles()[0]

    def close(self):
        for w in getattr(self, "waves", []):
            w.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Galerkin:
    """The Galerkin triple product A_c = P^T (A P) as a chain of two products.

    Construction transposes P (``spgemm_transpose``, values included),
    analyses A*P and R*(AP) with R = P^T, and runs both symbolic passes once
    (the structure of A and P must then stay fixed).  ``numeric()``
    recomputes A_c from the current values of A (P's values are those of
    construction); ``capture()`` records both numeric passes in one CUDA
    graph, ``replay()`` relaunches it.
    """

    def __init__(self, P: DeviceCSR, A: DeviceCSR, dtype=torch.float64, **opt_kw):
        self.P, self.A, self.dtype = P, A, dtype
        self.R, self.r_src = transpose(P, want_src=True, dtype=dtype)
        self.plan_ap = Plan(A, P, dtype=dtype, **opt_kw)
        self.ap_rp, ap_nnz = self.plan_ap.symbolic()
        self.ap_ci, self.ap_v = self.plan_ap.numeric(A.vals, P.vals)
        self.AP = DeviceCSR(A.nrows, P.ncols, self.ap_rp, self.ap_ci, self.ap_v)
        self.plan_c = Plan(self.R, self.AP, dtype=dtype, **opt_kw)
        self.c_rp, c_nnz = self.plan_c.symbolic()
        self.c_ci, self.c_v = self.plan_c.numeric(self.R.vals, self.ap_v)
        self.Ac = DeviceCSR(P.ncols, P.ncols, self.c_rp, self.c_ci, self.c_v)
        self.graph = None

    def numeric(self):
        self.plan_ap.numeric(self.A.vals, self.P.vals, col_idx=self.ap_ci, vals=self.ap_v)
        self.plan_c.numeric(self.R.vals, self.ap_v, col_idx=self.c_ci, vals=self.c_v)
        return self.Ac

    def capture(self):
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=self.A.row_ptr.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            saved = (self.plan_ap.stream, self.plan_c.stream)
            self.plan_ap.stream = self.plan_c.stream = int(s.cuda_stream)
            with torch.cuda.graph(g, stream=s):
                self.numeric()
            self.plan_ap.stream, self.plan_c.stream = saved
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.Ac
