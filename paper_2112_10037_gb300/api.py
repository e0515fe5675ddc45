"""Torch-facing helpers over the C ABI: device CSR containers, plans, and the
one-call product.  PyTorch supplies device memory (its caching allocator)
and the current CUDA stream; every step of the product runs in the CUDA
library through ``_native``.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _native as nat

_DT = {torch.float64: nat.SPGEMM_F64, torch.float32: nat.SPGEMM_F32}


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
              window_warp=0, window_block=0, split_min=0) -> nat.spgemm_opts:
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
        self.nnz: Optional[int] = None

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
        nat.spgemm_numeric(self.handle, a_vals.data_ptr() if a_vals.numel() else 0,
                           b_vals.data_ptr() if b_vals.numel() else 0, self.row_ptr.data_ptr(),
                           col_idx.data_ptr() if self.nnz else 0, vals.data_ptr() if self.nnz else 0,
                           self.stream)
        return col_idx, vals

    def stats(self):
        """(total products, largest row's products, rows per path
        [register-sort, hash, warp, block])."""
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


def spgemm(A: DeviceCSR, B: DeviceCSR, dtype=None, **opt_kw) -> DeviceCSR:
    """C = A*B on the device (analyse, symbolic, numeric)."""
    dtype = dtype or (A.vals.dtype if A.vals is not None else torch.float64)
    plan = Plan(A, B, dtype=dtype, **opt_kw)
    rp, nnz = plan.symbolic()
    ci, v = plan.numeric(A.vals, B.vals)
    plan.close()
    return DeviceCSR(plan.nrows, B.ncols, rp, ci, v)
