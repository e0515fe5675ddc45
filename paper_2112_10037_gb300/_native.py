"""ctypes binding of the C ABI in ``include/spgemm.h`` -- argument
marshalling only.  Every function here has the name of the C entry point it
calls; all computation runs in the CUDA library.

The library is loaded on first use.  If it has not been built, the call
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspgemm_gb300.so")

SPGEMM_F64 = 0
SPGEMM_F32 = 1

STATUS_NAMES = {
    0: "SPGEMM_OK", 1: "SPGEMM_ERR_INVALID_ARG", 2: "SPGEMM_ERR_DIM_MISMATCH",
    3: "SPGEMM_ERR_UNSORTED_INPUT", 4: "SPGEMM_ERR_INDEX_OVERFLOW", 5: "SPGEMM_ERR_WORKSPACE",
    6: "SPGEMM_ERR_TABLE_OVERFLOW", 7: "SPGEMM_ERR_CUDA", 8: "SPGEMM_ERR_INTERNAL",
    9: "SPGEMM_ERR_NOT_READY",
}


class SpgemmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(status, status),
                                          spgemm_status_string(status)))


class spgemm_csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p)]


class spgemm_opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("row_begin", ctypes.c_int64), ("row_end", ctypes.c_int64),
                ("warp_max", ctypes.c_int32), ("force_path", ctypes.c_int32),
                ("hash_max", ctypes.c_int32), ("window_warp", ctypes.c_int32),
                ("window_block", ctypes.c_int32), ("split_min", ctypes.c_int32),
                ("backward", ctypes.c_int32), ("num_block_min", ctypes.c_int32),
                ("block_warps", ctypes.c_int32), ("sort_max", ctypes.c_int32),
                ("rank_min", ctypes.c_int32), ("rank_accum", ctypes.c_int32),
                ("semiring", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_SIG = {
    "spgemm_opts_default": ([ctypes.POINTER(spgemm_opts)], None),
    "spgemm_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "spgemm_version": ([], ctypes.c_char_p),
    "spgemm_workspace_size": ([ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr),
                               ctypes.POINTER(spgemm_opts), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "spgemm_analyse": ([ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_opts),
                        _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "spgemm_rows_workspace_size": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "spgemm_analyse_rows": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t,
                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "spgemm_symbolic": ([_P, _P, _I64P, _P], ctypes.c_int),
    "spgemm_plan_adopt_row_ptr": ([_P, ctypes.c_int64, _P], ctypes.c_int),
    "spgemm_numeric": ([_P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "spgemm_plan_stats": ([_P, _P, _I64P, _I64P, _I64P], ctypes.c_int),
    "spgemm_plan_check": ([_P, _P], ctypes.c_int),
    "spgemm_plan_set_profiling": ([_P, ctypes.c_int], ctypes.c_int),
    "spgemm_plan_kernel_times": ([_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int], ctypes.c_int),
    "spgemm_plan_launches": ([_P, _I64P], ctypes.c_int),
    "spgemm_plan_destroy": ([_P], None),
    "spgemm_backward": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "spgemm_transpose_workspace_size": ([ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "spgemm_transpose": ([ctypes.POINTER(spgemm_csr), ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_size_t, _P],
                         ctypes.c_int),
    "spgemm_transpose_check": ([_P, _P], ctypes.c_int),
    "spgemm_transpose_noalloc": ([ctypes.POINTER(spgemm_csr), ctypes.c_int32, _P, _P, _P, _P, _P], ctypes.c_int),
    "spgemm_masked": ([ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr),
                       ctypes.c_int32, ctypes.c_int32, _P, _P], ctypes.c_int),
    "spgemm_semiring": ([ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr),
                         ctypes.c_int32, ctypes.c_int32, _P, _P], ctypes.c_int),
    "spgemm_batch_workspace_size": ([ctypes.c_int32, ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr),
                                     ctypes.POINTER(spgemm_opts), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "spgemm_batched": ([ctypes.c_int32, ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr),
                        ctypes.POINTER(spgemm_opts), _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "spgemm_batch_rows": ([_P, _I64P], ctypes.c_int),
    "spgemm_batch_symbolic": ([_P, _P, _I64P, _P], ctypes.c_int),
    "spgemm_batch_numeric": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "spgemm_batch_capture": ([_P, _P, _P, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "spgemm_graph_instantiate": ([_P, ctypes.POINTER(_P)], ctypes.c_int),
    "spgemm_graph_launch": ([_P, _P], ctypes.c_int),
    "spgemm_graph_destroy": ([_P, _P], None),
    "spgemm_batch_products_workspace_size": ([ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "spgemm_batch_products": ([ctypes.c_int32, ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr), _P, _P,
                               ctypes.c_size_t, _P], ctypes.c_int),
    "spgemm_batch_waves": ([ctypes.c_int32, ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr), _I64P,
                            ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_int32)],
                           ctypes.c_int),
    "spgemm_host_product_workspace_size": ([ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr),
                                            ctypes.POINTER(spgemm_opts), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "spgemm_host_product_begin": ([ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_csr), ctypes.POINTER(spgemm_opts),
                                   ctypes.c_int32, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P), _I64P], ctypes.c_int),
    "spgemm_host_product_staging_size": ([_P, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "spgemm_host_product_finish": ([_P, _P, _P, _P, _P, ctypes.c_size_t, _P, _P], ctypes.c_int),
    "spgemm_host_product_ranges": ([_P, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "spgemm_host_product_timeline": ([_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32], ctypes.c_int),
    "spgemm_host_product_destroy": ([_P], None),
    "spgemm_batch_plan": ([_P], _P),
    "spgemm_batch_destroy": ([_P], None),
}


def lib():
    """The loaded CUDA library; raises if it was not built."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError(
                        "CUDA library %s is missing: build it with "
                        "`python -m paper_2112_10037_gb300.build`" % LIB_PATH)
                handle = ctypes.CDLL(LIB_PATH)
                for name, (args, res) in _SIG.items():
                    fn = getattr(handle, name)
                    fn.argtypes = args
                    fn.restype = res
                _lib = handle
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise SpgemmError(status, where)


# ---------------------------------------------------------------- bindings
def spgemm_opts_default() -> spgemm_opts:
    o = spgemm_opts()
    lib().spgemm_opts_default(ctypes.byref(o))
    return o


def spgemm_status_string(status: int) -> str:
    return lib().spgemm_status_string(int(status)).decode()


def spgemm_version() -> str:
    return lib().spgemm_version().decode()


def spgemm_workspace_size(A: spgemm_csr, B: spgemm_csr, opts: spgemm_opts) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().spgemm_workspace_size(ctypes.byref(A), ctypes.byref(B), ctypes.byref(opts), ctypes.byref(n)),
           "spgemm_workspace_size")
    return n.value


def spgemm_analyse(A: spgemm_csr, B: spgemm_csr, opts: spgemm_opts, workspace: int, workspace_bytes: int,
                   stream: int) -> int:
    plan = _P(None)
    _check(lib().spgemm_analyse(ctypes.byref(A), ctypes.byref(B), ctypes.byref(opts), _P(workspace),
                                ctypes.c_size_t(workspace_bytes), _P(stream), ctypes.byref(plan)),
           "spgemm_analyse")
    return plan.value


def spgemm_rows_workspace_size(base: int, row_begin: int, row_end: int) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().spgemm_rows_workspace_size(_P(base), ctypes.c_int64(row_begin), ctypes.c_int64(row_end),
                                            ctypes.byref(n)), "spgemm_rows_workspace_size")
    return n.value


def spgemm_analyse_rows(base: int, row_begin: int, row_end: int, workspace: int, workspace_bytes: int,
                        stream: int) -> int:
    plan = _P(None)
    _check(lib().spgemm_analyse_rows(_P(base), ctypes.c_int64(row_begin), ctypes.c_int64(row_end), _P(workspace),
                                     ctypes.c_size_t(workspace_bytes), _P(stream), ctypes.byref(plan)),
           "spgemm_analyse_rows")
    return plan.value


def spgemm_plan_adopt_row_ptr(plan: int, nnz: int, stream: int) -> None:
    _check(lib().spgemm_plan_adopt_row_ptr(_P(plan), ctypes.c_int64(nnz), _P(stream)), "spgemm_plan_adopt_row_ptr")


def spgemm_symbolic(plan: int, c_row_ptr: int, stream: int) -> int:
    nnz = ctypes.c_int64(-1)
    _check(lib().spgemm_symbolic(_P(plan), _P(c_row_ptr), ctypes.byref(nnz), _P(stream)), "spgemm_symbolic")
    return nnz.value


def spgemm_numeric(plan: int, a_vals: int, b_vals: int, c_row_ptr: int, c_col_idx: int, c_vals: int,
                   stream: int) -> None:
    _check(lib().spgemm_numeric(_P(plan), _P(a_vals), _P(b_vals), _P(c_row_ptr), _P(c_col_idx), _P(c_vals),
                                _P(stream)), "spgemm_numeric")


def spgemm_plan_stats(plan: int, stream: int):
    tot, mx = ctypes.c_int64(0), ctypes.c_int64(0)
    rows = (ctypes.c_int64 * 4)()
    _check(lib().spgemm_plan_stats(_P(plan), _P(stream), ctypes.byref(tot), ctypes.byref(mx), rows),
           "spgemm_plan_stats")
    return tot.value, mx.value, list(rows)


def spgemm_plan_check(plan: int, stream: int) -> None:
    _check(lib().spgemm_plan_check(_P(plan), _P(stream)), "spgemm_plan_check")


SPGEMM_TIMER_COUNT = 11
TIMER_NAMES = ["analyse", "sym_tiny", "sym_hash", "sym_warp", "sym_block", "scan",
               "num_tiny", "num_hash", "num_warp", "num_block", "num_rank"]


def spgemm_plan_set_profiling(plan: int, on: bool) -> None:
    _check(lib().spgemm_plan_set_profiling(_P(plan), 1 if on else 0), "spgemm_plan_set_profiling")


def spgemm_plan_kernel_times(plan: int):
    ms = (ctypes.c_float * SPGEMM_TIMER_COUNT)()
    _check(lib().spgemm_plan_kernel_times(_P(plan), ms, SPGEMM_TIMER_COUNT), "spgemm_plan_kernel_times")
    return dict(zip(TIMER_NAMES, list(ms)))


def spgemm_plan_launches(plan: int) -> int:
    n = ctypes.c_int64(0)
    _check(lib().spgemm_plan_launches(_P(plan), ctypes.byref(n)), "spgemm_plan_launches")
    return n.value


def spgemm_plan_destroy(plan: int) -> None:
    if plan:
        lib().spgemm_plan_destroy(_P(plan))


def spgemm_backward(plan: int, a_vals: int, b_vals: int, c_row_ptr: int, c_col_idx: int, dc_vals: int,
                    da_vals: int, db_vals: int, stream: int) -> None:
    _check(lib().spgemm_backward(_P(plan), _P(a_vals), _P(b_vals), _P(c_row_ptr), _P(c_col_idx), _P(dc_vals),
                                 _P(da_vals), _P(db_vals), _P(stream)), "spgemm_backward")


def spgemm_transpose_workspace_size(nrows: int, ncols: int, nnz: int) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().spgemm_transpose_workspace_size(nrows, ncols, nnz, ctypes.byref(n)),
           "spgemm_transpose_workspace_size")
    return n.value


def spgemm_transpose(M: spgemm_csr, dtype: int, t_row_ptr: int, t_col_idx: int, t_vals: int, t_src: int,
                     workspace: int, workspace_bytes: int, stream: int) -> None:
    _check(lib().spgemm_transpose(ctypes.byref(M), dtype, _P(t_row_ptr), _P(t_col_idx), _P(t_vals), _P(t_src),
                                  _P(workspace), ctypes.c_size_t(workspace_bytes), _P(stream)), "spgemm_transpose")


def spgemm_transpose_check(workspace: int, stream: int) -> None:
    _check(lib().spgemm_transpose_check(_P(workspace), _P(stream)), "spgemm_transpose_check")


def spgemm_batch_workspace_size(As, Bs, opts: spgemm_opts) -> int:
    n = len(As)
    arrA, arrB = (spgemm_csr * max(n, 1))(*As), (spgemm_csr * max(n, 1))(*Bs)
    out = ctypes.c_size_t(0)
    _check(lib().spgemm_batch_workspace_size(n, arrA, arrB, ctypes.byref(opts), ctypes.byref(out)),
           "spgemm_batch_workspace_size")
    return out.value


def spgemm_batched(As, Bs, opts: spgemm_opts, workspace: int, workspace_bytes: int, stream: int) -> int:
    n = len(As)
    arrA, arrB = (spgemm_csr * max(n, 1))(*As), (spgemm_csr * max(n, 1))(*Bs)
    h = _P(None)
    _check(lib().spgemm_batched(n, arrA, arrB, ctypes.byref(opts), _P(workspace), ctypes.c_size_t(workspace_bytes),
                                _P(stream), ctypes.byref(h)), "spgemm_batched")
    return h.value


def spgemm_batch_rows(batch: int) -> int:
    r = ctypes.c_int64(0)
    _check(lib().spgemm_batch_rows(_P(batch), ctypes.byref(r)), "spgemm_batch_rows")
    return r.value


def spgemm_batch_symbolic(batch: int, n: int, c_row_ptr: int, stream: int):
    nnz = (ctypes.c_int64 * (n + 1))()
    _check(lib().spgemm_batch_symbolic(_P(batch), _P(c_row_ptr), nnz, _P(stream)), "spgemm_batch_symbolic")
    return list(nnz)


def spgemm_batch_numeric(batch: int, c_row_ptr: int, c_col_idx: int, c_vals: int, stream: int) -> None:
    _check(lib().spgemm_batch_numeric(_P(batch), _P(c_row_ptr), _P(c_col_idx), _P(c_vals), _P(stream)),
           "spgemm_batch_numeric")


def spgemm_batch_capture(batch: int, c_row_ptr: int, c_col_idx: int, c_vals: int, stream: int) -> int:
    """Handle of a new CUDA graph holding the batch numeric pass."""
    g = _P(None)
    _check(lib().spgemm_batch_capture(_P(batch), _P(c_row_ptr), _P(c_col_idx), _P(c_vals), _P(stream),
                                      ctypes.byref(g)), "spgemm_batch_capture")
    return g.value


def spgemm_graph_instantiate(graph: int) -> int:
    ge = _P(None)
    _check(lib().spgemm_graph_instantiate(_P(graph), ctypes.byref(ge)), "spgemm_graph_instantiate")
    return ge.value


def spgemm_graph_launch(exec_: int, stream: int) -> None:
    _check(lib().spgemm_graph_launch(_P(exec_), _P(stream)), "spgemm_graph_launch")


def spgemm_graph_destroy(graph: int, exec_: int) -> None:
    lib().spgemm_graph_destroy(_P(graph), _P(exec_))


def spgemm_batch_products_workspace_size(n: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().spgemm_batch_products_workspace_size(n, ctypes.byref(out)), "spgemm_batch_products_workspace_size")
    return out.value


def spgemm_batch_products(As, Bs, products: int, workspace: int, workspace_bytes: int, stream: int) -> None:
    n = len(As)
    arrA, arrB = (spgemm_csr * max(n, 1))(*As), (spgemm_csr * max(n, 1))(*Bs)
    _check(lib().spgemm_batch_products(n, arrA, arrB, _P(products), _P(workspace), ctypes.c_size_t(workspace_bytes),
                                       _P(stream)), "spgemm_batch_products")


def spgemm_batch_waves(As, Bs, products, max_products: int = 0, max_b_nnz: int = 0):
    """Wave boundaries [wave_first[w], wave_first[w+1]) of the instances."""
    n = len(As)
    arrA, arrB = (spgemm_csr * max(n, 1))(*As), (spgemm_csr * max(n, 1))(*Bs)
    prod = (ctypes.c_int64 * max(n, 1))(*[int(p) for p in products])
    first = (ctypes.c_int32 * (n + 1))()
    nw = ctypes.c_int32(0)
    _check(lib().spgemm_batch_waves(n, arrA, arrB, prod, ctypes.c_int64(max_products), ctypes.c_int64(max_b_nnz),
                                    first, ctypes.byref(nw)), "spgemm_batch_waves")
    return list(first)[:nw.value + 1]


def spgemm_batch_plan(batch: int) -> int:
    return lib().spgemm_batch_plan(_P(batch))


def spgemm_batch_destroy(batch: int) -> None:
    if batch:
        lib().spgemm_batch_destroy(_P(batch))


def spgemm_transpose_noalloc(M: spgemm_csr, dtype: int, t_row_ptr: int, t_col_idx: int, t_vals: int, t_src: int,
                             stream: int) -> None:
    _check(lib().spgemm_transpose_noalloc(ctypes.byref(M), dtype, _P(t_row_ptr), _P(t_col_idx), _P(t_vals),
                                          _P(t_src), _P(stream)), "spgemm_transpose_noalloc")


def spgemm_masked(A: spgemm_csr, B: spgemm_csr, M: spgemm_csr, dtype: int, use_mask_values: bool, c_vals: int,
                  stream: int) -> None:
    _check(lib().spgemm_masked(ctypes.byref(A), ctypes.byref(B), ctypes.byref(M), dtype,
                               1 if use_mask_values else 0, _P(c_vals), _P(stream)), "spgemm_masked")


SPGEMM_PLUS_TIMES, SPGEMM_MIN_PLUS, SPGEMM_MAX_PLUS, SPGEMM_OR_AND = 0, 1, 2, 3


def spgemm_semiring(A: spgemm_csr, B: spgemm_csr, M: spgemm_csr, dtype: int, semiring: int, c_vals: int,
                    stream: int) -> None:
    _check(lib().spgemm_semiring(ctypes.byref(A), ctypes.byref(B), ctypes.byref(M), dtype, semiring, _P(c_vals),
                                 _P(stream)), "spgemm_semiring")


def spgemm_host_product_workspace_size(A: spgemm_csr, B: spgemm_csr, opts: spgemm_opts) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().spgemm_host_product_workspace_size(ctypes.byref(A), ctypes.byref(B), ctypes.byref(opts),
                                                    ctypes.byref(n)), "spgemm_host_product_workspace_size")
    return n.value


def spgemm_host_product_begin(A: spgemm_csr, B: spgemm_csr, opts: spgemm_opts, chunks: int, workspace: int,
                              workspace_bytes: int, stream: int):
    """(handle, nnz(C))."""
    h = _P(None)
    nnz = ctypes.c_int64(-1)
    _check(lib().spgemm_host_product_begin(ctypes.byref(A), ctypes.byref(B), ctypes.byref(opts), int(chunks),
                                           _P(workspace), ctypes.c_size_t(workspace_bytes), _P(stream),
                                           ctypes.byref(h), ctypes.byref(nnz)), "spgemm_host_product_begin")
    return h.value, nnz.value


def spgemm_host_product_staging_size(product: int) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().spgemm_host_product_staging_size(_P(product), ctypes.byref(n)), "spgemm_host_product_staging_size")
    return n.value


def spgemm_host_product_finish(product: int, c_row_ptr: int, c_col_idx: int, c_vals: int, staging: int,
                               staging_bytes: int, stream: int, copy_stream: int) -> None:
    _check(lib().spgemm_host_product_finish(_P(product), _P(c_row_ptr), _P(c_col_idx), _P(c_vals), _P(staging),
                                            ctypes.c_size_t(staging_bytes), _P(stream), _P(copy_stream)),
           "spgemm_host_product_finish")


def spgemm_host_product_ranges(product: int) -> int:
    n = ctypes.c_int32(0)
    _check(lib().spgemm_host_product_ranges(_P(product), ctypes.byref(n)), "spgemm_host_product_ranges")
    return n.value


def spgemm_host_product_timeline(product: int, n: int):
    ms = (ctypes.c_float * max(n, 1))()
    _check(lib().spgemm_host_product_timeline(_P(product), ms, int(n)), "spgemm_host_product_timeline")
    return list(ms)[:n]


def spgemm_host_product_destroy(product: int) -> None:
    if product:
        lib().spgemm_host_product_destroy(_P(product))
