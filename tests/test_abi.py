"""The C-ABI library loads without a GPU and exports every function that
include/spgemm.h declares; host-side argument checks need no device."""
import ctypes
import os
import re

import pytest

from paper_2112_10037_gb300 import build as bld
from paper_2112_10037_gb300 import _native as nat

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "spgemm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spgemm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return bld.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("spgemm_analyse", "spgemm_symbolic", "spgemm_numeric", "spgemm_workspace_size",
                 "spgemm_plan_destroy", "spgemm_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    # every declared entry point has a same-named Python binding
    names = declared_functions()
    assert not [n for n in names if not hasattr(nat, n)]


def test_host_checks_without_gpu(libpath):
    o = nat.spgemm_opts_default()
    assert o.dtype == nat.SPGEMM_F64 and o.row_end == -1 and o.force_path == -1
    A = nat.spgemm_csr()
    A.nrows, A.ncols, A.nnz = 10, 20, 0
    A.row_ptr = 16  # never dereferenced by the size query
    B = nat.spgemm_csr()
    B.nrows, B.ncols, B.nnz = 20, 5, 0
    B.row_ptr = 16
    n = nat.spgemm_workspace_size(A, B, o)
    assert n > 0
    o.row_begin, o.row_end = 5, 3
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_workspace_size(A, B, o)
    assert ei.value.status == 2
    o = nat.spgemm_opts_default()
    # dimension mismatch is caught on the host before any device work
    A.ncols = 19
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_analyse(A, B, o, 256, 1 << 20, 0)
    assert ei.value.status == 2
    A.ncols = 20
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_analyse(A, B, o, 0, 0, 0)
    assert ei.value.status == 5  # workspace missing
    assert nat.spgemm_version().count(".") == 2
    for s in range(10):
        assert nat.spgemm_status_string(s)


def test_masked_and_semiring_host_checks_without_gpu(libpath):
    """Argument checks of spgemm_masked / spgemm_semiring happen on the host
    before any device work: shape mismatch, unknown semiring or dtype, a
    missing output; an empty mask is a no-op."""
    def csr(m, n, nnz=0):
        s = nat.spgemm_csr()
        s.nrows, s.ncols, s.nnz = m, n, nnz
        s.row_ptr = 16  # never dereferenced on the host
        s.col_idx = 16 if nnz else 0
        s.vals = 16 if nnz else 0
        return s
    A, B = csr(5, 4), csr(4, 6)
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_masked(A, B, csr(5, 7), nat.SPGEMM_F64, True, 0, 0)
    assert ei.value.status == 2
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_semiring(A, B, csr(6, 6), nat.SPGEMM_F64, nat.SPGEMM_MIN_PLUS, 0, 0)
    assert ei.value.status == 2
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_semiring(A, B, csr(5, 6), nat.SPGEMM_F64, 9, 0, 0)
    assert ei.value.status == 1
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_semiring(A, B, csr(5, 6), 7, nat.SPGEMM_OR_AND, 0, 0)
    assert ei.value.status == 1
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_masked(A, B, csr(5, 6, 3), nat.SPGEMM_F64, False, 0, 0)  # output missing
    assert ei.value.status == 1
    nat.spgemm_masked(A, B, csr(5, 6), nat.SPGEMM_F64, False, 0, 0)      # empty mask: nothing to do
    nat.spgemm_semiring(A, B, csr(5, 6), nat.SPGEMM_F32, nat.SPGEMM_MAX_PLUS, 0, 0)


def test_graph_calls_host_checks_without_gpu(libpath):
    """spgemm_batch_capture and the graph helpers reject missing handles on
    the host, before any CUDA call."""
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_batch_capture(0, 16, 16, 16, 16)
    assert ei.value.status == 1
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_graph_instantiate(0)
    assert ei.value.status == 1
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_graph_launch(0, 0)
    assert ei.value.status == 1
    nat.spgemm_graph_destroy(0, 0)  # NULL handles: nothing to free


def _desc(m, k, nnz):
    s = nat.spgemm_csr()
    s.nrows, s.ncols, s.nnz = m, k, nnz
    s.row_ptr = 16  # sizes only: never dereferenced by the wave split
    s.col_idx = 16 if nnz else 0
    return s


def test_batch_waves_host_only(libpath):
    """spgemm_batch_waves cuts consecutive instances into waves whose
    product sums stay within the bound and whose stacked counts fit int32;
    an oversized instance stands alone; everything is host logic."""
    As = [_desc(10, 10, 30) for _ in range(7)]
    Bs = [_desc(10, 10, 30) for _ in range(7)]
    prod = [40, 50, 30, 100, 5, 5, 90]
    assert nat.spgemm_batch_waves(As, Bs, prod, 100) == [0, 2, 3, 4, 7]  # 5 + 5 + 90 = 100 fits
    assert nat.spgemm_batch_waves(As, Bs, prod, 1000) == [0, 7]
    assert nat.spgemm_batch_waves(As, Bs, prod, 0) == [0, 7]            # default bound 2^31 - 1
    assert nat.spgemm_batch_waves(As, Bs, [250] + prod[1:], 100)[:3] == [0, 1, 3]  # 250 alone
    assert nat.spgemm_batch_waves(As, Bs, prod, 0, 90) == [0, 3, 6, 7]  # 30 B entries each, at most 90 a wave
    assert nat.spgemm_batch_waves(As, Bs, prod, 100, 60)[:4] == [0, 2, 3, 4]  # both bounds
    assert nat.spgemm_batch_waves([], [], [], 0) == [0]
    # the default bound keeps every wave's product sum (an upper bound of its nnz(C)) inside int32
    big = [1 << 30, 1 << 30, 1 << 30, 5]
    w = nat.spgemm_batch_waves(As[:4], Bs[:4], big, 0)
    assert w == [0, 1, 2, 4]
    for a, b in zip(w[:-1], w[1:]):
        assert sum(big[a:b]) < (1 << 31) - 1 or b - a == 1
    # stacked rows would reach 2^31 - 1: a new wave starts
    huge = [_desc((1 << 30) + 5, 10, 0), _desc((1 << 30) + 5, 10, 0)]
    assert nat.spgemm_batch_waves(huge, [_desc(10, 10, 0)] * 2, [0, 0], 0) == [0, 1, 2]
    with pytest.raises(nat.SpgemmError) as ei:  # shapes are checked
        nat.spgemm_batch_waves([_desc(4, 5, 0)], [_desc(6, 3, 0)], [0], 0)
    assert ei.value.status == 2
    with pytest.raises(nat.SpgemmError) as ei:  # negative product count
        nat.spgemm_batch_waves(As[:1], Bs[:1], [-1], 0)
    assert ei.value.status == 1


def test_batch_products_host_checks_without_gpu(libpath):
    assert nat.spgemm_batch_products_workspace_size(3) >= 3 * 8
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_batch_products([_desc(4, 5, 0)], [_desc(5, 3, 0)], 256, 0, 0, 0)
    assert ei.value.status == 5  # workspace missing
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_batch_products([_desc(4, 5, 0)], [_desc(6, 3, 0)], 256, 256, 1 << 12, 0)
    assert ei.value.status == 2
    nat.spgemm_batch_products([], [], 0, 0, 0, 0)  # nothing to count


def test_host_product_host_checks_without_gpu(libpath):
    """The host-buffer product sizes its workspace on the host (one copy of
    the inputs when B is A) and rejects bad arguments before any copy."""
    o = nat.spgemm_opts_default()

    def csr(m, n, nnz, base):
        M = nat.spgemm_csr()
        M.nrows, M.ncols, M.nnz = m, n, nnz
        M.row_ptr, M.col_idx, M.vals = base, base + 4096, base + 8192  # never dereferenced here
        return M

    A = csr(1000, 1000, 50000, 1 << 20)
    B = csr(1000, 1000, 50000, 1 << 24)
    same = nat.spgemm_host_product_workspace_size(A, A, o)
    both = nat.spgemm_host_product_workspace_size(A, B, o)
    # B's arrays (row pointer, columns, FP64 values) are the difference
    assert both - same >= 4 * 1001 + 12 * 50000
    o32 = nat.spgemm_opts_default()
    o32.dtype = nat.SPGEMM_F32
    assert nat.spgemm_host_product_workspace_size(A, B, o32) < both
    bad = csr(999, 1000, 50000, 1 << 26)
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_host_product_workspace_size(A, bad, o)
    assert ei.value.status == 2  # A.ncols != B.nrows
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_host_product_begin(A, B, o, 0, 1 << 30, both, 0)
    assert ei.value.status == 1  # chunks < 1
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_host_product_begin(A, B, o, 4, 0, both, 0)
    assert ei.value.status == 5  # no workspace
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_host_product_begin(A, B, o, 4, 1 << 30, both - 1, 0)
    assert ei.value.status == 5  # workspace too small
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_host_product_begin(A, B, o, 4, (1 << 30) + 8, both, 0)
    assert ei.value.status == 5  # workspace not 16-byte aligned
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_host_product_staging_size(0)
    assert ei.value.status == 1
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_host_product_finish(0, 1 << 20, 1 << 21, 1 << 22, 1 << 23, 1 << 20, 0, 0)
    assert ei.value.status == 1
    nat.spgemm_host_product_destroy(0)


def test_semiring_option_host_checks_without_gpu(libpath):
    """The plan option `semiring` is checked on the host before any device
    work: an unknown semiring, or a semiring plan that also asks for the
    backward pass, is refused."""
    A = nat.spgemm_csr()
    A.nrows, A.ncols, A.nnz = 10, 20, 0
    A.row_ptr = 16
    B = nat.spgemm_csr()
    B.nrows, B.ncols, B.nnz = 20, 5, 0
    B.row_ptr = 16
    o = nat.spgemm_opts_default()
    assert o.semiring == nat.SPGEMM_PLUS_TIMES
    for bad in (-1, 4, 7):
        o.semiring = bad
        with pytest.raises(nat.SpgemmError) as ei:
            nat.spgemm_analyse(A, B, o, 256, 1 << 20, 0)
        assert ei.value.status == 1
    o.semiring = nat.SPGEMM_MIN_PLUS
    o.backward = 1
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_analyse(A, B, o, 256, 1 << 20, 0)
    assert ei.value.status == 1


def test_semiring_workspace_uses_the_plan_defaults(libpath):
    """A semiring plan runs at the default window sizes whatever the options
    say, so its workspace size ignores them as the plan does."""
    A = nat.spgemm_csr()
    A.nrows, A.ncols, A.nnz = 1000, 2000, 50000
    A.row_ptr, A.col_idx = 16, 16
    B = nat.spgemm_csr()
    B.nrows, B.ncols, B.nnz = 2000, 3000, 80000
    B.row_ptr, B.col_idx = 16, 16
    o = nat.spgemm_opts_default()
    o.semiring = nat.SPGEMM_MIN_PLUS
    plain = nat.spgemm_workspace_size(A, B, o)
    o.window_warp, o.window_block, o.block_warps, o.split_min, o.sort_max = 4096, 2048, 4, 4096, 512
    assert nat.spgemm_workspace_size(A, B, o) == plain
