"""The benchmark workload at full size, in the launch configuration bench.py
times (R-MAT scale 18, edge factor 16, C = A*A, FP64, default options):
C's row pointer against the oracle's for every row (exact), every entry of C
against the oracle (range by range over host processes), the product
counts; the 3D stencil product at 96^3 entry by entry against the oracle and
its closed form."""
import numpy as np
import pytest
import torch

from paper_2112_10037_gb300 import gen
import fullcmp
from parity import RTOL_F64, stencil3d_square_closed_form

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10037_gb300 import build
    build.build()
    from paper_2112_10037_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def full(api):
    A = gen.rmat(18, 16)
    dA = api.DeviceCSR.from_host(A)
    plan = api.Plan(dA, dA)
    rp, nnz = plan.symbolic()
    ci, v = plan.numeric(dA.vals, dA.vals)
    torch.cuda.synchronize()
    plan.check()
    stats = plan.stats()
    plan.close()
    return A, rp, ci, v, nnz, stats


def test_fullsize_row_pointer_exact(full, oracle_mod):
    A, rp, _, _, nnz, _ = full
    ref = oracle_mod.spgemm_rowptr(A, A)
    assert nnz == int(ref[-1])
    np.testing.assert_array_equal(rp.cpu().numpy().astype(np.int64), ref)


def test_fullsize_product_counts(full, oracle_mod):
    A, _, _, _, _, stats = full
    prod = oracle_mod.row_products(A, A)
    total, largest, per_path = stats
    assert total == int(prod.sum())
    assert largest == int(prod.max())
    assert sum(per_path) == int((prod > 0).sum())


def _device_to_store(rp, ci, v):
    """The device's C copied into memory-mapped host files for the compare
    workers."""
    nnz = int(ci.numel())
    st = fullcmp.Store(12 * nnz + 8 * rp.numel())
    st.put("c_rp", rp.cpu().numpy().astype(np.int64))
    step = 1 << 27
    h_ci = st.empty("c_ci", (nnz,), np.int32)
    h_v = st.empty("c_v", (nnz,), np.float64)
    t_ci, t_v = torch.from_numpy(h_ci), torch.from_numpy(h_v)
    for off in range(0, nnz, step):
        n = min(step, nnz - off)
        t_ci[off:off + n].copy_(ci[off:off + n])
        t_v[off:off + n].copy_(v[off:off + n])
    return st


def test_fullsize_every_entry(full, oracle_mod):
    """Every row of C against the oracle: row sizes and all 1.28e9 column
    indices exact, every value within 1e-12 relative (R-MAT's values are
    positive, so each sum's terms share one sign and the bound is the plain
    relative error).  The oracle runs as independent single-threaded calls
    on row ranges, one host process per core."""
    A, rp, ci, v, nnz, _ = full
    prod = oracle_mod.row_products(A, A)
    st = _device_to_store(rp, ci, v)
    try:
        res = fullcmp.compare_product(A, A, st, prod, rtol=RTOL_F64)
    finally:
        st.close()
    ok, err, entries, msg = fullcmp.summarise(res)
    print("R-MAT 18 A*A: %d entries compared, max relative error %.3e" % (entries, err))
    assert entries == nnz
    assert ok, msg


def test_fullsize_stencil3d_96_square(api, oracle_mod):
    """The 3D stencil product A*A at 96^3 (the supplementary roofline
    workload, every row on the hash path) in bench.py's configuration: all
    21,732,480 entries bit-exact against the oracle and against the closed
    form (integer values, so every partial sum is exact)."""
    n = 96
    A = gen.laplacian_3d(n)
    dA = api.DeviceCSR.from_host(A)
    plan = api.Plan(dA, dA)
    rp, nnz = plan.symbolic()
    ci, v = plan.numeric(dA.vals, dA.vals)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    assert nnz == 21_732_480
    R = oracle_mod.spgemm(A, A)
    h_rp = rp.cpu().numpy().astype(np.int64)
    h_ci, h_v = ci.cpu().numpy(), v.cpu().numpy()
    np.testing.assert_array_equal(h_rp, R.row_ptr)
    np.testing.assert_array_equal(h_ci, R.col_idx)
    assert np.array_equal(h_v, R.vals)
    exp = stencil3d_square_closed_form(n, h_rp, h_ci)
    assert not np.isnan(exp).any(), "an entry at an offset the closed form does not allow"
    assert np.array_equal(h_v, exp)


def test_fullsize_triangle_counting_exact(api, oracle_mod):
    """The triangle-counting workload of bench.py at full size (masked
    product (L*L) .* L on the undirected R-MAT scale-18 graph's lower
    triangle): every one of the nnz(L) outputs exact against the oracle
    (integer sums), and the same triangle count."""
    L = gen.lower_triangle_undirected(gen.rmat(18, 16))
    dL = api.DeviceCSR.from_host(L)
    got = api.masked_spgemm(dL, dL, dL, use_mask_values=False).cpu().numpy()
    ref = oracle_mod.masked(L, L, L, use_mask_values=False)
    assert np.array_equal(got, ref)
    assert int(ref.sum()) > 0


def test_fullsize_omar(full, api, oracle_mod):
    """OMAR (Eq. 1) of the benchmark matrix at 2..32 computing units against
    the oracle's vector-by-vector count."""
    A = full[0]
    dA = api.DeviceCSR.from_host(A)
    for pes in (2, 4, 8, 16, 32):
        assert api.omar(dA, pes) == oracle_mod.omar(A, pes)
