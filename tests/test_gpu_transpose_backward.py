"""GPU parity of the CSR transpose and of the SDDMM-style adjoint kernels
(dA = dC*B^T on pattern(A), dB = A^T*dC on pattern(B)) against the oracle,
plus FP64 finite differences of L = sum W*C through the autograd Function."""
import numpy as np
import pytest

from paper_2112_10037_gb300 import gen
from parity import RTOL_F32, assert_structure_equal, long_column_matrix, max_rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10037_gb300 import build
    build.build()
    from paper_2112_10037_gb300 import api as a
    return a


@pytest.mark.parametrize("shape,density,seed", [((50, 70), 0.1, 1), ((300, 200), 0.05, 2), ((1, 1), 1.0, 3),
                                                ((0, 5), 0.5, 4), ((7, 0), 0.5, 5)])
def test_transpose_vs_oracle(api, oracle_mod, shape, density, seed):
    M = gen.random_csr(shape[0], shape[1], density, seed)
    T, src = api.transpose(api.DeviceCSR.from_host(M), want_src=True)
    torch.cuda.synchronize()
    R = oracle_mod.transpose(M)
    got = T.to_host()
    assert_structure_equal(got, R)
    assert np.array_equal(got.vals, R.vals)
    assert np.array_equal(M.vals[src.cpu().numpy()], R.vals)


def test_transpose_long_columns(api, oracle_mod):
    """A 20,000-entry column (its row of M^T spans several tiles of the
    counting scatter) among short ones."""
    rng = np.random.default_rng(0)
    m = 20000
    counts = rng.integers(1, 6, size=m)
    M = gen.random_rows(m, 64, counts, rng)
    rp = M.row_ptr.astype(np.int64)
    # force column 0 into every row: a 20000-entry column of the transpose
    rows = []
    for i in range(m):
        c = M.col_idx[rp[i]:rp[i + 1]]
        rows.append(np.unique(np.concatenate([[0], c])))
    ci = np.concatenate(rows).astype(np.int32)
    new_rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    M = gen.CSR(m, 64, new_rp, ci, rng.standard_normal(len(ci)))
    T = api.transpose(api.DeviceCSR.from_host(M))
    R = oracle_mod.transpose(M)
    got = T.to_host()
    assert_structure_equal(got, R)
    assert np.array_equal(got.vals, R.vals)


def test_transpose_long_column_spanning_windows(api, oracle_mod):
    M = long_column_matrix()
    T, src = api.transpose(api.DeviceCSR.from_host(M), want_src=True)
    R = oracle_mod.transpose(M)
    got = T.to_host()
    assert_structure_equal(got, R)
    assert np.array_equal(got.vals, R.vals)
    assert np.array_equal(M.vals[src.cpu().numpy()], R.vals)
    assert int(np.diff(R.row_ptr)[0]) == 12_000


def test_transpose_repeated_and_unsorted_columns(api):
    """The transpose is a stable sort of M's entries by column, so it needs
    neither ascending nor unique columns within a row of M: a repeated column
    gives its source row twice, adjacent, and every row of M^T is ascending
    by source row.  Checked against numpy's stable argsort."""
    rng = np.random.default_rng(5)
    m, n = 9000, 700
    rows = [rng.integers(0, n, size=rng.integers(0, 9)) for _ in range(m)]  # unsorted, repeats allowed
    rows[17] = np.array([0, 0, 5, 0])
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    ci = np.concatenate(rows).astype(np.int32)
    v = rng.standard_normal(len(ci))
    M = gen.CSR(m, n, rp, ci, v)
    T, src = api.transpose(api.DeviceCSR.from_host(M), want_src=True)
    order = np.argsort(ci, kind="stable")
    row_of = np.repeat(np.arange(m, dtype=np.int32), np.diff(rp))
    got = T.to_host()
    assert np.array_equal(got.row_ptr, np.concatenate([[0], np.cumsum(np.bincount(ci, minlength=n))]))
    assert np.array_equal(got.col_idx, row_of[order])
    assert np.array_equal(src.cpu().numpy(), order)
    assert np.array_equal(got.vals, v[order])
    first0 = got.col_idx[got.row_ptr[0]:got.row_ptr[1]]
    assert int((first0 == 17).sum()) == 3


def test_transpose_column_out_of_range_is_reported(api):
    M = gen.CSR(3, 4, np.array([0, 1, 2, 3], np.int32), np.array([1, 4, 2], np.int32), np.ones(3))
    from paper_2112_10037_gb300 import _native as nat
    with pytest.raises(nat.SpgemmError) as ei:
        api.transpose(api.DeviceCSR.from_host(M))
    assert ei.value.status == 3


@pytest.mark.parametrize("ncols", [1, 512, 513, 65536, 262144, 262145, 3_000_000])
def test_transpose_digit_passes(api, oracle_mod, ncols):
    """One to three counting-scatter passes (at most 9 bits of the column
    index each: 1 pass up to 512 columns, 2 up to 262,144, 3 above), with
    more entries than one 4096-entry tile and a ragged last tile."""
    rng = np.random.default_rng(ncols)
    m = 5000
    counts = rng.integers(0, 12, size=m)
    counts[::97] = 0
    M = gen.random_rows(m, ncols, np.minimum(counts, ncols), rng)
    T, src = api.transpose(api.DeviceCSR.from_host(M), want_src=True)
    R = oracle_mod.transpose(M)
    got = T.to_host()
    assert_structure_equal(got, R)
    assert np.array_equal(got.vals, R.vals)
    assert np.array_equal(M.vals[src.cpu().numpy()], R.vals)


def _grad_oracle(oracle_mod, A, B, W):
    C = oracle_mod.spgemm(A, B)
    da, db = oracle_mod.backward(A, B, C.row_ptr, C.col_idx, W)
    return C, da, db


def _scale_sums(oracle_mod, A, B, C, W):
    """Per-output magnitude sums for the gradient tolerance: |dC|*|B|^T and
    |A|^T*|dC| on the patterns (oracle backward on absolute values)."""
    from parity import abs_csr
    da_s, db_s = oracle_mod.backward(abs_csr(A), abs_csr(B), C.row_ptr, C.col_idx, np.abs(W))
    return da_s, db_s


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("row_range", [None, (40, 170)])
def test_backward_vs_oracle(api, oracle_mod, seed, row_range):
    A = gen.random_csr(200, 150, 0.06, seed)
    B = gen.random_csr(150, 180, 0.06, seed + 9)
    dA, dB = api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B)
    kw = {} if row_range is None else {"row_range": row_range}
    plan = api.Plan(dA, dB, backward=True, **kw)
    rp, nnz = plan.symbolic()
    ci, v = plan.numeric(dA.vals, dB.vals)
    W = np.random.default_rng(seed + 3).standard_normal(nnz)
    da, db = plan.backward(dA.vals, dB.vals, torch.from_numpy(W).cuda())
    torch.cuda.synchronize()
    plan.check()
    Asub = A if row_range is None else oracle_mod.select_rows(A, np.arange(*row_range))
    C, rda, rdb = _grad_oracle(oracle_mod, Asub, B, W)
    sa, sb = _scale_sums(oracle_mod, Asub, B, C, W)
    got_da = da.cpu().numpy()
    if row_range is not None:
        lo, hi = A.row_ptr[row_range[0]], A.row_ptr[row_range[1]]
        got_da = got_da[lo:hi]
    assert max_rel_err(got_da, rda, sa) <= 1e-12
    assert max_rel_err(db.cpu().numpy(), rdb, sb) <= 1e-12
    plan.close()


@pytest.mark.parametrize("row_range", [None, (100, 9000)])
def test_backward_power_law_rmat14(api, oracle_mod, row_range):
    """Gradients of the R-MAT scale-14 product (hub rows of A and B with
    thousands of entries, so sums of many more than 128 terms are split over
    the warp and sums of a few terms stay in one lane) against the oracle's
    gradient; a second call gives the same bits (fixed summation order)."""
    A = gen.rmat(14, 16)
    rng = np.random.default_rng(14)
    A = gen.CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx, rng.standard_normal(A.nnz))
    dA = api.DeviceCSR.from_host(A)
    kw = {} if row_range is None else {"row_range": row_range}
    plan = api.Plan(dA, dA, backward=True, **kw)
    rp, nnz = plan.symbolic()
    plan.numeric(dA.vals, dA.vals)
    W = rng.standard_normal(nnz)
    dW = torch.from_numpy(W).cuda()
    da, db = plan.backward(dA.vals, dA.vals, dW)
    da2, db2 = plan.backward(dA.vals, dA.vals, dW)
    torch.cuda.synchronize()
    plan.check()
    lo, hi = (0, A.nnz) if row_range is None else (int(A.row_ptr[row_range[0]]), int(A.row_ptr[row_range[1]]))
    assert torch.equal(da[lo:hi], da2[lo:hi]) and torch.equal(db, db2)  # entries outside the range are not written
    Asub = A if row_range is None else oracle_mod.select_rows(A, np.arange(*row_range))
    C, rda, rdb = _grad_oracle(oracle_mod, Asub, A, W)
    sa, sb = _scale_sums(oracle_mod, Asub, A, C, W)
    got_da = da[lo:hi].cpu().numpy()
    assert max_rel_err(got_da, rda, sa) <= 1e-12
    assert max_rel_err(db.cpu().numpy(), rdb, sb) <= 1e-12
    lens = np.diff(A.row_ptr.astype(np.int64))
    assert lens.max() > 128 * 5  # the long-sum path is exercised on both gradients
    plan.close()


def test_autograd_finite_differences_fp64(api, oracle_mod):
    """L = sum W*C is bilinear: (L(a + h e_p) - L(a)) / h = dA[p] up to rounding."""
    A = gen.random_csr(60, 50, 0.1, 11)
    B = gen.random_csr(50, 70, 0.1, 12)
    dA, dB = api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B)
    op = api.SparseMatmul(dA, dB)
    W = torch.from_numpy(np.random.default_rng(2).standard_normal(op.nnz)).cuda()
    a = dA.vals.clone().requires_grad_(True)
    b = dB.vals.clone().requires_grad_(True)
    L = (op(a, b) * W).sum()
    L.backward()
    with torch.no_grad():
        L0 = float((op(a, b) * W).sum())
        h = 1e-3
        for p in range(0, A.nnz, max(1, A.nnz // 10)):
            a2 = a.detach().clone()
            a2[p] += h
            fd = (float((op(a2, b) * W).sum()) - L0) / h
            assert abs(fd - float(a.grad[p])) <= 1e-9 * (1 + abs(float(a.grad[p])))
        for q in range(0, B.nnz, max(1, B.nnz // 10)):
            b2 = b.detach().clone()
            b2[q] += h
            fd = (float((op(a, b2) * W).sum()) - L0) / h
            assert abs(fd - float(b.grad[q])) <= 1e-9 * (1 + abs(float(b.grad[q])))
    # and the oracle's gradient
    C, rda, rdb = _grad_oracle(oracle_mod, A, B, W.cpu().numpy())
    sa, sb = _scale_sums(oracle_mod, A, B, C, W.cpu().numpy())
    assert max_rel_err(a.grad.cpu().numpy(), rda, sa) <= 1e-12
    assert max_rel_err(b.grad.cpu().numpy(), rdb, sb) <= 1e-12


def test_backward_fp32_vs_fp64_oracle(api, oracle_mod):
    A = gen.random_csr(300, 256, 0.03, 21)
    B = gen.random_csr(256, 300, 0.03, 22)
    A32 = gen.CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx, A.vals.astype(np.float32).astype(np.float64))
    B32 = gen.CSR(B.nrows, B.ncols, B.row_ptr, B.col_idx, B.vals.astype(np.float32).astype(np.float64))
    dA = api.DeviceCSR.from_host(A32, dtype=torch.float32)
    dB = api.DeviceCSR.from_host(B32, dtype=torch.float32)
    op = api.SparseMatmul(dA, dB, dtype=torch.float32)
    W = np.random.default_rng(5).standard_normal(op.nnz).astype(np.float32).astype(np.float64)
    a = dA.vals.clone().requires_grad_(True)
    b = dB.vals.clone().requires_grad_(True)
    (op(a, b) * torch.from_numpy(W).float().cuda()).sum().backward()
    C, rda, rdb = _grad_oracle(oracle_mod, A32, B32, W)
    sa, sb = _scale_sums(oracle_mod, A32, B32, C, W)
    assert max_rel_err(a.grad.double().cpu().numpy(), rda, sa) <= RTOL_F32
    assert max_rel_err(b.grad.double().cpu().numpy(), rdb, sb) <= RTOL_F32


@pytest.mark.slow
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_backward_full_size_65536(api, oracle_mod, dtype):
    """The differentiation workload at full size (A, B 65536^2, 32 random
    columns per row, the bench's seeds): forward C and both gradients against
    the FP64 oracle."""
    n = 65536
    A = gen.random_rows(n, n, np.full(n, 32), np.random.default_rng(0))
    B = gen.random_rows(n, n, np.full(n, 32), np.random.default_rng(1))
    dA, dB = api.DeviceCSR.from_host(A, dtype=dtype), api.DeviceCSR.from_host(B, dtype=dtype)
    plan = api.Plan(dA, dB, dtype=dtype, backward=True)
    rp, nnz = plan.symbolic()
    ci, v = plan.numeric(dA.vals, dB.vals)
    W = np.random.default_rng(2).standard_normal(nnz)
    da, db = plan.backward(dA.vals, dB.vals, torch.from_numpy(W).to(device="cuda", dtype=dtype))
    torch.cuda.synchronize()
    plan.check()
    Wq = W.astype(np.float32).astype(np.float64) if dtype == torch.float32 else W
    Aq = A if dtype == torch.float64 else gen.CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx,
                                                  A.vals.astype(np.float32).astype(np.float64))
    Bq = B if dtype == torch.float64 else gen.CSR(B.nrows, B.ncols, B.row_ptr, B.col_idx,
                                                  B.vals.astype(np.float32).astype(np.float64))
    C, rda, rdb = _grad_oracle(oracle_mod, Aq, Bq, Wq)
    assert nnz == C.nnz
    assert np.array_equal(rp.cpu().numpy().astype(np.int64), C.row_ptr.astype(np.int64))
    assert np.array_equal(ci.cpu().numpy(), C.col_idx)
    sa, sb = _scale_sums(oracle_mod, Aq, Bq, C, Wq)
    tol = 1e-12 if dtype == torch.float64 else RTOL_F32
    from parity import abs_csr
    S = oracle_mod.spgemm(abs_csr(Aq), abs_csr(Bq))
    assert max_rel_err(v.double().cpu().numpy(), C.vals, S.vals) <= tol
    assert max_rel_err(da.double().cpu().numpy(), rda, sa) <= tol
    assert max_rel_err(db.double().cpu().numpy(), rdb, sb) <= tol
    plan.close()


def test_golden_worked_example_product_and_gradient(api):
    """The hand-worked example of tests/golden (Sec. 2.2 row-wise
    Gustavson): C and the gradient of the sum of C's entries through the
    CUDA path, bit for bit (every value there is exact)."""
    import os
    from parity import load_golden
    g = load_golden(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                 "gustavson_worked_example.txt"))
    A, B = g["A"], g["B"]
    dA, dB = api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B)
    plan = api.Plan(dA, dB, backward=True)
    rp, nnz = plan.symbolic()
    ci, v = plan.numeric(dA.vals, dB.vals)
    da, db = plan.backward(dA.vals, dB.vals, torch.ones(nnz, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    assert np.array_equal(rp.cpu().numpy().astype(np.int64), g["C"].row_ptr.astype(np.int64))
    assert np.array_equal(ci.cpu().numpy(), g["C"].col_idx)
    assert np.array_equal(v.cpu().numpy(), g["C"].vals)
    assert np.array_equal(da.cpu().numpy(), g["dA"].vals)
    assert np.array_equal(db.cpu().numpy(), g["dB"].vals)
