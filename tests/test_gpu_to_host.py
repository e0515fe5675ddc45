"""Row-range plans sharing one preprocessing of B, and the pipelined
product into host memory, against the oracle."""
import numpy as np
import pytest
import torch

from paper_2112_10037_gb300 import gen
from parity import (abs_csr, assert_structure_equal, assert_values_close, assert_values_exact,
                    oracle_with_scale)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10037_gb300 import build
    build.build()
    from paper_2112_10037_gb300 import api as a
    return a


def _host_csr(nrows, ncols, rp, ci, v):
    return gen.CSR(nrows, ncols, np.asarray(rp), np.asarray(ci), np.asarray(v, dtype=np.float64))


@pytest.mark.parametrize("chunks", [1, 3, 8, 64])
def test_to_host_rmat_matches_oracle(api, oracle_mod, chunks):
    A = gen.rmat(11, 8)
    dA = api.DeviceCSR.from_host(A)
    rp, ci, v = api.spgemm_to_host(dA, dA, chunks=chunks)
    C = _host_csr(A.nrows, A.ncols, rp.numpy(), ci.numpy(), v.numpy())
    R, S = oracle_with_scale(oracle_mod, A, A)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)


def test_to_host_integer_exact_and_reused_output(api, oracle_mod):
    A = gen.laplacian_2d(40)
    B = gen.laplacian_2d(40)
    dA, dB = api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B)
    out = None
    for chunks in (5, 2):  # the second call reuses the first call's pinned buffers
        rp, ci, v = api.spgemm_to_host(dA, dB, chunks=chunks, out=out)
        out = (rp, ci, v) if out is None else out
        C = _host_csr(A.nrows, B.ncols, rp.numpy(), ci.numpy(), v.numpy())
        R = oracle_mod.spgemm(A, B)
        assert_structure_equal(C, R)
        assert_values_exact(C.vals, R.vals)


def test_to_host_empty_rows_and_rectangular(api, oracle_mod):
    rng = np.random.default_rng(7)
    counts = rng.integers(0, 6, size=300)
    counts[::7] = 0
    A = gen.random_rows(300, 120, counts, rng, values="int")
    B = gen.random_rows(120, 5000, rng.integers(0, 40, size=120), rng, values="int")
    dA, dB = api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B)
    rp, ci, v = api.spgemm_to_host(dA, dB, chunks=7)
    C = _host_csr(A.nrows, B.ncols, rp.numpy(), ci.numpy(), v.numpy())
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


def test_row_plans_share_b(api, oracle_mod):
    """Each row range of a product from plans derived from one base plan."""
    A = gen.rmat(10, 8)
    dA = api.DeviceCSR.from_host(A)
    base = api.Plan(dA, dA, row_range=(0, 0))
    R = oracle_mod.spgemm(A, A)
    S = oracle_mod.spgemm(abs_csr(A), abs_csr(A))
    for rb, re in [(0, 100), (100, 101), (500, 1024), (1024, 1024)]:
        pl = base.rows(rb, re)
        rp, nnz = pl.symbolic()
        ci, v = pl.numeric(dA.vals, dA.vals)
        torch.cuda.synchronize()
        pl.check()
        rows = np.arange(rb, re)
        sub, ssub = oracle_mod.select_rows(R, rows), oracle_mod.select_rows(S, rows)
        C = _host_csr(re - rb, A.ncols, rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy())
        assert_structure_equal(C, sub)
        assert_values_close(C.vals, sub.vals, ssub.vals)
        pl.close()
    base.close()


def test_adopt_refuses_split_rows(api):
    """Split rows take their per-window offsets from the symbolic pass, so a
    plan with split rows cannot be sized from a row pointer alone."""
    from paper_2112_10037_gb300 import _native as nat
    A = gen.rmat(11, 8)
    dA = api.DeviceCSR.from_host(A)
    base = api.Plan(dA, dA, split_min=128, num_block_min=-1)
    rp, nnz = base.symbolic()
    pl = base.rows(0, A.nrows)
    with pytest.raises(nat.SpgemmError):
        pl.adopt(rp, nnz)
    pl.close()
    base.close()


@pytest.mark.parametrize("chunks", [1, 4, 33])
def test_host_product_rmat_aliased(api, oracle_mod, chunks):
    """Host CSR in, host CSR out through spgemm_host_product_begin/finish,
    B aliased to A (one copy), against the oracle; the device timeline has
    one numeric and one copy interval per row range, computed and copied
    from the last range to the first."""
    A = gen.rmat(12, 8)
    tr = {}
    rp, ci, v = api.spgemm_host(A, chunks=chunks, trace=tr)
    C = _host_csr(A.nrows, A.ncols, rp.numpy(), ci.numpy(), v.numpy())
    R, S = oracle_with_scale(oracle_mod, A, A)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)
    d = tr["device_ms"]
    nr = len(d["numeric_start"])
    assert 1 <= nr <= chunks
    for r in range(nr):
        assert d["numeric_start"][r] <= d["numeric_end"][r] <= d["copy_start"][r] + 1e-3
        assert d["copy_start"][r] <= d["copy_end"][r]
        if r + 1 < nr:  # ranges are computed from the last to the first
            assert d["numeric_start"][r] >= d["numeric_end"][r + 1] - 1e-3
            assert d["copy_start"][r] >= d["copy_end"][r + 1] - 1e-3


def test_host_product_rectangular_pinned_reused(api, oracle_mod):
    """Distinct A and B (rectangular, empty rows, integer values: exact) from
    pinned host tensors; a second call fills the first call's output."""
    rng = np.random.default_rng(11)
    counts = rng.integers(0, 9, size=700)
    counts[::5] = 0
    A = gen.random_rows(700, 300, counts, rng, values="int")
    B = gen.random_rows(300, 9000, rng.integers(0, 60, size=300), rng, values="int")
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    HA = gen.CSR(A.nrows, A.ncols, pin(A.row_ptr), pin(A.col_idx), pin(A.vals))
    HB = gen.CSR(B.nrows, B.ncols, pin(B.row_ptr), pin(B.col_idx), pin(B.vals))
    R = oracle_mod.spgemm(A, B)
    out = None
    for chunks in (6, 2):
        rp, ci, v = api.spgemm_host(HA, HB, chunks=chunks, out=out)
        if out is None:
            out = (rp, ci, v)
        else:
            assert ci.data_ptr() == out[1].data_ptr()
        C = _host_csr(A.nrows, B.ncols, rp.numpy(), ci.numpy(), v.numpy())
        assert_structure_equal(C, R)
        assert_values_exact(C.vals, R.vals)


def test_host_product_fp32_and_empty(api, oracle_mod):
    """FP32 values (the oracle's FP64 result rounded, within FP32 error), and
    an empty product."""
    A = gen.laplacian_2d(30)
    A32 = gen.CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx, A.vals.astype(np.float32))
    rp, ci, v = api.spgemm_host(A32, dtype=torch.float32, chunks=3)
    R = oracle_mod.spgemm(A, A)
    C = _host_csr(A.nrows, A.ncols, rp.numpy(), ci.numpy(), v.numpy())
    assert_structure_equal(C, R)
    np.testing.assert_allclose(C.vals, R.vals, rtol=1e-6, atol=1e-6)
    E = gen.CSR(50, 40, np.zeros(51, np.int32), np.zeros(0, np.int32), np.zeros(0))
    F = gen.CSR(40, 30, np.zeros(41, np.int32), np.zeros(0, np.int32), np.zeros(0))
    rp, ci, v = api.spgemm_host(E, F, chunks=4)
    assert rp.numel() == 51 and int(rp.abs().sum()) == 0 and ci.numel() == 0 and v.numel() == 0


@pytest.mark.parametrize("semiring", ["min_plus", "or_and"])
def test_host_product_semiring(api, oracle_mod, semiring):
    """The host-buffer product with the plan option `semiring`: C's pattern
    from the symbolic pass, its values over the semiring, exact against the
    oracle's semiring values on that pattern."""
    A = gen.rmat(11, 8)
    rp, ci, v = api.spgemm_host(A, chunks=3, semiring=semiring)
    R = oracle_mod.spgemm(A, A)
    assert np.array_equal(rp.numpy(), R.row_ptr) and np.array_equal(ci.numpy(), R.col_idx)
    assert np.array_equal(v.numpy(), oracle_mod.masked_semiring(A, A, R, semiring))
