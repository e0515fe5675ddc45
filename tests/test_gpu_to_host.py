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
