"""GPU checks of two compositions of the CUDA path: the column-wise
Gustavson product (``api.spgemm_colwise``: transposes around a row-wise
product) against the oracle, and the OMAR statistic of Eq. 1
(``api.omar``: a symbolic pass of a grouping matrix times A) against the
oracle's vector-by-vector count."""
import numpy as np
import pytest

from paper_2112_10037_gb300 import gen
from parity import assert_structure_equal, assert_values_close, assert_values_exact, oracle_with_scale

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


def _colwise(api, A, B):
    C = api.spgemm_colwise(api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B))
    torch.cuda.synchronize()
    return C.to_host()


@pytest.mark.parametrize("shape,seed", [((300, 200, 500), 0), ((64, 900, 40), 1), ((1, 50, 1), 2)])
def test_colwise_integer_exact(api, oracle_mod, shape, seed):
    m, k, n = shape
    A = gen.random_csr(m, k, 0.05, seed, values="int", empty_rows=0.1)
    B = gen.random_csr(k, n, 0.05, seed + 7, values="int", empty_rows=0.1)
    C = _colwise(api, A, B)
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


def test_colwise_real_values_and_stencil(api, oracle_mod):
    A = gen.random_csr(400, 300, 0.04, 3)
    B = gen.random_csr(300, 350, 0.04, 4)
    C = _colwise(api, A, B)
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)
    L = gen.laplacian_3d(12)
    C = _colwise(api, L, L)
    R = oracle_mod.spgemm(L, L)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


@pytest.mark.parametrize("pes", [1, 2, 3, 4, 8, 16, 32])
def test_omar_matches_oracle(api, oracle_mod, pes):
    for A in (gen.random_csr(501, 300, 0.03, 5, empty_rows=0.1), gen.rmat(12, 16), gen.laplacian_2d(40)):
        got = api.omar(api.DeviceCSR.from_host(A), pes)
        assert got == oracle_mod.omar(A, pes)


def test_omar_closed_forms(api):
    # dense rows: every group of P rows shares all columns
    for m, n, pes in [(10, 7, 3), (12, 5, 4), (9, 1, 32)]:
        A = gen.from_dense(np.ones((m, n)))
        groups = -(-m // pes)
        assert api.omar(api.DeviceCSR.from_host(A), pes) == 100.0 * (m * n - groups * n) / (m * n)
    assert api.omar(api.DeviceCSR.from_host(gen.identity(50)), 8) == 0.0
