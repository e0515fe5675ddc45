"""GPU parity of the masked product C<M> = (A*B) .* M (``spgemm_masked``)
against the CPU oracle, through the C ABI: integer-valued inputs bit for
bit, real values within the sum-of-magnitudes criterion of parity.py,
triangle counts of graphs with known counts, mask rows longer than one
shared-memory slice, and the degenerate shapes."""
import numpy as np
import pytest

from paper_2112_10037_gb300 import gen
from parity import RTOL_F32, RTOL_F64, abs_csr, max_rel_err

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


def run(api, A, B, M, use_mask_values=True, dtype=torch.float64):
    dA = api.DeviceCSR.from_host(A, dtype=dtype)
    dB = api.DeviceCSR.from_host(B, dtype=dtype)
    dM = api.DeviceCSR.from_host(M, dtype=dtype)
    out = api.masked_spgemm(dA, dB, dM, use_mask_values=use_mask_values)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def scale(oracle_mod, A, B, M):
    """Per-entry magnitude sums |M(i,j)| * sum_k |A(i,k) B(k,j)|."""
    return oracle_mod.masked(abs_csr(A), abs_csr(B), abs_csr(M))


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("use_mask_values", [True, False])
def test_masked_integer_bit_exact(api, oracle_mod, seed, use_mask_values):
    A = gen.random_csr(300, 250, 0.05, seed, values="int", empty_rows=0.1)
    B = gen.random_csr(250, 400, 0.05, seed + 10, values="int", empty_rows=0.1)
    M = gen.random_csr(300, 400, 0.08, seed + 20, values="int", empty_rows=0.1)
    got = run(api, A, B, M, use_mask_values)
    ref = oracle_mod.masked(A, B, M, use_mask_values=use_mask_values)
    assert np.array_equal(got, ref)


def test_masked_real_values(api, oracle_mod):
    A = gen.random_csr(400, 300, 0.05, 5)
    B = gen.random_csr(300, 350, 0.05, 6)
    M = gen.random_csr(400, 350, 0.1, 7)
    got = run(api, A, B, M)
    ref = oracle_mod.masked(A, B, M)
    assert max_rel_err(got, ref, scale(oracle_mod, A, B, M)) <= RTOL_F64


def test_masked_fp32(api, oracle_mod):
    A = gen.random_csr(400, 300, 0.05, 8)
    B = gen.random_csr(300, 350, 0.05, 9)
    M = gen.random_csr(400, 350, 0.1, 10)
    got = run(api, A, B, M, dtype=torch.float32)
    ref = oracle_mod.masked(A, B, M)
    assert max_rel_err(got, ref, scale(oracle_mod, A, B, M)) <= RTOL_F32


def test_masked_long_mask_rows(api, oracle_mod):
    """Mask rows of up to 5000 columns (several 512-column slices, the last
    one ragged) next to short ones; A rows long enough for several chunks."""
    rng = np.random.default_rng(3)
    m, k, n = 40, 600, 6000
    M = gen.random_rows(m, n, np.concatenate([[5000, 512, 513, 1024, 1535], rng.integers(0, 300, m - 5)]), rng,
                        values="int")
    A = gen.random_rows(m, k, rng.integers(0, 100, m), rng, values="int")
    B = gen.random_rows(k, n, rng.integers(0, 200, k), rng, values="int")
    got = run(api, A, B, M)
    assert np.array_equal(got, oracle_mod.masked(A, B, M))


def _undirected(n, edges):
    d = np.zeros((n, n))
    for a, b in edges:
        d[a, b] = d[b, a] = 1.0
    return gen.lower_triangle_undirected(gen.from_dense(d))


@pytest.mark.parametrize("n,edges,triangles", [
    (40, [(a, b) for a in range(40) for b in range(a)], 9880),                          # K40: C(40,3)
    (31, [(a, (a + 1) % 30) for a in range(30)] + [(30, a) for a in range(30)], 30),   # wheel, 30-cycle rim
    (50, [(a, (a + 1) % 50) for a in range(50)], 0),                                    # cycle
])
def test_masked_triangle_counts(api, n, edges, triangles):
    L = _undirected(n, edges)
    assert float(run(api, L, L, L).sum()) == triangles


def test_masked_triangles_rmat_scale12(api, oracle_mod):
    """Triangle counting on an undirected R-MAT graph (scale 12): every
    entry of (L*L) .* L exact against the oracle."""
    L = gen.lower_triangle_undirected(gen.rmat(12, 16))
    got = run(api, L, L, L)
    ref = oracle_mod.masked(L, L, L)
    assert np.array_equal(got, ref)
    assert ref.sum() > 0


def test_masked_degenerate(api, oracle_mod):
    for (m, k, n) in [(0, 5, 7), (5, 0, 7), (5, 7, 0), (1, 1, 1), (6, 4, 5)]:
        A = gen.random_csr(m, k, 0.5, 1, values="int")
        B = gen.random_csr(k, n, 0.5, 2, values="int")
        M = gen.random_csr(m, n, 0.5, 3, values="int")
        got = run(api, A, B, M)
        assert np.array_equal(got, oracle_mod.masked(A, B, M))
    # a mask with entries but A*B empty: all zeros
    A = gen.CSR(3, 4, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = gen.random_csr(4, 5, 0.5, 4)
    M = gen.random_csr(3, 5, 0.6, 5)
    assert np.array_equal(run(api, A, B, M), np.zeros(M.nnz))


def test_masked_rejects_bad_shapes(api):
    from paper_2112_10037_gb300 import _native as nat
    A = api.DeviceCSR.from_host(gen.random_csr(5, 4, 0.5, 1))
    B = api.DeviceCSR.from_host(gen.random_csr(4, 6, 0.5, 2))
    M = api.DeviceCSR.from_host(gen.random_csr(5, 7, 0.5, 3))
    with pytest.raises(nat.SpgemmError) as ei:
        api.masked_spgemm(A, B, M)
    assert ei.value.status == 2
