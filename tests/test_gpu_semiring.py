"""GPU parity of the semiring products against the CPU oracle, through the
C ABI: the masked product (``spgemm_semiring``: min-plus, max-plus, or-and)
and the full product whose numeric pass accumulates over the semiring (the
plan option ``semiring``).
Min and max do not depend on the order of the sums, so every value is
compared bit for bit; FP32 results equal the oracle's FP64 result rounded to
FP32 (rounding is monotone, and the sums of FP32 inputs are exact in FP64).
All-pairs shortest paths by repeated min-plus squaring are checked against
scipy's Dijkstra."""
import numpy as np
import pytest

from paper_2112_10037_gb300 import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEMIRINGS = ["min_plus", "max_plus", "or_and"]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10037_gb300 import build
    build.build()
    from paper_2112_10037_gb300 import api as a
    return a


def run(api, A, B, M, semiring, dtype=torch.float64):
    dA = api.DeviceCSR.from_host(A, dtype=dtype)
    dB = api.DeviceCSR.from_host(B, dtype=dtype)
    dM = api.DeviceCSR.from_host(M, dtype=dtype)
    out = api.masked_semiring(dA, dB, dM, semiring)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("values", ["int", "normal"])
def test_semiring_exact(api, oracle_mod, semiring, values):
    A = gen.random_csr(300, 250, 0.05, 1, values=values, empty_rows=0.1)
    B = gen.random_csr(250, 400, 0.05, 2, values=values, empty_rows=0.1)
    M = gen.random_csr(300, 400, 0.08, 3, empty_rows=0.1)
    got = run(api, A, B, M, semiring)
    assert np.array_equal(got, oracle_mod.masked_semiring(A, B, M, semiring))


@pytest.mark.parametrize("semiring", SEMIRINGS)
def test_semiring_fp32(api, oracle_mod, semiring):
    A = gen.random_csr(300, 250, 0.05, 4).astype(np.float32).astype(np.float64)
    B = gen.random_csr(250, 400, 0.05, 5).astype(np.float32).astype(np.float64)
    M = gen.random_csr(300, 400, 0.08, 6)
    got = run(api, A, B, M, semiring, dtype=torch.float32)
    ref = oracle_mod.masked_semiring(A, B, M, semiring).astype(np.float32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("semiring", SEMIRINGS)
def test_semiring_long_mask_rows_and_full_pattern(api, oracle_mod, semiring):
    """Mask rows over several shared-memory slices, and the full pattern of
    A*B as the mask (the semiring product itself)."""
    rng = np.random.default_rng(3)
    m, k, n = 40, 600, 6000
    M = gen.random_rows(m, n, np.concatenate([[5000, 512, 513, 1024, 1535], rng.integers(0, 300, m - 5)]), rng)
    A = gen.random_rows(m, k, rng.integers(0, 100, m), rng, values="int")
    B = gen.random_rows(k, n, rng.integers(0, 200, k), rng, values="int")
    assert np.array_equal(run(api, A, B, M, semiring), oracle_mod.masked_semiring(A, B, M, semiring))
    C = api.spgemm_semiring(api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B), semiring)
    torch.cuda.synchronize()
    R = oracle_mod.spgemm(A, B)
    assert np.array_equal(C.col_idx.cpu().numpy(), R.col_idx)
    assert np.array_equal(C.vals.cpu().numpy(), oracle_mod.masked_semiring(A, B, R, semiring))


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_semiring_product_every_path(api, oracle_mod, semiring, dtype):
    """R-MAT scale 14 A*A through the numeric pass's own semiring
    accumulators: rows of at most 16 products in the register sort, up to 128
    in the warp hash table, up to 65,536 in the warp window, 102 rows above
    that in the block window.
    Structure equal to A*A's, every value exact against the oracle (FP32:
    inputs exact in FP32, the oracle's FP64 values rounded to FP32, since
    one rounding of a + b commutes with min and max)."""
    A = gen.rmat(14, 16).astype(np.float32).astype(np.float64)
    dA = api.DeviceCSR.from_host(A, dtype=dtype)
    C = api.spgemm_semiring(dA, dA, semiring)
    torch.cuda.synchronize()
    R = oracle_mod.spgemm(A, A)
    assert np.array_equal(C.row_ptr.cpu().numpy(), R.row_ptr)
    assert np.array_equal(C.col_idx.cpu().numpy(), R.col_idx)
    ref = oracle_mod.masked_semiring(A, A, R, semiring)
    assert np.array_equal(C.vals.cpu().numpy(), ref.astype(np.float32) if dtype == torch.float32 else ref)


@pytest.mark.parametrize("semiring", SEMIRINGS)
def test_semiring_product_stencil_lane_rows(api, oracle_mod, semiring):
    """3D 7-point Laplacian 20^3 squared: every row has at most 49 products,
    so the numeric pass takes the lane-per-row tables (and the register sort
    for boundary rows of at most 16)."""
    A = gen.laplacian_3d(20)
    dA = api.DeviceCSR.from_host(A)
    C = api.spgemm_semiring(dA, dA, semiring)
    torch.cuda.synchronize()
    R = oracle_mod.spgemm(A, A)
    assert np.array_equal(C.col_idx.cpu().numpy(), R.col_idx)
    assert np.array_equal(C.vals.cpu().numpy(), oracle_mod.masked_semiring(A, A, R, semiring))


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("force_path", [3, 4])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_semiring_product_forced_paths(api, oracle_mod, semiring, force_path, dtype):
    """Every non-empty row through the warp window (3) or the block window
    (4), rectangular with empty rows, in FP64 and FP32 (FP32 inputs whose
    sums are exact, so the result is the oracle's rounded to FP32)."""
    A = gen.random_csr(400, 300, 0.04, 11, empty_rows=0.1).astype(np.float32).astype(np.float64)
    B = gen.random_csr(300, 3000, 0.02, 12, empty_rows=0.1).astype(np.float32).astype(np.float64)
    dA = api.DeviceCSR.from_host(A, dtype=dtype)
    dB = api.DeviceCSR.from_host(B, dtype=dtype)
    C = api.spgemm_semiring(dA, dB, semiring, force_path=force_path)
    torch.cuda.synchronize()
    R = oracle_mod.spgemm(A, B)
    assert np.array_equal(C.col_idx.cpu().numpy(), R.col_idx)
    ref = oracle_mod.masked_semiring(A, B, R, semiring)
    if dtype == torch.float32:
        ref = ref.astype(np.float32)
    assert np.array_equal(C.vals.cpu().numpy(), ref)


def test_semiring_plan_rejects_backward_and_unknown(api):
    from paper_2112_10037_gb300 import _native as nat
    A = api.DeviceCSR.from_host(gen.random_csr(20, 20, 0.2, 1))
    with pytest.raises(nat.SpgemmError) as ei:
        api.Plan(A, A, semiring="min_plus", backward=True)
    assert ei.value.status == 1
    with pytest.raises(nat.SpgemmError) as ei:
        api.Plan(A, A, semiring=7)
    assert ei.value.status == 1


def test_min_plus_all_pairs_shortest_paths(api):
    """Repeated min-plus squaring on the GPU reaches scipy's Dijkstra
    distances on a weighted directed graph of 300 vertices."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    rng = np.random.default_rng(9)
    n = 300
    d = np.zeros((n, n))
    for _ in range(1200):
        a, b = rng.integers(0, n, 2)
        if a != b:
            d[a, b] = float(rng.integers(1, 50))
    P = gen.from_dense(d + np.eye(n))
    rows = np.repeat(np.arange(n), np.diff(np.asarray(P.row_ptr, np.int64)))
    W = gen.CSR(n, n, P.row_ptr, P.col_idx, np.where(rows == P.col_idx, 0.0, d[rows, P.col_idx]))
    D = api.DeviceCSR.from_host(W)
    for _ in range(12):
        Dn = api.spgemm_semiring(D, D, "min_plus")
        same = Dn.nnz == D.nnz and torch.equal(Dn.col_idx, D.col_idx) and torch.equal(Dn.vals, D.vals)
        D = Dn
        if same:
            break
    H = D.to_host()
    got = np.full((n, n), np.inf)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(H.row_ptr, np.int64)))
    got[rows, H.col_idx] = H.vals
    assert np.array_equal(got, shortest_path(csr_matrix(d), method="D", directed=True))


def test_semiring_degenerate_and_errors(api, oracle_mod):
    from paper_2112_10037_gb300 import _native as nat
    for (m, k, n) in [(0, 5, 7), (5, 0, 7), (5, 7, 0), (1, 1, 1)]:
        A = gen.random_csr(m, k, 0.5, 1, values="int")
        B = gen.random_csr(k, n, 0.5, 2, values="int")
        M = gen.random_csr(m, n, 0.5, 3)
        for sr in SEMIRINGS:
            assert np.array_equal(run(api, A, B, M, sr), oracle_mod.masked_semiring(A, B, M, sr))
    A = api.DeviceCSR.from_host(gen.random_csr(5, 4, 0.5, 1))
    B = api.DeviceCSR.from_host(gen.random_csr(4, 6, 0.5, 2))
    M = api.DeviceCSR.from_host(gen.random_csr(5, 6, 0.5, 3))
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_semiring(A.c_struct(), B.c_struct(), M.c_struct(), 0, 7, 0, 0)
    assert ei.value.status == 1
