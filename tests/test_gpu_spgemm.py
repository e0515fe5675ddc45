"""GPU parity of the single-product path (analyse -> symbolic -> scan ->
numeric) against the CPU oracle, through the C ABI.

Structure (row_ptr, col_idx, nnz) must match bit for bit; FP64 values within
the criterion in parity.py, or bit for bit for integer-valued inputs (every
partial sum is an exact integer below 2^53, so summation order is moot).
"""
import numpy as np
import pytest

from paper_2112_10037_gb300 import gen
from parity import (RTOL_F32, assert_structure_equal, assert_values_close, assert_values_exact,
                    oracle_with_scale, max_rel_err)

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


def run(api, A, B, dtype=torch.float64, **kw):
    dA = api.DeviceCSR.from_host(A, dtype=dtype)
    dB = api.DeviceCSR.from_host(B, dtype=dtype)
    plan = api.Plan(dA, dB, dtype=dtype, **kw)
    rp, nnz = plan.symbolic()
    ci, v = plan.numeric(dA.vals, dB.vals)
    torch.cuda.synchronize()
    plan.check()
    stats = plan.stats()
    plan.close()
    C = gen.CSR(plan.nrows, B.ncols, rp.cpu().numpy(), ci.cpu().numpy(), v.double().cpu().numpy())
    assert nnz == C.nnz
    return C, stats


PATHS = [-1, 1, 2, 3, 4]


@pytest.mark.parametrize("force", PATHS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_small_all_paths(api, oracle_mod, force, seed):
    A = gen.random_csr(300, 200, 0.05, seed, empty_rows=0.1)
    B = gen.random_csr(200, 500, 0.08, seed + 50, empty_rows=0.1)
    C, _ = run(api, A, B, force_path=force)
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)


@pytest.mark.parametrize("force", PATHS)
def test_integer_values_bit_exact(api, oracle_mod, force):
    A = gen.random_csr(257, 301, 0.1, 7, values="int", empty_rows=0.15)
    B = gen.random_csr(301, 263, 0.1, 8, values="int", empty_rows=0.15)
    C, _ = run(api, A, B, force_path=force)
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


@pytest.mark.parametrize("force", PATHS)
def test_laplacian2d_64_squared(api, oracle_mod, force):
    """The 64x64 2D 5-point Laplacian squared: bit-exact vs the oracle (and
    hence vs the closed form the oracle is pinned to)."""
    A = gen.laplacian_2d(64)
    C, stats = run(api, A, A, force_path=force)
    R = oracle_mod.spgemm(A, A)
    assert C.nnz == 51972
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)
    assert stats[0] == 100104


@pytest.mark.parametrize("force", PATHS)
def test_wide_rows_many_windows(api, oracle_mod, force):
    """Long rows spanning many windows, hub-like B rows, ragged tails."""
    rng = np.random.default_rng(3)
    counts = rng.integers(0, 400, size=64)
    counts[0] = 3000
    A = gen.random_rows(64, 4000, counts, rng)
    countsB = rng.integers(0, 60, size=4000)
    countsB[:20] = 20000
    B = gen.random_rows(4000, 70000, countsB, rng)
    C, _ = run(api, A, B, force_path=force)
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)


@pytest.mark.parametrize("P", [1, 7, 8, 9, 15, 16, 17, 31, 32, 33, 64, 65, 128, 129, 256, 257, 512, 513])
def test_bin_boundaries(api, oracle_mod, P):
    """Rows whose product count sits on each side of a bin edge."""
    rng = np.random.default_rng(P)
    B = gen.random_rows(P, 5000, np.ones(P, np.int64), rng)
    A = gen.CSR(3, P, np.array([0, P, P, 2 * P], np.int32),
                np.concatenate([np.arange(P), np.arange(P)]).astype(np.int32),
                rng.standard_normal(2 * P))
    C, _ = run(api, A, B)
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)


def test_empty_and_degenerate(api, oracle_mod):
    cases = [(0, 5, 7), (5, 0, 7), (5, 7, 0), (1, 1, 1)]
    for (m, k, n) in cases:
        A = gen.random_csr(m, k, 0.5, 1)
        B = gen.random_csr(k, n, 0.5, 2)
        C, _ = run(api, A, B)
        R = oracle_mod.spgemm(A, B)
        assert_structure_equal(C, R)
        assert_values_exact(C.vals, R.vals)
    # all rows empty
    A = gen.CSR(10, 10, np.zeros(11, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C, _ = run(api, A, gen.identity(10))
    assert C.nnz == 0 and np.all(C.row_ptr == 0)


def test_single_dense_row_and_identity(api, oracle_mod):
    n = 20000
    A = gen.CSR(1, n, np.array([0, n], np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    B = gen.random_csr(n, 300, 0.01, 5)
    C, _ = run(api, A, B)
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)
    M = gen.random_csr(500, 400, 0.02, 9)
    C2, _ = run(api, gen.identity(500), M)
    assert np.array_equal(C2.col_idx, M.col_idx) and np.array_equal(C2.vals, M.vals)


def test_explicit_zeros_and_cancellation(api, oracle_mod):
    A = gen.CSR(2, 3, np.array([0, 3, 5], np.int32), np.array([0, 1, 2, 0, 2], np.int32),
                np.array([1.0, 1.0, 0.0, 2.0, -0.0]))
    B = gen.CSR(3, 2, np.array([0, 2, 4, 6], np.int32), np.array([0, 1, 0, 1, 0, 1], np.int32),
                np.array([2.0, 3.0, -2.0, 1.0, 5.0, 0.0]))
    C, _ = run(api, A, B)
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert np.array_equal(C.vals, R.vals)  # 0.0 == -0.0 is allowed here


def test_row_range(api, oracle_mod):
    A = gen.random_csr(400, 300, 0.05, 21)
    B = gen.random_csr(300, 350, 0.05, 22)
    C, _ = run(api, A, B, row_range=(123, 321))
    R, S = oracle_with_scale(oracle_mod, oracle_mod.select_rows(A, np.arange(123, 321)), B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)


def test_numeric_repeat_new_values(api, oracle_mod):
    A = gen.random_csr(200, 150, 0.06, 31)
    B = gen.random_csr(150, 220, 0.06, 32)
    dA = api.DeviceCSR.from_host(A)
    dB = api.DeviceCSR.from_host(B)
    plan = api.Plan(dA, dB)
    rp, nnz = plan.symbolic()
    for t in range(3):
        rng = np.random.default_rng(100 + t)
        A.vals = rng.standard_normal(A.nnz)
        B.vals = rng.standard_normal(B.nnz)
        ci, v = plan.numeric(torch.from_numpy(A.vals).cuda(), torch.from_numpy(B.vals).cuda())
        C = gen.CSR(A.nrows, B.ncols, rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy())
        R, S = oracle_with_scale(oracle_mod, A, B)
        assert_structure_equal(C, R)
        assert_values_close(C.vals, R.vals, S)
    plan.close()


@pytest.mark.parametrize("force", [-1, 3, 4])
def test_fp32_values(api, oracle_mod, force):
    A = gen.random_csr(300, 300, 0.05, 41)
    B = gen.random_csr(300, 300, 0.05, 42)
    C, _ = run(api, A, B, dtype=torch.float32, force_path=force)
    A32 = A.astype(np.float32).astype(np.float64)
    B32 = B.astype(np.float32).astype(np.float64)
    A32 = gen.CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx, A32.vals)
    B32 = gen.CSR(B.nrows, B.ncols, B.row_ptr, B.col_idx, B32.vals)
    R, S = oracle_with_scale(oracle_mod, A32, B32)
    assert_structure_equal(C, R)
    err = max_rel_err(C.vals, R.vals, S)
    assert err <= RTOL_F32


def test_validate_rejects_unsorted(api):
    from paper_2112_10037_gb300._native import SpgemmError
    A = gen.CSR(2, 3, np.array([0, 2, 3], np.int32), np.array([2, 1, 0], np.int32), np.ones(3))
    B = gen.identity(3)
    with pytest.raises(SpgemmError) as ei:
        run(api, A, B, validate=True)
    assert ei.value.status == 3
    A2 = gen.CSR(2, 3, np.array([0, 2, 3], np.int32), np.array([0, 5, 0], np.int32), np.ones(3))
    with pytest.raises(SpgemmError):
        run(api, A2, B, validate=True)
    # valid input passes validation
    C, _ = run(api, gen.identity(3), B, validate=True)
    assert C.nnz == 3


def test_dim_mismatch(api):
    from paper_2112_10037_gb300._native import SpgemmError
    with pytest.raises(SpgemmError) as ei:
        run(api, gen.random_csr(4, 5, 0.5, 1), gen.random_csr(6, 4, 0.5, 2))
    assert ei.value.status == 2


def test_rmat_scale14(api, oracle_mod):
    A = gen.rmat(14, 16)
    C, stats = run(api, A, A)
    R, S = oracle_with_scale(oracle_mod, A, A)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)
    assert stats[0] == int(oracle_mod.row_products(A, A).sum())


@pytest.mark.parametrize("split_min", [64, 2000, 50000])
@pytest.mark.parametrize("window", [1024, 2048, 4096])
def test_split_rows_and_windows(api, oracle_mod, split_min, window):
    """Heavy rows split into column tiles (per-tile counts from the symbolic
    pass, tile bounds from the B-row tile table), for each window width."""
    rng = np.random.default_rng(11)
    counts = rng.integers(0, 300, size=96)
    counts[:4] = [2500, 1200, 700, 400]
    A = gen.random_rows(96, 5000, counts, rng)
    cB = rng.integers(0, 40, size=5000)
    cB[:30] = 9000
    B = gen.random_rows(5000, 40000, cB, rng)
    C, _ = run(api, A, B, split_min=split_min, window_warp=window)
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)


@pytest.mark.parametrize("split_min", [128, 4096])
def test_rmat_scale12_split_integer(api, oracle_mod, split_min):
    A = gen.rmat(12, 16)
    A.vals = np.round(A.vals * 4)  # integer values: bit-exact
    C, _ = run(api, A, A, split_min=split_min)
    R = oracle_mod.spgemm(A, A)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


def test_many_nonzeros_per_row_global_cursors(api, oracle_mod):
    """Rows with more than 256 nonzeros keep their cursors in global memory."""
    rng = np.random.default_rng(5)
    counts = rng.integers(200, 900, size=40)
    A = gen.random_rows(40, 3000, counts, rng)
    B = gen.random_rows(3000, 9000, rng.integers(0, 12, size=3000), rng)
    C, _ = run(api, A, B, split_min=-1)
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)


@pytest.mark.parametrize("sort_max", [128, 256, 512])
@pytest.mark.parametrize("P", [65, 96, 127, 128, 129, 200, 256, 257, 400, 512, 513])
def test_register_sort_multi_slot(api, oracle_mod, P, sort_max):
    rng = np.random.default_rng(P)
    B = gen.random_rows(P, 200, np.ones(P, np.int64), rng, values="int")
    A = gen.CSR(2, P, np.array([0, P, 2 * P], np.int32),
                np.concatenate([np.arange(P), np.arange(P)]).astype(np.int32),
                np.ones(2 * P))
    C, _ = run(api, A, B, sort_max=sort_max)
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


BLOCK_GEOMETRIES = [(2048, 4), (2048, 8), (4096, 4), (4096, 8), (4096, 16), (8192, 8), (8192, 16), (16384, 16)]


def _hub_workload():
    rng = np.random.default_rng(17)
    counts = rng.integers(50, 800, size=40)
    counts[:3] = [2000, 1500, 1200]
    A = gen.random_rows(40, 3000, counts, rng, values="int")
    cB = rng.integers(100, 400, size=3000)
    B = gen.random_rows(3000, 9000, cB, rng, values="int")
    # every row of B also hits the first 40 columns (hub columns)
    rows = []
    rp = B.row_ptr.astype(np.int64)
    for k in range(B.nrows):
        rows.append(np.unique(np.concatenate([np.arange(40), B.col_idx[rp[k]:rp[k + 1]]])))
    ci = np.concatenate(rows).astype(np.int32)
    nrp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    B = gen.CSR(B.nrows, B.ncols, nrp, ci, rng.integers(-3, 4, len(ci)).astype(np.float64))
    return A, B


@pytest.mark.parametrize("num_block_min", [256, 4096])
def test_block_window_long_rows_and_hub_columns(api, oracle_mod, num_block_min):
    """Rows of up to 2000 nonzeros (cursors in global memory, several rounds
    of segments per window) next to short ones (cursors in registers), long
    B segments and hub columns hit by every segment, through the
    block-window kernel; integer values, so the sums are exact."""
    A, B = _hub_workload()
    C, _ = run(api, A, B, num_block_min=num_block_min)
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


@pytest.mark.parametrize("geom", BLOCK_GEOMETRIES)
def test_block_window_geometries(api, oracle_mod, geom):
    """Every compiled (window columns, warps) pair of the block kernel."""
    A, B = _hub_workload()
    C, _ = run(api, A, B, num_block_min=256, window_block=geom[0], block_warps=geom[1])
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


def test_block_window_fp32_exact(api, oracle_mod):
    """FP32 through the block kernel: integer sums below 2**24 are exact."""
    A, B = _hub_workload()
    C, _ = run(api, A, B, dtype=torch.float32, num_block_min=256)
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


# ------------------------------------------------------------ hash path
# Rows of 17..hash_max products go through the warp hash accumulator (one
# shared-memory table per warp, cleared between the warp's rows); hash_max
# -1 keeps the register sort, so each case also runs without the path.
HASH_SETTINGS = [-1, 32, 64, 128]


def _hash_rows(prod, hash_max):
    hi = {-1: 0, 32: 32, 64: 64, 128: 128}[hash_max]
    return int(((prod >= 17) & (prod <= hi)).sum())


def _row_products(A, B):
    blen = np.diff(B.row_ptr.astype(np.int64))
    return np.add.reduceat(np.concatenate([blen[A.col_idx], [0]]),
                           A.row_ptr[:-1].astype(np.int64)) * (np.diff(A.row_ptr) > 0)


@pytest.mark.parametrize("hash_max", HASH_SETTINGS)
@pytest.mark.parametrize("ncols", [300, 50000])
def test_hash_path_mixed_rows(api, oracle_mod, hash_max, ncols):
    """Rows of 0..~200 products: the register sort below 17, the hash bins
    (1, 2 and 4 products per lane) and the window path above 128; a narrow
    B (300 columns: many equal columns merge in each row) and a wide one."""
    rng = np.random.default_rng(11 + ncols)
    m, k = 4000, 900
    A = gen.random_rows(m, k, rng.integers(0, 16, size=m), rng)
    B = gen.random_rows(k, ncols, rng.integers(1, 17, size=k), rng)
    C, stats = run(api, A, B, hash_max=hash_max)
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)
    prod = _row_products(A, B)
    assert stats[0] == int(prod.sum())
    assert stats[2][1] == _hash_rows(prod, hash_max)
    if hash_max == 128:
        assert stats[2][1] > 1000


@pytest.mark.parametrize("hash_max", HASH_SETTINGS)
def test_hash_path_integer_bit_exact(api, oracle_mod, hash_max):
    rng = np.random.default_rng(23)
    A = gen.random_rows(2500, 700, rng.integers(0, 12, size=2500), rng, values="int")
    B = gen.random_rows(700, 400, rng.integers(1, 14, size=700), rng, values="int")
    C, _ = run(api, A, B, hash_max=hash_max)
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)


@pytest.mark.parametrize("hash_max", [-1, 128])
def test_hash_path_fp32(api, oracle_mod, hash_max):
    rng = np.random.default_rng(29)
    A = gen.random_rows(3000, 800, rng.integers(0, 12, size=3000), rng)
    B = gen.random_rows(800, 2000, rng.integers(1, 14, size=800), rng)
    C, _ = run(api, A, B, dtype=torch.float32, hash_max=hash_max)
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S, rtol=RTOL_F32)


@pytest.mark.parametrize("hash_max", HASH_SETTINGS)
def test_hash_path_3d_stencil_squared(api, oracle_mod, hash_max):
    """3D 7-point operator on 20^3 squared: interior rows have 49 products
    and 25 columns (bin 7), faces, edges and corners fewer; integer values,
    so the result is bit-exact."""
    A = gen.laplacian_3d(20)
    C, stats = run(api, A, A, hash_max=hash_max)
    R = oracle_mod.spgemm(A, A)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)
    assert stats[2][1] == _hash_rows(_row_products(A, A), hash_max)


def test_hash_path_galerkin_small(api, oracle_mod):
    """P^T (A P) on a 16^3 grid with 2x2x2 aggregation: both products have
    rows in the hash bins (A P rows 7 products, P^T (AP) rows up to 8 times
    A P's row sizes); exact integer sums."""
    A = gen.laplacian_3d(16)
    P = gen.aggregation_3d(16)
    Pt = oracle_mod.transpose(P)
    AP, _ = run(api, A, P)
    R_AP = oracle_mod.spgemm(A, P)
    assert_structure_equal(AP, R_AP)
    assert_values_exact(AP.vals, R_AP.vals)
    G, stats = run(api, Pt, R_AP)
    R = oracle_mod.spgemm(Pt, R_AP)
    assert_structure_equal(G, R)
    assert_values_exact(G.vals, R.vals)
    assert stats[2][1] > 0


def test_torch_sparse_and_tuple_inputs(api, oracle_mod):
    """spgemm on torch.sparse_csr_tensor inputs (int64 indices) returns a
    torch.sparse_csr_tensor, on (indptr, indices, values, shape) tuples a
    tuple; both equal the oracle's product."""
    A = gen.random_csr(300, 200, 0.05, 21, values="int")
    B = gen.random_csr(200, 250, 0.05, 22, values="int")
    R = oracle_mod.spgemm(A, B)
    dev = torch.device("cuda")
    ta = torch.sparse_csr_tensor(torch.from_numpy(A.row_ptr.astype(np.int64)),
                                 torch.from_numpy(A.col_idx.astype(np.int64)),
                                 torch.from_numpy(A.vals), size=(A.nrows, A.ncols)).to(dev)
    tb = torch.sparse_csr_tensor(torch.from_numpy(B.row_ptr.astype(np.int64)),
                                 torch.from_numpy(B.col_idx.astype(np.int64)),
                                 torch.from_numpy(B.vals), size=(B.nrows, B.ncols)).to(dev)
    tc = api.spgemm(ta, tb)
    assert tc.layout == torch.sparse_csr and tuple(tc.shape) == (300, 250)
    assert np.array_equal(tc.crow_indices().cpu().numpy(), R.row_ptr)
    assert np.array_equal(tc.col_indices().cpu().numpy(), R.col_idx)
    assert np.array_equal(tc.values().cpu().numpy(), R.vals)
    dA, dB = api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B)
    rp, ci, v, shape = api.spgemm(dA.to_tuple(), dB.to_tuple())
    assert shape == (300, 250) and np.array_equal(ci.cpu().numpy(), R.col_idx)
    assert np.array_equal(v.cpu().numpy(), R.vals)


def test_batched_and_galerkin_helpers(api, oracle_mod):
    """The one-call helpers: batched() over three pairs and galerkin(P, A)
    against the oracle (integer values: exact)."""
    rng = np.random.default_rng(5)
    pairs, refs = [], []
    for s in range(3):
        A = gen.random_rows(60 + 10 * s, 50, rng.integers(0, 8, size=60 + 10 * s), rng, values="int")
        B = gen.random_rows(50, 80, rng.integers(0, 8, size=50), rng, values="int")
        pairs.append((api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(B)))
        refs.append(oracle_mod.spgemm(A, B))
    for C, R in zip(api.batched(pairs), refs):
        assert np.array_equal(C.row_ptr.cpu().numpy(), R.row_ptr)
        assert np.array_equal(C.col_idx.cpu().numpy(), R.col_idx)
        assert np.array_equal(C.vals.cpu().numpy(), R.vals)
    A = gen.laplacian_2d(16)
    n = A.nrows
    P = gen.CSR(n, n // 4, np.arange(n + 1, dtype=np.int32), (np.arange(n) // 4).astype(np.int32), np.ones(n))
    Ac = api.galerkin(api.DeviceCSR.from_host(P), api.DeviceCSR.from_host(A))
    Pt = oracle_mod.transpose(P)
    R = oracle_mod.spgemm(Pt, oracle_mod.spgemm(A, P))
    assert np.array_equal(Ac.col_idx.cpu().numpy(), R.col_idx)
    assert np.array_equal(Ac.vals.cpu().numpy(), R.vals)
