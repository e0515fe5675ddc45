"""GPU parity of the rank-compacted numeric accumulator (rows of more than
rank_min products: a presence bitmap over up to 2^18 columns ranks the
output columns, values accumulate in an array of the row's outputs) against
the oracle, through the C ABI: with rank_min = 1024 (rows of 1025..65536
products),
with every row above the register sort forced onto it (value chunks of more
than 6144 outputs, rows of more than 512 nonzeros listed in rounds), with
the values reduced into C in global memory or summed in shared memory, on
column spans wider than one 2^18-column window, on both sides of the
rank_min bin edge, in FP64 and FP32."""
import numpy as np
import pytest

from paper_2112_10037_gb300 import gen
from parity import (RTOL_F32, assert_structure_equal, assert_values_close, assert_values_exact,
                    oracle_with_scale, max_rel_err)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# every row above 128 products (register sort below) on the rank path (no
# block window, no split of heavy rows, which would keep them on the warp path)
RANK_ALL = dict(hash_max=-1, rank_min=1, num_block_min=-1, split_min=-1)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10037_gb300 import build
    build.build()
    from paper_2112_10037_gb300 import api as a
    return a


def run(api, A, B, dtype=torch.float64, **kw):
    from paper_2112_10037_gb300 import _native as nat
    dA = api.DeviceCSR.from_host(A, dtype=dtype)
    dB = api.DeviceCSR.from_host(B, dtype=dtype)
    plan = api.Plan(dA, dB, dtype=dtype, **kw)
    nat.spgemm_plan_set_profiling(plan.handle, True)
    rp, nnz = plan.symbolic()
    ci, v = plan.numeric(dA.vals, dB.vals)
    torch.cuda.synchronize()
    plan.check()
    times = nat.spgemm_plan_kernel_times(plan.handle)
    plan.close()
    C = gen.CSR(plan.nrows, B.ncols, rp.cpu().numpy(), ci.cpu().numpy(), v.double().cpu().numpy())
    assert nnz == C.nnz
    return C, times


def _check(oracle_mod, A, B, C):
    R, S = oracle_with_scale(oracle_mod, A, B)
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S)


ACCUM = [0, 1]  # values reduced in C (L2 atomics) / summed in shared-memory chunks


@pytest.mark.parametrize("accum", ACCUM)
@pytest.mark.parametrize("seed", [0, 1])
def test_random_rows_forced_rank(api, oracle_mod, seed, accum):
    A = gen.random_csr(300, 200, 0.05, seed, empty_rows=0.1)
    B = gen.random_csr(200, 500, 0.08, seed + 50, empty_rows=0.1)
    C, times = run(api, A, B, rank_accum=accum, **RANK_ALL)
    _check(oracle_mod, A, B, C)
    assert times["num_rank"] > 0 and times["num_warp"] == 0 and times["num_block"] == 0


@pytest.mark.parametrize("accum", ACCUM)
def test_integer_values_bit_exact_forced_rank(api, oracle_mod, accum):
    A = gen.random_csr(257, 301, 0.1, 7, values="int", empty_rows=0.15)
    B = gen.random_csr(301, 263, 0.1, 8, values="int", empty_rows=0.15)
    C, times = run(api, A, B, rank_accum=accum, **RANK_ALL)
    R = oracle_mod.spgemm(A, B)
    assert_structure_equal(C, R)
    assert_values_exact(C.vals, R.vals)
    assert times["num_rank"] > 0


@pytest.mark.parametrize("accum", ACCUM)
def test_chunks_and_rounds(api, oracle_mod, accum):
    """Rows of 3000 nonzeros (six rounds of the 512-entry segment list) and
    hub B rows of 20000 entries (rows of far more than 6144 outputs, so the
    values accumulate in several chunks)."""
    rng = np.random.default_rng(3)
    counts = rng.integers(0, 400, size=64)
    counts[0] = 3000
    A = gen.random_rows(64, 4000, counts, rng)
    countsB = rng.integers(0, 60, size=4000)
    countsB[:20] = 20000
    B = gen.random_rows(4000, 70000, countsB, rng)
    C, times = run(api, A, B, rank_accum=accum, **RANK_ALL)
    _check(oracle_mod, A, B, C)
    assert np.diff(C.row_ptr).max() > 3 * 6144
    assert times["num_rank"] > 0 and times["num_warp"] == 0


@pytest.mark.parametrize("accum", ACCUM)
def test_spans_wider_than_one_window(api, oracle_mod, accum):
    """Rows whose columns span 700,000 columns: three windows of 2^18
    columns, each nonzero's part of its B row found by binary search; by
    with rank_min = 1024 and forced."""
    rng = np.random.default_rng(17)
    A = gen.random_rows(80, 3000, rng.integers(1, 40, size=80), rng)
    B = gen.random_rows(3000, 700_000, rng.integers(50, 1500, size=3000), rng)
    for kw in (dict(rank_min=1024), RANK_ALL):
        C, times = run(api, A, B, rank_accum=accum, **kw)
        _check(oracle_mod, A, B, C)
        assert times["num_rank"] > 0


@pytest.mark.parametrize("P", [1024, 1025, 2048, 2049, 65536, 65537])
def test_rank_min_bin_edges(api, oracle_mod, P):
    """Rows of P products on each side of rank_min = 1024 and of the block
    window's edge (65536): whichever kernel takes them, the same product."""
    rng = np.random.default_rng(P)
    B = gen.random_rows(P, 300_000, np.ones(P, np.int64), rng)
    A = gen.CSR(3, P, np.array([0, P, P, 2 * P], np.int32),
                np.concatenate([np.arange(P), np.arange(P)]).astype(np.int32),
                rng.standard_normal(2 * P))
    C, times = run(api, A, B, rank_min=1024)
    _check(oracle_mod, A, B, C)
    assert (times["num_rank"] > 0) == (1024 < P <= 65536)


@pytest.mark.parametrize("accum", ACCUM)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kw", [dict(rank_min=1024), RANK_ALL], ids=["above1024", "forced"])
def test_rmat_scale14(api, oracle_mod, dtype, kw, accum):
    A = gen.rmat(14, 16)
    C, times = run(api, A, A, dtype=dtype, rank_accum=accum, **kw)
    R, S = oracle_with_scale(oracle_mod, A, A)
    assert_structure_equal(C, R)
    if dtype == torch.float64:
        assert_values_close(C.vals, R.vals, S)
    else:
        assert max_rel_err(C.vals, R.vals, S) <= RTOL_F32
    assert times["num_rank"] > 0
