"""The benchmark workload at full size, in the launch configuration bench.py
times (R-MAT scale 18, edge factor 16, C = A*A, FP64, default options):
C's row pointer against the oracle's for every row (exact), rows sampled from
every accumulator path against the oracle element by element, the product
counts, and structural properties of all of C."""
import numpy as np
import pytest
import torch

from paper_2112_10037_gb300 import gen
from parity import abs_csr, assert_structure_equal, assert_values_close

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


def _sample_rows(prod, rng):
    order = np.argsort(prod, kind="stable")
    nz = order[prod[order] > 0]
    pick = [nz[-16:]]  # the heaviest rows (block window)
    for edge in (128, 8192, 32768, 65536):  # both sides of each path boundary
        i = np.searchsorted(prod[nz], edge)
        pick.append(nz[max(0, i - 8):i + 8])
    pick.append(rng.choice(nz, 64, replace=False))
    pick.append(order[prod[order] == 0][:4])  # empty rows
    return np.unique(np.concatenate(pick))


def test_fullsize_sampled_rows(full, oracle_mod):
    A, rp, ci, v, _, _ = full
    prod = oracle_mod.row_products(A, A)
    rows = _sample_rows(prod, np.random.default_rng(2112))
    R = oracle_mod.spgemm(oracle_mod.select_rows(A, rows), A)
    S = oracle_mod.spgemm(oracle_mod.select_rows(abs_csr(A), rows), abs_csr(A))
    h_rp = rp.cpu().numpy().astype(np.int64)
    parts_c, parts_v, lens = [], [], []
    for r in rows:
        lo, hi = int(h_rp[r]), int(h_rp[r + 1])
        parts_c.append(ci[lo:hi].cpu().numpy())
        parts_v.append(v[lo:hi].cpu().numpy())
        lens.append(hi - lo)
    C = gen.CSR(len(rows), A.ncols, np.concatenate([[0], np.cumsum(lens)]).astype(np.int32),
                np.concatenate(parts_c).astype(np.int32), np.concatenate(parts_v).astype(np.float64))
    assert_structure_equal(C, R)
    assert_values_close(C.vals, R.vals, S.vals)


def test_fullsize_structure(full):
    """Columns in range and strictly ascending inside every row; values finite."""
    A, rp, ci, v, nnz, _ = full
    dev = ci.device
    rp64 = rp.long()
    lens = rp64[1:] - rp64[:-1]
    start = torch.zeros(nnz + 1, dtype=torch.bool, device=dev)
    start[rp64[:-1][lens > 0]] = True
    step = 1 << 28
    for off in range(0, nnz - 1, step):
        n = min(step, nnz - 1 - off)
        c = ci[off:off + n + 1]
        ok = (c[1:] > c[:-1]) | start[off + 1:off + n + 1]
        assert bool(ok.all()), "columns not ascending inside a row near entry %d" % off
    assert int(ci.min()) >= 0 and int(ci.max()) < A.ncols
    assert bool(torch.isfinite(v).all())


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
