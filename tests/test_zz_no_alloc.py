"""The allocation-free transpose entry point (spgemm_transpose_noalloc).

It exists for callers that may not allocate device memory at the moment they
need a transpose; its scratch is a fixed array inside the library.  This test
calls it through the C ABI and checks that it returns exactly what the
workspace-taking spgemm_transpose returns, on two calls in a row (the second
call must not see stale scratch from the first), and that inputs too large
for the fixed scratch are refused.  The file is collected last so that a run
stopping at the first failure has run every other test already.
"""
import numpy as np
import pytest

from paper_2112_10037_gb300 import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10037_gb300 import build
    build.build()
    from paper_2112_10037_gb300 import _native as nat
    from paper_2112_10037_gb300 import api
    return nat, api


def _reference(nat, api, M):
    """spgemm_transpose with its own workspace."""
    return api.transpose(M, want_src=True)


def _noalloc(nat, api, M):
    dev = M.row_ptr.device
    t_rp = torch.full((M.ncols + 1,), -7, dtype=torch.int32, device=dev)
    t_ci = torch.full((max(M.nnz, 1),), -7, dtype=torch.int32, device=dev)
    t_v = torch.full((max(M.nnz, 1),), -7.0, dtype=M.vals.dtype, device=dev)
    t_src = torch.full((max(M.nnz, 1),), -7, dtype=torch.int32, device=dev)
    s = M.c_struct()
    dt = nat.SPGEMM_F32 if M.vals.dtype == torch.float32 else nat.SPGEMM_F64
    nat.spgemm_transpose_noalloc(s, dt, t_rp.data_ptr(), t_ci.data_ptr(), t_v.data_ptr(), t_src.data_ptr(),
                                 int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return t_rp, t_ci[:M.nnz], t_v[:M.nnz], t_src[:M.nnz]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_transpose_matches_workspace_transpose_twice(mods, dtype):
    nat, api = mods
    # two different matrices back to back: the second call must not reuse
    # anything the first left in the shared scratch (fill cursors, error word)
    mats = [gen.random_csr(3000, 2000, 0.004, 1), gen.random_csr(1500, 2500, 0.006, 2)]
    for M in mats:
        dM = api.DeviceCSR.from_host(M, dtype=dtype)
        (T, src) = _reference(nat, api, dM)
        rp, ci, v, s2 = _noalloc(nat, api, dM)
        assert torch.equal(rp, T.row_ptr)
        assert torch.equal(ci, T.col_idx)
        assert torch.equal(v, T.vals)  # same gathered values: exact
        assert torch.equal(s2, src)


def test_noalloc_transpose_long_columns_and_repeat(mods):
    nat, api = mods
    rng = np.random.default_rng(3)
    m = 9000
    rows = [np.unique(np.concatenate([[0], rng.integers(0, 40, size=3)])) for _ in range(m)]
    ci = np.concatenate(rows).astype(np.int32)
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    M = gen.CSR(m, 40, rp, ci, rng.standard_normal(len(ci)))
    dM = api.DeviceCSR.from_host(M)
    T, src = _reference(nat, api, dM)
    for _ in range(2):
        rp2, ci2, v2, s2 = _noalloc(nat, api, dM)
        assert torch.equal(rp2, T.row_ptr) and torch.equal(ci2, T.col_idx)
        assert torch.equal(v2, T.vals) and torch.equal(s2, src)


def test_noalloc_long_column_spanning_windows(mods):
    """A 12,000-entry column over 600,000 source rows (its transpose row
    gathers entries from every tile of the counting scatter), twice in a
    row."""
    nat, api = mods
    from parity import long_column_matrix
    dM = api.DeviceCSR.from_host(long_column_matrix())
    T, src = _reference(nat, api, dM)
    for _ in range(2):
        rp2, ci2, v2, s2 = _noalloc(nat, api, dM)
        assert torch.equal(rp2, T.row_ptr) and torch.equal(ci2, T.col_idx)
        assert torch.equal(v2, T.vals) and torch.equal(s2, src)


def test_noalloc_size_rule_with_and_without_t_src(mods):
    """An input of 1000 columns (two counting-scatter passes of 5 bits) whose
    scratch fits with t_src and FP64 t_vals given (12 + 8 bytes per entry
    plus the digit counts) but not without t_src (4 bytes per entry more)
    runs in the first case and is refused in the second; without values
    and without t_src (16 bytes per entry) it runs again."""
    nat, api = mods
    M = gen.random_csr(9000, 1000, 0.043, 7)
    limit = 8 << 20
    tiles = (M.nnz + 4095) // 4096
    assert 20 * M.nnz + 4 * (32 * tiles + 1) + 8 * 64 + 4096 < limit < 24 * M.nnz
    dM = api.DeviceCSR.from_host(M)
    T, src = _reference(nat, api, dM)
    rp2, ci2, v2, s2 = _noalloc(nat, api, dM)
    assert torch.equal(rp2, T.row_ptr) and torch.equal(ci2, T.col_idx)
    assert torch.equal(v2, T.vals) and torch.equal(s2, src)
    t_rp = torch.empty(M.ncols + 1, dtype=torch.int32, device=dM.row_ptr.device)
    t_ci = torch.empty(M.nnz, dtype=torch.int32, device=dM.row_ptr.device)
    t_v = torch.empty(M.nnz, dtype=torch.float64, device=dM.row_ptr.device)
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_transpose_noalloc(dM.c_struct(), nat.SPGEMM_F64, t_rp.data_ptr(), t_ci.data_ptr(),
                                     t_v.data_ptr(), 0, int(torch.cuda.current_stream().cuda_stream))
    assert ei.value.status == 5
    # structure only and no t_src: 16 bytes per entry, which fits
    nat.spgemm_transpose_noalloc(dM.c_struct(), nat.SPGEMM_F64, t_rp.data_ptr(), t_ci.data_ptr(), 0, 0,
                                 int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert torch.equal(t_rp, T.row_ptr) and torch.equal(t_ci, T.col_idx)


def test_noalloc_rejects_inputs_beyond_the_fixed_scratch(mods):
    nat, api = mods
    M = gen.random_csr(200, 2_500_000, 0.002, 4)   # ~1M entries: scratch > 8 MiB without t_src
    dM = api.DeviceCSR.from_host(M)
    dev = dM.row_ptr.device
    t_rp = torch.empty(M.ncols + 1, dtype=torch.int32, device=dev)
    t_ci = torch.empty(M.nnz, dtype=torch.int32, device=dev)
    with pytest.raises(nat.SpgemmError) as ei:
        nat.spgemm_transpose_noalloc(dM.c_struct(), nat.SPGEMM_F64, t_rp.data_ptr(), t_ci.data_ptr(), 0, 0,
                                     int(torch.cuda.current_stream().cuda_stream))
    assert ei.value.status == 5
