"""Host-side conversions of the Python layer: torch.sparse_csr_tensor and
(indptr, indices, values, shape) tuples to the library's int32 CSR and back
(no device work)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2112_10037_gb300 import api, gen


def test_from_torch_and_back():
    M = gen.random_csr(40, 70, 0.1, 3)
    t = torch.sparse_csr_tensor(torch.from_numpy(M.row_ptr.astype(np.int64)),
                                torch.from_numpy(M.col_idx.astype(np.int64)),
                                torch.from_numpy(M.vals), size=(M.nrows, M.ncols))
    d = api.DeviceCSR.from_torch(t)
    assert (d.nrows, d.ncols, d.nnz) == (40, 70, M.nnz)
    assert d.row_ptr.dtype == torch.int32 and d.col_idx.dtype == torch.int32
    assert np.array_equal(d.row_ptr.numpy(), M.row_ptr) and np.array_equal(d.col_idx.numpy(), M.col_idx)
    back = d.to_torch()
    assert back.layout == torch.sparse_csr and tuple(back.shape) == (40, 70)
    dense = np.zeros((40, 70))
    for i in range(40):
        for p in range(M.row_ptr[i], M.row_ptr[i + 1]):
            dense[i, M.col_idx[p]] = M.vals[p]
    assert np.array_equal(back.to_dense().numpy(), dense)


def test_tuple_round_trip_and_errors():
    M = gen.random_csr(10, 12, 0.3, 4)
    d = api.DeviceCSR(M.nrows, M.ncols, torch.from_numpy(M.row_ptr), torch.from_numpy(M.col_idx),
                      torch.from_numpy(M.vals))
    e = api.DeviceCSR.from_tuple(d.to_tuple())
    assert (e.nrows, e.ncols) == (10, 12) and torch.equal(e.col_idx, d.col_idx) and torch.equal(e.vals, d.vals)
    with pytest.raises(TypeError):
        api.DeviceCSR.from_torch(torch.zeros(3, 3))
    with pytest.raises(TypeError):
        api._as_csr([1, 2])
