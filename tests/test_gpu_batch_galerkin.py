"""Batched products (one stacked launch per pass) and the Galerkin chain
P^T (A P), eager and replayed from a CUDA graph, against the oracle and
against one-by-one plain calls."""
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


def _host(dc):
    return dc.to_host()


def _small_batch(count=16, scale=0.01):
    return list(gen.batched_instances(count=count, scale_rows=scale))


def test_batch_matches_oracle_and_single_calls(api, oracle_mod):
    insts = _small_batch(16, 0.01)
    pairs = []
    for inst in insts:
        dA = api.DeviceCSR.from_host(inst.A)
        dB = dA if inst.B is inst.A else api.DeviceCSR.from_host(inst.B)
        pairs.append((dA, dB))
    batch = api.Batch(pairs)
    nnz = batch.symbolic()
    batch.numeric()
    torch.cuda.synchronize()
    res = batch.results()
    for inst, (dA, dB), C in zip(insts, pairs, res):
        got = _host(C)
        R, S = oracle_with_scale(oracle_mod, inst.A, inst.B)
        assert_structure_equal(got, R)
        if inst.kind == "random":
            assert_values_close(got.vals, R.vals, S)
        else:
            assert_values_exact(got.vals, R.vals)
        single = _host(api.spgemm(dA, dB))
        assert_structure_equal(got, single)
    assert sum(nnz[:-1]) == nnz[-1]
    batch.close()


def test_batch_graph_replay_new_values(api, oracle_mod):
    """The batch numeric pass recorded by spgemm_batch_capture (the C ABI's
    capture call) and launched three times with new values written in
    place into the instances' value buffers."""
    insts = [i for i in _small_batch(10, 0.01)]
    pairs = [(api.DeviceCSR.from_host(i.A), api.DeviceCSR.from_host(i.B)) for i in insts]
    batch = api.Batch(pairs)
    batch.symbolic()
    batch.numeric()
    batch.capture()
    for rep in range(3):
        rng = np.random.default_rng(rep)
        for (dA, dB), inst in zip(pairs, insts):
            va = rng.standard_normal(inst.A.nnz)
            vb = rng.standard_normal(inst.B.nnz)
            dA.vals.copy_(torch.from_numpy(va))
            dB.vals.copy_(torch.from_numpy(vb))
            inst.A = gen.CSR(inst.A.nrows, inst.A.ncols, inst.A.row_ptr, inst.A.col_idx, va)
            inst.B = gen.CSR(inst.B.nrows, inst.B.ncols, inst.B.row_ptr, inst.B.col_idx, vb)
        batch.replay()
        torch.cuda.synchronize()
        for inst, C in zip(insts, batch.results()):
            got = _host(C)
            R, S = oracle_with_scale(oracle_mod, inst.A, inst.B)
            assert_structure_equal(got, R)
            assert_values_close(got.vals, R.vals, S)
    batch.close()


def test_batch_empty_instances(api, oracle_mod):
    A0 = gen.CSR(5, 4, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B0 = gen.random_csr(4, 6, 0.5, 1)
    A1 = gen.random_csr(7, 3, 0.5, 2)
    B1 = gen.random_csr(3, 9, 0.5, 3)
    pairs = [(api.DeviceCSR.from_host(A0), api.DeviceCSR.from_host(B0)),
             (api.DeviceCSR.from_host(A1), api.DeviceCSR.from_host(B1))]
    batch = api.Batch(pairs)
    nnz = batch.symbolic()
    batch.numeric()
    res = batch.results()
    assert nnz[0] == 0
    R = oracle_mod.spgemm(A1, B1)
    got = _host(res[1])
    assert_structure_equal(got, R)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_galerkin_chain_closed_form(api, oracle_mod, n):
    A = gen.laplacian_3d(n)
    P = gen.aggregation_3d(n)
    g = api.Galerkin(api.DeviceCSR.from_host(P), api.DeviceCSR.from_host(A))
    Ac = _host(g.numeric())
    ref = gen.laplacian_3d(n // 2)
    assert np.array_equal(Ac.row_ptr.astype(np.int64), ref.row_ptr.astype(np.int64))
    assert np.array_equal(Ac.col_idx, ref.col_idx)
    assert np.array_equal(Ac.vals, np.where(ref.vals == 6.0, 24.0, -4.0))
    # graph replay gives the same bits, and follows new values of A
    g.capture()
    g.A.vals.mul_(2.0)
    Ac2 = _host(g.replay())
    torch.cuda.synchronize()
    assert np.array_equal(Ac2.vals, 2.0 * Ac.vals)


def test_galerkin_96_matches_two_plain_calls(api, oracle_mod):
    A = gen.laplacian_3d(96)
    P = gen.aggregation_3d(96)
    dA, dP = api.DeviceCSR.from_host(A), api.DeviceCSR.from_host(P)
    g = api.Galerkin(dP, dA)
    g.capture()
    Ac = _host(g.replay())
    torch.cuda.synchronize()
    assert Ac.nnz == 760320
    R = api.transpose(dP)
    AP = api.spgemm(dA, dP)
    plain = _host(api.spgemm(R, AP))
    assert_structure_equal(Ac, plain)
    assert_values_exact(Ac.vals, plain.vals)
    assert g.AP.nnz == 3483648
    # and against the oracle at this full size (integer values: exact)
    ref = oracle_mod.spgemm(oracle_mod.transpose(P), oracle_mod.spgemm(A, P))
    assert_structure_equal(Ac, ref)
    assert_values_exact(Ac.vals, ref.vals)
