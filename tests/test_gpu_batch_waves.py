"""Batches split into waves (spgemm_batch_products + spgemm_batch_waves):
instances cut into runs whose stacked product count fits int32, each run
one spgemm_batched call.  A small batch forced into several waves against
the single-wave batch and the oracle, eager and from the captured graphs;
the batched workload at its stated size (512 instances, rows log-uniform in
[1024, 200000], about 9.8e9 products, C of about 9.5e9 entries, more than
one wave) against the oracle: every stencil instance bit-exact, 32 seeded
random instances and the largest one entry by entry."""
import numpy as np
import pytest

from paper_2112_10037_gb300 import gen
from parity import assert_structure_equal, assert_values_close, oracle_with_scale, RTOL_F64
import fullcmp

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


def _pairs(api, insts):
    out = []
    for inst in insts:
        dA = api.DeviceCSR.from_host(inst.A)
        dB = dA if inst.B is inst.A else api.DeviceCSR.from_host(inst.B)
        out.append((dA, dB))
    return out


def _host_products(inst):
    lens = np.diff(np.asarray(inst.B.row_ptr, np.int64))
    return int(lens[np.asarray(inst.A.col_idx, np.int64)].sum())


def test_forced_waves_match_single_wave_and_oracle(api, oracle_mod):
    insts = list(gen.batched_instances(count=16, scale_rows=0.01))
    pairs = _pairs(api, insts)
    one = api.Batch(pairs)
    assert len(one.waves) == 1
    assert one.products == [_host_products(i) for i in insts]
    n1 = one.symbolic()
    one.numeric()
    bound = sum(one.products) // 8 + 1
    many = api.Batch(pairs, max_products=bound)
    assert len(many.waves) >= 3
    for a, b in zip(many.wave_first[:-1], many.wave_first[1:]):
        assert sum(many.products[a:b]) <= bound or b - a == 1
    nm = many.symbolic()
    assert nm == n1
    many.numeric()
    torch.cuda.synchronize()
    for inst, C1, C2 in zip(insts, one.results(), many.results()):
        g1, g2 = C1.to_host(), C2.to_host()
        R, S = oracle_with_scale(oracle_mod, inst.A, inst.B)
        assert_structure_equal(g2, R)
        assert_structure_equal(g1, g2)
        assert_values_close(g2.vals, R.vals, S)
    # every wave's numeric pass captured (spgemm_batch_capture) and replayed with new values
    many.capture()
    rng = np.random.default_rng(11)
    for (dA, dB), inst in zip(pairs, insts):
        if inst.B is inst.A:
            continue
        va, vb = rng.standard_normal(inst.A.nnz), rng.standard_normal(inst.B.nnz)
        dA.vals.copy_(torch.from_numpy(va))
        dB.vals.copy_(torch.from_numpy(vb))
        inst.A = gen.CSR(inst.A.nrows, inst.A.ncols, inst.A.row_ptr, inst.A.col_idx, va)
        inst.B = gen.CSR(inst.B.nrows, inst.B.ncols, inst.B.row_ptr, inst.B.col_idx, vb)
    many.replay()
    torch.cuda.synchronize()
    for inst, C in zip(insts, many.results()):
        got = C.to_host()
        R, S = oracle_with_scale(oracle_mod, inst.A, inst.B)
        assert_structure_equal(got, R)
        assert_values_close(got.vals, R.vals, S)
    one.close()
    many.close()


@pytest.mark.slow
def test_batched_workload_at_stated_size(api, oracle_mod):
    insts = gen.batched_instances_parallel(512, 1.0)
    assert len(insts) == 512 and min(i.rows for i in insts) >= 1000 and max(i.rows for i in insts) <= 200_000
    pairs = _pairs(api, insts)
    batch = api.Batch(pairs)
    host_prod = [_host_products(i) for i in insts]
    assert batch.products == host_prod
    total_products = sum(host_prod)
    assert total_products > 9e9
    assert len(batch.waves) >= 5  # 2^31 - 1 products per wave at most
    for a, b in zip(batch.wave_first[:-1], batch.wave_first[1:]):
        assert sum(host_prod[a:b]) < 2 ** 31
    nnz = batch.symbolic()
    batch.numeric()
    torch.cuda.synchronize()
    for w in batch.waves:
        from paper_2112_10037_gb300 import _native as nat
        nat.spgemm_plan_check(nat.spgemm_batch_plan(w.handle), w.stream)
    assert sum(nnz[:-1]) == nnz[-1] and nnz[-1] > 9e9
    res = batch.results()
    rng = np.random.default_rng(2112_10037)
    rand = [i for i in range(256, 512)]
    sample = sorted(set(rng.choice(rand, 32, replace=False).tolist()) | {int(np.argmax(host_prod))})
    chosen = list(range(256)) + sample
    need = sum(12 * nnz[i] + 8 * (insts[i].rows + 1) for i in chosen)
    st = fullcmp.Store(need)
    items = []
    try:
        for i in chosen:
            C, inst = res[i], insts[i]
            px = "i%d_" % i
            st.put(px + "c_rp", C.row_ptr.cpu().numpy().astype(np.int64))
            st.put(px + "c_ci", C.col_idx.cpu().numpy())
            st.put(px + "c_v", C.vals.cpu().numpy())
            lens = np.diff(np.asarray(inst.B.row_ptr, np.int64))
            cs = np.concatenate([[0], np.cumsum(lens[np.asarray(inst.A.col_idx, np.int64)])])
            rp = np.asarray(inst.A.row_ptr, np.int64)
            prod = cs[rp[1:]] - cs[rp[:-1]]
            items.append((px, inst.A, inst.B, prod, RTOL_F64, inst.kind != "random"))
        out = fullcmp.compare_many(items, st)
    finally:
        st.close()
    ok, err, entries, msg = fullcmp.summarise(out)
    print("batched 512: %d waves, %d products, nnz(C) %d; compared %d entries of %d instances, max error %.3e"
          % (len(batch.waves), total_products, nnz[-1], entries, len(chosen), err))
    assert ok, msg
    assert entries == sum(nnz[i] for i in chosen)
    batch.close()
