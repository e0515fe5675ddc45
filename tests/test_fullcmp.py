"""The whole-product comparison helper (tests/fullcmp.py) on the CPU: an
oracle product compared with itself passes, and a value, a column or a row
size planted wrong in the copy under test is reported."""
import numpy as np
import pytest

from paper_2112_10037_gb300 import gen
import fullcmp


def _store_of(C):
    st = fullcmp.Store(12 * C.nnz + 8 * (C.nrows + 1))
    st.put("c_rp", np.asarray(C.row_ptr, np.int64))
    st.empty("c_ci", (C.nnz,), np.int32)[...] = C.col_idx
    st.empty("c_v", (C.nnz,), np.float64)[...] = C.vals
    return st


@pytest.mark.parametrize("signed", [False, True])
def test_compare_detects_planted_errors(oracle_mod, signed):
    A = gen.rmat(10, 8)
    if signed:  # mixed signs: the magnitude-sum product is used
        rng = np.random.default_rng(5)
        A = gen.CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx, rng.standard_normal(A.nnz))
    C = oracle_mod.spgemm(A, A)
    prod = oracle_mod.row_products(A, A)
    st = _store_of(C)
    try:
        ok, err, n, msg = fullcmp.summarise(fullcmp.compare_product(A, A, st, prod, processes=2))
        assert ok and err == 0.0 and n == C.nnz, msg
        v = np.memmap(st.specs["c_v"][0], dtype=np.float64, mode="r+", shape=(C.nnz,))
        j = C.nnz // 3
        v[j] = v[j] * (1 + 1e-9) + 1e-9
        v.flush()
        ok, err, _, msg = fullcmp.summarise(fullcmp.compare_product(A, A, st, prod, processes=2))
        assert not ok and "values" in msg and err > 1e-12
        v[j] = C.vals[j]
        ci = np.memmap(st.specs["c_ci"][0], dtype=np.int32, mode="r+", shape=(C.nnz,))
        ci[j] += 1
        ci.flush()
        ok, _, _, msg = fullcmp.summarise(fullcmp.compare_product(A, A, st, prod, processes=2))
        assert not ok and "columns" in msg
        ci[j] = C.col_idx[j]
        rp = np.memmap(st.specs["c_rp"][0], dtype=np.int64, mode="r+", shape=(C.nrows + 1,))
        r = int(np.searchsorted(C.row_ptr, j, side="right")) - 1
        rp[r + 1] += 1
        rp.flush()
        ok, _, _, msg = fullcmp.summarise(fullcmp.compare_product(A, A, st, prod, processes=2))
        assert not ok and "row sizes" in msg
    finally:
        st.close()


def test_compare_exact_mode(oracle_mod):
    A = gen.laplacian_2d(16)
    C = oracle_mod.spgemm(A, A)
    st = _store_of(C)
    try:
        res = fullcmp.compare_product(A, A, st, oracle_mod.row_products(A, A), exact=True, processes=2)
        ok, err, n, msg = fullcmp.summarise(res)
        assert ok and n == C.nnz, msg
        v = np.memmap(st.specs["c_v"][0], dtype=np.float64, mode="r+", shape=(C.nnz,))
        v[7] = np.nextafter(v[7], np.inf)
        v.flush()
        ok, _, _, msg = fullcmp.summarise(fullcmp.compare_product(A, A, st, oracle_mod.row_products(A, A),
                                                                  exact=True, processes=2))
        assert not ok and "values" in msg
    finally:
        st.close()


def test_compare_many_reports_the_item(oracle_mod):
    """Several products in one pool: all pass as stored, and a value planted
    wrong in the second item's copy is reported with that item's tag."""
    items, st = [], fullcmp.Store(1 << 24)
    try:
        for k, (A, B) in enumerate([(gen.laplacian_2d(12), None), (gen.random_csr(60, 50, 0.1, 3),
                                                                    gen.random_csr(50, 70, 0.1, 4))]):
            B = A if B is None else B
            C = oracle_mod.spgemm(A, B)
            px = "i%d_" % k
            st.put(px + "c_rp", np.asarray(C.row_ptr, np.int64))
            st.put(px + "c_ci", C.col_idx)
            st.put(px + "c_v", C.vals)
            items.append((px, A, B, oracle_mod.row_products(A, B), 1e-12, k == 0))
        ok, err, n, msg = fullcmp.summarise(fullcmp.compare_many(items, st, processes=2))
        assert ok, msg
        v = np.memmap(st.specs["i1_c_v"][0], dtype=np.float64, mode="r+", shape=st.specs["i1_c_v"][1])
        v[5] = v[5] + 1.0
        v.flush()
        ok, err, n, msg = fullcmp.summarise(fullcmp.compare_many(items, st, processes=2))
        assert not ok and "i1_" in msg and "values" in msg
    finally:
        st.close()
