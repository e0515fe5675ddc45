"""Pins for the CPU oracle: each test checks it against something other than
itself -- dense brute force, special products with a known answer, stencil
closed forms, the associativity invariant, finite differences.  No GPU.

Each pin is chosen so that a plausible slip in the oracle fails it: a dropped
product or wrong index (brute force, closed forms), a transposed operand
(non-square brute force), a sign error (Laplacian closed form), unsorted or
repeated output columns (structure checks), a lost pattern entry on
cancellation (explicit-zero test).
"""
import os

import numpy as np
import pytest

from paper_2112_10037_gb300 import gen

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _dense(m):
    return gen.to_dense(m)


def _pattern(m):
    d = np.zeros((m.nrows, m.ncols), bool)
    rows = np.repeat(np.arange(m.nrows), np.diff(np.asarray(m.row_ptr, np.int64)))
    d[rows, m.col_idx] = True
    return d


def _assert_sorted_unique(C):
    rp = np.asarray(C.row_ptr, np.int64)
    for i in range(C.nrows):
        seg = C.col_idx[rp[i]:rp[i + 1]]
        assert np.all(np.diff(seg) > 0), f"row {i} not strictly ascending"


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("shape,density,seed", [
    ((1, 1, 1), 1.0, 0), ((7, 5, 9), 0.4, 1), ((33, 17, 40), 0.2, 2),
    ((64, 64, 64), 0.1, 3), ((20, 64, 3), 0.3, 4), ((50, 1, 50), 0.5, 5),
])
def test_brute_force_integer_exact(oracle_mod, shape, density, seed):
    """Integer-valued inputs: every partial sum is an exact integer, so the
    oracle must equal the dense product bit for bit (Sec. 2.2 definition)."""
    m, k, n = shape
    A = gen.random_csr(m, k, density, seed, values="int", empty_rows=0.2)
    B = gen.random_csr(k, n, density, seed + 100, values="int", empty_rows=0.2)
    C = oracle_mod.spgemm(A, B)
    _assert_sorted_unique(C)
    dense = _dense(A) @ _dense(B)
    struct = (_pattern(A).astype(np.int64) @ _pattern(B).astype(np.int64)) > 0
    assert np.array_equal(_pattern(C), struct)
    assert np.array_equal(_dense(C), np.where(struct, dense, 0.0))
    assert np.array_equal(np.asarray(C.row_ptr, np.int64), oracle_mod.spgemm_rowptr(A, B))


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_real_values(oracle_mod, seed):
    A = gen.random_csr(40, 30, 0.25, seed, values="normal", empty_rows=0.1)
    B = gen.random_csr(30, 50, 0.25, seed + 7, values="normal", empty_rows=0.1)
    C = oracle_mod.spgemm(A, B)
    ref = _dense(A) @ _dense(B)
    scale = np.abs(_dense(A)) @ np.abs(_dense(B))
    got = _dense(C)
    assert np.all(np.abs(got - ref) <= 1e-14 * scale + 1e-300)


def test_non_square_operand_order(oracle_mod):
    """A (3x2) * B (2x4): swapping the operands or transposing one cannot
    even produce a 3x4 result, and the values are asymmetric."""
    A = gen.from_dense(np.array([[1.0, 2.0], [0.0, 3.0], [4.0, 0.0]]))
    B = gen.from_dense(np.array([[1.0, 0.0, 5.0, 0.0], [0.0, 6.0, 7.0, 1.0]]))
    C = oracle_mod.spgemm(A, B)
    assert (C.nrows, C.ncols) == (3, 4)
    expect = np.array([[1.0, 12.0, 19.0, 2.0], [0.0, 18.0, 21.0, 3.0], [4.0, 0.0, 20.0, 0.0]])
    assert np.array_equal(_dense(C), expect)
    assert list(np.diff(C.row_ptr)) == [4, 3, 2]


def test_cancellation_keeps_structure(oracle_mod):
    """Products that cancel to 0.0 stay in the pattern (structural C)."""
    A = gen.from_dense(np.array([[1.0, 1.0]]))
    B = gen.from_dense(np.array([[2.0, 3.0], [-2.0, 1.0]]))
    C = oracle_mod.spgemm(A, B)
    assert list(C.col_idx) == [0, 1]
    assert C.vals[0] == 0.0 and C.vals[1] == 4.0


def test_empty_shapes(oracle_mod):
    for (m, k, n) in [(0, 0, 0), (0, 5, 3), (4, 0, 3), (4, 5, 0), (3, 3, 3)]:
        A = gen.random_csr(m, k, 0.5, 1)
        B = gen.random_csr(k, n, 0.5, 2)
        if (m, k, n) == (3, 3, 3):
            A = gen.CSR(3, 3, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0))
        C = oracle_mod.spgemm(A, B)
        assert C.nrows == m and C.ncols == n and C.nnz == 0


# ------------------------------------------------------- special products
def test_identity_products(oracle_mod):
    A = gen.random_csr(57, 43, 0.2, 11)
    I_l, I_r = gen.identity(57), gen.identity(43)
    for C in (oracle_mod.spgemm(I_l, A), oracle_mod.spgemm(A, I_r)):
        assert np.array_equal(C.row_ptr, A.row_ptr.astype(np.int64))
        assert np.array_equal(C.col_idx, A.col_idx)
        assert np.array_equal(C.vals, A.vals)


def test_permutation_products(oracle_mod):
    rng = np.random.default_rng(5)
    A = gen.random_csr(30, 30, 0.2, 12)
    perm = rng.permutation(30)
    P = gen.permutation(perm)
    # P*A: row i of the result is row perm[i] of A.
    C = oracle_mod.spgemm(P, A)
    assert np.array_equal(_dense(C), _dense(A)[perm, :])
    _assert_sorted_unique(C)
    # A*P: column perm[c] of A moves to column c (entries re-sorted).
    C2 = oracle_mod.spgemm(A, P)
    # (A*P)[:, c] = A[:, i] with perm[i] = c, i.e. A[:, argsort(perm)].
    assert np.array_equal(_dense(C2), _dense(A)[:, np.argsort(perm)])
    _assert_sorted_unique(C2)


def test_power_of_two_diagonal_scaling(oracle_mod):
    A = gen.random_csr(25, 25, 0.3, 13)
    d = 2.0 ** np.random.default_rng(1).integers(-4, 5, 25)
    C = oracle_mod.spgemm(gen.diagonal(d), A)
    rows = np.repeat(np.arange(25), np.diff(A.row_ptr))
    assert np.array_equal(C.vals, A.vals * d[rows])
    assert np.array_equal(C.col_idx, A.col_idx)


# ---------------------------------------------------------- closed forms
def _lap2d_square_expected(nx):
    """Closed form of (2D 5-point Laplacian)^2 on an nx x nx grid: 16 + deg(i)
    on the diagonal, -8 at distance 1, 2 at the four diagonal neighbours, 1
    at axial distance 2 (all restricted to the grid)."""
    exp = {}
    for y in range(nx):
        for x in range(nx):
            i = y * nx + x
            deg = (x > 0) + (x < nx - 1) + (y > 0) + (y < nx - 1)
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    if abs(dx) + abs(dy) > 2:
                        continue
                    xx, yy = x + dx, y + dy
                    if not (0 <= xx < nx and 0 <= yy < nx):
                        continue
                    j = yy * nx + xx
                    if dx == 0 and dy == 0:
                        v = 16.0 + deg
                    elif abs(dx) + abs(dy) == 1:
                        v = -8.0
                    elif abs(dx) == 1 and abs(dy) == 1:
                        v = 2.0
                    else:
                        v = 1.0
                    exp[(i, j)] = v
    return exp


@pytest.mark.parametrize("nx", [1, 2, 3, 8, 64])
def test_laplacian2d_squared_closed_form(oracle_mod, nx):
    A = gen.laplacian_2d(nx)
    C = oracle_mod.spgemm(A, A)
    _assert_sorted_unique(C)
    exp = _lap2d_square_expected(nx)
    assert C.nnz == len(exp)
    rows = np.repeat(np.arange(C.nrows), np.diff(C.row_ptr))
    got = {(int(r), int(c)): float(v) for r, c, v in zip(rows, C.col_idx, C.vals)}
    assert got == exp
    if nx == 64:
        # nnz = sum over the 13 offsets of (64-|dx|)(64-|dy|) = 51,972
        offs = [(dx, dy) for dx in range(-2, 3) for dy in range(-2, 3) if abs(dx) + abs(dy) <= 2]
        assert C.nnz == sum((64 - abs(dx)) * (64 - abs(dy)) for dx, dy in offs) == 51972
        interior = 20 * 64 + 20
        assert got[(interior, interior)] == 20.0


@pytest.mark.parametrize("n", [2, 4, 8])
def test_galerkin_coarse_operator_closed_form(oracle_mod, n):
    """P^T (A P) for the 3D 7-point operator (6 / -1) and 2x2x2 aggregation
    is the coarse 7-point operator with 24 on the diagonal and -4 to each
    face-neighbour aggregate (4 fine edges cross each aggregate face; the
    12 edges inside an aggregate cancel 24 of the 8*6 = 48)."""
    A = gen.laplacian_3d(n)
    P = gen.aggregation_3d(n)
    R = oracle_mod.transpose(P)
    AP = oracle_mod.spgemm(A, P)
    Ac = oracle_mod.spgemm(R, AP)
    nc = n // 2
    ref = gen.laplacian_3d(nc)
    assert np.array_equal(np.asarray(Ac.row_ptr, np.int64), ref.row_ptr.astype(np.int64))
    assert np.array_equal(Ac.col_idx, ref.col_idx)
    assert np.array_equal(Ac.vals, np.where(ref.vals == 6.0, 24.0, -4.0))


def test_galerkin_full_size_counts(oracle_mod):
    """nnz(A P) and nnz(P^T A P) at the 96^3 workload (7-point stencil on
    the 48^3 coarse grid: 7*48^3 - 6*48^2 entries)."""
    A = gen.laplacian_3d(96)
    P = gen.aggregation_3d(96)
    AP_rp = oracle_mod.spgemm_rowptr(A, P)
    assert AP_rp[-1] == 3_483_648
    assert 7 * 48 ** 3 - 6 * 48 ** 2 == 760_320


def test_laplacian3d_squared_diagonal(oracle_mod):
    A = gen.laplacian_3d(6)
    C = oracle_mod.spgemm(A, A)
    d = _dense(C)
    deg = np.diff(A.row_ptr) - 1
    assert np.array_equal(np.diag(d), 36.0 + deg)


@pytest.mark.parametrize("n", [1, 2, 3, 8])
def test_laplacian3d_squared_closed_form(oracle_mod, n):
    """A*A for the 3D 7-point operator against its closed form entry by
    entry (36 + deg on the diagonal, -12 at distance 1, 2 at diagonal
    offsets, 1 at distance-2 axial offsets; the same helper checks the
    device's 96^3 product)."""
    from parity import stencil3d_square_closed_form
    A = gen.laplacian_3d(n)
    C = oracle_mod.spgemm(A, A)
    _assert_sorted_unique(C)
    exp = stencil3d_square_closed_form(n, C.row_ptr, C.col_idx)
    assert not np.isnan(exp).any()
    assert np.array_equal(C.vals, exp)
    # every in-grid position of each of the 25 offsets is an entry
    offs = [(a, b, c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)
            if abs(a) + abs(b) + abs(c) <= 2]
    assert len(offs) == 25
    assert C.nnz == sum(max(n - abs(a), 0) * max(n - abs(b), 0) * max(n - abs(c), 0) for a, b, c in offs)


def test_laplacian3d_squared_nnz_96():
    offs = [(a, b, c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)
            if abs(a) + abs(b) + abs(c) <= 2]
    assert sum((96 - abs(a)) * (96 - abs(b)) * (96 - abs(c)) for a, b, c in offs) == 21_732_480


# ------------------------------------------------------------- invariant
@pytest.mark.parametrize("seed", [0, 1])
def test_associativity_invariant(oracle_mod, seed):
    A = gen.random_csr(300, 200, 0.03, seed)
    B = gen.random_csr(200, 250, 0.03, seed + 1)
    x = np.random.default_rng(seed).standard_normal(250)
    C = oracle_mod.spgemm(A, B)
    lhs = oracle_mod.spmv(C, x)
    rhs = oracle_mod.spmv(A, oracle_mod.spmv(B, x))
    scale = np.abs(_dense(A)) @ (np.abs(_dense(B)) @ np.abs(x))
    assert np.all(np.abs(lhs - rhs) <= 1e-13 * scale + 1e-300)


def test_spmv_and_transpose_vs_dense(oracle_mod):
    A = gen.random_csr(37, 23, 0.2, 3)
    x = np.arange(23, dtype=np.float64) - 5
    assert np.allclose(oracle_mod.spmv(A, x), _dense(A) @ x, rtol=1e-14, atol=1e-14)
    T = oracle_mod.transpose(A)
    assert np.array_equal(_dense(T), _dense(A).T)
    _assert_sorted_unique(T)
    TT = oracle_mod.transpose(T)
    assert np.array_equal(TT.col_idx, A.col_idx) and np.array_equal(TT.vals, A.vals)


def test_row_products(oracle_mod):
    A = gen.random_csr(40, 30, 0.2, 4)
    B = gen.random_csr(30, 60, 0.2, 5)
    lens = np.diff(B.row_ptr).astype(np.int64)
    expect = np.array([lens[A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]].sum() for i in range(40)])
    assert np.array_equal(oracle_mod.row_products(A, B), expect)


def test_rmat_generator_counts():
    """Workload recipe check (input side only): R-MAT scale 10 is
    deterministic and self-loop free, with hubs at low ids."""
    A = gen.rmat(10, 16).check()
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    assert not np.any(rows == A.col_idx)
    lens = np.diff(A.row_ptr)
    assert lens[0] == lens.max()
    B = gen.rmat(10, 16)
    assert np.array_equal(A.col_idx, B.col_idx) and np.array_equal(A.vals, B.vals)


# -------------------------------------------------------------- gradient
def _loss(oracle_mod, A, B, W_of):
    C = oracle_mod.spgemm(A, B)
    return float(np.sum(W_of(C) * C.vals))


def test_backward_vs_dense(oracle_mod):
    A = gen.random_csr(30, 25, 0.2, 21)
    B = gen.random_csr(25, 35, 0.2, 22)
    C = oracle_mod.spgemm(A, B)
    W = np.random.default_rng(3).standard_normal(C.nnz)
    da, db = oracle_mod.backward(A, B, C.row_ptr, C.col_idx, W)
    Wd = _dense(gen.CSR(C.nrows, C.ncols, C.row_ptr.astype(np.int32), C.col_idx, W))
    dA_dense = Wd @ _dense(B).T
    dB_dense = _dense(A).T @ Wd
    ra = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    rb = np.repeat(np.arange(B.nrows), np.diff(B.row_ptr))
    assert np.allclose(da, dA_dense[ra, A.col_idx], rtol=1e-13, atol=1e-13)
    assert np.allclose(db, dB_dense[rb, B.col_idx], rtol=1e-13, atol=1e-13)


def test_backward_finite_differences(oracle_mod):
    """L = sum W*C is bilinear in (A, B), so a one-sided difference
    (L(A + h e_p) - L(A)) / h equals dA[p] up to rounding, for any h."""
    A = gen.random_csr(20, 15, 0.3, 31)
    B = gen.random_csr(15, 18, 0.3, 32)
    C = oracle_mod.spgemm(A, B)
    W = np.random.default_rng(4).standard_normal(C.nnz)
    key = {(int(r), int(c)): t for t, (r, c) in enumerate(
        zip(np.repeat(np.arange(C.nrows), np.diff(C.row_ptr)), C.col_idx))}

    def W_of(Cn):
        rows = np.repeat(np.arange(Cn.nrows), np.diff(Cn.row_ptr))
        return np.array([W[key[(int(r), int(c))]] for r, c in zip(rows, Cn.col_idx)])

    da, db = oracle_mod.backward(A, B, C.row_ptr, C.col_idx, W)
    L0 = _loss(oracle_mod, A, B, W_of)
    h = 1e-3
    for p in range(0, A.nnz, max(1, A.nnz // 12)):
        A2 = gen.CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx, A.vals.copy())
        A2.vals[p] += h
        fd = (_loss(oracle_mod, A2, B, W_of) - L0) / h
        assert abs(fd - da[p]) <= 1e-9 * (1 + abs(da[p]))
    for q in range(0, B.nnz, max(1, B.nnz // 12)):
        B2 = gen.CSR(B.nrows, B.ncols, B.row_ptr, B.col_idx, B.vals.copy())
        B2.vals[q] += h
        fd = (_loss(oracle_mod, A, B2, W_of) - L0) / h
        assert abs(fd - db[q]) <= 1e-9 * (1 + abs(db[q]))


# ------------------------------------------------------- hand-worked example
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gustavson_worked_example.txt")


def test_golden_worked_example(oracle_mod):
    """The oracle against a product worked out by hand from the row-wise
    Gustavson definition (Sec. 2.2): exact structure (a cancelled entry
    stays, an empty row, an A entry whose B row is empty) and exact values,
    and the gradient of the sum of C's entries."""
    from parity import load_golden
    g = load_golden(GOLDEN)
    A, B, Cref = g["A"], g["B"], g["C"]
    C = oracle_mod.spgemm(A, B)
    assert np.array_equal(np.asarray(C.row_ptr, np.int64), np.asarray(Cref.row_ptr, np.int64))
    assert np.array_equal(C.col_idx, Cref.col_idx)
    assert np.array_equal(C.vals, Cref.vals)
    da, db = oracle_mod.backward(A, B, C.row_ptr, C.col_idx, np.ones(C.nnz))
    assert np.array_equal(da, g["dA"].vals) and np.array_equal(g["dA"].col_idx, A.col_idx)
    assert np.array_equal(db, g["dB"].vals) and np.array_equal(g["dB"].col_idx, B.col_idx)


# ------------------------------------------------------------ masked product
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_masked_brute_force(oracle_mod, seed):
    """C<M> = (A*B) .* M against dense brute force on M's pattern (integer
    values: exact), with and without M's values; rows and columns of M that
    no product reaches included."""
    A = gen.random_csr(37, 23, 0.2, seed, values="int", empty_rows=0.2)
    B = gen.random_csr(23, 41, 0.2, seed + 10, values="int", empty_rows=0.2)
    M = gen.random_csr(37, 41, 0.3, seed + 20, values="int")
    P = _dense(A) @ _dense(B)
    rows = np.repeat(np.arange(M.nrows), np.diff(np.asarray(M.row_ptr, np.int64)))
    got = oracle_mod.masked(A, B, M)
    assert np.array_equal(got, P[rows, M.col_idx] * M.vals)
    got1 = oracle_mod.masked(A, B, M, use_mask_values=False)
    assert np.array_equal(got1, P[rows, M.col_idx])


def test_masked_real_values_and_full_mask(oracle_mod):
    """Real values: within rounding of the dense product; with M = the
    pattern of A*B the masked product is the product itself."""
    A = gen.random_csr(50, 40, 0.15, 4)
    B = gen.random_csr(40, 60, 0.15, 5)
    C = oracle_mod.spgemm(A, B)
    M = gen.CSR(C.nrows, C.ncols, C.row_ptr, C.col_idx, np.ones(C.nnz))
    got = oracle_mod.masked(A, B, M)
    rows = np.repeat(np.arange(M.nrows), np.diff(np.asarray(M.row_ptr, np.int64)))
    dense = (_dense(A) @ _dense(B))[rows, M.col_idx]
    scale = (np.abs(_dense(A)) @ np.abs(_dense(B)))[rows, M.col_idx]
    assert np.all(np.abs(got - dense) <= 1e-14 * scale)
    assert np.array_equal(got, C.vals)


def _undirected(n, edges):
    d = np.zeros((n, n))
    for a, b in edges:
        d[a, b] = d[b, a] = 1.0
    return gen.lower_triangle_undirected(gen.from_dense(d))


@pytest.mark.parametrize("name,n,edges,triangles", [
    ("K12", 12, [(a, b) for a in range(12) for b in range(a)], 220),      # C(12,3)
    ("K4 minus an edge", 4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)], 2),
    ("cycle C9", 9, [(a, (a + 1) % 9) for a in range(9)], 0),
    ("wheel W10", 11, [(a, (a + 1) % 10) for a in range(10)] + [(10, a) for a in range(10)], 10),
    ("3x4 grid", 12, [(r * 4 + c, r * 4 + c + 1) for r in range(3) for c in range(3)] +
                     [(r * 4 + c, (r + 1) * 4 + c) for r in range(2) for c in range(4)], 0),
])
def test_masked_triangle_counts(oracle_mod, name, n, edges, triangles):
    """Triangle counting (Sec. 1 lists it among SpGEMM's applications):
    sum((L*L) .* L) over the strictly lower triangle L of the adjacency
    matrix equals the graph's number of triangles (closed forms: C(n,3) for
    K_n, n for the wheel with an n-cycle rim, none in a cycle or a grid)."""
    L = _undirected(n, edges)
    assert float(oracle_mod.masked(L, L, L).sum()) == triangles


# ------------------------------------------------------------------- OMAR
def test_omar_hand_example(oracle_mod):
    """Eq. 1 by hand: rows {0,1}, {1,2}, {0,3}, {3} with two computing
    units: vectors (group 0: column 0 x1, column 1 x2, column 2 x1;
    group 1: column 0 x1, column 3 x2) give (2-1) + (2-1) = 2 shared reads
    out of 7 nonzeros."""
    d = np.zeros((4, 4))
    for r, cs in enumerate([(0, 1), (1, 2), (0, 3), (3,)]):
        d[r, list(cs)] = 1.0
    A = gen.from_dense(d)
    assert abs(oracle_mod.omar(A, 2) - 100.0 * 2 / 7) < 1e-12
    assert oracle_mod.omar(A, 1) == 0.0
    assert abs(oracle_mod.omar(A, 4) - 100.0 * 3 / 7) < 1e-12   # columns 0,1,3 read twice each


@pytest.mark.parametrize("m,n,pes", [(10, 7, 3), (12, 5, 4), (9, 1, 32), (1, 6, 8)])
def test_omar_closed_forms(oracle_mod, m, n, pes):
    """Dense rows (every group shares all n columns): 1 - ceil(m/P)/m;
    a diagonal: no sharing at all."""
    A = gen.from_dense(np.ones((m, n)))
    groups = -(-m // pes)
    assert abs(oracle_mod.omar(A, pes) - 100.0 * (1 - groups / m)) < 1e-12
    assert oracle_mod.omar(gen.identity(m), pes) == 0.0


# ------------------------------------------------------------ semirings
def _semiring_brute(A, B, M, semiring):
    """Entry by entry from the definition, on dense arrays: for (i,j) in M,
    reduce over the k where A(i,k) and B(k,j) are both stored."""
    Ad, Bd = _dense(A), _dense(B)
    Ap, Bp = _pattern(A), _pattern(B)
    rows = np.repeat(np.arange(M.nrows), np.diff(np.asarray(M.row_ptr, np.int64)))
    out = []
    for i, j in zip(rows, M.col_idx):
        ks = np.flatnonzero(Ap[i] & Bp[:, j])
        a, b = Ad[i, ks], Bd[ks, j]
        if semiring == "min_plus":
            out.append((a + b).min() if len(ks) else np.inf)
        elif semiring == "max_plus":
            out.append((a + b).max() if len(ks) else -np.inf)
        else:
            out.append(1.0 if np.any((a != 0) & (b != 0)) else 0.0)
    return np.array(out)


@pytest.mark.parametrize("semiring", ["min_plus", "max_plus", "or_and"])
@pytest.mark.parametrize("seed", [0, 1])
def test_semiring_brute_force(oracle_mod, semiring, seed):
    """Integer values in [-3, 3] (stored zeros included, which or-and must
    treat as false), empty rows, mask entries no product reaches."""
    A = gen.random_csr(23, 17, 0.25, seed, values="int", empty_rows=0.2)
    B = gen.random_csr(17, 29, 0.25, seed + 5, values="int", empty_rows=0.2)
    M = gen.random_csr(23, 29, 0.4, seed + 9)
    assert np.array_equal(oracle_mod.masked_semiring(A, B, M, semiring), _semiring_brute(A, B, M, semiring))


def _with_zero_diagonal(d):
    """CSR of the positive weights in d (zero diagonal) plus a stored 0.0 on
    every diagonal entry (a path may stay put at no cost)."""
    n = d.shape[0]
    P = gen.from_dense(d + np.eye(n))
    rows = np.repeat(np.arange(n), np.diff(np.asarray(P.row_ptr, np.int64)))
    return gen.CSR(n, n, P.row_ptr, P.col_idx, np.where(rows == P.col_idx, 0.0, d[rows, P.col_idx]))


def _square_to_fixpoint(oracle_mod, D, semiring):
    """D <- D (x) D over the pattern of D*D until nothing changes (the
    pattern of D*D contains D's because D's diagonal is stored)."""
    for _ in range(20):
        P = oracle_mod.spgemm(D, D)
        vals = oracle_mod.masked_semiring(D, D, P, semiring)
        Dn = gen.CSR(P.nrows, P.ncols, P.row_ptr, P.col_idx, vals)
        if Dn.nnz == D.nnz and np.array_equal(Dn.col_idx, D.col_idx) and np.array_equal(Dn.vals, D.vals):
            return Dn
        D = Dn
    raise AssertionError("no fixpoint")


def test_min_plus_all_pairs_shortest_paths(oracle_mod):
    """Repeated min-plus squaring of the weighted adjacency (zero diagonal)
    reaches the all-pairs shortest-path distances: checked against scipy's
    Dijkstra; pairs outside the final pattern are unreachable there."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    rng = np.random.default_rng(4)
    n = 60
    d = np.zeros((n, n))
    for _ in range(150):
        a, b = rng.integers(0, n, 2)
        if a != b:
            d[a, b] = float(rng.integers(1, 20))
    D = _square_to_fixpoint(oracle_mod, _with_zero_diagonal(d), "min_plus")
    ref = shortest_path(csr_matrix(d), method="D", directed=True)
    got = np.full((n, n), np.inf)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(D.row_ptr, np.int64)))
    got[rows, D.col_idx] = D.vals
    assert np.array_equal(got, ref)


def test_max_plus_longest_paths_in_a_dag(oracle_mod):
    """Repeated max-plus squaring of a DAG's weighted adjacency (zero
    diagonal) gives the longest path between every connected pair: checked
    against dynamic programming over the topological order."""
    rng = np.random.default_rng(7)
    n = 40
    d = np.zeros((n, n))
    edges = []
    for _ in range(90):
        a, b = sorted(rng.integers(0, n, 2))
        if a != b:
            d[a, b] = float(rng.integers(1, 9))
            edges.append((a, b))
    D = _square_to_fixpoint(oracle_mod, _with_zero_diagonal(d), "max_plus")
    best = np.full((n, n), -np.inf)
    for s in range(n):
        best[s, s] = 0.0
        for u in range(s, n):          # vertices in topological (index) order
            if best[s, u] == -np.inf:
                continue
            for v in np.flatnonzero(d[u]):
                best[s, v] = max(best[s, v], best[s, u] + d[u, v])
    got = np.full((n, n), -np.inf)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(D.row_ptr, np.int64)))
    got[rows, D.col_idx] = D.vals
    assert np.array_equal(got, best)


def test_or_and_is_the_boolean_product(oracle_mod):
    """Or-and over the full product pattern: 1 exactly where some product
    has both factors nonzero, i.e. the Boolean matrix product of the
    nonzero patterns."""
    A = gen.random_csr(30, 20, 0.2, 3, values="int")
    B = gen.random_csr(20, 25, 0.2, 4, values="int")
    C = oracle_mod.spgemm(A, B)
    got = oracle_mod.masked_semiring(A, B, C, "or_and")
    boolean = ((_dense(A) != 0).astype(int) @ (_dense(B) != 0).astype(int)) > 0
    rows = np.repeat(np.arange(C.nrows), np.diff(np.asarray(C.row_ptr, np.int64)))
    assert np.array_equal(got, boolean[rows, C.col_idx].astype(float))
