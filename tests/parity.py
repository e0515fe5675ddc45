"""Comparison helpers for GPU-vs-oracle parity (imported by the tests)."""
import numpy as np

from paper_2112_10037_gb300 import gen

# FP64 criterion: |c - c*| <= RTOL_F64 * max(|c*|, sum_k |A(i,k) B(k,j)|).
# With all terms of one sign this is the plain 1e-12 relative bound; the
# sum-of-magnitudes form keeps near-cancelling sums of N(0,1) products from
# failing on a tiny |c*|.
RTOL_F64 = 1e-12
# FP32 values (accumulated in FP32) against the FP64 oracle: a row of m
# products carries at most about m * 2^-24 relative error of the magnitude
# sum; the tests use the bound below for rows of up to a few thousand terms.
RTOL_F32 = 2e-4


def abs_csr(m):
    return gen.CSR(m.nrows, m.ncols, m.row_ptr, m.col_idx, np.abs(np.asarray(m.vals, np.float64)))


def oracle_with_scale(oracle, A, B):
    """Oracle product and the per-entry magnitude sum (the oracle applied to
    |A| and |B|, which has the same pattern)."""
    C = oracle.spgemm(A, B)
    S = oracle.spgemm(abs_csr(A), abs_csr(B))
    return C, S.vals


def assert_structure_equal(got, ref):
    assert got.nrows == ref.nrows and got.ncols == ref.ncols
    assert np.array_equal(np.asarray(got.row_ptr, np.int64), np.asarray(ref.row_ptr, np.int64)), "row_ptr differs"
    assert np.array_equal(np.asarray(got.col_idx, np.int64), np.asarray(ref.col_idx, np.int64)), "col_idx differs"


def max_rel_err(got_vals, ref_vals, scale):
    got = np.asarray(got_vals, np.float64)
    ref = np.asarray(ref_vals, np.float64)
    den = np.maximum(np.abs(ref), np.asarray(scale, np.float64))
    den = np.where(den == 0, 1.0, den)
    return float(np.max(np.abs(got - ref) / den)) if len(ref) else 0.0


def assert_values_close(got_vals, ref_vals, scale, rtol=RTOL_F64):
    err = max_rel_err(got_vals, ref_vals, scale)
    assert err <= rtol, "max relative error %.3e > %.1e" % (err, rtol)
    return err


def assert_values_exact(got_vals, ref_vals):
    assert np.array_equal(np.asarray(got_vals, np.float64), np.asarray(ref_vals, np.float64))


def load_golden(path):
    """Matrices of a text fixture under tests/golden/ (format in the file's
    header): {name: CSR}."""
    mats, cur = {}, None
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("matrix "):
                _, name, m, n = line.split()
                cur = {"name": name, "m": int(m), "n": int(n), "rows": []}
                mats[name] = cur
                continue
            head, _, rest = line.partition(":")
            assert head.split()[0] == "row" and int(head.split()[1]) == len(cur["rows"]), line
            cur["rows"].append([(int(c), float(v)) for c, v in (t.split(":") for t in rest.split())])
    out = {}
    for name, d in mats.items():
        assert len(d["rows"]) == d["m"], name
        rp = np.zeros(d["m"] + 1, np.int32)
        rp[1:] = np.cumsum([len(r) for r in d["rows"]])
        ci = np.array([c for r in d["rows"] for c, _ in r], np.int32)
        v = np.array([x for r in d["rows"] for _, x in r], np.float64)
        out[name] = gen.CSR(d["m"], d["n"], rp, ci, v)
    return out


def stencil3d_square_closed_form(n, rp, ci):
    """Expected values of A*A for the 3D 7-point operator (6 on the
    diagonal, -1 to each face neighbour, Dirichlet) on an n^3 grid, from the
    offset between row and column: 36 + deg(i) on the diagonal (deg = the
    row's face neighbours, 6 in the interior), -12 at distance 1, 2 at the
    diagonal offsets (two paths), 1 at distance 2 along an axis; nnz is the
    sum over the 25 offsets of the in-grid positions."""
    rp = np.asarray(rp, np.int64)
    rows = np.repeat(np.arange(n ** 3, dtype=np.int64), np.diff(rp))
    cols = np.asarray(ci, np.int64)
    def coords(x):
        return x // (n * n), (x // n) % n, x % n
    zi, yi, xi = coords(rows)
    zj, yj, xj = coords(cols)
    d = np.abs(zi - zj) + np.abs(yi - yj) + np.abs(xi - xj)
    axis = (zi == zj).astype(int) + (yi == yj) + (xi == xj)
    deg = sum(((c > 0).astype(np.int64) + (c < n - 1)) for c in (zi, yi, xi))
    exp = np.full(len(rows), np.nan)
    exp[d == 0] = 36 + deg[d == 0]
    exp[d == 1] = -12
    exp[(d == 2) & (axis == 1)] = 2   # two coordinates differ by one
    exp[(d == 2) & (axis == 2)] = 1   # one coordinate differs by two
    return exp


def long_column_matrix(m=600_000, every=50, seed=6):
    """Column 0 set in every `every`-th row (12,000 entries over 600,000
    source rows, so its transpose row spans more than one 262,144-key
    window of the long-row sort), plus one random column in [1, 64) in every
    third row."""
    rng = np.random.default_rng(seed)
    i = np.arange(m)
    c0 = i % every == 0
    c1 = i % 3 == 0
    other = rng.integers(1, 64, size=m)
    counts = c0.astype(np.int64) + c1
    rp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    ci = np.empty(int(rp[-1]), np.int32)
    ci[rp[:-1][c0]] = 0
    ci[(rp[1:] - 1)[c1]] = other[c1]
    return gen.CSR(m, 64, rp, ci, rng.standard_normal(len(ci))).check()
