"""Pins for the oracle's non-symmetric path (pivot-free A = L D U' and the
full Algorithm 1 with step 4): each check compares it with something fixed
independently of the oracle -- numpy's dense inverse, sympy's exact rational
inverse, Usmani's closed form for tridiagonal inverses, the diagonal
similarity that maps upwind convection-diffusion to a symmetric separable
operator, the product L D U' itself, numpy's slogdet and solve.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def lower_pair_from_dense(A):
    """(colptr, rowind, lower, upper) of a matrix with a symmetric pattern."""
    n = A.shape[0]
    mask = (A != 0) | (A.T != 0) | np.eye(n, dtype=bool)
    rows, cols = np.nonzero(np.tril(mask))
    cp, ri, lo = synth.lower_csc_from_coo(n, rows, cols, A[rows, cols])
    c = np.repeat(np.arange(n), np.diff(cp))
    up = A[c, ri]
    return cp, ri, lo, up


def random_unsym(n, density, seed, cplx=False):
    rng = np.random.default_rng(seed)
    mask = np.triu(rng.random((n, n)) < density, 1)
    mask = mask | mask.T
    off = rng.normal(size=(n, n))
    if cplx:
        off = off + 1j * rng.normal(size=(n, n))
    off = off * mask
    diag = np.maximum(np.abs(off).sum(0), np.abs(off).sum(1)) + rng.uniform(0.5, 1.5, n)
    if cplx:
        diag = diag + 1j * rng.uniform(-1, 1, n)
    return off + np.diag(diag)


def entries_on_pattern(Ainv, lcp, lri):
    """(X_ij, X_ji, X_jj) of a dense inverse at the L positions (i, j)."""
    n = len(lcp) - 1
    cols = np.repeat(np.arange(n), np.diff(lcp))
    return Ainv[lri, cols], Ainv[cols, lri], np.diag(Ainv)


def check_against(Ainv, res, tol):
    sym, lv, uv, d, xv, xu, xd, lcp, lri = res
    post = sym["post"]
    Ap = Ainv[np.ix_(post, post)]
    ev, eu, ed = entries_on_pattern(Ap, lcp, lri)
    scale = np.abs(Ainv).max()
    assert np.max(np.abs(xd - ed)) / scale < tol
    if xv.size:
        assert np.max(np.abs(xv - ev)) / scale < tol
        assert np.max(np.abs(xu - eu)) / scale < tol


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("seed", range(10))
def test_lu_tiny_random_vs_dense_inverse(seed, cplx):
    n = 2 + seed % 11
    A = random_unsym(n, 0.35, 300 + seed, cplx)
    # a random relabelling makes some stored entries change sides (flip)
    perm = np.random.default_rng(seed).permutation(n)
    cp0, ri0, lo0, up0 = lower_pair_from_dense(A)
    cp, ri, lo, up, _, flip = synth.permute_lower_unsym(n, cp0, ri0, lo0, up0, perm)
    Ap = A[np.ix_(perm, perm)]
    assert np.array_equal(oracle.dense_from_lower_lu(n, cp, ri, lo, up), Ap)
    Ainv = np.linalg.inv(Ap)
    for wmax, relax, pat in ((0, 0, "exact"), (0, 0, "supernodal"), (3, 1, "supernodal")):
        check_against(Ainv, oracle.selected_inverse_lu(n, cp, ri, lo, up, wmax, relax, pat), 1e-13)


def test_lu_exact_rational_inverse():
    """Integer non-symmetric matrices inverted exactly in rational arithmetic."""
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(11)
    for n in (3, 5, 8):
        mask = np.triu(rng.random((n, n)) < 0.5, 1)
        mask = mask | mask.T
        off = rng.integers(-3, 4, size=(n, n)) * mask
        off[mask & (off == 0)] = 1
        A = off + np.diag(np.maximum(np.abs(off).sum(0), np.abs(off).sum(1)) + rng.integers(1, 3, n))
        exact = sympy.Matrix(A.tolist()).inv()
        Ainv = np.array([[float(exact[i, j]) for j in range(n)] for i in range(n)])
        cp, ri, lo, up = lower_pair_from_dense(A.astype(np.float64))
        check_against(Ainv, oracle.selected_inverse_lu(n, cp, ri, lo, up, 0, 0, "exact"), 1e-14)


def usmani_inverse(b, a, c):
    """Exact inverse entries of tridiagonal T (diagonal b, T_{i+1,i} = a_i,
    T_{i,i+1} = c_i; 0-based lists of Fractions) from Usmani's recurrences:
    theta_i = b_i theta_{i-1} - a_{i-1} c_{i-1} theta_{i-2},
    phi_i = b_i phi_{i+1} - a_i c_i phi_{i+2}, and
    (T^-1)_ij = (-1)^(i+j) c_i..c_{j-1} theta_{i-1} phi_{j+1} / theta_n (i <= j),
    (T^-1)_ij = (-1)^(i+j) a_j..a_{i-1} theta_{j-1} phi_{i+1} / theta_n (i > j).
    Returns (diag, sub = X_{i+1,i}, super = X_{i,i+1})."""
    n = len(b)
    th = [Fraction(1), b[0]]                     # theta_0, theta_1 (1-based)
    for i in range(2, n + 1):
        th.append(b[i - 1] * th[i - 1] - a[i - 2] * c[i - 2] * th[i - 2])
    ph = [Fraction(0)] * (n + 2)
    ph[n + 1] = Fraction(1)
    ph[n] = b[n - 1]
    for i in range(n - 1, 0, -1):
        ph[i] = b[i - 1] * ph[i + 1] - a[i - 1] * c[i - 1] * ph[i + 2]
    det = th[n]
    diag = [th[i - 1] * ph[i + 1] / det for i in range(1, n + 1)]
    sup = [-c[i - 1] * th[i - 1] * ph[i + 2] / det for i in range(1, n)]
    sub = [-a[j - 1] * th[j - 1] * ph[j + 2] / det for j in range(1, n)]
    return diag, sub, sup


def test_lu_tridiagonal_usmani_closed_form():
    rng = np.random.default_rng(5)
    n = 60
    b = [Fraction(int(x)) for x in rng.integers(6, 10, n)]
    a = [Fraction(int(x)) for x in rng.integers(-3, 3, n - 1)]
    c = [Fraction(int(x)) for x in rng.integers(-3, 3, n - 1)]
    a = [x if x != 0 else Fraction(1) for x in a]
    c = [x if x != 0 else Fraction(-1) for x in c]
    diag, sub, sup = usmani_inverse(b, a, c)
    A = np.diag([float(x) for x in b]) + np.diag([float(x) for x in a], -1) + np.diag([float(x) for x in c], 1)
    cp, ri, lo, up = lower_pair_from_dense(A)
    sym, lv, uv, d, xv, xu, xd, lcp, lri = oracle.selected_inverse_lu(n, cp, ri, lo, up, 0, 0, "exact")
    assert np.array_equal(sym["post"], np.arange(n))
    assert np.array_equal(lri, np.arange(1, n, dtype=np.int32))    # L is bidiagonal
    f = lambda xs: np.array([float(x) for x in xs])
    scale = np.abs(f(diag)).max()
    assert np.max(np.abs(xd - f(diag))) / scale < 1e-14
    assert np.max(np.abs(xv - f(sub))) / scale < 1e-14
    assert np.max(np.abs(xu - f(sup))) / scale < 1e-14
    # the pivots telescope: prod d_j = theta_n = det T
    assert abs(oracle.logdet(d)[0] - math.log(abs(float(_det(b, a, c))))) < 1e-12


def _det(b, a, c):
    th0, th1 = Fraction(1), b[0]
    for i in range(1, len(b)):
        th0, th1 = th1, b[i] * th1 - a[i - 1] * c[i - 1] * th0
    return th1


@pytest.mark.parametrize("cplx", [False, True])
def test_ldu_reproduces_A(cplx):
    """L D U' multiplied out equals A on a supernodal pattern (the factor is
    checked directly, not through the inverse)."""
    A = random_unsym(40, 0.1, 77, cplx)
    n = A.shape[0]
    cp, ri, lo, up = lower_pair_from_dense(A)
    sym = oracle.analyse(n, cp, ri, 4, 1)
    post = sym["post"]
    _, _, lo2, up2, _, _ = synth.permute_lower_unsym(n, cp, ri, lo, up, post)
    lcp, lri = oracle.supernodal_pattern(n, sym["sn_start"], sym["rcount"], sym["rrows"])
    lv, uv, d = oracle.ldu(n, sym["colptr"], sym["rowind"], lo2, up2, lcp, lri)
    cols = np.repeat(np.arange(n), np.diff(lcp))
    L = np.eye(n, dtype=lv.dtype)
    L[lri, cols] = lv
    U = np.eye(n, dtype=lv.dtype)
    U[cols, lri] = uv
    Ap = A[np.ix_(post, post)]
    assert np.max(np.abs(L @ np.diag(d) @ U - Ap)) < 1e-13 * np.abs(A).max()


def test_lu_reduces_to_the_symmetric_form_bitwise():
    """On symmetric input the LDU path takes the same operations in the same
    order as the LDL^T path, so the results agree bit for bit."""
    p = synth.grid3d(side=7)
    res_s = oracle.selected_inverse(p.n, p.colptr, p.rowind, p.values, 8, 1)
    res_u = oracle.selected_inverse_lu(p.n, p.colptr, p.rowind, p.values, p.values, 8, 1)
    _, lv, d, xv, xd, _, _ = res_s
    _, lv2, uv2, d2, xv2, xu2, xd2, _, _ = res_u
    assert np.array_equal(lv, lv2) and np.array_equal(lv, uv2) and np.array_equal(d, d2)
    assert np.array_equal(xv, xv2) and np.array_equal(xv, xu2) and np.array_equal(xd, xd2)


def test_convdiff_closed_form_is_the_inverse():
    """Pin the similarity-transformed eigen-expansion itself on a dense inverse."""
    dims, beta, shift = (5, 4, 3), (0.3, -0.2, 0.1), 0.4
    n, cp, ri, lo, up = synth.convdiff_grid(dims, 0, beta_const=beta, shift_const=shift)
    Ainv = np.linalg.inv(oracle.dense_from_lower_lu(n, cp, ri, lo, up))
    rng = np.random.default_rng(9)
    pairs = rng.integers(0, n, size=(60, 2))
    got = oracle.convdiff_inverse_entries(dims, beta, shift, pairs)
    want = Ainv[pairs[:, 0], pairs[:, 1]]
    assert np.max(np.abs(got - want)) < 1e-14 * np.abs(Ainv).max()


def test_lu_oracle_vs_convdiff_closed_form_nd_order():
    """12^3 constant-coefficient convection-diffusion in ND order: every
    selected entry (both triangles) against the closed form."""
    beta, shift = (0.3, 0.2, 0.1), 0.05
    p = synth.convdiff_problem(12, beta_const=beta, shift_const=shift)
    sym, lv, uv, d, xv, xu, xd, lcp, lri = oracle.selected_inverse_lu(
        p.n, p.colptr, p.rowind, p.values, p.values_up, 16, 1)
    # internal index t -> natural node p.perm[sym.post[t]]
    nat = np.asarray(p.perm)[sym["post"]]
    cols = np.repeat(np.arange(p.n), np.diff(lcp))
    rng = np.random.default_rng(4)
    pick = rng.choice(len(lri), size=150, replace=False)
    pr = np.stack([nat[lri[pick]], nat[cols[pick]]], 1)
    want_lo = oracle.convdiff_inverse_entries(p.dims, beta, shift, pr)
    want_up = oracle.convdiff_inverse_entries(p.dims, beta, shift, pr[:, ::-1])
    dg = rng.choice(p.n, size=40, replace=False)
    want_d = oracle.convdiff_inverse_entries(p.dims, beta, shift, np.stack([nat[dg], nat[dg]], 1))
    scale = np.abs(want_d).max()
    assert np.max(np.abs(xv[pick] - want_lo)) / scale < 1e-12
    assert np.max(np.abs(xu[pick] - want_up)) / scale < 1e-12
    assert np.max(np.abs(xd[dg] - want_d)) / scale < 1e-12


@pytest.mark.parametrize("cplx", [False, True])
def test_lu_solve_and_logdet_vs_numpy(cplx):
    A = random_unsym(30, 0.15, 21, cplx)
    n = A.shape[0]
    cp, ri, lo, up = lower_pair_from_dense(A)
    sym, lv, uv, d, xv, xu, xd, lcp, lri = oracle.selected_inverse_lu(n, cp, ri, lo, up, 0, 0, "exact")
    post = sym["post"]
    Ap = A[np.ix_(post, post)]
    rhs = np.random.default_rng(2).normal(size=n)
    x = oracle.solve_lu(n, lcp, lri, lv, uv, d, rhs)
    assert np.max(np.abs(x - np.linalg.solve(Ap, rhs))) < 1e-12
    sign, ld = np.linalg.slogdet(Ap)
    got = oracle.logdet(d)
    assert abs(got[0] - ld) < 1e-11
    if cplx:
        assert abs(np.exp(1j * got[1]) - sign) < 1e-11
    else:
        assert (-1) ** int(got[1]) == sign


def test_lu_zero_pivot_is_reported():
    A = np.array([[1.0, 2.0, 0.0], [3.0, 6.0, 1.0], [0.0, 1.0, 4.0]])   # d_1 = 6 - 3*2 = 0
    cp, ri, lo, up = lower_pair_from_dense(A)
    with pytest.raises(ZeroDivisionError, match="column 1"):
        oracle.selected_inverse_lu(3, cp, ri, lo, up, 0, 0, "exact")
