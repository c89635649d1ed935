"""Pins for the oracle's symmetric-indefinite path (Bunch-Kaufman 1x1/2x2
pivots inside supernodes, then the selected inversion): the block
factorisation against LAPACK's Bunch-Kaufman (scipy.linalg.ldl, xSYTRF),
the selected inverse against numpy's dense inverse on indefinite grids, a
saddle-point matrix the pivot-free path cannot factor, the reduction to the
pivot-free path on diagonally dominant matrices, and slogdet.  CPU only."""
import numpy as np
import pytest

import oracle
import synth


def sym_random(n, seed, cplx=False):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n))
    if cplx:
        A = A + 1j * rng.normal(size=(n, n))
    return A + A.T


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 2, 7, 33, 96, 128])
def test_bk_block_matches_lapack_bunch_kaufman(n, cplx):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    A = sym_random(n, 1000 + n, cplx)
    p, L, d, e, pt = oracle.bk_block(A)
    D = oracle.block_d(d, e, pt)
    lu, dd, perm = scipy_linalg.ldl(A, lower=True, hermitian=False)
    assert np.array_equal(perm, p)                     # same interchanges, same 1x1/2x2 choices
    assert np.max(np.abs(dd - D)) <= 1e-12 * np.abs(A).max()
    assert np.max(np.abs(lu[perm] - L)) <= 1e-12
    assert np.max(np.abs(A[np.ix_(p, p)] - L @ D @ L.T)) <= 1e-12 * np.abs(A).max()
    if n >= 33:
        assert (pt == 1).any()                         # 2x2 pivots are exercised


def indefinite_grid(dims, shift, cplx=False):
    n, cp, ri, v = synth.grid_laplacian(dims, 0, 0, 0, shift_const=shift)
    if cplx:
        v = v + 0.05j * (np.asarray(ri) == np.repeat(np.arange(n), np.diff(cp)))
    return synth.Problem("ind", n, cp, ri, v, synth.nd_order(dims))


def check_vs_dense(p, wmax, relax, tol):
    sym, X, fac = oracle.selected_inverse_bk(p.n, p.colptr, p.rowind, p.values, wmax, relax)
    post = sym["post"]
    A = oracle.dense_from_lower(p.n, p.colptr, p.rowind, p.values)
    Ai = np.linalg.inv(A)[np.ix_(post, post)]
    lcp, lri = oracle.supernodal_pattern(p.n, sym["sn_start"], sym["rcount"], sym["rrows"])
    cols = np.repeat(np.arange(p.n), np.diff(lcp))
    scale = np.abs(Ai).max()
    assert np.max(np.abs(X[lri, cols] - Ai[lri, cols])) / scale <= tol
    assert np.max(np.abs(np.diag(X) - np.diag(Ai))) / scale <= tol
    return sym, X, fac, A


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("dims,shift", [((7, 6, 5), -2.5), ((9, 8), -1.7), ((5, 5, 4), -4.1)])
def test_bk_selected_inverse_vs_dense_on_indefinite_grids(dims, shift, cplx):
    p = indefinite_grid(dims, shift, cplx)
    n2x2 = 0
    for wmax, relax in ((0, 0), (16, 1), (128, 1)):
        sym, X, fac, A = check_vs_dense(p, wmax, relax, 1e-11)
        n2x2 += sum(int((F["ptype"] == 1).sum()) for F in fac)
    if not cplx:
        assert n2x2 > 0                                             # 2x2 pivots occurred
    ld = oracle.logdet_bk(fac)
    sign, ld0 = np.linalg.slogdet(A)
    assert abs(ld[0] - ld0) <= 1e-10 * max(1.0, abs(ld0))
    if cplx:
        assert abs(np.exp(1j * ld[1]) - sign) <= 1e-9
    else:
        assert (-1) ** int(ld[1]) == sign


def test_bk_factors_a_saddle_point_matrix_the_pivot_free_path_cannot():
    """[[H, B^T], [B, 0]] with the constraint rows interleaved inside one
    supernode: exact zero pivots stop the pivot-free LDL^T; 2x2 pivots do not."""
    rng = np.random.default_rng(3)
    m, k = 6, 3
    H = rng.normal(size=(m, m)); H = H @ H.T + m * np.eye(m)
    B = rng.normal(size=(k, m))
    K = np.block([[H, B.T], [B, np.zeros((k, k))]])
    order = np.array([6, 0, 1, 7, 2, 3, 8, 4, 5])      # a zero-diagonal row first
    A = K[np.ix_(order, order)]
    n = A.shape[0]
    rows, cols = np.nonzero(np.tril(np.ones((n, n), bool)))
    cp, ri, v = synth.lower_csc_from_coo(n, rows, cols, A[rows, cols])
    with pytest.raises(ZeroDivisionError):
        oracle.selected_inverse(n, cp, ri, v, 16, 1)
    p = synth.Problem("kkt", n, cp, ri, v, np.arange(n))
    sym, X, fac, _ = check_vs_dense(p, 16, 1, 1e-12)
    F = fac[0]
    assert len(fac) == 1 and ((F["ptype"] == 1).any() or not np.array_equal(F["p"], np.arange(n)))


def test_bk_on_diagonally_dominant_matrices_takes_no_pivoting_steps():
    p = synth.grid3d(side=6)
    sym, X, fac = oracle.selected_inverse_bk(p.n, p.colptr, p.rowind, p.values, 8, 1)
    assert all(np.array_equal(F["p"], np.arange(len(F["p"]))) and not F["ptype"].any() for F in fac)
    sym2, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(p.n, p.colptr, p.rowind, p.values, 8, 1)
    cols = np.repeat(np.arange(p.n), np.diff(lcp))
    assert np.max(np.abs(X[lri, cols] - xv)) <= 1e-14 * np.abs(xd).max()
    assert np.max(np.abs(np.diag(X) - xd)) <= 1e-14 * np.abs(xd).max()
