"""Edge cases of the non-symmetric and the Bunch-Kaufman paths on the GPU:
order 1, diagonal and dense matrices, batches sharing a pattern, uneven
batches, and the pivoted factor of one dense block against LAPACK's
Bunch-Kaufman (scipy.linalg.ldl).  Tolerance 1e-10 of max |X|."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1404_0447_gb300 as P
    return P


def dev(v):
    import torch
    v = np.ascontiguousarray(v)
    return torch.tensor(v, dtype=torch.complex128 if np.iscomplexobj(v) else torch.float64, device="cuda")


def lower_pair(A):
    """(colptr, rowind, lower, upper) of a matrix with a symmetric pattern."""
    n = A.shape[0]
    mask = (A != 0) | (A.T != 0) | np.eye(n, dtype=bool)
    rows, cols = np.nonzero(np.tril(mask))
    cp, ri, lo = synth.lower_csc_from_coo(n, rows, cols, A[rows, cols])
    c = np.repeat(np.arange(n), np.diff(cp))
    return cp, ri, lo, A[c, ri]


def unsym_random(n, density, seed):
    rng = np.random.default_rng(seed)
    mask = np.triu(rng.random((n, n)) < density, 1)
    mask = mask | mask.T
    off = rng.normal(size=(n, n)) * mask
    return off + np.diag(np.maximum(np.abs(off).sum(0), np.abs(off).sum(1)) + rng.uniform(0.5, 1.5, n))


def check_unsym_dense(P, A, **opts):
    n = A.shape[0]
    cp, ri, lo, up = lower_pair(A)
    h = P.SelInv(n, cp, ri, unsym=1, **opts)
    h.factor_unsym(dev(lo), dev(up))
    h.selinv(P.LEVEL)
    Xi = np.linalg.inv(A)
    c = np.repeat(np.arange(n), np.diff(cp))
    s = np.abs(Xi).max()
    assert np.max(np.abs(h.selected()[0].cpu().numpy() - Xi[ri, c])) / s <= TOL
    assert np.max(np.abs(h.selected_upper()[0].cpu().numpy() - Xi[c, ri])) / s <= TOL


@pytest.mark.parametrize("case", ["order1", "diagonal", "dense40", "dense200", "sparse300"])
def test_unsym_shapes(P, case):
    if case == "order1":
        A = np.array([[3.0]])
    elif case == "diagonal":
        A = np.diag(np.random.default_rng(0).uniform(1, 2, 50))
    elif case == "dense40":
        A = unsym_random(40, 1.0, 1)
    elif case == "dense200":
        A = unsym_random(200, 1.0, 2)          # one dense block split into supernodes of <= 128
    else:
        A = unsym_random(300, 0.02, 3)
    check_unsym_dense(P, A)


def test_unsym_batch_sharing_a_pattern(P):
    p = synth.convdiff_problem(dims=(9, 8, 7))
    rng = np.random.default_rng(4)
    B = 3
    lo = np.stack([p.values * (1 + 0.1 * b) + 0.05 * rng.uniform(size=p.nnz) * (b > 0) for b in range(B)])
    up = np.stack([p.values_up * (1 + 0.1 * b) for b in range(B)])
    diag = np.asarray(p.colptr[:-1])
    lo[:, diag] += 1.0
    h = P.SelInv(p.n, p.colptr, p.rowind, unsym=1, batch=B)
    h.factor_unsym(dev(lo.ravel()), dev(up.ravel()))
    h.selinv(P.LEVEL)
    sel = h.selected().cpu().numpy()
    selu = h.selected_upper().cpu().numpy()
    c = np.repeat(np.arange(p.n), np.diff(p.colptr))
    for b in range(B):
        Xi = np.linalg.inv(oracle.dense_from_lower_lu(p.n, p.colptr, p.rowind, lo[b], up[b]))
        s = np.abs(Xi).max()
        assert np.max(np.abs(sel[b] - Xi[p.rowind, c])) / s <= TOL
        assert np.max(np.abs(selu[b] - Xi[c, p.rowind])) / s <= TOL


def test_unsym_uneven_batch(P):
    mats = [unsym_random(n, 0.05, 10 + n) for n in (30, 1, 75, 140)]
    pairs = [lower_pair(A) for A in mats]
    h = P.SelInv([A.shape[0] for A in mats], [q[0] for q in pairs], [q[1] for q in pairs], unsym=1)
    h.factor_unsym(dev(np.concatenate([q[2] for q in pairs])), dev(np.concatenate([q[3] for q in pairs])))
    h.selinv(P.GRAPH)
    sel = h.selected()[0].cpu().numpy()
    selu = h.selected_upper()[0].cpu().numpy()
    off = 0
    for A, (cp, ri, lo, up) in zip(mats, pairs):
        n = A.shape[0]
        Xi = np.linalg.inv(A)
        c = np.repeat(np.arange(n), np.diff(cp))
        s = np.abs(Xi).max()
        assert np.max(np.abs(sel[off:off + len(ri)] - Xi[ri, c])) / s <= TOL
        assert np.max(np.abs(selu[off:off + len(ri)] - Xi[c, ri])) / s <= TOL
        off += len(ri)


def dense_sym_lower(A):
    n = A.shape[0]
    rows, cols = np.nonzero(np.tril(np.ones((n, n), bool)))
    return synth.lower_csc_from_coo(n, rows, cols, A[rows, cols])


@pytest.mark.parametrize("A", [np.array([[-2.0]]), np.array([[0.0, 1.0], [1.0, 0.0]]),
                               np.array([[0.0, 2.0, 0.0], [2.0, 0.0, 1.0], [0.0, 1.0, 0.0]]) + 1e-3 * np.eye(3)])
def test_bk_tiny(P, A):
    n = A.shape[0]
    cp, ri, v = dense_sym_lower(A)
    h = P.SelInv(n, cp, ri)
    h.factor_bk(dev(v))
    h.selinv(P.LEVEL)
    Xi = np.linalg.inv(A)
    c = np.repeat(np.arange(n), np.diff(cp))
    assert np.max(np.abs(h.selected()[0].cpu().numpy() - Xi[ri, c])) / np.abs(Xi).max() <= TOL


@pytest.mark.parametrize("cplx", [False, True])
def test_bk_dense_block_matches_lapack_pivots(P, cplx):
    """One supernode of width 128: the GPU's interchanges and 1x1/2x2 choices
    equal LAPACK's Bunch-Kaufman on the same block."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(7)
    n = 128
    A = rng.normal(size=(n, n))
    if cplx:
        A = A + 1j * rng.normal(size=(n, n))
    A = A + A.T
    cp, ri, v = dense_sym_lower(A)
    h = P.SelInv(n, cp, ri, dtype=P.C128 if cplx else P.F64)
    assert h.info["nsn"] == 1
    h.factor_bk(dev(v))
    piv, ty = h.pivots()
    lu, d, perm = scipy_linalg.ldl(A, lower=True, hermitian=False)
    assert np.array_equal(piv[0], perm)
    two = np.abs(np.diag(d, -1)) > 0
    assert np.array_equal(ty[0][:-1] == 1, two)
    h.selinv(P.LEVEL)
    c = np.repeat(np.arange(n), np.diff(cp))
    sel = h.selected()[0].cpu().numpy()
    _, Xo, _ = oracle.selected_inverse_bk(n, cp, ri, v, 128, 1)     # same pivots (checked above)
    assert np.max(np.abs(sel - Xo[ri, c])) / np.abs(Xo).max() <= TOL
    Xi = np.linalg.inv(A)                                            # sanity: the inverse itself
    assert np.max(np.abs(sel - Xi[ri, c])) / np.abs(Xi).max() <= 1e-9


def test_bk_uneven_batch(P):
    rng = np.random.default_rng(9)
    mats = []
    for n in (20, 64, 3):
        A = rng.normal(size=(n, n)); A = A + A.T
        mats.append(A)
    low = [dense_sym_lower(A) for A in mats]
    h = P.SelInv([A.shape[0] for A in mats], [q[0] for q in low], [q[1] for q in low])
    h.factor_bk(dev(np.concatenate([q[2] for q in low])))
    h.selinv(P.PERSISTENT)
    h.sync_status()
    sel = h.selected()[0].cpu().numpy()
    off = 0
    for A, (cp, ri, v) in zip(mats, low):
        n = A.shape[0]
        c = np.repeat(np.arange(n), np.diff(cp))
        _, Xo, _ = oracle.selected_inverse_bk(n, cp, ri, v, 128, 1)
        assert np.max(np.abs(sel[off:off + len(ri)] - Xo[ri, c])) / np.abs(Xo).max() <= TOL
        Xi = np.linalg.inv(A)                                        # sanity: the inverse itself
        assert np.max(np.abs(sel[off:off + len(ri)] - Xi[ri, c])) / np.abs(Xi).max() <= 1e-9
        off += len(ri)
