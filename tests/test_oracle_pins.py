"""Pins for the CPU oracle: every check compares it with something fixed
independently of the oracle (a dense or exact rational inverse, a textbook
closed form, the paper's worked example, brute-force boolean elimination,
numpy's slogdet / solve, finite differences).  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

def lower_from_dense(A):
    n = A.shape[0]
    rows, cols = np.nonzero(np.tril(A != 0) | np.eye(n, dtype=bool))
    return synth.lower_csc_from_coo(n, rows, cols, A[rows, cols])


def random_symmetric(n, density, seed, cplx=False):
    rng = np.random.default_rng(seed)
    mask = np.triu(rng.random((n, n)) < density, 1)
    mask = mask | mask.T
    if cplx:
        off = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    else:
        off = rng.normal(size=(n, n))
    off = np.triu(off, 1)
    off = (off + off.T) * mask
    diag = np.abs(off).sum(1) + rng.uniform(0.5, 1.5, n)
    if cplx:
        diag = diag + 1j * rng.uniform(-1, 1, n)
    return off + np.diag(diag)


def x_on_pattern(Ainv, lcp, lri):
    n = len(lcp) - 1
    cols = np.repeat(np.arange(n), np.diff(lcp))
    return Ainv[lri, cols], np.diag(Ainv)


def rel_err(a, b, scale):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / scale


# --------------------------------------------------------------------------
# values on tiny inputs against dense inverses
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("seed", range(12))
def test_tiny_random_vs_dense_inverse(seed, cplx):
    n = 1 + seed % 12
    A = random_symmetric(n, 0.35, 100 + seed, cplx)
    cp, ri, v = lower_from_dense(A)
    Ainv = np.linalg.inv(A)
    scale = np.abs(Ainv).max()
    for wmax, relax, pat in ((0, 0, "exact"), (0, 0, "supernodal"), (3, 1, "supernodal")):
        sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp, ri, v, wmax, relax, pat)
        post = sym["post"]
        Ap = Ainv[np.ix_(post, post)]
        ev, ed = x_on_pattern(Ap, lcp, lri)
        assert rel_err(xv, ev, scale) < 1e-13 if xv.size else True
        assert rel_err(xd, ed, scale) < 1e-13


def test_exact_rational_inverse():
    """Integer SPD matrices inverted exactly in rational arithmetic."""
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(7)
    for n in (3, 5, 8):
        mask = np.triu(rng.random((n, n)) < 0.5, 1)
        off = -rng.integers(1, 4, size=(n, n)) * mask
        off = off + off.T
        A = off + np.diag(np.abs(off).sum(1) + rng.integers(1, 3, n))
        exact = sympy.Matrix(A.tolist()).inv()
        Ainv = np.array([[float(exact[i, j]) for j in range(n)] for i in range(n)])
        cp, ri, v = lower_from_dense(A.astype(np.float64))
        sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp, ri, v, 0, 0, "exact")
        post = sym["post"]
        ev, ed = x_on_pattern(Ainv[np.ix_(post, post)], lcp, lri)
        scale = np.abs(Ainv).max()
        assert rel_err(xd, ed, scale) < 1e-14
        if xv.size:
            assert rel_err(xv, ev, scale) < 1e-14


# --------------------------------------------------------------------------
# textbook closed forms
# --------------------------------------------------------------------------

def test_laplacian_1d_closed_form_and_linear_work():
    n = 400
    nn, cp, ri, v = synth.laplacian_1d(n)
    sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp, ri, v, 0, 0, "exact")
    T = oracle.laplacian_1d_inverse(n)
    # struct(j) = {j+1}: the etree is a path and L is bidiagonal
    assert np.array_equal(np.diff(lcp), np.r_[np.ones(n - 1, int), 0])
    assert np.array_equal(lri, np.arange(1, n, dtype=np.int32))
    assert np.array_equal(sym["parent"][:-1], np.arange(1, n))
    ev, ed = x_on_pattern(T, lcp, lri)
    assert rel_err(xv, ev, T.max()) < 1e-13
    assert rel_err(xd, ed, T.max()) < 1e-13
    # O(n) work (Section 4.2's tridiagonal remark): sum over supernodes of
    # the algorithmic flop count grows linearly with n.
    s = np.diff(sym["sn_start"]).astype(float)
    r = sym["rcount"].astype(float)
    f = np.sum(2 * r * r * s + 3 * r * s * s + 2 / 3 * s ** 3)
    assert f <= 6 * n


def test_grid_closed_form_is_the_inverse():
    """Pin the separable eigen-expansion itself against a dense inverse."""
    dims = (5, 4, 3)
    n, cp, ri, v = synth.grid_laplacian(dims, 0, 0, 0, shift_const=0.3)
    Ainv = oracle.dense_inverse(n, cp, ri, v)
    rng = np.random.default_rng(3)
    pairs = rng.integers(0, n, size=(40, 2))
    got = oracle.grid_inverse_entries(dims, 0.3, pairs)
    want = Ainv[pairs[:, 0], pairs[:, 1]]
    assert np.max(np.abs(got - want)) < 1e-14


def test_oracle_vs_grid_closed_form_nd_order():
    """31x31 grid (the smallest workload's shape) with a constant shift."""
    p = synth.grid2d_31(shift_const=0.55)
    sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(p.n, p.colptr, p.rowind, p.values,
                                                           0, 0, "supernodal")
    assert np.array_equal(sym["post"], np.arange(p.n))
    cols = np.repeat(np.arange(p.n), np.diff(lcp))
    rng = np.random.default_rng(11)
    pick = rng.choice(len(lri), 300, replace=False)
    pairs = np.stack([p.perm[lri[pick]], p.perm[cols[pick]]], 1)
    want = oracle.grid_inverse_entries(p.dims, 0.55, pairs)
    wd = oracle.grid_inverse_entries(p.dims, 0.55, np.stack([p.perm[:50], p.perm[:50]], 1))
    scale = np.abs(xd).max()
    assert rel_err(xv[pick], want, scale) < 1e-13
    assert rel_err(xd[:50], wd, scale) < 1e-13


# --------------------------------------------------------------------------
# symbolic analysis
# --------------------------------------------------------------------------

def brute_force_pattern(Apat):
    """Boolean Gaussian elimination: the exact fill pattern of L."""
    M = Apat.copy()
    n = M.shape[0]
    for k in range(n):
        nz = np.nonzero(M[k + 1:, k])[0] + k + 1
        M[np.ix_(nz, nz)] = True
    return np.tril(M, -1)


@pytest.mark.parametrize("seed", range(10))
def test_symbolic_vs_brute_force(seed):
    n = 6 + 3 * seed
    A = random_symmetric(n, 0.15, 500 + seed)
    cp, ri, v = lower_from_dense(A)
    parent, lcp, lri = oracle.column_structure(n, cp, ri)
    Lpat = brute_force_pattern(A != 0)
    cols = np.repeat(np.arange(n), np.diff(lcp))
    got = np.zeros((n, n), bool)
    got[lri, cols] = True
    assert np.array_equal(got, Lpat)
    for j in range(n):
        below = np.nonzero(Lpat[:, j])[0]
        assert parent[j] == (below.min() if below.size else -1)


def test_postorder_of_random_forest():
    rng = np.random.default_rng(5)
    n = 200
    parent = np.array([rng.integers(j + 1, n) if j < n - 1 and rng.random() < 0.9 else -1
                       for j in range(n)], np.int32)
    post = oracle.postorder(parent)
    assert np.array_equal(np.sort(post), np.arange(n))
    pos = np.empty(n, int)
    pos[post] = np.arange(n)
    # every subtree occupies a contiguous range ending at its root
    size = np.ones(n, int)
    for j in range(n):
        if parent[j] >= 0:
            size[parent[j]] += size[j]
    for j in range(n):
        members = [j]
        stack = [j]
        while stack:
            u = stack.pop()
            ch = np.nonzero(parent == u)[0]
            members.extend(ch)
            stack.extend(ch)
        assert sorted(pos[members]) == list(range(pos[j] - size[j] + 1, pos[j] + 1))


def _read_fig1():
    part, blocks, fill, snp, levels = None, [], [], None, []
    with open(os.path.join(GOLDEN, "fig1_worked_example.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            key, *rest = line.split()
            if key == "partition":
                part = np.array(list(map(int, rest)), np.int32)
            elif key in ("A", "fill"):
                br, bc, _, *rows = rest
                (blocks if key == "A" else fill).append((int(br), int(bc), list(map(int, rows))))
            elif key == "sn_parent":
                snp = list(map(int, rest))
            elif key == "level":
                levels.append(set(map(int, rest)))
    return part, blocks, fill, snp, levels


def test_figure1_worked_example():
    part, blocks, fill, snp, levels = _read_fig1()
    n = int(part[-1])
    M = np.zeros((n, n), bool)
    for k in range(len(part) - 1):
        M[part[k]:part[k + 1], part[k]:part[k + 1]] = True
    for br, bc, rows in blocks:
        M[np.ix_(rows, range(part[bc - 1], part[bc]))] = True
    M = M | M.T
    cp, ri, v = lower_from_dense(np.where(M, 1.0, 0.0))
    parent, lcp, lri = oracle.column_structure(n, cp, ri)
    cols = np.repeat(np.arange(n), np.diff(lcp))
    L = np.zeros((n, n), bool)
    L[lri, cols] = True
    fillpos = L & ~np.tril(M, -1)
    want = np.zeros((n, n), bool)
    for br, bc, rows in fill:
        want[np.ix_(rows, range(part[bc - 1], part[bc]))] = True
    assert np.array_equal(fillpos, want)          # only block (10,8), rows 25, 26, 28
    snp_got, sigma, rc, rr = oracle.sn_struct(n, lcp, lri, part)
    assert list(snp_got[:-1] + 1) == snp and snp_got[-1] == -1
    got_levels = [set(np.nonzero(sigma == k)[0] + 1) for k in range(1, sigma.max() + 1)]
    assert got_levels == levels
    # the figure's partition is not the fundamental one: 9 and 10 chain up
    fund = oracle.supernodes(parent, lcp, 0, 0)
    assert 23 in fund and 25 not in fund


def test_supernode_rule_properties():
    p = synth.grid3d(side=10)
    parent, lcp, lri = oracle.column_structure(p.n, p.colptr, p.rowind)
    cnt = np.diff(lcp)
    fund = oracle.supernodes(parent, lcp, 0, 0)
    for k in range(len(fund) - 1):
        f, l = fund[k], fund[k + 1]
        for j in range(f, l - 1):           # identical structure below the block
            sj = set(lri[lcp[j]:lcp[j + 1]])
            assert sj == {j + 1} | set(lri[lcp[j + 1]:lcp[j + 2]])
        if l < p.n:                          # maximal
            nxt = l
            ok = (parent[l - 1] == nxt and np.sum(parent == nxt) == 1
                  and cnt[l - 1] == cnt[nxt] + 1)
            assert not ok
    for wmax in (4, 16, 64):
        sn = oracle.supernodes(parent, lcp, wmax, 1)
        w = np.diff(sn)
        assert w.max() <= wmax
        # merging only removes fundamental boundaries; a boundary that is not a
        # fundamental one comes from the split, a multiple of wmax after the
        # first column of its merged supernode
        fset = set(fund.tolist())
        starts = [b for b in sn.tolist() if b in fset]
        for b in sn.tolist():
            if b not in fset:
                a = max(x for x in starts if x < b)
                assert (b - a) % wmax == 0, (wmax, a, b)
        snp, sig, rc, rr = oracle.sn_struct(p.n, lcp, lri, sn)
        roff = np.r_[0, np.cumsum(rc)]
        for k in range(len(sn) - 1):
            f, l = sn[k], sn[k + 1]
            R = rr[roff[k]:roff[k + 1]]
            # closure: R(K) is the structure of K's last column
            assert np.array_equal(R, lri[lcp[l - 1]:lcp[l]])
            s = l - f
            stored = s * (s + 1) // 2 + s * len(R)
            true = np.sum(1 + cnt[f:l])
            # every stored panel is either narrow or has at most 5% zeros,
            # unless it is a piece of a split fundamental supernode
            inside_fund = np.searchsorted(fund, f, "right") == np.searchsorted(fund, l - 1, "right")
            assert s <= 8 or 20 * (stored - true) <= stored or inside_fund


def test_relative_indices_definition():
    p = synth.grid3d(side=9)
    sym = oracle.analyse(p.n, p.colptr, p.rowind, 16, 1)
    sn, rc, rr, rel = sym["sn_start"], sym["rcount"], sym["rrows"], sym["relidx"]
    col2sn = np.repeat(np.arange(len(sn) - 1), np.diff(sn))
    roff = np.r_[0, np.cumsum(rc)]
    t = 0
    for k in range(len(sn) - 1):
        C = rr[roff[k]:roff[k + 1]]
        p0 = 0
        nb = 0
        while p0 < len(C):
            J = col2sn[C[p0]]
            q = p0
            while q < len(C) and col2sn[C[q]] == J:
                q += 1
            rowsJ = np.r_[np.arange(sn[J], sn[J + 1]), rr[roff[J]:roff[J + 1]]]
            seg = rel[t:t + len(C) - p0]
            assert np.array_equal(rowsJ[seg], C[p0:])
            t += len(C) - p0
            p0 = q
            nb += 1
        assert sym["nblk"][k] == nb
    assert t == len(rel)


# --------------------------------------------------------------------------
# logdet, solves, trace identity, adjoint formula
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cplx", [False, True])
def test_logdet_vs_slogdet(cplx):
    A = random_symmetric(60, 0.1, 42, cplx)
    cp, ri, v = lower_from_dense(A)
    sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(60, cp, ri, v, 0, 0, "exact")
    got = oracle.logdet(d)
    sign, ld = np.linalg.slogdet(A)
    assert abs(got[0] - ld) < 1e-11 * abs(ld)
    if cplx:
        # imaginary part modulo 2 pi
        diff = (got[1] - np.angle(sign) + np.pi) % (2 * np.pi) - np.pi
        assert abs(diff) < 1e-10
    else:
        assert got[1] == 0


@pytest.mark.parametrize("cplx", [False, True])
def test_solve_vs_numpy(cplx):
    A = random_symmetric(40, 0.15, 9, cplx)
    cp, ri, v = lower_from_dense(A)
    sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(40, cp, ri, v, 0, 0, "exact")
    b = np.random.default_rng(1).normal(size=40)
    post = sym["post"]
    x = oracle.solve(40, lcp, lri, lv, d, b[post])
    want = np.linalg.solve(A, b)[post]
    assert np.max(np.abs(x - want)) < 1e-13 * np.max(np.abs(want))


def test_trace_identity_grid2d_31():
    p = synth.grid2d_31()
    sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(p.n, p.colptr, p.rowind, p.values,
                                                           0, 0, "exact")
    # X at A's positions: diagonal from xd, off-diagonals looked up in the L pattern
    cols = np.repeat(np.arange(p.n), np.diff(p.colptr))
    lcols = np.repeat(np.arange(p.n), np.diff(lcp))
    keys = lcols.astype(np.int64) * p.n + lri
    xa = np.empty(p.nnz)
    dg = p.rowind == cols
    xa[dg] = xd[cols[dg]]
    pos = np.searchsorted(keys, cols[~dg].astype(np.int64) * p.n + p.rowind[~dg])
    xa[~dg] = xv[pos]
    assert oracle.trace_error(p.n, p.colptr, p.rowind, p.values, xa) < 1e-13


def test_dense_adjoint_against_finite_differences():
    """d/dt <G, P_S(A(t)^{-1})> along symmetric directions."""
    n = 7
    A = random_symmetric(n, 0.4, 77)
    cp, ri, v = lower_from_dense(A)
    parent, lcp, lri = oracle.column_structure(n, cp, ri)
    S = np.eye(n, dtype=bool)
    cols = np.repeat(np.arange(n), np.diff(lcp))
    S[lri, cols] = True
    S = S | S.T
    rng = np.random.default_rng(2)
    G = rng.normal(size=(n, n))
    G = (G + G.T) * S
    J = lambda M: np.sum(G * np.linalg.inv(M))
    grad = oracle.dense_adjoint(np.linalg.inv(A), G)
    h = 1e-6
    for p, q in [(0, 0), (3, 3)] + [tuple(x) for x in np.argwhere(np.tril(A != 0, -1))[:4]]:
        E = np.zeros((n, n))
        E[p, q] = E[q, p] = 1.0
        fd = (J(A + h * E) - J(A - h * E)) / (2 * h)
        want = grad[p, q] * (1 if p == q else 2)
        assert abs(fd - want) < 1e-7 * max(1.0, abs(want))


def test_complex_config_small_pole_block_matrix():
    """A 2x2x2-element DG-like block matrix: complex-symmetric shifts against
    the dense inverse on the supernodal pattern."""
    n, cp, ri, hv, z = synth.dg_block_matrix((2, 2, 2), 6, 3, seed=5)
    vals = synth.shifted_values(n, cp, ri, hv, z)
    perm = synth.block_nd_order((2, 2, 2), 6)
    cp2, ri2, v2, _ = synth.permute_lower(n, cp, ri, vals, perm)
    for l in range(3):
        Ainv = oracle.dense_inverse(n, cp2, ri2, v2[l])
        sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp2, ri2, v2[l], 8, 1)
        post = sym["post"]
        ev, ed = x_on_pattern(Ainv[np.ix_(post, post)], lcp, lri)
        scale = np.abs(Ainv).max()
        assert rel_err(xv, ev, scale) < 1e-13
        assert rel_err(xd, ed, scale) < 1e-13


@pytest.mark.parametrize("cplx", [False, True])
def test_panel_layouts_against_the_dense_inverse(cplx):
    """``panels_from_columns`` (column-form X of the sweep) and
    ``panels_from_dense`` (numpy's dense inverse) lay X out on the same
    supernodal panels: a wrong row, column or mirror index in either would
    make them differ.  Relaxed supernodes of width <= 4, so the diagonal
    blocks hold entries mirrored above the diagonal."""
    n = 40
    A = random_symmetric(n, 0.15, 321, cplx)
    cp, ri, v = lower_from_dense(A)
    sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp, ri, v, 4, 1, "supernodal")
    post = sym["post"]
    Ap = np.linalg.inv(A)[np.ix_(post, post)]
    off, Xc = oracle.panels_from_columns(n, sym["sn_start"], sym["rcount"], sym["rrows"], lcp, xv, xd)
    Xd = oracle.panels_from_dense(sym, Ap)
    assert off[-1] == Xd.size
    assert np.max(np.abs(np.diff(sym["sn_start"]))) > 1          # some supernode has a mirrored block
    assert rel_err(Xc, Xd, np.abs(Ap).max()) < 1e-13
