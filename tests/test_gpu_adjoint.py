"""The hand-written adjoint of the selected inversion (and of the LDL^T),
through the C ABI, against the dense-gradient formula -(X G X) on A's
pattern (oracle definitions, numpy dense inverse) and against central
finite differences.  Gradients are with respect to the stored lower-CSC
values: -(XGX)_jj on the diagonal, -2 (XGX)_ij off it."""
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


def panel_positions(sym):
    """(rows, cols) in internal numbering of every panel entry, panel order."""
    rows, cols = [], []
    for k in range(sym["nsn"]):
        f, l = sym["sn_start"][k], sym["sn_start"][k + 1]
        R = sym["rows"][sym["rowptr"][k]:sym["rowptr"][k + 1]]
        prow = np.r_[np.arange(f, l), R]
        for c in range(l - f):
            rows.append(prow)
            cols.append(np.full(prow.size, f + c))
    return np.concatenate(rows), np.concatenate(cols)


def dense_G_from_panels(n, sym, gpan, rows, cols):
    """Symmetric dense G from the lower panel entries (rows >= cols)."""
    G = np.zeros((n, n), dtype=gpan.dtype)
    low = rows >= cols
    G[rows[low], cols[low]] = gpan[low]
    G[cols[low], rows[low]] = gpan[low]
    return G


def expected_grad(n, cp, ri, A_user, G_int, perm):
    """dJ/d(stored values), J = <G, A^{-1}>, in user order."""
    Ainv = np.linalg.inv(A_user)
    Gu = np.zeros_like(G_int)
    Gu[np.ix_(perm, perm)] = G_int                      # internal -> user numbering
    XGX = Ainv @ Gu @ Ainv
    cols = np.repeat(np.arange(n), np.diff(cp))
    g = -XGX[ri, cols]
    return np.where(ri == cols, g, 2 * g)


def run_case(P, n, cp, ri, vals, perm=None, wmax=16, cplx=False, seed=0):
    import torch
    dt = torch.complex128 if cplx else torch.float64
    h = P.SelInv(n, cp, ri, perm=perm, max_sn_width=wmax, dtype=P.C128 if cplx else P.F64)
    h.factor(torch.tensor(vals, dtype=dt, device="cuda"))
    h.selinv(P.LEVEL)
    sym = h.symbolic()
    rows, cols = panel_positions(sym)
    rng = np.random.default_rng(seed)
    gpan = rng.normal(size=rows.size) + (1j * rng.normal(size=rows.size) if cplx else 0)
    grad = h.adjoint(torch.tensor(gpan, dtype=dt, device="cuda"))[0].cpu().numpy()
    G = dense_G_from_panels(n, sym, gpan, rows, cols)
    A = oracle.dense_from_lower(n, cp, ri, vals)
    want = expected_grad(n, cp, ri, A, G, sym["perm"])
    err = np.max(np.abs(grad - want)) / np.max(np.abs(want))
    assert err <= TOL, err
    return h


def test_adjoint_random_pattern_with_permutation(P):
    rng = np.random.default_rng(21)
    n = 160
    mask = np.triu(rng.random((n, n)) < 0.04, 1)
    r_, c_ = np.nonzero(mask.T)
    off = rng.normal(size=r_.size)
    diag = np.bincount(r_, np.abs(off), n) + np.bincount(c_, np.abs(off), n) + rng.uniform(0.5, 1.5, n)
    cp, ri, v = synth.lower_csc_from_coo(n, np.r_[np.arange(n), r_], np.r_[np.arange(n), c_], np.r_[diag, off])
    run_case(P, n, cp, ri, v, perm=rng.permutation(n), wmax=8)


@pytest.mark.parametrize("side,wmax", [(9, 16), (11, 128)])
def test_adjoint_3d_grid(P, side, wmax):
    p = synth.grid_problem((side, side, side - 2), 0.01, 0.1, 9)
    run_case(P, p.n, p.colptr, p.rowind, p.values, wmax=wmax)


def test_adjoint_bitwise_reproducible(P):
    """Two adjoint sweeps with the same seed give bitwise the same gradient:
    the scatter of -(Yb Lhat^T + Lhat Yb^T) into the ancestors runs per
    group of supernodes with disjoint targets, without atomics."""
    import torch
    p = synth.grid3d(side=18)
    h = P.SelInv(p.n, p.colptr, p.rowind)
    h.factor(torch.tensor(p.values, dtype=torch.float64, device="cuda"))
    h.selinv(P.LEVEL)
    G = torch.randn(h.info["panel_entries"], dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(7))
    g1 = h.adjoint(G)[0].clone()
    g2 = h.adjoint(G)[0]
    assert torch.equal(g1, g2)


def test_adjoint_dense_single_supernode_and_split(P):
    rng = np.random.default_rng(4)
    n = 200
    G = rng.normal(size=(n, n))
    A = G @ G.T / n + np.eye(n)
    rows, cols = np.tril_indices(n)
    cp, ri, v = synth.lower_csc_from_coo(n, rows, cols, A[rows, cols])
    run_case(P, n, cp, ri, v, wmax=128)


def test_adjoint_complex_symmetric_poles(P):
    n, cp, ri, hv, z = synth.dg_block_matrix((3, 3, 2), 6, 1, seed=3)
    perm = synth.block_nd_order((3, 3, 2), 6)
    vals = synth.shifted_values(n, cp, ri, hv, z)[0]
    cp2, ri2, v2, _ = synth.permute_lower(n, cp, ri, vals, perm)
    run_case(P, n, cp2, ri2, v2, wmax=12, cplx=True)


def test_selected_inverse_autograd_against_finite_differences(P):
    """J(theta) = sum_e W_e X_e over the X panels of the graph Laplacian
    A(theta); autograd through pselinv_selinv_adjoint vs central differences."""
    import torch
    gl = synth.GraphLaplacian((7, 6, 5), seed=8)
    perm = synth.nd_order(gl.dims)
    h = P.SelInv(gl.n, gl.colptr, gl.rowind, perm=perm, max_sn_width=16)
    theta = torch.tensor(gl.theta, dtype=torch.float64, device="cuda", requires_grad=True)
    W = torch.tensor(np.random.default_rng(1).normal(size=h.info["panel_entries"]), device="cuda")
    J = lambda t: (P.selected_inverse(gl.assemble_torch(t).unsqueeze(0), h)[0] * W).sum()
    J(theta).backward()
    g = theta.grad.cpu().numpy()
    hstep = 1e-6
    with torch.no_grad():
        for e in np.random.default_rng(2).choice(gl.ei.size, 8, replace=False):
            tp = theta.detach().clone(); tp[e] += hstep
            tm = theta.detach().clone(); tm[e] -= hstep
            fd = (J(tp).item() - J(tm).item()) / (2 * hstep)
            assert abs(fd - g[e]) <= 1e-6 * max(1.0, abs(g[e])), (e, fd, g[e])


@pytest.mark.slow
def test_full_size_48cubed_adjoint_fd_32_edges(P):
    """The 48^3 graph-Laplacian workload: J(theta) = <G, P_S(X(theta))> with
    G ~ N(0,1) symmetric on the selected pattern; dJ/dtheta from the adjoint
    against central differences (h = 1e-6) on 32 random edges."""
    import torch
    gl = synth.GraphLaplacian((48, 48, 48))
    perm = synth.nd_order(gl.dims)
    h = P.SelInv(gl.n, gl.colptr, gl.rowind, perm=perm)
    sym = h.symbolic()
    rows, cols = panel_positions(sym)
    rng = np.random.default_rng(48)
    gpan = rng.normal(size=rows.size)
    Gt = torch.tensor(gpan, device="cuda")
    # <G, X> over the full symmetric pattern as a weight on the panel entries
    wts = np.where(rows > cols, 2.0, np.where(rows == cols, 1.0, 0.0))
    Wt = torch.tensor(gpan * wts, device="cuda")
    theta = torch.tensor(gl.theta, dtype=torch.float64, device="cuda")
    vals = gl.assemble_torch(theta)
    h.factor(vals)
    h.selinv(P.LEVEL)
    gradA = h.adjoint(Gt)[0]
    thr = theta.clone().requires_grad_(True)
    g = torch.autograd.grad(gl.assemble_torch(thr), thr, grad_outputs=gradA)[0].cpu().numpy()

    def J(t):
        h.factor(gl.assemble_torch(t))
        h.selinv(P.LEVEL)
        return float((h.panels(0)[0] * Wt).sum().item())

    hstep = 1e-6
    errs = []
    for e in rng.choice(gl.ei.size, 32, replace=False):
        tp = theta.clone(); tp[e] += hstep
        tm = theta.clone(); tm[e] -= hstep
        fd = (J(tp) - J(tm)) / (2 * hstep)
        errs.append(abs(fd - g[e]) / max(1e-3, abs(g[e])))
    assert max(errs) <= 1e-4, max(errs)
