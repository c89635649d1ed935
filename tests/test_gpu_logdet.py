"""Differentiable log det (torch.autograd.Function over the C ABI) on the
anisotropic graph-Laplacian family A(theta) = sum_e theta_e (e_i - e_j)(e_i - e_j)^T
+ 0.05 I: value against the oracle, gradient against the exact formula
d logdet / d theta_e = X_ii + X_jj - 2 X_ij with X from the oracle, and
central finite differences (h = 1e-6)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1404_0447_gb300 as P
    return P


def setup_problem(P, side):
    import torch
    gl = synth.GraphLaplacian((side, side, side))
    perm = synth.nd_order(gl.dims)
    h = P.SelInv(gl.n, gl.colptr, gl.rowind, perm=perm)
    theta = torch.tensor(gl.theta, dtype=torch.float64, device="cuda", requires_grad=True)
    return gl, perm, h, theta


def test_logdet_gradient_matches_oracle_exact_formula(P):
    import torch
    gl, perm, h, theta = setup_problem(P, 12)
    vals = gl.assemble_torch(theta)
    ld = P.logdet(vals, h)
    ld.backward()
    g = theta.grad.cpu().numpy()
    # oracle: logdet and X on the L pattern (ND order) -> X_ii + X_jj - 2 X_ij
    cp, ri, v, _ = synth.permute_lower(gl.n, gl.colptr, gl.rowind, gl.assemble(), perm)
    sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(gl.n, cp, ri, v, 128, 1, "exact")
    assert np.array_equal(sym["post"], np.arange(gl.n))
    want_ld = oracle.logdet(d)[0]
    assert abs(ld.item() - want_ld) <= 1e-12 * abs(want_ld)
    inv = np.empty(gl.n, np.int64)
    inv[perm] = np.arange(gl.n)
    a, b = inv[gl.ei], inv[gl.ej]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    lcols = np.repeat(np.arange(gl.n), np.diff(lcp))
    keys = lcols.astype(np.int64) * gl.n + lri
    pos = np.searchsorted(keys, lo * gl.n + hi)
    assert np.array_equal(keys[pos], lo * gl.n + hi)
    want = xd[a] + xd[b] - 2 * xv[pos]
    assert np.max(np.abs(g - want)) <= 1e-10 * np.max(np.abs(want))


def test_logdet_gradient_finite_differences_small(P):
    import torch
    gl, perm, h, theta = setup_problem(P, 10)
    ld = P.logdet(gl.assemble_torch(theta), h)
    ld.backward()
    g = theta.grad.cpu().numpy()
    rng = np.random.default_rng(3)
    hstep = 1e-6
    with torch.no_grad():
        for e in rng.choice(gl.ei.size, 8, replace=False):
            tp = theta.detach().clone(); tp[e] += hstep
            tm = theta.detach().clone(); tm[e] -= hstep
            fd = (P.logdet(gl.assemble_torch(tp), h).item() - P.logdet(gl.assemble_torch(tm), h).item()) / (2 * hstep)
            assert abs(fd - g[e]) <= 1e-5 * max(1.0, abs(g[e]))


@pytest.mark.slow
def test_full_size_48cubed_fd_32_edges_and_trace(P):
    """The 48^3 workload (n = 110,592): central differences (h = 1e-6) on 32
    random theta_e against the autograd gradient.  The differences carry
    roughly eps |logdet| / h ~ 1e-5 absolute error (|logdet| ~ 1e5)."""
    import torch
    gl, perm, h, theta = setup_problem(P, 48)
    ld = P.logdet(gl.assemble_torch(theta), h)
    ld.backward()
    g = theta.grad.cpu().numpy()
    xa = h.selected()[0].cpu().numpy()
    assert oracle.trace_error(gl.n, gl.colptr, gl.rowind, gl.assemble(), xa) < 1e-11
    rng = np.random.default_rng(48)
    hstep = 1e-6
    errs = []
    with torch.no_grad():
        for e in rng.choice(gl.ei.size, 32, replace=False):
            tp = theta.detach().clone(); tp[e] += hstep
            tm = theta.detach().clone(); tm[e] -= hstep
            fd = (P.logdet(gl.assemble_torch(tp), h).item() - P.logdet(gl.assemble_torch(tm), h).item()) / (2 * hstep)
            errs.append(abs(fd - g[e]) / max(1.0, abs(g[e])))
    assert max(errs) <= 1e-4
