"""Complex-symmetric batches (poles H - z_l I sharing one pattern) on the
GPU against the oracle, through the C ABI.  Plain transposes throughout
(complex symmetric, not Hermitian).  Tolerance 1e-10 relative to max|X|."""
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


def poles_problem(elems, nb, npoles, seed):
    n, cp, ri, hv, z = synth.dg_block_matrix(elems, nb, npoles, seed=seed)
    perm = synth.block_nd_order(elems, nb)
    vals = synth.shifted_values(n, cp, ri, hv, z)
    cp2, ri2, v2, _ = synth.permute_lower(n, cp, ri, vals, perm)
    return n, cp2, ri2, v2, z, hv


def tvals(v):
    import torch
    return torch.tensor(np.ascontiguousarray(v), dtype=torch.complex128, device="cuda")


@pytest.mark.parametrize("elems,nb,wmax", [((3, 3, 2), 8, 16), ((4, 4, 3), 12, 128), ((5, 4, 3), 6, 32)])
def test_pole_batch_matches_oracle(P, elems, nb, wmax):
    n, cp, ri, v, z, hv = poles_problem(elems, nb, 4, seed=31 + nb)
    h = P.SelInv(n, cp, ri, dtype=P.C128, batch=len(z), max_sn_width=wmax, relax=P.RELAX_AMALG)
    h.factor(tvals(v))
    for mode in (P.LEVEL, P.PLAIN, P.PERSISTENT):
        h.selinv(mode)
        X = h.panels(0).cpu().numpy()
        for l in range(len(z)):
            sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp, ri, v[l], wmax, 1)
            off, Xo = oracle.panels_from_columns(n, sym["sn_start"], sym["rcount"], sym["rrows"], lcp, xv, xd)
            err = np.max(np.abs(X[l] - Xo)) / np.max(np.abs(Xo))
            assert err <= TOL, (mode, l, err)


def test_conjugate_pole_gives_conjugate_inverse(P):
    """H is real, so X(conj z) = conj(X(z)).  The complex kernels mirror every
    real operation (conjugated inputs give negated imaginary parts, rounded
    symmetrically) and the factorisation runs in a fixed order, so the two
    members are exact conjugates."""
    n, cp, ri, hv, z = synth.dg_block_matrix((4, 3, 3), 10, 1, seed=7)
    perm = synth.block_nd_order((4, 3, 3), 10)
    zz = np.array([z[0], np.conj(z[0])])
    vals = synth.shifted_values(n, cp, ri, hv, zz)
    cp2, ri2, v2, _ = synth.permute_lower(n, cp, ri, vals, perm)
    h = P.SelInv(n, cp2, ri2, dtype=P.C128, batch=2)
    h.factor(tvals(v2))
    h.selinv(P.GRAPH)
    X = h.panels(0).cpu().numpy()
    assert np.array_equal(X[1], np.conj(X[0]))


def test_complex_logdet_and_selected_entries(P):
    n, cp, ri, v, z, hv = poles_problem((3, 3, 3), 6, 3, seed=5)
    h = P.SelInv(n, cp, ri, dtype=P.C128, batch=3, max_sn_width=24)
    h.factor(tvals(v))
    h.selinv(P.LEVEL)
    sel = h.selected().cpu().numpy()
    ld = h.logdet()
    cols = np.repeat(np.arange(n), np.diff(cp))
    for l in range(3):
        A = oracle.dense_from_lower(n, cp, ri, v[l])
        Ainv = np.linalg.inv(A)
        assert np.max(np.abs(sel[l] - Ainv[ri, cols])) <= TOL * np.max(np.abs(Ainv))
        sign, want = np.linalg.slogdet(A)
        assert abs(ld[l, 0] - want) <= 1e-12 * abs(want)
        dphi = (ld[l, 1] - np.angle(sign) + np.pi) % (2 * np.pi) - np.pi
        assert abs(dphi) < 1e-9
        # the oracle's sum of principal logs agrees without wrapping
        sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp, ri, v[l], 24, 1)
        assert abs(oracle.logdet(d)[1] - ld[l, 1]) < 1e-9


def test_pole_sum_and_trace_error_per_pole(P):
    """Gamma = sum_l w_l X_l (the pole expansion of Section 4.4) against the
    same sum over the oracle's selected inverse of each pole, and E(z_l) of
    Eq. (16) per pole against the oracle's E."""
    import torch
    n, cp, ri, v, z, hv = poles_problem((4, 3, 3), 8, 5, seed=17)
    h = P.SelInv(n, cp, ri, dtype=P.C128, batch=5, max_sn_width=32)
    vt = tvals(v)
    h.factor(vt)
    h.selinv(P.LEVEL)
    w = np.random.default_rng(2).normal(size=5) + 1j * np.random.default_rng(3).normal(size=5)
    G = h.pole_sum(w).cpu().numpy()
    assert np.array_equal(G, h.pole_sum(w).cpu().numpy())   # fixed order over the poles: reproducible
    want = 0
    for l in range(5):
        sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp, ri, v[l], 32, 1)
        off, Xo = oracle.panels_from_columns(n, sym["sn_start"], sym["rcount"], sym["rrows"], lcp, xv, xd)
        want = want + w[l] * Xo
    assert np.max(np.abs(G - want)) <= TOL * np.max(np.abs(want))
    E = h.trace_error(vt)
    sel = h.selected().cpu().numpy()
    for l in range(5):
        assert abs(E[l] - oracle.trace_error(n, cp, ri, v[l], sel[l])) < 1e-13
        assert E[l] < 1e-12


@pytest.mark.parametrize("wmax", [32, 8])
def test_pole_sum_fused_into_the_sweep(P, wmax):
    """pselinv_selinv_pole_sum: Gamma accumulated in the write step of the
    batched sweep (Section 4.4's pole expansion) against the sum over the
    oracle's selected inverse of each pole, bitwise reproducible, equal to the
    separate pass over the same X, and the X panels of every pole as a plain
    selinv leaves them.  Two tile policies (wide and narrow supernodes), so
    the finish shares cover X_{C,K} rows and diagonal blocks of several sizes."""
    import torch
    n, cp, ri, v, z, hv = poles_problem((4, 3, 3), 8, 5, seed=23)
    h = P.SelInv(n, cp, ri, dtype=P.C128, batch=5, max_sn_width=wmax)
    h.factor(tvals(v))
    w = np.random.default_rng(5).normal(size=5) + 1j * np.random.default_rng(6).normal(size=5)
    G = h.selinv_pole_sum(w).cpu().numpy()
    X1 = h.panels().cpu().numpy()
    want = 0
    for l in range(5):
        sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp, ri, v[l], wmax, 1)
        off, Xo = oracle.panels_from_columns(n, sym["sn_start"], sym["rcount"], sym["rrows"], lcp, xv, xd)
        want = want + w[l] * Xo
        assert np.max(np.abs(X1[l] - Xo)) <= TOL * np.max(np.abs(Xo))
    assert np.max(np.abs(G - want)) <= TOL * np.max(np.abs(want))
    assert np.array_equal(G, h.selinv_pole_sum(w).cpu().numpy())      # fixed pole order: reproducible
    sep = h.pole_sum(w).cpu().numpy()
    assert np.max(np.abs(G - sep)) <= 1e-14 * np.max(np.abs(sep))      # same sums as the separate pass
    h.selinv(P.LEVEL)
    assert np.array_equal(X1, h.panels().cpu().numpy())               # X as a plain selinv leaves it


def test_pole_sum_fused_rejects_pivoted_and_unsym(P):
    """The fused pole sum needs a pivot-free symmetric factor."""
    import torch
    n, cp, ri, v, z, hv = poles_problem((3, 3, 2), 4, 2, seed=29)
    h = P.SelInv(n, cp, ri, dtype=P.C128, batch=2, max_sn_width=16)
    w = np.ones(2, np.complex128)
    with pytest.raises(P.PselinvError, match="ERR_STATE"):
        h.selinv_pole_sum(w)                                           # no factor yet
    h.factor_bk(tvals(v))
    with pytest.raises(P.PselinvError, match="ERR_STATE"):
        h.selinv_pole_sum(w)


@pytest.mark.slow
def test_full_size_dg_two_poles_trace_identity_and_batch_equivalence(P):
    """The 12^3-element, 48-dof DG-like matrix (n = 82,944) with its first two
    poles: the trace identity E(z) of Eq. (16) per pole, and the batched run
    bitwise equal to a single-pole run of the same pole (the schedule does
    not depend on the batch size and the factorisation runs in a fixed
    order)."""
    import torch
    n, cp, ri, hv, z = synth.dg_block_matrix((12, 12, 12), 48, 16)
    perm = synth.block_nd_order((12, 12, 12), 48)
    vals = synth.shifted_values(n, cp, ri, hv, z[:2])
    h = P.SelInv(n, cp, ri, perm=perm, dtype=P.C128, batch=2)
    h.factor(tvals(vals))
    h.selinv(P.LEVEL)
    sel = h.selected().cpu().numpy()
    for l in range(2):
        assert oracle.trace_error(n, cp, ri, vals[l], sel[l]) < 1e-11
    x_batch = h.panels(0)[1].clone()
    h.close()
    del h
    torch.cuda.empty_cache()
    h1 = P.SelInv(n, cp, ri, perm=perm, dtype=P.C128, batch=1)
    h1.factor(tvals(vals[1:2]))
    h1.selinv(P.LEVEL)
    x1 = h1.panels(0)[0]
    assert torch.equal(x1, x_batch)
