"""GPU parity of the non-symmetric path (A = L D U' and Algorithm 1 with
step 4) against the oracle, through the C ABI.  Tolerance as for the
symmetric path: max |X_gpu - X_oracle| / max |X_oracle| <= 1e-10 over every
panel entry of both the XL and the XU panels (FP64 throughout)."""
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


def dev(v, cplx=False):
    import torch
    return torch.tensor(np.ascontiguousarray(v), dtype=torch.complex128 if cplx else torch.float64, device="cuda")


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def panel_masks(sym, off):
    """(on or below the diagonal of each diagonal block, strictly below)."""
    low = np.ones(int(off[-1]), bool)
    strict = np.ones(int(off[-1]), bool)
    sn = sym["sn_start"]
    for k in range(len(sn) - 1):
        s = int(sn[k + 1] - sn[k]); r = int(sym["rcount"][k]); ld = s + r
        for j in range(s):
            low[off[k] + j * ld: off[k] + j * ld + j] = False
            strict[off[k] + j * ld: off[k] + j * ld + j + 1] = False
    return low, strict


def oracle_panels_lu(n, cp, ri, lo, up, wmax, relax, perm=None):
    if perm is not None:
        cp, ri, lo, up, _, _ = synth.permute_lower_unsym(n, cp, ri, lo, up, perm)
    sym, lv, uv, d, xv, xu, xd, lcp, lri = oracle.selected_inverse_lu(n, cp, ri, lo, up, wmax, relax)
    args = (n, sym["sn_start"], sym["rcount"], sym["rrows"], lcp)
    off, XL, XU = oracle.panels_from_columns_lu(*args, xv, xu, xd)
    _, Lp = oracle.panels_from_columns(*args, lv, d)
    _, Up = oracle.panels_from_columns(*args, uv, d)
    return sym, off, XL, XU, Lp, Up, d


def check_unsym(P, n, cp, ri, lo, up, wmax=128, relax=1, perm=None, modes=(1,), cplx=False, **opts):
    h = P.SelInv(n, cp, ri, perm=perm, max_sn_width=wmax, relax=relax, unsym=1, dtype=P.C128 if cplx else P.F64,
                 **opts)
    h.factor_unsym(dev(lo, cplx), dev(up, cplx))
    wm = min(wmax, 112) if cplx else wmax
    sym, off, XLo, XUo, Lo, Uo, do = oracle_panels_lu(n, cp, ri, lo, up, wm, relax, perm)
    assert np.array_equal(h.symbolic()["panel_off"], off)
    low, strict = panel_masks(sym, off)
    assert rel(h.panels(1)[0].cpu().numpy()[low], Lo[low]) <= 1e-12
    assert rel(h.panels(3)[0].cpu().numpy()[strict], Uo[strict]) <= 1e-12
    outs = {}
    for mode in modes:
        h.selinv(mode)
        XL = h.panels(0)[0].cpu().numpy()
        XU = h.panels(2)[0].cpu().numpy()
        assert rel(XL, XLo) <= TOL, (mode, rel(XL, XLo))
        assert rel(XU, XUo) <= TOL, (mode, rel(XU, XUo))
        outs[mode] = (XL, XU)
    return h, outs


def test_unsym_convdiff_all_schedules_bitwise_equal(P):
    p = synth.convdiff_problem(dims=(12, 11, 10))
    h, outs = check_unsym(P, p.n, p.colptr, p.rowind, p.values, p.values_up, modes=(0, 1, 2, 1, 2))
    for m in (1, 2):
        assert np.array_equal(outs[0][0], outs[m][0]) and np.array_equal(outs[0][1], outs[m][1])
    assert h.info["flops_gemm1"] > 0


@pytest.mark.parametrize("split,cutoff,wmax", [(0, -1, 128), (48, -1, 64), (100, 32, 64), (16, 0, 16)])
def test_unsym_split_step2_step4_and_tile_policies(P, split, cutoff, wmax):
    p = synth.convdiff_problem(dims=(14, 13, 12))
    h, outs = check_unsym(P, p.n, p.colptr, p.rowind, p.values, p.values_up, wmax=wmax, modes=(1, 0),
                          split_k_rows=split, small_cutoff=cutoff)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_unsym_user_ordering_flips_entries(P):
    """A random user ordering moves stored entries across the diagonal; the
    gathered X_ij / X_ji at A's stored positions must match a dense inverse."""
    import torch
    n, cp, ri, lo, up = synth.convdiff_grid((9, 8, 7), 17)
    perm = np.random.default_rng(1).permutation(n).astype(np.int32)
    h = P.SelInv(n, cp, ri, perm=perm, unsym=1)
    h.factor_unsym(dev(lo), dev(up))
    h.selinv(P.LEVEL)
    Xi = np.linalg.inv(oracle.dense_from_lower_lu(n, cp, ri, lo, up))
    cols = np.repeat(np.arange(n), np.diff(cp))
    g_lo = h.selected()[0].cpu().numpy()
    g_up = h.selected_upper()[0].cpu().numpy()
    scale = np.abs(Xi).max()
    assert np.max(np.abs(g_lo - Xi[ri, cols])) / scale <= TOL
    assert np.max(np.abs(g_up - Xi[cols, ri])) / scale <= TOL
    # also against the oracle's panels under the same ordering
    check_unsym(P, n, cp, ri, lo, up, perm=perm, modes=(1,))


def test_unsym_complex_values_and_width_cap(P):
    p = synth.convdiff_problem(dims=(10, 9, 11))
    rng = np.random.default_rng(3)
    lo = p.values + 1j * rng.uniform(-0.2, 0.2, p.nnz)
    up = p.values_up + 1j * rng.uniform(-0.2, 0.2, p.nnz)
    h, outs = check_unsym(P, p.n, p.colptr, p.rowind, lo, up, wmax=128, cplx=True, modes=(1, 0))
    assert h.info["max_width"] <= 112


def test_unsym_on_symmetric_values_matches_symmetric_path(P):
    import torch
    p = synth.grid3d(side=14)
    hs = P.SelInv(p.n, p.colptr, p.rowind)
    hs.factor(dev(p.values))
    hs.selinv(P.LEVEL)
    hu = P.SelInv(p.n, p.colptr, p.rowind, unsym=1)
    hu.factor_unsym(dev(p.values), dev(p.values))
    hu.selinv(P.LEVEL)
    Xs = hs.panels(0)[0].cpu().numpy()
    XL = hu.panels(0)[0].cpu().numpy()
    XU = hu.panels(2)[0].cpu().numpy()
    assert rel(XL, Xs) <= 1e-13 and rel(XU, Xs) <= 1e-13
    assert np.allclose(hs.logdet(), hu.logdet(), rtol=1e-14, atol=0)


def test_unsym_logdet_vs_slogdet(P):
    n, cp, ri, lo, up = synth.convdiff_grid((7, 6, 5), 23)
    h = P.SelInv(n, cp, ri, unsym=1)
    h.factor_unsym(dev(lo), dev(up))
    sign, ld = np.linalg.slogdet(oracle.dense_from_lower_lu(n, cp, ri, lo, up))
    got = h.logdet()[0]
    assert abs(got[0] - ld) <= 1e-10 * abs(ld) and (-1) ** int(got[1]) == sign


def test_unsym_errors_and_symmetric_only_entry_points(P):
    import torch
    n, cp, ri, lo, up = synth.convdiff_grid((5, 5, 4), 2)
    h = P.SelInv(n, cp, ri, unsym=1)
    with pytest.raises(P.PselinvError, match="ERR_STATE"):
        h.factor(dev(lo))
    hs = P.SelInv(n, cp, ri)
    with pytest.raises(P.PselinvError, match="ERR_STATE"):
        hs.factor_unsym(dev(lo), dev(up))
    h.factor_unsym(dev(lo), dev(up))
    with pytest.raises(P.PselinvError, match="ERR_ARG"):
        h.selinv(P.PERSISTENT)
    h.selinv(P.LEVEL)
    with pytest.raises(P.PselinvError, match="ERR_STATE"):
        h.logdet_grad()
    with pytest.raises(P.PselinvError, match="ERR_STATE"):
        h.adjoint(torch.zeros(h.info["panel_entries"], dtype=torch.float64, device="cuda"))
    with pytest.raises(P.PselinvError, match="ERR_ARG"):
        hs.panels(2)
    # [[1, 2], [3, 6]]: d_1 = 6 - 3 * 2 = 0 exactly; then the handle recovers
    cp2 = np.array([0, 2, 3], np.int64)
    ri2 = np.array([0, 1, 1], np.int32)
    h2 = P.SelInv(2, cp2, ri2, relax=0, unsym=1)
    h2.factor_unsym(dev([1.0, 3.0, 6.0]), dev([0.0, 2.0, 0.0]))
    with pytest.raises(P.PselinvError, match="ERR_ZERO_PIVOT"):
        h2.sync_status()
    h2.factor_unsym(dev([np.nan, 3.0, 6.0]), dev([0.0, 2.0, 0.0]))
    with pytest.raises(P.PselinvError, match="ERR_NONFINITE"):
        h2.sync_status()
    h2.factor_unsym(dev([2.0, 4.0, 3.0]), dev([0.0, 1.0, 0.0]))
    h2.selinv(P.LEVEL)
    inv = np.linalg.inv(np.array([[2.0, 1.0], [4.0, 3.0]]))
    XL = h2.panels(0)[0].cpu().numpy()
    XU = h2.panels(2)[0].cpu().numpy()
    assert np.allclose(XL, [inv[0, 0], inv[1, 0], inv[0, 1], inv[1, 1]], rtol=1e-14, atol=0)
    assert np.allclose(XU, [inv[0, 0], inv[0, 1], inv[1, 0], inv[1, 1]], rtol=1e-14, atol=0)


@pytest.mark.slow
def test_unsym_full_size_closed_form_and_row_identities(P):
    """80^3 constant-coefficient convection-diffusion (the bench workload's
    pattern): sampled selected entries against the closed form, and for every
    row (A X)_jj = (X A)_jj = 1 using only selected entries."""
    import torch
    beta, shift = (0.3, 0.2, 0.1), 0.05
    p = synth.convdiff_problem(80, beta_const=beta, shift_const=shift)
    h = P.SelInv(p.n, p.colptr, p.rowind, unsym=1)
    lo, up = dev(p.values), dev(p.values_up)
    h.factor_unsym(lo, up)
    h.selinv(P.LEVEL)
    xl = h.selected()[0]
    xu = h.selected_upper()[0]
    cols = torch.repeat_interleave(torch.arange(p.n, device="cuda"),
                                   torch.tensor(np.diff(p.colptr), device="cuda"))
    rows = torch.tensor(p.rowind.astype(np.int64), device="cuda")
    off = rows != cols
    ax = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    xa = torch.zeros_like(ax)
    diag = ~off
    ax.index_add_(0, cols[diag], (lo * xl)[diag])
    xa.index_add_(0, cols[diag], (lo * xl)[diag])
    ax.index_add_(0, cols[off], (up * xl)[off])      # A_ji X_ij -> (AX)_jj
    ax.index_add_(0, rows[off], (lo * xu)[off])      # A_ij X_ji -> (AX)_ii
    xa.index_add_(0, cols[off], (xu * lo)[off])      # X_ji A_ij -> (XA)_jj
    xa.index_add_(0, rows[off], (xl * up)[off])      # X_ij A_ji -> (XA)_ii
    assert float((ax - 1).abs().max()) <= 1e-10
    assert float((xa - 1).abs().max()) <= 1e-10
    rng = np.random.default_rng(8)
    pick = rng.choice(p.nnz, size=200, replace=False)
    nat = np.asarray(p.perm)
    i_nat, j_nat = nat[p.rowind[pick]], nat[np.asarray(cols.cpu())[pick]]
    want_lo = oracle.convdiff_inverse_entries(p.dims, beta, shift, np.stack([i_nat, j_nat], 1))
    want_up = oracle.convdiff_inverse_entries(p.dims, beta, shift, np.stack([j_nat, i_nat], 1))
    got_lo = xl.cpu().numpy()[pick]
    got_up = xu.cpu().numpy()[pick]
    scale = np.abs(want_lo).max()
    assert np.max(np.abs(got_lo - want_lo)) / scale <= TOL
    assert np.max(np.abs(got_up - want_up)) / scale <= TOL
