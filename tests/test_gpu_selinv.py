"""GPU parity of the factorisation and the selected inversion against the
oracle, through the C ABI.  Tolerance: max |X_gpu - X_oracle| over every
panel entry divided by max |X_oracle| <= 1e-10 (FP64 throughout)."""
import math

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


def torch_vals(v):
    import torch
    return torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def oracle_panels(n, cp, ri, vals, wmax, relax, perm=None):
    """Oracle X (and L, D) laid out as the library's panels."""
    if perm is not None:
        cp, ri, vals, _ = synth.permute_lower(n, cp, ri, vals, perm)
    sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(n, cp, ri, vals, wmax, relax, "supernodal")
    off, X = oracle.panels_from_columns(n, sym["sn_start"], sym["rcount"], sym["rrows"], lcp, xv, xd)
    _, Lp = oracle.panels_from_columns(n, sym["sn_start"], sym["rcount"], sym["rrows"], lcp, lv, d)
    return sym, off, X, Lp, d


def lower_mask(sym, off):
    """Panel entries on or below the diagonal of each diagonal block."""
    m = np.ones(int(off[-1]), bool)
    sn = sym["sn_start"]
    for k in range(len(sn) - 1):
        s = int(sn[k + 1] - sn[k]); r = int(sym["rcount"][k]); ld = s + r
        for j in range(1, s):
            m[off[k] + j * ld: off[k] + j * ld + j] = False
    return m


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def check_problem(P, n, cp, ri, vals, wmax=128, relax=1, perm=None, modes=(1,), **opts):
    import torch
    h = P.SelInv(n, cp, ri, perm=perm, max_sn_width=wmax, relax=relax, **opts)
    h.factor(torch_vals(vals))
    sym, off, Xo, Lo, do = oracle_panels(n, cp, ri, vals, wmax, relax, perm)
    assert np.array_equal(h.symbolic()["panel_off"], off)
    Lg = h.panels(1)[0].cpu().numpy()
    msk = lower_mask(sym, off)
    assert rel(Lg[msk], Lo[msk]) <= 1e-12
    outs = {}
    for mode in modes:
        h.selinv(mode)
        outs[mode] = h.panels(0)[0].cpu().numpy()
        assert rel(outs[mode], Xo) <= TOL, (mode, rel(outs[mode], Xo))
    return h, outs, sym, Xo


def test_grid2d_31_all_schedules_bitwise_equal(P):
    p = synth.grid2d_31()
    h, outs, sym, Xo = check_problem(P, p.n, p.colptr, p.rowind, p.values, 128, 0, modes=(0, 1, 2, 3, 1, 2, 3))
    # the schedules run identical per-supernode arithmetic: bitwise equal
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    assert np.array_equal(outs[1], outs[3])


@pytest.mark.parametrize("side,wmax,relax", [(12, 16, 1), (16, 128, 1), (13, 128, 0), (24, 128, 1)])
def test_3d_grids_tiles_and_ragged_tails(P, side, wmax, relax):
    p = synth.grid_problem((side, side + 1, side - 1), 0.01, 0.1, 77 + side)
    h, outs, sym, Xo = check_problem(P, p.n, p.colptr, p.rowind, p.values, wmax, relax, modes=(1, 0, 3))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[3])
    if side == 24:
        assert h.info["max_r"] > 512   # several step-3 row chunks, several 64-row tiles


@pytest.mark.parametrize("split,cutoff", [(0, -1), (48, -1), (100, 32), (333, 64), (16, 0)])
def test_split_step2_and_tile_policies(P, split, cutoff):
    """Step 2 split into slices of `split` rows of C (reduced in order) and the
    wide-tile policy for supernodes of width >= `cutoff` give the oracle's X."""
    p = synth.grid_problem((14, 13, 12), 0.01, 0.1, 91)
    h, outs, sym, Xo = check_problem(P, p.n, p.colptr, p.rowind, p.values, 64, 1, modes=(1, 0, 2, 3),
                                     split_k_rows=split, small_cutoff=cutoff)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    assert np.array_equal(outs[1], outs[3])


def test_autotune_keeps_a_correct_schedule(P):
    import torch
    p = synth.grid_problem((18, 17, 16), 0.01, 0.1, 5)
    h = P.SelInv(p.n, p.colptr, p.rowind)
    h.factor(torch_vals(p.values))
    best = h.autotune()
    assert best["split_k_rows"] in (0, 512, 1024, 2048, 4096) and best["small_cutoff"] in (-1, 32, 64)
    assert best["level_tiles"] in (4864, 9728, 19456)
    assert best["mode"] in (P.LEVEL, P.GRAPH, P.PERSISTENT)
    assert best["ms"] > 0
    sym, off, Xo, Lo, do = oracle_panels(p.n, p.colptr, p.rowind, p.values, 128, 1)
    for mode in (P.GRAPH, P.LEVEL, P.PLAIN, P.PERSISTENT):
        h.selinv(mode)
        assert rel(h.panels(0)[0].cpu().numpy(), Xo) <= TOL


def test_persistent_wait_times_out_and_handle_recovers(P):
    """Failure detection without a GPU fault: one dependency wait of the
    persistent schedule is armed with a completion that never comes; the
    launch must end by the 2 ms spin limit and report ERR_TIMEOUT, and the
    same handle must then give correct results."""
    import time
    import torch
    p = synth.grid_problem((12, 11, 10), 0.01, 0.1, 3)
    h = P.SelInv(p.n, p.colptr, p.rowind, spin_limit_ns=2_000_000)
    h.factor(torch_vals(p.values))
    h.selinv(P.PERSISTENT)
    h.sync_status()
    good = h.panels(0)[0].cpu().numpy()
    h.set_debug(2)
    t0 = time.time()
    h.selinv(P.PERSISTENT)
    with pytest.raises(P.PselinvError) as e:
        h.sync_status()
    assert e.value.code == -7
    assert time.time() - t0 < 10.0
    h.selinv(P.PERSISTENT)
    h.sync_status()
    assert np.array_equal(h.panels(0)[0].cpu().numpy(), good)


def test_random_pattern_with_permutation(P):
    rng = np.random.default_rng(12)
    n = 300
    mask = np.triu(rng.random((n, n)) < 0.02, 1)
    rows, cols = np.nonzero(mask.T)
    off = rng.normal(size=rows.size)
    diag = np.bincount(rows, np.abs(off), n) + np.bincount(cols, np.abs(off), n) + rng.uniform(0.5, 1.5, n)
    cp, ri, v = synth.lower_csc_from_coo(n, np.r_[np.arange(n), rows], np.r_[np.arange(n), cols], np.r_[diag, off])
    perm = rng.permutation(n)
    check_problem(P, n, cp, ri, v, 8, 1, perm=perm, modes=(1, 0))


def test_batch_of_shifts_shares_one_analysis(P):
    import torch
    p = synth.grid2d_31()
    cols = np.repeat(np.arange(p.n), np.diff(p.colptr))
    dg = p.rowind == cols
    vals = np.stack([p.values + dg * sh for sh in (0.0, 0.3, 2.0)])
    h = P.SelInv(p.n, p.colptr, p.rowind, batch=3, max_sn_width=128, relax=1)
    h.factor(torch_vals(vals))
    h.selinv(P.LEVEL)
    X = h.panels(0).cpu().numpy()
    for b in range(3):
        sym, off, Xo, Lo, do = oracle_panels(p.n, p.colptr, p.rowind, vals[b], 128, 1)
        assert rel(X[b], Xo) <= TOL


@pytest.mark.parametrize("kind", ["n1", "diagonal", "tridiagonal", "dense100", "dense200"])
def test_edge_cases(P, kind):
    rng = np.random.default_rng(3)
    if kind == "n1":
        n, cp, ri, v = 1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([4.0])
    elif kind == "diagonal":
        n = 77
        cp, ri, v = np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), rng.uniform(1, 2, n)
    elif kind == "tridiagonal":
        n, cp, ri, v = synth.laplacian_1d(300)
    else:
        n = 100 if kind == "dense100" else 200
        G = rng.normal(size=(n, n))
        A = G @ G.T / n + np.eye(n)
        rows, cols = np.tril_indices(n)
        cp, ri, v = synth.lower_csc_from_coo(n, rows, cols, A[rows, cols])
    check_problem(P, n, cp, ri, v, 128, 1, modes=(1, 0, 2, 3))


def test_bad_pivots_are_reported_and_handle_recovers(P):
    import torch
    # [[1, 1], [1, 1]]: d_1 = 0 exactly
    cp = np.array([0, 2, 3], np.int64)
    ri = np.array([0, 1, 1], np.int32)
    h = P.SelInv(2, cp, ri, relax=0)
    h.factor(torch_vals([1.0, 1.0, 1.0]))          # asynchronous: reported by sync_status
    with pytest.raises(P.PselinvError) as e:
        h.sync_status()
    assert e.value.code == -3 and "column 1" in str(e.value)
    with pytest.raises(P.PselinvError) as e:
        h.selinv(P.LEVEL)
    assert e.value.code == -8
    h.factor(torch_vals([np.nan, 1.0, 3.0]))
    with pytest.raises(P.PselinvError) as e:
        h.logdet()                                   # logdet synchronises and reports it too
    assert e.value.code == -4
    h.factor(torch_vals([2.0, 1.0, 3.0]))
    h.selinv(P.LEVEL)
    X = h.panels(0)[0].cpu().numpy()
    inv = np.linalg.inv(np.array([[2.0, 1.0], [1.0, 3.0]]))
    assert np.allclose(X, [inv[0, 0], inv[1, 0], inv[0, 1], inv[1, 1]], rtol=1e-14, atol=0)


def test_logdet_and_selected_entries(P):
    import torch
    p = synth.grid_problem((9, 8, 7), 0.1, 1.0, 5)
    rng = np.random.default_rng(0)
    perm = rng.permutation(p.n)        # user-supplied ordering on top of the ND one
    cp, ri, v, _ = synth.permute_lower(p.n, p.colptr, p.rowind, p.values, np.argsort(perm))
    h = P.SelInv(p.n, cp, ri, perm=perm, max_sn_width=32, relax=1)
    h.factor(torch_vals(v))
    h.selinv(P.GRAPH)
    sel = h.selected()[0].cpu().numpy()
    Ainv = oracle.dense_inverse(p.n, cp, ri, v)
    cols = np.repeat(np.arange(p.n), np.diff(cp))
    assert rel(sel, Ainv[ri, cols]) <= TOL
    ld = h.logdet()[0]
    sign, want = np.linalg.slogdet(oracle.dense_from_lower(p.n, cp, ri, v))
    assert abs(ld[0] - want) <= 1e-12 * abs(want) and ld[1] == 0


def test_panels_into_pinned_host_memory(P):
    import torch
    p = synth.grid2d_31()
    h = P.SelInv(p.n, p.colptr, p.rowind)
    h.factor(torch_vals(p.values))
    h.selinv(P.LEVEL)
    host = torch.empty(h.info["panel_entries"], dtype=torch.float64).pin_memory()
    h.panels(0, out=host)
    torch.cuda.synchronize()
    assert torch.equal(host, h.panels(0)[0].cpu())


@pytest.mark.parametrize("case", ["grid48", "poles", "unsym"])
def test_selinv_to_host_matches_device_panels(P, case):
    """pselinv_selinv_to_host: the level-by-level host copies (including the
    deferred tail of levels with more than 1024 runs of panels, which 48^3
    has) reproduce the device panels bit for bit and cover every entry."""
    import torch
    if case == "grid48":
        p = synth.grid3d(side=48)
        h = P.SelInv(p.n, p.colptr, p.rowind)
        h.factor(torch_vals(p.values))
    elif case == "poles":
        p = synth.grid_problem((14, 13, 12), 0.01, 0.1, 4)
        z = np.array([0.3 + 0.2j, -0.1 + 0.05j])
        vals = np.stack([p.values.astype(np.complex128) for _ in z])
        diag = np.asarray(p.colptr[:-1])
        vals[:, diag] -= z[:, None]
        h = P.SelInv(p.n, p.colptr, p.rowind, dtype=P.C128, batch=2)
        h.factor(torch.tensor(vals, device="cuda").view(-1))
    else:
        p = synth.convdiff_problem(dims=(20, 18, 16))
        h = P.SelInv(p.n, p.colptr, p.rowind, unsym=1)
        h.factor_unsym(torch_vals(p.values), torch_vals(p.values_up))
    n = h.opts.batch * h.info["panel_entries"]
    out = torch.full((n,), float("nan"), dtype=h.torch_dtype).pin_memory()
    out_u = torch.full((n,), float("nan"), dtype=h.torch_dtype).pin_memory() if case == "unsym" else None
    for _ in range(2):
        h.selinv_to_host(out, out_u)
        torch.cuda.synchronize()
        assert torch.equal(out, h.panels(0).view(-1).cpu())
        if out_u is not None:
            assert torch.equal(out_u, h.panels(2).view(-1).cpu())
        out.fill_(float("nan"))
        if out_u is not None:
            out_u.fill_(float("nan"))


def test_runs_are_bitwise_deterministic(P):
    import torch
    p = synth.grid3d(side=20)
    h = P.SelInv(p.n, p.colptr, p.rowind)
    h.factor(torch_vals(p.values))
    h.selinv(P.LEVEL)
    a = h.panels(0).clone()
    h.selinv(P.LEVEL)
    b = h.panels(0)
    h.selinv(P.GRAPH)
    c = h.panels(0)
    assert torch.equal(a, b) and torch.equal(a, c)


@pytest.mark.parametrize("case", ["grid3d_24", "graph_laplacian", "poles", "unsym", "bk"])
def test_factor_and_selinv_bitwise_reproducible(P, case):
    """Two factorisations of the same values give bitwise the same L (and D)
    and, after the selected inversion, the same X: the Schur updates of a
    level run in groups with disjoint targets, in a fixed order, without
    atomics.  Levels of these cases hold many supernodes that update shared
    ancestors."""
    import torch
    kw, factor = {}, "factor"
    if case == "grid3d_24":
        p = synth.grid3d(side=24)
        n, cp, ri, v = p.n, p.colptr, p.rowind, p.values
    elif case == "graph_laplacian":
        gl = synth.GraphLaplacian((18, 17, 16), seed=3)
        n, cp, ri, v = gl.n, gl.colptr, gl.rowind, gl.assemble()
        kw["perm"] = synth.nd_order(gl.dims)
    elif case == "poles":
        n, cp0, ri0, hv, z = synth.dg_block_matrix((4, 4, 3), 8, 3, seed=5)
        vals = synth.shifted_values(n, cp0, ri0, hv, z)
        cp, ri, v, _ = synth.permute_lower(n, cp0, ri0, vals, synth.block_nd_order((4, 4, 3), 8))
        kw.update(dtype=P.C128, batch=3)
    elif case == "unsym":
        p = synth.convdiff_problem(dims=(14, 13, 12))
        n, cp, ri, v, up = p.n, p.colptr, p.rowind, p.values, p.values_up
        kw["unsym"] = 1
        factor = "factor_unsym"
    else:
        p = synth.grid3d(20, shift_const=-0.5)
        n, cp, ri, v = p.n, p.colptr, p.rowind, p.values
        factor = "factor_bk"
    h = P.SelInv(n, cp, ri, **kw)
    dt = torch.complex128 if kw.get("dtype") == P.C128 else torch.float64
    vt = torch.tensor(np.ascontiguousarray(v), dtype=dt, device="cuda")
    args = (vt, torch.tensor(np.ascontiguousarray(up), dtype=dt, device="cuda")) if factor == "factor_unsym" else (vt,)
    runs = []
    for _ in range(2):
        getattr(h, factor)(*args)
        h.sync_status()
        L = h.panels(1).clone()
        h.selinv(P.LEVEL)
        runs.append((L, h.panels(0).clone()))
    assert torch.equal(runs[0][0], runs[1][0])
    assert torch.equal(runs[0][1], runs[1][1])


@pytest.mark.slow
def test_full_size_80cubed_against_closed_form_and_trace(P):
    """The benchmark workload (80^3 7-point grid, n = 512,000, relaxed
    supernodes of width <= 128, level schedule) at full size.  With a
    constant shift the inverse has a separable closed form: sampled panel
    entries are checked against it; with the random shifts the trace
    identity E of Eq. (16) is checked over all of A's entries."""
    import torch
    side = 80
    p = synth.grid3d(side, shift_const=0.055)
    h = P.SelInv(p.n, p.colptr, p.rowind)
    s = h.symbolic()
    h.factor(torch_vals(p.values))
    h.selinv(P.LEVEL)
    X = h.panels(0)[0]
    rng = np.random.default_rng(2024)
    nsn = s["nsn"]
    # sample entries: supernodes spread over all levels (root chain included)
    ks = np.unique(np.r_[rng.integers(0, nsn, 120), s["level_sn"][:10]])
    pos, pairs = [], []
    for k in ks:
        f, l = s["sn_start"][k], s["sn_start"][k + 1]
        sw = l - f
        R = s["rows"][s["rowptr"][k]:s["rowptr"][k + 1]]
        rowsK = np.r_[np.arange(f, l), R]
        for _ in range(2):
            c = int(rng.integers(0, sw)); rr = int(rng.integers(c, sw + len(R)))
            pos.append(s["panel_off"][k] + c * (sw + len(R)) + rr)
            # internal index -> ND-ordered input (library perm) -> natural grid index
            pairs.append((p.perm[s["perm"][rowsK[rr]]], p.perm[s["perm"][f + c]]))
    got = X[torch.tensor(np.array(pos), device="cuda")].cpu().numpy()
    want = oracle.grid_inverse_entries(p.dims, 0.055, np.array(pairs))
    scale = float(torch.max(torch.abs(X)).item())
    assert np.max(np.abs(got - want)) / scale <= TOL
    # random shifts: trace identity on the selected entries at A's positions
    q = synth.grid3d(side)
    h.factor(torch_vals(q.values))
    h.selinv(P.LEVEL)
    xa = h.selected()[0].cpu().numpy()
    assert oracle.trace_error(q.n, q.colptr, q.rowind, q.values, xa) < 1e-11
