"""GPU parity of step 2 with its FP64 arithmetic emulated on the bf16 tensor
cores (opts.fp64_emulation = 1, mma.sync: scaled X and Lhat
cut into 8-bit slices, exact integer accumulation of the slice products)
against the oracle,
through the C ABI: SPD grids and graph Laplacians over the tile widths,
k-slices and ragged tails, the PLAIN / LEVEL / GRAPH schedules, batches,
and the report of an X that is not positive definite.  Tolerance 1e-10 of
max |X| (the FP64 path's); the emulated and the FP64 GPU results are also
compared with each other."""
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
    return torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def oracle_x(p, wmax, relax):
    """Oracle X panels of a synth.Problem (whose arrays are already in ND order)."""
    sym, lv, d, xv, xd, lcp, lri = oracle.selected_inverse(p.n, p.colptr, p.rowind, p.values, wmax, relax,
                                                           "supernodal")
    off, X = oracle.panels_from_columns(p.n, sym["sn_start"], sym["rcount"], sym["rrows"], lcp, xv, xd)
    return off, X


def run(P, p, wmax=128, relax=1, modes=(1,), emulate=1, **opts):
    h = P.SelInv(p.n, p.colptr, p.rowind, max_sn_width=wmax, relax=relax, fp64_emulation=emulate, **opts)
    h.factor(dev(p.values))
    outs = {}
    for mode in modes:
        h.selinv(mode)
        h.sync_status()
        outs[mode] = h.panels(0)[0].cpu().numpy()
    return h, outs


VARIANTS = [pytest.param(1, id="mma_sync")]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case,wmax,relax,opts", [
    ("grid2d_31", 128, 0, {}),
    ("grid3d_12", 16, 1, {}),
    ("grid3d_16", 128, 1, {}),
    ("grid3d_13", 128, 0, {"small_cutoff": 0}),       # 64-column tiles wherever possible
    ("grid3d_20", 128, 1, {"split_k_rows": 48}),      # k-slices of C with ordered reductions
    ("graphlap_10", 128, 1, {}),                      # random weights, uneven degrees
])
def test_emulated_step2_against_oracle_and_fp64_path(P, case, wmax, relax, opts, variant):
    if case == "grid2d_31":
        p = synth.grid2d_31()
    elif case.startswith("grid3d"):
        p = synth.grid3d(int(case.split("_")[1]))
    else:
        p = synth.graph_laplacian3d(int(case.split("_")[1]))
    off, Xo = oracle_x(p, wmax, relax)
    h, outs = run(P, p, wmax, relax, modes=(0, 1, 2), emulate=variant, **opts)
    assert np.array_equal(h.symbolic()["panel_off"], off)
    for m, x in outs.items():
        assert rel(x, Xo) <= TOL, (m, rel(x, Xo))
    # the schedules run the same per-tile arithmetic: bitwise equal
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    _, f64 = run(P, p, wmax, relax, modes=(1,), emulate=0, **opts)
    d = rel(outs[1], f64[1])
    print(case, "emulated vs FP64 path", d, "emulated vs oracle", rel(outs[1], Xo), "FP64 vs oracle",
          rel(f64[1], Xo))
    assert d <= 1e-12


@pytest.mark.parametrize("variant", VARIANTS)
def test_emulated_batch_members(P, variant):
    gl = synth.GraphLaplacian((9, 8, 7))
    base = gl.assemble()
    diag = np.asarray(gl.colptr[:-1])
    perm = synth.nd_order(gl.dims)
    probs = []
    for sh in (0.0, 0.3, 5.0):
        v = base.copy()
        v[diag] += sh
        probs.append(synth.Problem("gl", gl.n, gl.colptr, gl.rowind, v, perm))
    p0 = probs[0]
    h = P.SelInv(p0.n, p0.colptr, p0.rowind, batch=3, fp64_emulation=variant)
    h.factor(dev(np.concatenate([q.values for q in probs])))
    h.selinv(P.LEVEL)
    h.sync_status()
    X = h.panels(0).cpu().numpy()
    for b, q in enumerate(probs):
        _, Xo = oracle_x(q, 128, 1)
        assert rel(X[b], Xo) <= TOL


@pytest.mark.parametrize("variant", VARIANTS)
def test_not_positive_definite_is_reported_and_the_handle_recovers(P, variant):
    """A = -(SPD): every X_pp < 0, so the scaling has no exponent; the
    selinv is reported as ERR_RANGE and its X is not offered.  The same
    handle then inverts an SPD matrix correctly."""
    p = synth.grid3d(10)
    h = P.SelInv(p.n, p.colptr, p.rowind, fp64_emulation=variant)
    h.factor(dev(-p.values))
    h.selinv(P.LEVEL)
    with pytest.raises(P.PselinvError, match="ERR_RANGE"):
        h.sync_status()
    with pytest.raises(P.PselinvError, match="ERR_STATE"):
        h.panels(0)
    h.factor(dev(p.values))
    h.selinv(P.LEVEL)
    h.sync_status()
    _, Xo = oracle_x(p, 128, 1)
    assert rel(h.panels(0)[0].cpu().numpy(), Xo) <= TOL


def test_persistent_schedule_is_refused(P):
    p = synth.grid3d(6)
    h = P.SelInv(p.n, p.colptr, p.rowind, fp64_emulation=1)
    h.factor(dev(p.values))
    with pytest.raises(P.PselinvError, match="ERR_ARG"):
        h.selinv(P.PERSISTENT)


@pytest.mark.slow
@pytest.mark.parametrize("variant", VARIANTS)
def test_full_size_80cubed_emulated_against_closed_form_and_fp64(P, variant):
    """The benchmark workload at full size (n = 512,000) with the emulated
    step 2: sampled entries against the separable closed form, and every X
    panel entry against the FP64 path."""
    import torch
    p = synth.grid3d(80, shift_const=0.055)
    h = P.SelInv(p.n, p.colptr, p.rowind, fp64_emulation=variant)
    s = h.symbolic()
    h.factor(dev(p.values))
    h.selinv(P.LEVEL)
    h.sync_status()
    X = h.panels(0)[0]
    rng = np.random.default_rng(2024)
    ks = np.unique(np.r_[rng.integers(0, s["nsn"], 120), s["level_sn"][:10]])
    pos, pairs = [], []
    for k in ks:
        f, l = s["sn_start"][k], s["sn_start"][k + 1]
        R = s["rows"][s["rowptr"][k]:s["rowptr"][k + 1]]
        rowsK = np.r_[np.arange(f, l), R]
        for _ in range(2):
            c = int(rng.integers(0, l - f)); rr = int(rng.integers(c, l - f + len(R)))
            pos.append(s["panel_off"][k] + c * (l - f + len(R)) + rr)
            pairs.append((p.perm[s["perm"][rowsK[rr]]], p.perm[s["perm"][f + c]]))
    got = X[torch.tensor(np.array(pos), device="cuda")].cpu().numpy()
    want = oracle.grid_inverse_entries(p.dims, 0.055, np.array(pairs))
    scale = float(torch.max(torch.abs(X)).item())
    err = np.max(np.abs(got - want)) / scale
    h64 = P.SelInv(p.n, p.colptr, p.rowind)
    h64.factor(dev(p.values))
    h64.selinv(P.LEVEL)
    X64 = h64.panels(0)[0]
    d = float(torch.max(torch.abs(X - X64)).item()) / scale
    print("full-size emulated", variant, ": closed-form error", err, "max |X_em - X_fp64| / max|X|", d)
    assert err <= TOL and d <= 1e-12
