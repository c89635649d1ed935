"""Host-side checks of the C-ABI library (no GPU work): the library loads,
exports every symbol the header declares, and its symbolic analysis matches
the oracle's bit for bit (elimination tree, supernodes, supernodal tree,
Algorithm 2 priorities, row lists, relative indices)."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build_library()
    import paper_1404_0447_gb300 as P
    return P


def test_exports_every_declared_symbol(P):
    hdr = open(os.path.join(ROOT, "include", "pselinv.h")).read()
    declared = set(re.findall(r"\b(pselinv_[a-z_]+)\s*\(", hdr))
    lib = P.load_library()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(P.EXPORTED)


def _compare(P, n, cp, ri, wmax, relax, perm=None):
    h = P.SelInv(n, cp, ri, perm=perm, max_sn_width=wmax, relax=relax)
    s = h.symbolic()
    if perm is not None:
        cp2, ri2, _, _ = synth.permute_lower(n, cp, ri, np.zeros(len(ri)), perm)
    else:
        cp2, ri2 = cp, ri
    o = oracle.analyse(n, cp2, ri2, wmax, 1 if relax else 0)
    base = np.arange(n) if perm is None else np.asarray(perm)
    assert np.array_equal(s["perm"], base[o["post"]])
    for a, b in [("parent", "parent"), ("sn_start", "sn_start"), ("sn_parent", "sn_parent"),
                 ("sigma", "sigma"), ("rows", "rrows"), ("relidx", "relidx"), ("nblk", "nblk")]:
        assert np.array_equal(np.asarray(s[a], np.int64), np.asarray(o[b], np.int64)), a
    assert np.array_equal(np.diff(s["rowptr"]), o["rcount"])
    # levels are the sets of Algorithm 2
    for lv in range(s["nlevels"]):
        members = s["level_sn"][s["level_ptr"][lv]:s["level_ptr"][lv + 1]]
        assert np.all(o["sigma"][members] == lv + 1)
    info = h.info
    sw = np.diff(o["sn_start"]).astype(np.int64)
    assert info["panel_entries"] == int(np.sum((sw + o["rcount"]) * sw))
    return h


@pytest.mark.parametrize("wmax,relax", [(128, 0), (16, 1), (128, 1), (5, 1)])
def test_structure_parity_grids(P, wmax, relax):
    for prob in (synth.grid2d_31(), synth.grid3d(side=11), synth.grid_problem((7, 9, 5), .1, 1, 3)):
        _compare(P, prob.n, prob.colptr, prob.rowind, wmax, relax)


def test_structure_parity_random_perm_and_postorder(P):
    rng = np.random.default_rng(4)
    for trial in range(6):
        n = 30 + 17 * trial
        mask = np.triu(rng.random((n, n)) < 0.06, 1)
        rows, cols = np.nonzero(mask.T)
        cp, ri, _ = synth.lower_csc_from_coo(
            n, np.r_[np.arange(n), rows], np.r_[np.arange(n), cols], np.ones(n + rows.size))
        perm = rng.permutation(n)
        _compare(P, n, cp, ri, 8, 1, perm=perm)


def test_structure_parity_block_matrix(P):
    n, cp, ri, hv, z = synth.dg_block_matrix((3, 3, 2), 6, 1, seed=1)
    perm = synth.block_nd_order((3, 3, 2), 6)
    cp2, ri2, _, _ = synth.permute_lower(n, cp, ri, hv, perm)
    _compare(P, n, cp2, ri2, 32, 1)


def test_analyze_rejects_bad_input(P):
    cp = np.array([0, 2, 3], np.int64)
    ri = np.array([1, 0, 1], np.int32)           # diagonal not first in column 0
    with pytest.raises(P.PselinvError) as e:
        P.SelInv(2, cp, ri)
    assert e.value.code == -2
    cp = np.array([0, 1, 2], np.int64)
    ri = np.array([0, 1], np.int32)
    with pytest.raises(P.PselinvError) as e:
        P.SelInv(2, cp, ri, perm=np.array([0, 0]))
    assert e.value.code == -2
    with pytest.raises(P.PselinvError) as e:
        P.SelInv(2, cp, ri, max_sn_width=500)
    assert e.value.code == -1
    # FP64 emulation of steps 2 and 3 (opt-in): real symmetric handles only
    for kw in ({"fp64_emulation": 2}, {"fp64_emulation": -1}, {"fp64_emulation": 1, "dtype": P.C128},
               {"fp64_emulation": 1, "unsym": 1}):
        with pytest.raises(P.PselinvError) as e:
            P.SelInv(2, cp, ri, **kw)
        assert e.value.code == -1, kw
    P.SelInv(2, cp, ri, fp64_emulation=1)
    with pytest.raises(TypeError):
        P.SelInv(2, cp, ri, no_such_option=1)


def test_figure1_partition_levels_match_algorithm2(P):
    """The library's priority lists on the Figure 1 pattern (its own
    supernodes) agree with Algorithm 2 applied by the oracle."""
    from tests.test_oracle_pins import _read_fig1, lower_from_dense
    part, blocks, fill, snp, levels = _read_fig1()
    n = int(part[-1])
    M = np.zeros((n, n), bool)
    for k in range(len(part) - 1):
        M[part[k]:part[k + 1], part[k]:part[k + 1]] = True
    for br, bc, rows in blocks:
        M[np.ix_(rows, range(part[bc - 1], part[bc]))] = True
    M = M | M.T
    cp, ri, v = lower_from_dense(np.where(M, 1.0, 0.0))
    _compare(P, n, cp, ri, 128, 0)


def test_opts_structure_matches_the_c_layout(P):
    """pselinv_default_opts zeroes exactly sizeof(pselinv_opts) bytes and sets
    its defaults: run it on a sentinel-filled buffer larger than the ctypes
    Opts and check the extent it wrote and the fields at the ctypes offsets."""
    import ctypes
    n = ctypes.sizeof(P.Opts)
    buf = (ctypes.c_uint8 * (n + 64))(*([0xA5] * (n + 64)))
    P.load_library().pselinv_default_opts(ctypes.cast(buf, ctypes.POINTER(P.Opts)))
    assert all(b == 0xA5 for b in buf[n:]), "the C structure is larger than the ctypes one"
    o = P.Opts.from_buffer(buf)
    assert (o.dtype, o.batch, o.max_sn_width, o.relax, o.small_cutoff, o.split_k_rows) == (P.F64, 1, 128,
                                                                                          P.RELAX_AMALG, -1, 1024)
    assert (o.debug_checks, o.unsym, o.spin_limit_ns, o.level_tiles, o.min_slice_rows, o.fp64_emulation) == (
        0, 0, 1000000000, 0, 0, 0)


def test_pole_sum_state_checks_run_on_the_host(P):
    """pselinv_selinv_pole_sum and pselinv_pole_sum check their arguments and
    the handle's state before any device work (called through the C ABI with
    a NULL stream, no GPU needed): NULL output -> ERR_ARG, no factor ->
    ERR_STATE, a non-symmetric handle -> ERR_STATE."""
    import ctypes
    lib = P.load_library()
    cp = np.array([0, 2, 4, 5], np.int64)
    ri = np.array([0, 1, 1, 2, 2], np.int32)
    h = P.SelInv(3, cp, ri, dtype=P.C128, batch=2)
    w = np.ones(4, np.float64)                     # two complex weights as (re, im) pairs
    out = np.zeros(2 * h.info["panel_entries"], np.float64)
    wp, op = ctypes.c_void_p(w.ctypes.data), ctypes.c_void_p(out.ctypes.data)
    for fn in (lib.pselinv_selinv_pole_sum, lib.pselinv_pole_sum):
        assert fn(h._h, wp, None, None) == -1      # ERR_ARG
        assert fn(h._h, wp, op, None) == -8        # ERR_STATE: nothing factored / inverted
    hu = P.SelInv(3, cp, ri, unsym=1)
    assert lib.pselinv_selinv_pole_sum(hu._h, wp, op, None) == -8


@pytest.mark.parametrize("case", ["grid3d_12", "graphlap_10", "random_perm"])
def test_schur_groups_have_disjoint_targets(P, case):
    """The factorisation's Schur update runs the supernodes of a level in
    groups, each group one launch with plain read-modify-writes (no atomics).
    That is race-free only if no two supernodes of a group update the same
    ancestor entry, i.e. (the analysis's sufficient condition) their sets C
    are disjoint.  Checked on the exported groups: every group lies in one
    level, its C sets are pairwise disjoint, and every supernode with a
    non-empty C is in exactly one group of its level."""
    if case == "grid3d_12":
        p = synth.grid3d(12)
        h = P.SelInv(p.n, p.colptr, p.rowind, max_sn_width=16, relax=P.RELAX_AMALG)
    elif case == "graphlap_10":
        gl = synth.GraphLaplacian((10, 10, 10))
        h = P.SelInv(gl.n, gl.colptr, gl.rowind, perm=synth.nd_order(gl.dims), max_sn_width=8)
    else:
        p = synth.grid3d(9)
        perm = np.random.default_rng(4).permutation(p.n).astype(np.int32)
        h = P.SelInv(p.n, p.colptr, p.rowind, perm=perm, max_sn_width=32)
    sym = h.symbolic()
    lp, ls, gp = sym["level_ptr"], sym["level_sn"], sym["group_ptr"]
    gsp, gsn, rp, rows = sym["group_sn_ptr"], sym["group_sn"], sym["rowptr"], sym["rows"]
    assert gp[0] == 0 and gp[-1] == len(gsp) - 1
    seen = np.zeros(sym["nsn"], int)
    ngroups_max = 0
    for l in range(sym["nlevels"]):
        level = set(ls[lp[l]:lp[l + 1]].tolist())
        ngroups_max = max(ngroups_max, gp[l + 1] - gp[l])
        for g in range(gp[l], gp[l + 1]):
            members = gsn[gsp[g]:gsp[g + 1]]
            assert set(members.tolist()) <= level
            covered = set()
            for k in members:
                C = set(rows[rp[k]:rp[k + 1]].tolist())
                assert not (C & covered), (l, g, k)
                covered |= C
                seen[k] += 1
    r = np.diff(rp)
    assert np.all(seen[r > 0] == 1) and np.all(seen <= 1)
    assert ngroups_max > 1          # the cases do have levels whose supernodes conflict
