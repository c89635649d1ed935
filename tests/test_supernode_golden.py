"""The supernode rule pinned to hand-derived partitions
(tests/golden/relaxed_supernodes.txt: a tridiagonal chain, a 5 x 5 grid in
natural order, and a pattern on either side of the 5% explicit-zero
threshold, with its equality case).  Both the oracle's orc_supernodes and
the library's host analysis (pselinv_analyze, no GPU work) must produce
exactly the derived sn_start arrays."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "relaxed_supernodes.txt")


def read_cases():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "case":
            kw = dict(x.split("=") for x in f[4:])
            cur = {"name": f[1], "kind": f[2], "arg": int(f[3]), "wmax": int(kw["wmax"]),
                   "relax": int(kw["relax"])}
        elif f[0] == "sn_start":
            cur["sn_start"] = [int(x) for x in f[1:]]
            cases.append(cur)
            cur = None
    return cases


CASES = read_cases()


def pattern(kind, arg):
    """Lower CSC pattern (values 1) of each case's matrix."""
    rows, cols = [], []
    if kind == "chain":
        n = arg
        for j in range(n):
            rows.append(j), cols.append(j)
            if j + 1 < n:
                rows.append(j + 1), cols.append(j)
    elif kind == "grid5":
        n = 25
        for y in range(5):
            for x in range(5):
                i = x + 5 * y
                rows.append(i), cols.append(i)
                if x < 4:
                    rows.append(i + 1), cols.append(i)
                if y < 4:
                    rows.append(i + 5), cols.append(i)
    elif kind in ("thresh15", "thresh15k1"):
        n, t = 15, arg
        sk = 2 if kind == "thresh15" else 1      # width of K
        S = range(sk, sk + t)
        for j in range(n):
            rows.append(j), cols.append(j)
        if sk == 2:
            rows.append(1), cols.append(0)
        for i in S:
            for j in range(sk):
                rows.append(i), cols.append(j)
        for j in range(sk, n):
            for i in range(j + 1, n):
                rows.append(i), cols.append(j)
    else:
        raise ValueError(kind)
    cp, ri, _ = synth.lower_csc_from_coo(n, rows, cols, np.ones(len(rows)))
    return n, cp, ri


def test_golden_file_has_every_case():
    assert {c["name"] for c in CASES} == {"chain10", "chain10_w4", "chain20_w16", "grid5", "grid5_w128",
                                           "grid5_w4", "thresh15_t10_w32", "thresh15_t9_w32",
                                           "thresh15_t10_w14", "thresh15_t10_w8", "thresh15k1_t7_w32",
                                           "thresh15k1_t8_w32"}


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_oracle_supernodes_match_hand_derivation(case):
    n, cp, ri = pattern(case["kind"], case["arg"])
    parent, lcp, lri = oracle.column_structure(n, cp, ri)
    assert np.array_equal(parent[:-1], np.arange(1, n))      # a path: postorder is the identity
    sn = oracle.supernodes(parent, lcp, case["wmax"], case["relax"])
    assert sn.tolist() == case["sn_start"]


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build_library()
    import paper_1404_0447_gb300 as P
    return P


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_library_analysis_matches_hand_derivation(P, case):
    n, cp, ri = pattern(case["kind"], case["arg"])
    relax = P.RELAX_AMALG if case["relax"] else P.RELAX_NONE
    h = P.SelInv(n, cp, ri, max_sn_width=case["wmax"] if case["wmax"] else 128, relax=relax)
    s = h.symbolic()
    assert np.array_equal(s["perm"], np.arange(n))
    assert s["sn_start"].tolist() == case["sn_start"]
