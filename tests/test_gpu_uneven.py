"""Uneven batches: independent matrices with their own patterns analysed as
one block-diagonal matrix (pselinv_analyze_batch), so each level of
Algorithm 2 is one grouped launch over every member."""
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


def members_small():
    rng = np.random.default_rng(44)
    out = []
    for b in range(7):
        if b % 2 == 0:
            m = int(rng.integers(6, 21))
            out.append(synth.grid_problem((m, m), 0.1, 1.0, 500 + b))
        else:
            m = int(rng.integers(4, 8))
            out.append(synth.grid_problem((m, m, m), 0.1, 1.0, 500 + b))
    return out


def test_small_uneven_batch_against_oracle(P):
    import torch
    mem = members_small()
    h = P.SelInv([m.n for m in mem], [m.colptr for m in mem], [m.rowind for m in mem], max_sn_width=16)
    vals = np.concatenate([m.values for m in mem])
    h.factor(torch.tensor(vals, dtype=torch.float64, device="cuda"))
    levels = h.info["nlevels"]
    assert levels == max(P.SelInv(m.n, m.colptr, m.rowind, max_sn_width=16).info["nlevels"] for m in mem)
    for mode in (P.GRAPH, P.PLAIN, P.PERSISTENT):
        h.selinv(mode)
        sel = h.selected()[0].cpu().numpy()
        q0 = 0
        for m in mem:
            Ainv = oracle.dense_inverse(m.n, m.colptr, m.rowind, m.values)
            cols = np.repeat(np.arange(m.n), np.diff(m.colptr))
            got = sel[q0:q0 + m.nnz]
            assert np.max(np.abs(got - Ainv[m.rowind, cols])) <= TOL * np.max(np.abs(Ainv))
            q0 += m.nnz
    ld = h.logdet()[0, 0]
    want = sum(np.linalg.slogdet(oracle.dense_from_lower(m.n, m.colptr, m.rowind, m.values))[1] for m in mem)
    assert abs(ld - want) <= 1e-12 * abs(want)


@pytest.mark.slow
def test_full_uneven_batch_48_members_against_single_handles(P):
    """The 48-member uneven batch (2D sides U{64..512}, 3D sides U{16..48}),
    merged and graph-replayed, against each member inverted on its own
    handle (same kernels, one matrix): every member's selected entries at
    A's positions agree to rounding (a merged level can cut step 2 into other
    slices than the member's own level, so the sums differ in order), and
    every member satisfies the trace identity E of Eq. (16)."""
    import torch
    specs = synth.uneven_batch_specs()
    mem = [synth.uneven_member(s) for s in specs]
    h = P.SelInv([m.n for m in mem], [m.colptr for m in mem], [m.rowind for m in mem])
    vals = np.concatenate([m.values for m in mem])
    h.factor(torch.tensor(vals, dtype=torch.float64, device="cuda"))
    h.selinv(P.GRAPH)
    sel = h.selected()[0].cpu().numpy()
    h.close()
    q0 = 0
    rng = np.random.default_rng(0)
    check = set(rng.choice(len(mem), 6, replace=False).tolist())
    for b, m in enumerate(mem):
        got = sel[q0:q0 + m.nnz]
        q0 += m.nnz
        assert oracle.trace_error(m.n, m.colptr, m.rowind, m.values, got) < 1e-11
        if b in check:
            h1 = P.SelInv(m.n, m.colptr, m.rowind)
            h1.factor(torch.tensor(m.values, dtype=torch.float64, device="cuda"))
            h1.selinv(P.LEVEL)
            ref = h1.selected()[0].cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
            h1.close()
