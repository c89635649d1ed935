"""The allocation-free entry point pselinv_block_inverse_static, called
through the C ABI.  It exists for callers that cannot call cudaMalloc or
cudaFree: code that runs inside another framework's memory pool or under a
fixed memory budget, and loops that must never block on the allocator
(cudaFree synchronises the device, cudaMalloc can stall).  Its only scratch
is a fixed device array inside the library.

Each block's result is checked against numpy's inverse of that block and
against the selected inversion of the regular entry points on the same
factor, on two calls in a row with different inputs; a further check
shows that a call allocates nothing (free device memory and torch's
allocation counters unchanged).  Collected last on purpose."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1404_0447_gb300 as P
    return P


def dense_batch(s, count, seed):
    """count SPD s x s blocks and their lower-CSC pattern and values."""
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(count):
        G = rng.normal(size=(s, s))
        mats.append(G @ G.T / s + np.eye(s))
    rows, cols = np.tril_indices(s)
    cp, ri, _ = synth.lower_csc_from_coo(s, rows, cols, np.ones(rows.size))
    c = np.repeat(np.arange(s), np.diff(cp))
    vals = np.stack([A[ri, c] for A in mats])
    return mats, cp, ri, vals


def factor_blocks(P, s, count, seed):
    """LDL^T of each block through the regular entry points: (A_b list, L panels
    [count, s*s] with the pivots on the diagonal, pivots [count, s], X panels)."""
    import torch
    mats, cp, ri, vals = dense_batch(s, count, seed)
    h = P.SelInv(s, cp, ri, batch=count, max_sn_width=128, relax=P.RELAX_AMALG)
    assert h.info["nsn"] == 1                               # one dense supernode
    h.factor(torch.tensor(vals, dtype=torch.float64, device="cuda"))
    h.selinv(P.LEVEL)
    X = h.panels(0).clone()                                 # A^{-1} from the regular path
    Lp = h.panels(1).contiguous().clone()
    d = torch.diagonal(Lp.view(count, s, s), dim1=1, dim2=2).contiguous()
    torch.cuda.synchronize()
    return mats, Lp, d, X


@pytest.mark.parametrize("s,count", [(100, 3), (128, 2), (7, 5)])
def test_two_calls_match_numpy_inverse_and_selinv(P, s, count):
    import torch
    for call, seed in enumerate((11, 12)):                 # two calls in a row, different inputs
        mats, Lp, d, X = factor_blocks(P, s, count, seed + s)
        M = P.block_inverse_static(Lp, d)
        torch.cuda.synchronize()
        Mh = M.cpu().numpy().reshape(count, s, s).transpose(0, 2, 1)   # column-major blocks
        for b, A in enumerate(mats):
            Ai = np.linalg.inv(A)
            err = np.max(np.abs(Mh[b] - Ai)) / np.max(np.abs(Ai))
            assert err <= TOL, (call, b, err)
        err = (torch.max(torch.abs(M - X)) / torch.max(torch.abs(X))).item()
        assert err <= TOL, (call, err)


def test_a_call_allocates_nothing(P):
    import torch
    s, count = 64, 4
    mats, Lp, d, X = factor_blocks(P, s, count, 5)
    out = torch.empty(count, s * s, dtype=torch.float64, device="cuda")
    P.block_inverse_static(Lp, d, out=out)                 # first call: per-device set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = torch.cuda.memory_stats()
    for _ in range(3):
        P.block_inverse_static(Lp, d, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    stats1 = torch.cuda.memory_stats()
    for key in ("allocation.all.allocated", "segment.all.allocated"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    Ai = np.linalg.inv(mats[0])
    M0 = out[0].cpu().numpy().reshape(s, s).T
    assert np.max(np.abs(M0 - Ai)) / np.max(np.abs(Ai)) <= TOL


def test_rejects_sizes_beyond_the_static_scratch(P):
    import torch
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = P.load_library()
    ptr = P.ctypes.c_void_p(L.data_ptr())
    rc = lib.pselinv_block_inverse_static(128, 129, ptr, ptr, ptr, None)   # 129 * 128^2 > 2^21 doubles
    assert P.ERRORS[rc] == "ERR_ARG" and "static scratch" in lib.pselinv_last_error(None).decode()
    rc = lib.pselinv_block_inverse_static(129, 1, ptr, ptr, ptr, None)     # order above 128
    assert P.ERRORS[rc] == "ERR_ARG"
