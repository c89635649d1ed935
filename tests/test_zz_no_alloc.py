"""The allocation-free entry point pselinv_block_inverse_static, called
through the C ABI, against the selected inversion of the regular entry
points on the same matrices.  It exists for callers that may not call
cudaMalloc/cudaFree (another framework's memory pool, a fixed memory budget,
loops that must not block on the allocator); its scratch is a fixed device
array inside the library.  Collected last on purpose."""
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
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(count):
        G = rng.normal(size=(s, s))
        mats.append(G @ G.T / s + np.eye(s))
    rows, cols = np.tril_indices(s)
    cp, ri, _ = synth.lower_csc_from_coo(s, rows, cols, np.ones(rows.size))
    order = np.lexsort((rows, cols))                      # CSC order: by column, then row
    vals = np.stack([A[rows[order], cols[order]] for A in mats])
    return cp, ri, vals


@pytest.mark.parametrize("s,count", [(100, 3), (128, 2), (7, 5)])
def test_matches_selinv_on_two_calls(P, s, count):
    import torch
    outs = []
    for call, seed in enumerate((11, 12)):
        cp, ri, vals = dense_batch(s, count, seed + s)
        h = P.SelInv(s, cp, ri, batch=count, max_sn_width=128, relax=P.RELAX_AMALG)
        assert h.info["nsn"] == 1                          # one dense supernode
        h.factor(torch.tensor(vals, dtype=torch.float64, device="cuda"))
        h.selinv(P.LEVEL)
        X = h.panels(0)                                    # [count, s*s]: A^{-1} from the regular path
        Lp = h.panels(1).contiguous()                      # L with the pivots on the diagonal slots
        d = torch.diagonal(Lp.view(count, s, s), dim1=1, dim2=2).contiguous()
        M = P.block_inverse_static(Lp, d)
        torch.cuda.synchronize()
        err = (torch.max(torch.abs(M - X)) / torch.max(torch.abs(X))).item()
        assert err <= TOL, (call, err)
        outs.append(M.clone())
    assert not torch.equal(outs[0], outs[1])               # the second call did not reuse stale data


def test_rejects_sizes_beyond_the_static_scratch(P):
    import torch
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PselinvError) as e:
        rc = P.load_library().pselinv_block_inverse_static(
            128, 129, P.ctypes.c_void_p(L.data_ptr()), P.ctypes.c_void_p(L.data_ptr()),
            P.ctypes.c_void_p(L.data_ptr()), None)
        if rc != 0:
            raise P.PselinvError(rc, P.load_library().pselinv_last_error(None).decode())
    assert e.value.code == -1 and "static scratch" in str(e.value)
    with pytest.raises(P.PselinvError):
        rc = P.load_library().pselinv_block_inverse_static(
            129, 1, P.ctypes.c_void_p(L.data_ptr()), P.ctypes.c_void_p(L.data_ptr()),
            P.ctypes.c_void_p(L.data_ptr()), None)
        if rc != 0:
            raise P.PselinvError(rc, P.load_library().pselinv_last_error(None).decode())
