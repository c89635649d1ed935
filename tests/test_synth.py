"""The seeded generators: orderings are permutations, separators separate,
matrices have the stated structure.  CPU only."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import synth


def test_nd_order_is_permutation_and_separates():
    dims = (9, 7, 5)
    perm = synth.nd_order(dims)
    n = int(np.prod(dims))
    assert np.array_equal(np.sort(perm), np.arange(n))
    # the last plane in the order is the top separator: removing it splits
    # the grid into the two halves numbered before it
    ei, ej = synth.grid_edges(dims)
    mx, my, mz = dims
    sep = perm[-(my * mz):]                      # x is the longest axis: a y-z plane
    xs = sep % mx
    assert np.all(xs == (mx - 1) // 2)
    keep = np.ones(n, bool)
    keep[sep] = False
    m = sp.coo_matrix((np.ones(ei.size), (ei, ej)), shape=(n, n)).tocsr()
    m = m[keep][:, keep]
    ncomp, lab = csg.connected_components(m, directed=False)
    assert ncomp == 2


def test_grid_laplacian_structure():
    n, cp, ri, v = synth.grid_laplacian((4, 3), 0.1, 1.0, 123)
    A = sp.csc_matrix((v, ri, cp), shape=(n, n)).toarray()
    A = A + np.tril(A, -1).T
    assert np.all((np.diag(A) >= 4.1) & (np.diag(A) <= 5.0))
    off = A - np.diag(np.diag(A))
    assert set(np.unique(off)) <= {0.0, -1.0}
    assert np.sum(off == -1) == 2 * (3 * 3 + 4 * 2)


def test_graph_laplacian_assembly():
    gl = synth.GraphLaplacian((3, 3, 2), seed=9)
    v = gl.assemble()
    A = sp.csc_matrix((v, gl.rowind, gl.colptr), shape=(gl.n, gl.n)).toarray()
    A = A + np.tril(A, -1).T
    want = 0.05 * np.eye(gl.n)
    for t, i, j in zip(gl.theta, gl.ei, gl.ej):
        e = np.zeros(gl.n); e[i] = 1; e[j] = -1
        want += t * np.outer(e, e)
    assert np.allclose(A, want, rtol=0, atol=1e-15)


def test_permute_lower_roundtrip():
    n, cp, ri, v = synth.grid_laplacian((5, 4), 0.1, 1.0, 1)
    perm = synth.nd_order((5, 4))
    cp2, ri2, v2, src = synth.permute_lower(n, cp, ri, v, perm)
    A = sp.csc_matrix((v, ri, cp), shape=(n, n)).toarray(); A = A + np.tril(A, -1).T
    B = sp.csc_matrix((v2, ri2, cp2), shape=(n, n)).toarray(); B = B + np.tril(B, -1).T
    assert np.array_equal(B, A[np.ix_(perm, perm)])
    assert np.array_equal(v2, v[src])


def test_dg_block_matrix_and_poles():
    n, cp, ri, hv, z = synth.dg_block_matrix((3, 2, 2), 4, 5, seed=3)
    assert n == 48
    assert np.all(np.diff(np.angle(z - 0.5)) > 0)   # t_l sorted ascending
    assert np.allclose(np.abs(z - 0.5), 0.5)
    vals = synth.shifted_values(n, cp, ri, hv, z)
    cols = np.repeat(np.arange(n), np.diff(cp))
    dg = ri == cols
    assert np.allclose(vals[:, dg], hv[dg][None, :] - z[:, None])
    assert np.array_equal(vals[:, ~dg].imag, np.zeros_like(vals[:, ~dg].imag))


def test_uneven_batch_specs():
    specs = synth.uneven_batch_specs()
    assert len(specs) == 48
    for b, (dims, seed) in enumerate(specs):
        if b % 2 == 0:
            assert len(dims) == 2 and 64 <= dims[0] <= 512
        else:
            assert len(dims) == 3 and 16 <= dims[0] <= 48
