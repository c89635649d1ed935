"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only builds matrices and orderings: grids, geometric nested
dissection, the anisotropic graph Laplacian, the block-sparse DG-like matrix
with its pole shifts, and the uneven batch.  It contains none of the
selected-inversion arithmetic (no factorisation, no inverse, no symbolic
elimination) and imports neither the CUDA package nor the oracle.

Conventions
-----------
* A matrix is returned as the lower triangle (diagonal included) in CSC form:
  ``colptr`` int64[n+1], ``rowind`` int32[nnz] (sorted inside each column,
  diagonal first), ``values`` float64 or complex128 [nnz] (or [batch, nnz]).
* An ordering ``perm`` lists old indices in new order: new index ``k`` is old
  index ``perm[k]``, so the permuted matrix is ``B[k, l] = A[perm[k], perm[l]]``.
* Random numbers come from ``numpy.random.Generator(PCG64(seed))`` and are
  drawn in the order stated in each function's docstring.

The matrix families stand in for the paper's test problems (Section 4,
Tables 1-2): 2D/3D grid operators for the FEM-class matrices (pwtk,
parabolic_fem, ecology2, audikw_1) and a 48-dof-per-element block matrix for
DG_Graphene_2048 (n = 82,944), whose pole set follows the pole expansion of
Section 4.4.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

BASE_SEED = 20140447


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# sparse helpers (index manipulation only)
# --------------------------------------------------------------------------

def lower_csc_from_coo(n, rows, cols, vals):
    """Lower-triangular CSC (diagonal first, rows sorted) from COO triplets.

    Duplicate (row, col) pairs are summed, as in an assembly.  Entries with
    row < col are mirrored into the lower triangle.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    lo = np.maximum(rows, cols)
    hi = np.minimum(rows, cols)
    m = sp.coo_matrix((vals, (lo, hi)), shape=(n, n)).tocsc()
    m.sum_duplicates()
    m.sort_indices()
    return (m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.copy())


def permute_lower(n, colptr, rowind, values, perm):
    """Lower CSC of P A P^T given the lower CSC of A and ``perm`` (new -> old).

    ``values`` may be [nnz] or [batch, nnz].  Returns (colptr, rowind,
    values, src) where ``src[q]`` is the position in the input arrays that
    output position ``q`` was taken from.
    """
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n, dtype=np.int64)
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    r2 = inv[np.asarray(rowind, dtype=np.int64)]
    c2 = inv[cols]
    lo = np.maximum(r2, c2)
    hi = np.minimum(r2, c2)
    order = np.lexsort((lo, hi))            # by new column, then new row
    newcolptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(newcolptr, hi + 1, 1)
    newcolptr = np.cumsum(newcolptr)
    vals = np.asarray(values)
    newvals = vals[..., order]
    return newcolptr, lo[order].astype(np.int32), np.ascontiguousarray(newvals), order


def permute_lower_unsym(n, colptr, rowind, lower, upper, perm):
    """``permute_lower`` for a non-symmetric matrix with a symmetric pattern,
    held as ``lower`` (A_ij) and ``upper`` (A_ji) at the stored lower
    positions (i, j), i >= j.  An entry whose two indices swap order under
    the permutation lands transposed, so its two values trade places.
    Returns (colptr, rowind, lower, upper, src, flip) with ``flip[q]`` true
    where output position ``q`` was transposed."""
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n, dtype=np.int64)
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    flip_in = inv[np.asarray(rowind, dtype=np.int64)] < inv[cols]
    cp, ri, _, src = permute_lower(n, colptr, rowind, np.zeros(len(rowind)), perm)
    flip = flip_in[src]
    lo, up = np.asarray(lower), np.asarray(upper)
    new_lo = np.where(flip, up[..., src], lo[..., src])
    new_up = np.where(flip, lo[..., src], up[..., src])
    return cp, ri, np.ascontiguousarray(new_lo), np.ascontiguousarray(new_up), src, flip


def to_scipy_full_unsym(n, colptr, rowind, lower, upper):
    """Full scipy CSC matrix from the lower/upper value pair on a lower pattern."""
    lo = sp.csc_matrix((lower, rowind, colptr), shape=(n, n))
    up = sp.csc_matrix((upper, rowind, colptr), shape=(n, n))
    return (lo + up.T - sp.diags(up.diagonal())).tocsc()


def to_scipy_full(n, colptr, rowind, values):
    """Full symmetric scipy CSC matrix from the lower CSC (plain transpose)."""
    lower = sp.csc_matrix((values, rowind, colptr), shape=(n, n))
    diag = sp.diags(lower.diagonal())
    return (lower + lower.T - diag).tocsc()


# --------------------------------------------------------------------------
# geometric nested dissection (the reading of the paper's ordering step used
# here: ParMETIS / PT-Scotch are replaced by a deterministic geometric rule)
# --------------------------------------------------------------------------

def _lex(box, dims):
    """Old indices of the nodes of ``box`` in lexicographic order, x fastest."""
    (x0, x1), (y0, y1), (z0, z1) = box
    xs = np.arange(x0, x1)
    ys = np.arange(y0, y1)
    zs = np.arange(z0, z1)
    mx, my, _ = dims
    zz, yy, xx = np.meshgrid(zs, ys, xs, indexing="ij")
    return (xx + mx * (yy + my * zz)).ravel()


def nd_order(dims, leaf_volume: int = 8):
    """Geometric nested dissection of a box grid of extents ``dims`` (x, y, z).

    Rule: a box is a leaf if its volume is <= ``leaf_volume`` or its longest
    extent is < 3; a leaf's nodes are numbered lexicographically (x fastest).
    Otherwise the box is cut along its longest axis (ties: x before y before
    z) by the plane at local index floor((m-1)/2); the order is [left part,
    right part, separator plane], the plane's nodes lexicographic.
    Returns ``perm`` (new -> old), int64.
    """
    dims = tuple(int(d) for d in dims) + (1,) * (3 - len(dims))
    out = []

    def rec(box):
        ext = [b[1] - b[0] for b in box]
        vol = ext[0] * ext[1] * ext[2]
        if vol == 0:
            return
        if vol <= leaf_volume or max(ext) < 3:
            out.append(_lex(box, dims))
            return
        ax = int(np.argmax(ext))            # argmax returns the first maximum
        lo, hi = box[ax]
        c = lo + (ext[ax] - 1) // 2
        left = list(box); left[ax] = (lo, c)
        sep = list(box); sep[ax] = (c, c + 1)
        right = list(box); right[ax] = (c + 1, hi)
        rec(tuple(left))
        rec(tuple(right))
        out.append(_lex(tuple(sep), dims))

    rec(((0, dims[0]), (0, dims[1]), (0, dims[2])))
    perm = np.concatenate(out).astype(np.int64)
    assert perm.size == dims[0] * dims[1] * dims[2]
    return perm


# --------------------------------------------------------------------------
# matrix families
# --------------------------------------------------------------------------

def grid_edges(dims):
    """Nearest-neighbour edges of a Dirichlet-truncated box grid.

    Ordered x-edges, then y-edges, then z-edges; inside each group by the
    lower endpoint's lexicographic index (x fastest).  Returns (i, j) int64
    arrays with i < j.
    """
    dims = tuple(int(d) for d in dims) + (1,) * (3 - len(dims))
    mx, my, mz = dims
    idx = np.arange(mx * my * mz, dtype=np.int64).reshape(mz, my, mx)
    ei, ej = [], []
    if mx > 1:
        ei.append(idx[:, :, :-1].ravel()); ej.append(idx[:, :, 1:].ravel())
    if my > 1:
        ei.append(idx[:, :-1, :].ravel()); ej.append(idx[:, 1:, :].ravel())
    if mz > 1:
        ei.append(idx[:-1, :, :].ravel()); ej.append(idx[1:, :, :].ravel())
    if not ei:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(ei), np.concatenate(ej)


def grid_laplacian(dims, shift_lo, shift_hi, seed, shift_const=None):
    """Dirichlet-truncated 2D/3D Laplacian: off-diagonals -1 between in-grid
    neighbours, diagonal 2*d + s_i (d = number of axes with extent > 1).

    s_i ~ U(shift_lo, shift_hi) drawn once per node in natural lexicographic
    order (x fastest) before any permutation; ``shift_const`` replaces the
    draw by a constant (used for the separable closed-form check).
    Returns (n, colptr, rowind, values) in natural order.
    """
    dims = tuple(int(d) for d in dims)
    d = sum(1 for m in dims if m > 1)
    n = int(np.prod(dims))
    if shift_const is None:
        s = rng_for(seed).uniform(shift_lo, shift_hi, size=n)
    else:
        s = np.full(n, float(shift_const))
    ei, ej = grid_edges(dims)
    rows = np.concatenate([np.arange(n), ej])
    cols = np.concatenate([np.arange(n), ei])
    vals = np.concatenate([2.0 * d + s, -np.ones(ei.size)])
    colptr, rowind, values = lower_csc_from_coo(n, rows, cols, vals)
    return n, colptr, rowind, values


def convdiff_grid(dims, seed, beta=0.5, shift_lo=0.01, shift_hi=0.1, beta_const=None, shift_const=None):
    """Upwind convection-diffusion on a Dirichlet box grid: a non-symmetric
    matrix with the symmetric 2D/3D nearest-neighbour pattern.

    Along an edge (i, j), i < j, the lower entry is A_ji = -(1 + b_e) and the
    upper entry A_ij = -(1 - b_e).  Random form: b_e ~ U(-beta, beta) drawn
    per edge in ``grid_edges`` order, then s_i ~ U(shift_lo, shift_hi) per
    node; the diagonal is sum over the node's edges of (1 + |b_e|) plus s_i,
    so A is strictly diagonally dominant by rows and by columns (no pivoting
    needed).  Constant form (``beta_const`` = one b per axis, x y z, and
    ``shift_const``): b_e = b_axis and the diagonal is 2 d + shift_const,
    a Kronecker sum of Toeplitz tridiagonals with a closed-form inverse.
    Returns (n, colptr, rowind, lower, upper) in natural order.
    """
    dims = tuple(int(m) for m in dims)
    d = sum(1 for m in dims if m > 1)
    n = int(np.prod(dims))
    ei, ej = grid_edges(dims)
    if beta_const is None:
        g = rng_for(seed)
        b = g.uniform(-beta, beta, size=ei.size)
        s = g.uniform(shift_lo, shift_hi, size=n)
        diag = s.copy()
        np.add.at(diag, ei, 1.0 + np.abs(b))
        np.add.at(diag, ej, 1.0 + np.abs(b))
    else:
        bc = np.asarray(beta_const, dtype=np.float64)
        b = bc[_edge_axes(dims, ei, ej)]
        diag = np.full(n, 2.0 * d + float(shift_const if shift_const is not None else 0.0))
    rows = np.concatenate([np.arange(n), ej])
    cols = np.concatenate([np.arange(n), ei])
    colptr, rowind, lower = lower_csc_from_coo(n, rows, cols, np.concatenate([diag, -(1.0 + b)]))
    _, _, upper = lower_csc_from_coo(n, rows, cols, np.concatenate([diag, -(1.0 - b)]))
    return n, colptr, rowind, lower, upper


def _edge_axes(dims, ei, ej):
    """Axis (0 = x, 1 = y, 2 = z) of every grid edge."""
    dd = tuple(int(m) for m in dims) + (1,) * (3 - len(dims))
    mx, my, _ = dd
    xi, yi, zi = ei % mx, (ei // mx) % my, ei // (mx * my)
    xj, yj, zj = ej % mx, (ej // mx) % my, ej // (mx * my)
    return np.where(xi != xj, 0, np.where(yi != yj, 1, 2)).astype(np.int64)


def laplacian_1d(n):
    """tridiag(-1, 2, -1) of order n, lower CSC."""
    i = np.arange(n - 1)
    rows = np.concatenate([np.arange(n), i + 1])
    cols = np.concatenate([np.arange(n), i])
    vals = np.concatenate([np.full(n, 2.0), -np.ones(n - 1)])
    return (n,) + lower_csc_from_coo(n, rows, cols, vals)


class GraphLaplacian:
    """A(theta) = sum_e theta_e (e_i - e_j)(e_i - e_j)^T + shift * I on a
    Dirichlet-truncated grid (no boundary edges), natural order.

    theta_e = exp(N(0, sigma^2)) drawn per edge in ``grid_edges`` order.
    ``assemble(theta)`` gives the lower-CSC values for any theta; the
    position of each edge's off-diagonal entry and of both endpoint
    diagonals is kept for the chain rule d/dtheta_e.
    """

    def __init__(self, dims, sigma=0.5, shift=0.05, seed=BASE_SEED + 2):
        self.dims = tuple(int(m) for m in dims)
        self.n = int(np.prod(self.dims))
        self.ei, self.ej = grid_edges(self.dims)
        self.shift = float(shift)
        self.theta = np.exp(rng_for(seed).normal(0.0, sigma, size=self.ei.size))
        n = self.n
        rows = np.concatenate([np.arange(n), self.ej])
        cols = np.concatenate([np.arange(n), self.ei])
        pat = sp.coo_matrix((np.ones(rows.size), (rows, cols)), shape=(n, n)).tocsc()
        pat.sort_indices()
        self.colptr = pat.indptr.astype(np.int64)
        self.rowind = pat.indices.astype(np.int32)
        # position lookup: diag of node k, and the (ej, ei) entry of each edge
        self.pos_diag = self._pos(np.arange(n), np.arange(n))
        self.pos_edge = self._pos(self.ej, self.ei)

    def _pos(self, r, c):
        r = np.asarray(r, np.int64); c = np.asarray(c, np.int64)
        # global key = col * n + row is increasing along the sorted CSC order
        cols = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.colptr))
        keys = cols * self.n + self.rowind.astype(np.int64)
        out = np.searchsorted(keys, c * self.n + r)
        assert np.all(keys[out] == c * self.n + r)
        return out

    def assemble_torch(self, theta):
        """Differentiable torch version of ``assemble`` (theta: float64 tensor)."""
        import torch
        dev = theta.device
        idx = lambda a: torch.as_tensor(a, dtype=torch.int64, device=dev)
        v = torch.zeros(self.rowind.size, dtype=theta.dtype, device=dev)
        v = v.index_add(0, idx(self.pos_diag), torch.full((self.n,), self.shift, dtype=theta.dtype, device=dev))
        v = v.index_add(0, idx(self.pos_diag[self.ei]), theta)
        v = v.index_add(0, idx(self.pos_diag[self.ej]), theta)
        v = v.index_add(0, idx(self.pos_edge), -theta)
        return v

    def assemble(self, theta=None):
        theta = self.theta if theta is None else np.asarray(theta, np.float64)
        v = np.zeros(self.rowind.size)
        np.add.at(v, self.pos_diag, self.shift)
        np.add.at(v, self.pos_diag[self.ei], theta)
        np.add.at(v, self.pos_diag[self.ej], theta)
        v[self.pos_edge] -= theta
        return v


def dg_block_matrix(elems=(12, 12, 12), nb=48, npoles=16, seed=BASE_SEED + 3):
    """DG-like block-sparse Hamiltonian H and complex shifts z_l.

    Elements on a non-periodic box grid, ``nb`` basis functions each; element
    e couples to its face neighbours.  Draw order: for each element e in
    lexicographic order a G_e (nb x nb, iid N(0,1)); then for each face edge
    (x-edges, then y, then z, as in ``grid_edges``) a B (nb x nb, iid N(0,1));
    then t_l ~ U(0, pi) for the poles, sorted ascending.
    H_ee = (G_e + G_e^T) / (2 sqrt(nb)) + 2 I,  H_{e'e} = 0.1 B / sqrt(nb),
    z_l = 0.5 (1 + cos t_l) + 0.5 i sin t_l,  A_l = H - z_l I.
    Degrees of freedom of one element are contiguous (dof = e * nb + a).
    Returns (n, colptr, rowind, Hvalues, z) in natural order.
    """
    rng = rng_for(seed)
    ne = int(np.prod(elems))
    n = ne * nb
    sq = np.sqrt(nb)
    rows, cols, vals = [], [], []
    a = np.arange(nb)
    ii, jj = np.meshgrid(a, a, indexing="ij")
    for e in range(ne):
        g = rng.normal(0.0, 1.0, size=(nb, nb))
        h = (g + g.T) / (2.0 * sq) + 2.0 * np.eye(nb)
        m = ii >= jj
        rows.append(e * nb + ii[m]); cols.append(e * nb + jj[m]); vals.append(h[m])
    ei, ej = grid_edges(elems)
    for e1, e2 in zip(ei, ej):
        b = rng.normal(0.0, 1.0, size=(nb, nb)) * (0.1 / sq)
        rows.append(e2 * nb + ii.ravel()); cols.append(e1 * nb + jj.ravel()); vals.append(b.ravel())
    t = np.sort(rng.uniform(0.0, np.pi, size=npoles))
    z = 0.5 * (1.0 + np.cos(t)) + 0.5j * np.sin(t)
    colptr, rowind, values = lower_csc_from_coo(
        n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return n, colptr, rowind, values, z


def block_nd_order(elems, nb, leaf_volume=8):
    """Nested dissection on the element grid; each element's dofs stay
    contiguous in basis order."""
    eperm = nd_order(elems, leaf_volume)
    return (eperm[:, None] * nb + np.arange(nb)[None, :]).ravel()


def shifted_values(n, colptr, rowind, hvalues, z):
    """Lower-CSC values of H - z_l I for every pole: complex128 [npoles, nnz]."""
    cols = np.repeat(np.arange(n), np.diff(colptr))
    isdiag = rowind.astype(np.int64) == cols
    out = np.repeat(hvalues[None, :].astype(np.complex128), len(z), axis=0)
    out[:, isdiag] -= np.asarray(z)[:, None]
    return out


def uneven_batch_specs(count=48, seed=BASE_SEED + 4):
    """Member b even: 2D grid, side ~ U{64..512}; b odd: 3D grid, side ~
    U{16..48} (inclusive).  One draw per member, in member order; each
    member's shifts come from seed + 1000 + b."""
    rng = rng_for(seed)
    specs = []
    for b in range(count):
        if b % 2 == 0:
            m = int(rng.integers(64, 513))
            specs.append(((m, m), BASE_SEED + 4 + 1000 + b))
        else:
            m = int(rng.integers(16, 49))
            specs.append(((m, m, m), BASE_SEED + 4 + 1000 + b))
    return specs


# --------------------------------------------------------------------------
# the five workloads, permuted by nested dissection
# --------------------------------------------------------------------------

class Problem:
    """One symmetric matrix (or a batch sharing a pattern) in ND order."""

    def __init__(self, name, n, colptr, rowind, values, perm, dims=None, extra=None):
        self.name = name
        self.n = n
        self.perm = perm
        self.colptr, self.rowind, self.values, self.src = permute_lower(
            n, colptr, rowind, values, perm)
        self.dims = dims
        self.extra = extra or {}

    @property
    def nnz(self):
        return int(self.rowind.size)


def grid_problem(dims, shift_lo, shift_hi, seed, shift_const=None, name=None):
    n, cp, ri, v = grid_laplacian(dims, shift_lo, shift_hi, seed, shift_const)
    return Problem(name or f"grid{'x'.join(map(str, dims))}", n, cp, ri, v,
                   nd_order(dims), dims=tuple(dims))


def grid2d_31(shift_const=None):
    """31x31 5-point grid, diag 4 + U(0.1, 1)."""
    return grid_problem((31, 31), 0.1, 1.0, BASE_SEED + 0, shift_const, "grid2d_31")


def grid3d(side=80, shift_const=None):
    """80^3 7-point grid, diag 6 + U(0.01, 0.1); ``side`` gives smaller
    members of the same family."""
    return grid_problem((side, side, side), 0.01, 0.1, BASE_SEED + 1, shift_const,
                        f"grid3d_{side}")


def graph_laplacian3d(side=48):
    gl = GraphLaplacian((side, side, side))
    perm = nd_order(gl.dims)
    p = Problem(f"graphlap3d_{side}", gl.n, gl.colptr, gl.rowind, gl.assemble(), perm,
                dims=gl.dims, extra={"graph": gl})
    return p


def dg_poles(elems=(12, 12, 12), nb=48, npoles=16):
    n, cp, ri, hv, z = dg_block_matrix(elems, nb, npoles)
    vals = shifted_values(n, cp, ri, hv, z)
    perm = block_nd_order(elems, nb)
    return Problem(f"dg{'x'.join(map(str, elems))}_nb{nb}", n, cp, ri, vals, perm,
                   dims=tuple(elems), extra={"z": z, "H": hv})


def uneven_member(spec):
    dims, seed = spec
    return grid_problem(dims, 0.1, 1.0, seed, None, f"grid{'x'.join(map(str, dims))}")


class UnsymProblem:
    """One non-symmetric matrix with a symmetric pattern, in ND order:
    ``values`` holds A_ij and ``values_up`` A_ji at the stored lower
    positions; ``flip`` marks entries the ordering transposed."""

    def __init__(self, name, n, colptr, rowind, lower, upper, perm, dims=None, extra=None):
        self.name = name
        self.n = n
        self.perm = perm
        (self.colptr, self.rowind, self.values, self.values_up, self.src,
         self.flip) = permute_lower_unsym(n, colptr, rowind, lower, upper, perm)
        self.dims = dims
        self.extra = extra or {}

    @property
    def nnz(self):
        return int(self.rowind.size)


def convdiff_problem(side=80, beta_const=None, shift_const=None, dims=None):
    """Upwind convection-diffusion on a side^3 grid (or ``dims``), random
    per-edge convection b_e ~ U(-0.5, 0.5) unless ``beta_const`` is given;
    same ND ordering as the symmetric grid workloads."""
    dims = tuple(dims) if dims is not None else (side, side, side)
    n, cp, ri, lo, up = convdiff_grid(dims, BASE_SEED + 5, beta_const=beta_const, shift_const=shift_const)
    return UnsymProblem(f"convdiff{'x'.join(map(str, dims))}", n, cp, ri, lo, up, nd_order(dims),
                        dims=dims, extra={"beta_const": beta_const, "shift_const": shift_const})
