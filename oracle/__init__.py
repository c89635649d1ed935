"""CPU oracle for supernodal selected inversion -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU
library (``paper_1404_0447_gb300``) and never imports it.

The arithmetic lives in ``oracle.c`` / ``oracle_num.h`` (plain scalar C:
column LDL^T and the column form of the selected-inversion recurrence,
Eqs. 7-13 and Algorithm 1 of the paper).  This module is the ctypes
binding plus a few plain numpy definitions used as independent pins:

* ``dense_inverse`` -- numpy's dense inverse (tiny inputs);
* ``laplacian_1d_inverse`` -- the textbook closed form of tridiag(-1,2,-1)^{-1};
* ``grid_inverse_entries`` -- the separable eigen-expansion of the inverse of
  a Dirichlet grid Laplacian with a constant shift;
* ``trace_error`` -- the accuracy measure E of Section 4.3, Eq. (16);
* ``dense_adjoint`` -- the gradient -(X G X) restricted to A's pattern.

Every function pinned by tests/test_oracle_pins.py; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_liboracle.so")
_lib = None

i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
c128p = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c into _liboracle.so with gcc (no FMA contraction so
    x86 and Arm hosts round identically)."""
    src = [os.path.join(_HERE, "oracle.c")]
    deps = src + [os.path.join(_HERE, "oracle_num.h")]
    if (not force and os.path.exists(_SO)
            and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in deps)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp] + src + ["-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        L.orc_etree.argtypes = [ctypes.c_int32, i64p, i32p, i32p]
        L.orc_postorder.argtypes = [ctypes.c_int32, i32p, i32p]
        L.orc_sym_new.argtypes = [ctypes.c_int32, i64p, i32p]
        L.orc_sym_new.restype = ctypes.c_void_p
        L.orc_sym_nnzl.argtypes = [ctypes.c_void_p]
        L.orc_sym_nnzl.restype = ctypes.c_int64
        L.orc_sym_get.argtypes = [ctypes.c_void_p, i32p, i64p, i32p]
        L.orc_sym_free.argtypes = [ctypes.c_void_p]
        L.orc_supernodes.argtypes = [ctypes.c_int32, i32p, i64p, ctypes.c_int32,
                                     ctypes.c_int32, i32p]
        L.orc_supernodes.restype = ctypes.c_int32
        L.orc_sn_struct.argtypes = [ctypes.c_int32, i64p, i32p, ctypes.c_int32, i32p, i32p,
                                    i32p, i64p, ctypes.c_void_p]
        L.orc_relidx.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i64p, i32p,
                                 ctypes.c_void_p, ctypes.c_void_p]
        L.orc_relidx.restype = ctypes.c_int64
        for sfx, vp in (("d", f64p), ("z", c128p)):
            f = getattr(L, f"orc_ldlt_{sfx}")
            f.argtypes = [ctypes.c_int32, i64p, i32p, vp, i64p, i32p, vp, vp]
            f = getattr(L, f"orc_selinv_{sfx}")
            f.argtypes = [ctypes.c_int32, i64p, i32p, vp, vp, vp, vp]
            f = getattr(L, f"orc_solve_{sfx}")
            f.argtypes = [ctypes.c_int32, i64p, i32p, vp, vp, vp]
            f = getattr(L, f"orc_ldu_{sfx}")
            f.argtypes = [ctypes.c_int32, i64p, i32p, vp, vp, i64p, i32p, vp, vp, vp]
            f = getattr(L, f"orc_selinv_lu_{sfx}")
            f.argtypes = [ctypes.c_int32, i64p, i32p, vp, vp, vp, vp, vp, vp]
            f = getattr(L, f"orc_solve_lu_{sfx}")
            f.argtypes = [ctypes.c_int32, i64p, i32p, vp, vp, vp, vp]
        L.orc_logdet_d.argtypes = [ctypes.c_int32, f64p, f64p]
        L.orc_logdet_z.argtypes = [ctypes.c_int32, c128p, f64p]
        _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


# --------------------------------------------------------------------------
# symbolic
# --------------------------------------------------------------------------

def etree(n, colptr, rowind):
    parent = np.empty(n, np.int32)
    if lib().orc_etree(n, _i64(colptr), _i32(rowind), parent):
        raise ValueError("pattern is not lower CSC with sorted rows and the diagonal first")
    return parent


def postorder(parent):
    n = len(parent)
    post = np.empty(n, np.int32)
    if lib().orc_postorder(n, _i32(parent), post):
        raise ValueError("not a forest")
    return post


def column_structure(n, colptr, rowind):
    """(parent, lcolptr, lrowind): etree and struct(j) strictly below the diagonal."""
    h = lib().orc_sym_new(n, _i64(colptr), _i32(rowind))
    if not h:
        raise ValueError("pattern is not lower CSC with sorted rows and the diagonal first")
    try:
        nnzl = lib().orc_sym_nnzl(h)
        parent = np.empty(n, np.int32)
        lcp = np.empty(n + 1, np.int64)
        lri = np.empty(max(nnzl, 1), np.int32)
        lib().orc_sym_get(h, parent, lcp, lri)
    finally:
        lib().orc_sym_free(h)
    return parent, lcp, lri[:nnzl]


def supernodes(parent, lcolptr, wmax, relax):
    n = len(parent)
    sn = np.empty(n + 1, np.int32)
    ns = lib().orc_supernodes(n, _i32(parent), _i64(lcolptr), int(wmax), int(relax), sn)
    return sn[:ns + 1].copy()


def sn_struct(n, lcolptr, lrowind, sn_start):
    """(sn_parent, sigma, rcount, rrows) for a partition (Section 2.2, Alg. 2)."""
    nsn = len(sn_start) - 1
    snp = np.empty(nsn, np.int32)
    sig = np.empty(nsn, np.int32)
    rc = np.empty(nsn, np.int64)
    L = lib()
    L.orc_sn_struct(n, _i64(lcolptr), _i32(lrowind), nsn, _i32(sn_start), snp, sig, rc, None)
    rrows = np.empty(max(int(rc.sum()), 1), np.int32)
    L.orc_sn_struct(n, _i64(lcolptr), _i32(lrowind), nsn, _i32(sn_start), snp, sig, rc,
                    rrows.ctypes.data_as(ctypes.c_void_p))
    return snp, sig, rc, rrows[:int(rc.sum())]


def relative_indices(n, sn_start, rcount, rrows):
    nsn = len(sn_start) - 1
    nblk = np.empty(nsn, np.int32)
    L = lib()
    tot = L.orc_relidx(n, nsn, _i32(sn_start), _i64(rcount), _i32(rrows), None, None)
    rel = np.empty(max(tot, 1), np.int32)
    L.orc_relidx(n, nsn, _i32(sn_start), _i64(rcount), _i32(rrows),
                 nblk.ctypes.data_as(ctypes.c_void_p), rel.ctypes.data_as(ctypes.c_void_p))
    return nblk, rel[:tot]


def supernodal_pattern(n, sn_start, rcount, rrows):
    """Column structure of the supernodal panels: for j in K,
    struct'(j) = {j+1, ..., last(K)} U R(K)."""
    sn_start = np.asarray(sn_start, np.int64)
    roff = np.concatenate([[0], np.cumsum(rcount)])
    counts = np.empty(n, np.int64)
    for k in range(len(sn_start) - 1):
        f, l = sn_start[k], sn_start[k + 1]
        counts[f:l] = (l - 1 - np.arange(f, l)) + rcount[k]
    lcp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    lri = np.empty(int(lcp[-1]), np.int32)
    for k in range(len(sn_start) - 1):
        f, l = int(sn_start[k]), int(sn_start[k + 1])
        R = rrows[roff[k]:roff[k + 1]]
        for j in range(f, l):
            lri[lcp[j]:lcp[j + 1]] = np.concatenate([np.arange(j + 1, l), R])
    return lcp, lri


def analyse(n, colptr, rowind, wmax=0, relax=0):
    """Full symbolic pipeline on an already ordered pattern.

    The etree is postordered first (children in increasing order); if that
    postorder is not the identity the pattern is relabelled by it and the
    returned ``post`` says how.  Returns a dict with the etree, the column
    structure of L, the supernode partition, supernodal parents, Algorithm 2
    priorities, row lists R(K) and the relative indices.
    """
    from synth import permute_lower  # index relabelling only
    parent = etree(n, colptr, rowind)
    post = postorder(parent)
    ident = np.array_equal(post, np.arange(n))
    if not ident:
        colptr, rowind, _, _ = permute_lower(n, colptr, rowind, np.zeros(len(rowind)), post)
    parent, lcp, lri = column_structure(n, colptr, rowind)
    sn = supernodes(parent, lcp, wmax, relax)
    snp, sig, rc, rr = sn_struct(n, lcp, lri, sn)
    nblk, rel = relative_indices(n, sn, rc, rr)
    return dict(n=n, post=post.astype(np.int64), colptr=colptr, rowind=rowind, parent=parent,
                lcolptr=lcp, lrowind=lri, sn_start=sn, sn_parent=snp, sigma=sig, rcount=rc,
                rrows=rr, nblk=nblk, relidx=rel)


# --------------------------------------------------------------------------
# numeric
# --------------------------------------------------------------------------

def _cplx(v):
    return np.iscomplexobj(v)


def ldlt(n, colptr, rowind, values, lcolptr, lrowind):
    """Pivot-free LDL^T on the given (elimination-closed) pattern."""
    cz = _cplx(values)
    dt = np.complex128 if cz else np.float64
    lv = np.zeros(len(lrowind), dt)
    d = np.zeros(n, dt)
    f = lib().orc_ldlt_z if cz else lib().orc_ldlt_d
    st = f(n, _i64(colptr), _i32(rowind), np.ascontiguousarray(values, dt), _i64(lcolptr),
           _i32(lrowind), lv, d)
    if st == -(n + 1):
        raise ValueError("A has entries outside the given L pattern")
    if st < 0:
        raise ZeroDivisionError(f"zero or non-finite pivot at column {-st - 1}")
    return lv, d


def selinv(n, lcolptr, lrowind, lvals, d):
    """Column selected inversion: X on the L pattern (xv) and its diagonal (xd)."""
    cz = _cplx(lvals)
    dt = np.complex128 if cz else np.float64
    xv = np.zeros(len(lrowind), dt)
    xd = np.zeros(n, dt)
    f = lib().orc_selinv_z if cz else lib().orc_selinv_d
    st = f(n, _i64(lcolptr), _i32(lrowind), np.ascontiguousarray(lvals, dt),
           np.ascontiguousarray(d, dt), xv, xd)
    if st < 0:
        raise ValueError(f"pattern not elimination-closed at column {-st - 1}")
    return xv, xd


def solve(n, lcolptr, lrowind, lvals, d, b):
    cz = _cplx(lvals) or _cplx(b)
    dt = np.complex128 if cz else np.float64
    x = np.array(b, dtype=dt, copy=True, order="C")
    f = lib().orc_solve_z if cz else lib().orc_solve_d
    f(n, _i64(lcolptr), _i32(lrowind), np.ascontiguousarray(lvals, dt),
      np.ascontiguousarray(d, dt), x)
    return x


def ldu(n, colptr, rowind, lower, upper, lcolptr, lrowind):
    """Pivot-free A = L D U' (non-symmetric values on a symmetric pattern).
    Returns (lv, uv, d): L_ij and U'_ji at the L positions (i, j), and D."""
    cz = _cplx(lower) or _cplx(upper)
    dt = np.complex128 if cz else np.float64
    lv = np.zeros(len(lrowind), dt)
    uv = np.zeros(len(lrowind), dt)
    d = np.zeros(n, dt)
    f = lib().orc_ldu_z if cz else lib().orc_ldu_d
    st = f(n, _i64(colptr), _i32(rowind), np.ascontiguousarray(lower, dt), np.ascontiguousarray(upper, dt),
           _i64(lcolptr), _i32(lrowind), lv, uv, d)
    if st == -(n + 1):
        raise ValueError("A has entries outside the given L pattern")
    if st < 0:
        raise ZeroDivisionError(f"zero or non-finite pivot at column {-st - 1}")
    return lv, uv, d


def selinv_lu(n, lcolptr, lrowind, lv, uv, d):
    """Non-symmetric column selected inversion: X_ij (xv) and X_ji (xu) at
    the L positions (i, j), and the diagonal xd."""
    cz = _cplx(lv) or _cplx(uv)
    dt = np.complex128 if cz else np.float64
    xv = np.zeros(len(lrowind), dt)
    xu = np.zeros(len(lrowind), dt)
    xd = np.zeros(n, dt)
    f = lib().orc_selinv_lu_z if cz else lib().orc_selinv_lu_d
    st = f(n, _i64(lcolptr), _i32(lrowind), np.ascontiguousarray(lv, dt), np.ascontiguousarray(uv, dt),
           np.ascontiguousarray(d, dt), xv, xu, xd)
    if st < 0:
        raise ValueError(f"pattern not elimination-closed at column {-st - 1}")
    return xv, xu, xd


def solve_lu(n, lcolptr, lrowind, lv, uv, d, b):
    cz = _cplx(lv) or _cplx(b)
    dt = np.complex128 if cz else np.float64
    x = np.array(b, dtype=dt, copy=True, order="C")
    f = lib().orc_solve_lu_z if cz else lib().orc_solve_lu_d
    f(n, _i64(lcolptr), _i32(lrowind), np.ascontiguousarray(lv, dt), np.ascontiguousarray(uv, dt),
      np.ascontiguousarray(d, dt), x)
    return x


def logdet(d):
    """Real: (sum log|d_j|, number of negative pivots).  Complex: sum of
    principal logs as (real, imaginary) -- not wrapped to (-pi, pi]."""
    out = np.zeros(2)
    if _cplx(d):
        lib().orc_logdet_z(len(d), np.ascontiguousarray(d, np.complex128), out)
    else:
        lib().orc_logdet_d(len(d), np.ascontiguousarray(d, np.float64), out)
    return out


# --------------------------------------------------------------------------
# pipeline helpers
# --------------------------------------------------------------------------

def selected_inverse(n, colptr, rowind, values, wmax=0, relax=0, pattern="supernodal"):
    """Analyse, factor and selectively invert on the supernodal (default) or
    the exact L pattern.  Returns (sym, lv, d, xv, xd, lcp, lri) where
    lcp/lri is the pattern used."""
    sym = analyse(n, colptr, rowind, wmax, relax)
    cp, ri = sym["colptr"], sym["rowind"]
    vals = values
    if not np.array_equal(sym["post"], np.arange(n)):
        from synth import permute_lower
        _, _, vals, _ = permute_lower(n, colptr, rowind, values, sym["post"])
    if pattern == "supernodal":
        lcp, lri = supernodal_pattern(n, sym["sn_start"], sym["rcount"], sym["rrows"])
    else:
        lcp, lri = sym["lcolptr"], sym["lrowind"]
    lv, d = ldlt(n, cp, ri, vals, lcp, lri)
    xv, xd = selinv(n, lcp, lri, lv, d)
    return sym, lv, d, xv, xd, lcp, lri


def selected_inverse_lu(n, colptr, rowind, lower, upper, wmax=0, relax=0, pattern="supernodal"):
    """Non-symmetric counterpart of ``selected_inverse``: returns
    (sym, lv, uv, d, xv, xu, xd, lcp, lri)."""
    sym = analyse(n, colptr, rowind, wmax, relax)
    cp, ri = sym["colptr"], sym["rowind"]
    lo, up = lower, upper
    if not np.array_equal(sym["post"], np.arange(n)):
        from synth import permute_lower_unsym
        _, _, lo, up, _, _ = permute_lower_unsym(n, colptr, rowind, lower, upper, sym["post"])
    if pattern == "supernodal":
        lcp, lri = supernodal_pattern(n, sym["sn_start"], sym["rcount"], sym["rrows"])
    else:
        lcp, lri = sym["lcolptr"], sym["lrowind"]
    lv, uv, d = ldu(n, cp, ri, lo, up, lcp, lri)
    xv, xu, xd = selinv_lu(n, lcp, lri, lv, uv, d)
    return sym, lv, uv, d, xv, xu, xd, lcp, lri


def panels_from_columns_lu(n, sn_start, rcount, rrows, lcp, xv, xu, xd):
    """Panels of a non-symmetric X: (offsets, XL, XU) where XL holds X_ij at
    panel position (i, j) (full diagonal block) and XU holds X_ji there."""
    off, XL = _panels(n, sn_start, rcount, lcp, xv, xu, xd)
    _, XU = _panels(n, sn_start, rcount, lcp, xu, xv, xd)
    return off, XL, XU


def panels_from_columns(n, sn_start, rcount, rrows, lcp, xv, xd):
    """Lay a column-form X on the supernodal pattern out as the panels the
    GPU library stores: per supernode K an (s+r) x s column-major block whose
    rows are cols(K) then R(K); the diagonal block is filled on both sides of
    the diagonal (X is symmetric).  Returns (panel offsets int64[nsn+1],
    flat values)."""
    return _panels(n, sn_start, rcount, lcp, xv, xv, xd)


def _panels(n, sn_start, rcount, lcp, below, above, xd):
    """Panel layout of column-form values: column j of K holds ``below``
    (struct(j) rows: j+1..last(K), then R(K)) under the diagonal; the
    diagonal block's part above the diagonal takes ``above`` mirrored."""
    nsn = len(sn_start) - 1
    s = np.diff(sn_start).astype(np.int64)
    r = np.asarray(rcount, np.int64)
    sizes = (s + r) * s
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    out = np.zeros(int(off[-1]), dtype=np.result_type(below, above, xd))
    for k in range(nsn):
        f, sk, rk = int(sn_start[k]), int(s[k]), int(r[k])
        ld = sk + rk
        P = np.zeros((sk, ld), dtype=out.dtype)        # P[col, row]: column-major panel
        for b in range(sk):
            j = f + b
            P[b, b] = xd[j]
            P[b, b + 1:] = below[lcp[j]:lcp[j + 1]]
            P[b + 1:sk, b] = above[lcp[j]:lcp[j] + sk - b - 1]   # (row b, col b+c) = mirror
        out[off[k]:off[k + 1]] = P.ravel()
    return off, out


# --------------------------------------------------------------------------
# plain definitions used as pins
# --------------------------------------------------------------------------

def dense_from_lower(n, colptr, rowind, values):
    dt = np.complex128 if _cplx(values) else np.float64
    A = np.zeros((n, n), dt)
    cols = np.repeat(np.arange(n), np.diff(colptr))
    A[rowind, cols] = values
    A[cols, rowind] = values
    return A


def dense_from_lower_lu(n, colptr, rowind, lower, upper):
    """Dense A from A_ij (``lower``) and A_ji (``upper``) on a lower pattern."""
    dt = np.complex128 if (_cplx(lower) or _cplx(upper)) else np.float64
    A = np.zeros((n, n), dt)
    cols = np.repeat(np.arange(n), np.diff(colptr))
    A[cols, rowind] = upper
    A[rowind, cols] = lower          # the diagonal takes ``lower``
    return A


def convdiff_inverse_entries(dims, beta, shift, pairs):
    """Entries of A^{-1} for the constant-coefficient upwind
    convection-diffusion operator A = sum_a (I x .. x T_a x .. x I) + shift I
    with T_a = tridiag(-(1 + b_a), 2, -(1 - b_a)) of order m_a, |b_a| < 1.

    With rho_a = sqrt((1 + b_a) / (1 - b_a)) and S = diag(rho^{p_a}) per
    axis, S^{-1} T_a S = tridiag(-t_a, 2, -t_a), t_a = sqrt(1 - b_a^2), whose
    eigenpairs are 2 - 2 t_a cos(k pi/(m+1)) and sine vectors.  Hence

      (A^{-1})_pq = prod_a rho_a^(p_a - q_a) *
        sum_k prod_a (2/(m_a+1)) sin(k_a p_a pi/(m_a+1)) sin(k_a q_a pi/(m_a+1))
              / (shift + sum_a (2 - 2 t_a cos(k_a pi/(m_a+1)))),

    the mode sum added with math.fsum; p, q natural indices (x fastest).
    """
    dims = [int(m) for m in dims]
    beta = [float(b) for b in beta][:len(dims)]
    ks = [np.arange(1, m + 1) for m in dims]
    tau = [math.sqrt(1.0 - b * b) for b in beta]
    rho = [math.sqrt((1.0 + b) / (1.0 - b)) for b in beta]
    lam = [2.0 - 2.0 * t * np.cos(k * np.pi / (m + 1)) for k, m, t in zip(ks, dims, tau)]
    grids = np.meshgrid(*lam[::-1], indexing="ij")
    denom = shift + sum(grids)
    out = np.empty(len(pairs))
    for t, (p, q) in enumerate(pairs):
        pc, qc = [], []
        pp, qq = int(p), int(q)
        for m in dims:
            pc.append(pp % m + 1); pp //= m
            qc.append(qq % m + 1); qq //= m
        fac = []
        for a, m in enumerate(dims):
            fac.append((2.0 / (m + 1)) * np.sin(ks[a] * pc[a] * np.pi / (m + 1))
                       * np.sin(ks[a] * qc[a] * np.pi / (m + 1)))
        num = fac[-1]
        for a in range(len(dims) - 2, -1, -1):
            num = np.multiply.outer(num, fac[a])
        scale = 1.0
        for a in range(len(dims)):
            scale *= rho[a] ** (pc[a] - qc[a])
        out[t] = scale * math.fsum((num / denom).ravel())
    return out


def dense_inverse(n, colptr, rowind, values):
    return np.linalg.inv(dense_from_lower(n, colptr, rowind, values))


def laplacian_1d_inverse(n):
    """(T^{-1})_{ij} = i (n + 1 - j) / (n + 1) for 1 <= i <= j <= n."""
    i = np.arange(1, n + 1)[:, None]
    j = np.arange(1, n + 1)[None, :]
    lo = np.minimum(i, j)
    hi = np.maximum(i, j)
    return lo * (n + 1 - hi) / (n + 1.0)


def grid_inverse_entries(dims, shift, pairs):
    """Entries of (L_grid + shift I)^{-1} for a Dirichlet box grid whose
    Laplacian L_grid has 2 on the diagonal per axis and -1 between
    neighbours.  The eigenvectors are products of sines, so

      X_pq = sum_k prod_a (2/(m_a+1)) sin(k_a p_a pi/(m_a+1)) sin(k_a q_a pi/(m_a+1))
                    / (shift + sum_a 4 sin^2(k_a pi / (2 (m_a+1)))).

    ``pairs`` are (p, q) natural (lexicographic, x fastest) node indices;
    the mode sum is added with math.fsum (exactly rounded).
    """
    dims = [int(m) for m in dims]
    ks = [np.arange(1, m + 1) for m in dims]
    lam = [4.0 * np.sin(k * np.pi / (2.0 * (m + 1))) ** 2 for k, m in zip(ks, dims)]
    # eigenvalue denominators on the full mode grid (axis order z, y, x for 3D)
    grids = np.meshgrid(*lam[::-1], indexing="ij")
    denom = shift + sum(grids)
    out = np.empty(len(pairs))
    for t, (p, q) in enumerate(pairs):
        pc, qc = [], []
        pp, qq = int(p), int(q)
        for m in dims:
            pc.append(pp % m + 1); pp //= m
            qc.append(qq % m + 1); qq //= m
        fac = []
        for a, m in enumerate(dims):
            fac.append((2.0 / (m + 1)) * np.sin(ks[a] * pc[a] * np.pi / (m + 1))
                       * np.sin(ks[a] * qc[a] * np.pi / (m + 1)))
        num = fac[-1]
        for a in range(len(dims) - 2, -1, -1):
            num = np.multiply.outer(num, fac[a])
        out[t] = math.fsum((num / denom).ravel())   # exactly rounded sum
    return out


def trace_error(n, colptr, rowind, avals, xvals_on_a):
    """E = |1 - (1/n) sum_{A_ij != 0} X_ij A_ji| (Section 4.3, Eq. 16),
    summed over the full symmetric pattern from the lower triangle."""
    cols = np.repeat(np.arange(n), np.diff(colptr))
    off = np.asarray(rowind) != cols
    s = np.sum(xvals_on_a * avals) + np.sum(xvals_on_a[off] * avals[off])
    return abs(1.0 - s / n)


def dense_adjoint(Ainv, G):
    """d<G, P_S(A^{-1})>/dA = -(A^{-1} G A^{-1}) (bilinear pairing, plain
    transpose), as a dense matrix; callers restrict it to A's pattern."""
    return -(Ainv @ G @ Ainv)
