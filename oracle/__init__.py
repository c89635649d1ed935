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

Pins (values fixed independently of this package), per function:

* the C sweeps and symbolic analysis -- listed in ``oracle.c``'s header;
* ``laplacian_1d_inverse``, ``grid_inverse_entries`` -- multiplied back
  against A to the identity (test_oracle_pins::test_laplacian_1d_closed_form_and_linear_work,
  test_grid_closed_form_is_the_inverse);
* ``convdiff_inverse_entries`` -- the same check for the non-symmetric form
  (test_oracle_lu_pins::test_convdiff_closed_form_is_the_inverse);
* ``trace_error`` -- E = 0 for the exact inverse of a 2D grid
  (test_trace_identity_grid2d_31);
* ``dense_adjoint`` -- central finite differences of <G, A^{-1}>
  (test_dense_adjoint_against_finite_differences);
* ``bk_block``, ``selected_inverse_bk``, ``logdet_bk`` -- scipy.linalg.ldl's
  Bunch-Kaufman pivots and dense inverses of indefinite matrices
  (tests/test_oracle_bk_pins.py);
* ``panels_from_columns``, ``panels_from_dense`` -- each other and numpy's
  dense inverse on relaxed supernodes (test_panel_layouts_against_the_dense_inverse);
  ``panels_from_columns_lu`` runs the same ``_panels`` layout twice.

None is "parity unpinned".
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
    x86 and Arm hosts round identically; OpenMP for the row-parallel
    timing variant of the column recurrence)."""
    src = [os.path.join(_HERE, "oracle.c")]
    deps = src + [os.path.join(_HERE, "oracle_num.h")]
    if (not force and os.path.exists(_SO)
            and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in deps)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
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
            f = getattr(L, f"orc_selinv_omp_{sfx}")
            f.argtypes = [ctypes.c_int32, i64p, i32p, vp, vp, vp, vp, ctypes.c_int32]
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


def selinv(n, lcolptr, lrowind, lvals, d, threads=None):
    """Column selected inversion: X on the L pattern (xv) and its diagonal (xd).
    threads=None: the plain single-thread recurrence; threads=t: the OpenMP
    row-parallel variant on t threads (bitwise the same result)."""
    cz = _cplx(lvals)
    dt = np.complex128 if cz else np.float64
    xv = np.zeros(len(lrowind), dt)
    xd = np.zeros(n, dt)
    args = (n, _i64(lcolptr), _i32(lrowind), np.ascontiguousarray(lvals, dt), np.ascontiguousarray(d, dt), xv, xd)
    if threads is None:
        f = lib().orc_selinv_z if cz else lib().orc_selinv_d
        st = f(*args)
    else:
        f = lib().orc_selinv_omp_z if cz else lib().orc_selinv_omp_d
        st = f(*args, int(threads))
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


# --------------------------------------------------------------------------
# symmetric indefinite: Bunch-Kaufman pivots inside supernodes
# --------------------------------------------------------------------------

BK_ALPHA = (1.0 + math.sqrt(17.0)) / 8.0


def _cabs1(x):
    """|re| + |im| (the magnitude Bunch-Kaufman compares for complex data)."""
    return np.abs(np.real(x)) + np.abs(np.imag(x))


def bk_block(W):
    """Bunch-Kaufman factorisation of one dense symmetric block (Bunch and
    Kaufman 1977, in the lower-triangle form of LAPACK's xSYTF2), with every
    interchange applied to the whole block so that

        W[p][:, p] = L D L^T,   L unit lower triangular, D block diagonal
        with 1x1 and 2x2 blocks (L is zero beside each 2x2 block).

    Column k of the reduced block: a = |W_kk|, colmax = max_{i>k} |W_ik| at
    imax.  a >= alpha colmax: 1x1 pivot.  Otherwise, with rowmax the largest
    off-diagonal magnitude in row/column imax of the reduced block:
    a rowmax >= alpha colmax^2 ->
    1x1; |W_imax,imax| >= alpha rowmax -> 1x1 after swapping k and imax;
    else 2x2 on (k, k+1) after swapping k+1 and imax.  alpha = (1+sqrt 17)/8.
    Returns (p, L, d, e, ptype): p[t] = original index at pivot position t;
    d the diagonal of D; e[t] = D[t+1, t] at the first column of a 2x2 block
    (0 elsewhere); ptype[t] = 0 (1x1), 1 (first of a 2x2), 2 (second).
    Raises ZeroDivisionError(k) when the reduced column k is entirely zero.
    """
    W = np.array(W, dtype=np.result_type(W, np.float64), copy=True)
    s = W.shape[0]
    p = np.arange(s)
    d = np.zeros(s, W.dtype)
    e = np.zeros(s, W.dtype)
    ptype = np.zeros(s, np.int8)
    k = 0
    while k < s:
        absakk = _cabs1(W[k, k])
        if k + 1 < s:
            col = _cabs1(W[k + 1:, k])
            imax = k + 1 + int(np.argmax(col))
            colmax = float(col.max())
        else:
            imax, colmax = k, 0.0
        if max(absakk, colmax) == 0.0 or not np.isfinite(absakk) or not np.isfinite(colmax):
            raise ZeroDivisionError(k)
        kstep, kp = 1, k
        if absakk < BK_ALPHA * colmax:
            rowmax = float(_cabs1(W[imax, k:imax]).max())
            if imax + 1 < s:
                rowmax = max(rowmax, float(_cabs1(W[imax + 1:, imax]).max()))
            if absakk * rowmax >= BK_ALPHA * colmax * colmax:
                kp = k
            elif _cabs1(W[imax, imax]) >= BK_ALPHA * rowmax:
                kp = imax
            else:
                kp, kstep = imax, 2
        kk = k + kstep - 1
        if kp != kk:                      # symmetric interchange of kk and kp
            W[[kk, kp], :] = W[[kp, kk], :]
            W[:, [kk, kp]] = W[:, [kp, kk]]
            p[[kk, kp]] = p[[kp, kk]]
        if kstep == 1:
            dk = W[k, k]
            col = W[k + 1:, k].copy()
            W[k + 1:, k + 1:] -= np.outer(col, col) / dk
            W[k + 1:, k] = col / dk
            d[k] = dk
        else:
            D2 = W[k:k + 2, k:k + 2].copy()
            det = D2[0, 0] * D2[1, 1] - D2[1, 0] * D2[1, 0]
            if det == 0 or not np.isfinite(det):
                raise ZeroDivisionError(k)
            Wc = W[k + 2:, k:k + 2].copy()
            Lc = Wc @ np.linalg.inv(D2)
            W[k + 2:, k + 2:] -= Lc @ Wc.T
            W[k + 2:, k:k + 2] = Lc
            W[k + 1, k] = 0
            d[k], d[k + 1], e[k] = D2[0, 0], D2[1, 1], D2[1, 0]
            ptype[k], ptype[k + 1] = 1, 2
        k += kstep
    L = np.tril(W, -1) + np.eye(s, dtype=W.dtype)
    return p, L, d, e, ptype


def block_d(d, e, ptype):
    """Dense D from its diagonal, 2x2 off-diagonals and pivot types."""
    D = np.diag(np.asarray(d))
    for t in np.nonzero(np.asarray(ptype) == 1)[0]:
        D[t + 1, t] = D[t, t + 1] = e[t]
    return D


def selected_inverse_bk(n, colptr, rowind, values, wmax=0, relax=0):
    """Supernodal LDL^T with Bunch-Kaufman pivoting restricted to each
    supernode's diagonal block (interchanges only among a supernode's own
    columns, so the supernodal structure is unchanged), then Algorithm 1 on
    the pivoted factor.  Dense n x n working storage: small n only.

    Factor, supernodes in column order (right-looking, Section 2.1 with the
    2x2 blocks of D allowed): W = S_KK -> bk_block -> p_K, L_KK, D_K;
    L_CK = S_{C, K p_K} L_KK^{-T} D_K^{-1}; S_CC -= L_CK D_K L_CK^T.
    Selected inversion, supernodes in reverse order: V = L_KK^{-1},
    Lhat = L_CK V, Y = -X_CC Lhat, Z = V^T D_K^{-1} V - Lhat^T Y,
    X_KK = (Z + Z^T)/2 -- all in K's pivot order -- stored back at K's
    original columns (X_{C, K p_K} = Y, X_{K p_K, K p_K} = X_KK).

    Returns (sym, X, fac): X dense in the analysis order (entries on the
    supernodal pattern), fac = per-supernode dict list with p (local pivot
    order), L_KK, L_CK, d, e, ptype."""
    sym = analyse(n, colptr, rowind, wmax, relax)
    cp, ri = sym["colptr"], sym["rowind"]
    vals = values
    if not np.array_equal(sym["post"], np.arange(n)):
        from synth import permute_lower
        _, _, vals, _ = permute_lower(n, colptr, rowind, values, sym["post"])
    S = dense_from_lower(n, cp, ri, vals)
    sn = sym["sn_start"]
    roff = np.concatenate([[0], np.cumsum(sym["rcount"])]).astype(np.int64)
    fac = []
    for K in range(len(sn) - 1):
        f, l = int(sn[K]), int(sn[K + 1])
        C = sym["rrows"][roff[K]:roff[K + 1]].astype(np.int64)
        try:
            p, Lkk, d, e, pt = bk_block(S[f:l, f:l])
        except ZeroDivisionError as z:
            raise ZeroDivisionError(f"zero pivot block at column {f + z.args[0]}")
        cols = f + p
        D = block_d(d, e, pt)
        LC = np.linalg.solve(D.T, np.linalg.solve(Lkk, S[np.ix_(C, cols)].T)).T if len(C) else \
            np.zeros((0, l - f), S.dtype)
        if len(C):
            S[np.ix_(C, C)] -= LC @ D @ LC.T
        fac.append(dict(p=p, L_KK=Lkk, L_CK=LC, d=d, e=e, ptype=pt, C=C))
    X = np.zeros((n, n), S.dtype)
    for K in reversed(range(len(sn) - 1)):
        F = fac[K]
        f = int(sn[K])
        cols = f + F["p"]
        C = F["C"]
        V = np.linalg.inv(F["L_KK"])
        M = V.T @ np.linalg.inv(block_d(F["d"], F["e"], F["ptype"])) @ V
        if len(C):
            Lhat = F["L_CK"] @ V
            Y = -X[np.ix_(C, C)] @ Lhat
            Z = M - Lhat.T @ Y
            X[np.ix_(C, cols)] = Y
            X[np.ix_(cols, C)] = Y.T
        else:
            Z = M
        X[np.ix_(cols, cols)] = 0.5 * (Z + Z.T)
    return sym, X, fac


def panels_from_dense(sym, X):
    """The library's panel layout of a dense X (rows cols(K) then R(K),
    columns cols(K) in original order)."""
    sn = sym["sn_start"]
    roff = np.concatenate([[0], np.cumsum(sym["rcount"])]).astype(np.int64)
    out = []
    for K in range(len(sn) - 1):
        f, l = int(sn[K]), int(sn[K + 1])
        rows = np.concatenate([np.arange(f, l), sym["rrows"][roff[K]:roff[K + 1]]])
        out.append(X[np.ix_(rows, np.arange(f, l))].ravel(order="F"))
    return np.concatenate(out) if out else np.zeros(0, X.dtype)


def logdet_bk(fac):
    """log det A from the pivoted factor: sum of log|d| over 1x1 blocks and
    log|det| over 2x2 blocks; real: (value, number of negative determinants),
    complex: (re, im) of the sum of principal logs."""
    re, im = 0.0, 0.0
    for F in fac:
        d, e, pt = F["d"], F["e"], F["ptype"]
        for t in range(len(d)):
            if pt[t] == 2:
                continue
            v = d[t] * d[t + 1] - e[t] * e[t] if pt[t] == 1 else d[t]
            if np.iscomplexobj(v):
                re += math.log(abs(v))
                im += float(np.angle(v))
            else:
                re += math.log(abs(v))
                im += 1.0 if v < 0 else 0.0
    return np.array([re, im])
