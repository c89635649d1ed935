"""Python binding of the pselinv C ABI (include/pselinv.h).

Argument marshalling only: every step of the factorisation and of the
selected inversion runs in the library's CUDA kernels.  PyTorch provides
device memory and streams.  There is no CPU fallback: if the compiled
library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpselinv.so")

PSELINV_OK = 0
ERRORS = {-1: "ERR_ARG", -2: "ERR_NOT_LOWER", -3: "ERR_ZERO_PIVOT", -4: "ERR_NONFINITE",
          -5: "ERR_OOM", -6: "ERR_CUDA", -7: "ERR_TIMEOUT", -8: "ERR_STATE", -9: "ERR_RANGE"}
F64, C128 = 0, 1
RELAX_NONE, RELAX_AMALG = 0, 1
PLAIN, LEVEL, GRAPH, PERSISTENT = 0, 1, 2, 3
G_SYMMETRIC, G_PANEL = 0, 1

EXPORTED = ["pselinv_default_opts", "pselinv_analyze", "pselinv_analyze_batch", "pselinv_factor",
            "pselinv_factor_unsym", "pselinv_factor_bk", "pselinv_get_pivots", "pselinv_selinv",
            "pselinv_selinv_to_host", "pselinv_get_panels", "pselinv_pole_sum", "pselinv_selinv_pole_sum",
            "pselinv_trace_sum",
            "pselinv_sync_status", "pselinv_set_debug", "pselinv_get_selected", "pselinv_get_selected_upper",
            "pselinv_logdet_grad", "pselinv_logdet",
            "pselinv_selinv_adjoint",
            "pselinv_set_timing", "pselinv_get_timing", "pselinv_autotune", "pselinv_get_info",
            "pselinv_export_symbolic",
            "pselinv_destroy", "pselinv_last_error", "pselinv_block_inverse_static"]


class PselinvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("batch", ctypes.c_int32), ("max_sn_width", ctypes.c_int32),
                ("relax", ctypes.c_int32), ("small_cutoff", ctypes.c_int32), ("split_k_rows", ctypes.c_int32),
                ("debug_checks", ctypes.c_int32), ("unsym", ctypes.c_int32), ("spin_limit_ns", ctypes.c_int64),
                ("level_tiles", ctypes.c_int32), ("min_slice_rows", ctypes.c_int32),
                ("fp64_emulation", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz_a", ctypes.c_int64), ("nnz_l", ctypes.c_int64),
                ("panel_entries", ctypes.c_int64), ("relidx_len", ctypes.c_int64), ("nsn", ctypes.c_int32),
                ("nlevels", ctypes.c_int32), ("max_width", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("max_r", ctypes.c_int64), ("flops_selinv", ctypes.c_double), ("flops_gemm1", ctypes.c_double),
                ("bytes_selinv", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


_P32 = ctypes.POINTER(ctypes.c_int32)
_P64 = ctypes.POINTER(ctypes.c_int64)


class Symbolic(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nsn", ctypes.c_int32), ("nlevels", ctypes.c_int32),
                ("perm", _P32), ("parent", _P32), ("sn_start", _P32), ("sn_parent", _P32), ("sigma", _P32),
                ("rowptr", _P64), ("rows", _P32), ("panel_off", _P64), ("relptr", _P64), ("relidx", _P32),
                ("nblk", _P32), ("level_ptr", _P32), ("level_sn", _P32),
                ("ngroups", ctypes.c_int32), ("group_ptr", _P32), ("group_sn_ptr", _P32), ("group_sn", _P32)]


_lib = None


def load_library():
    """Load the compiled library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"pselinv library not built ({LIB_PATH} missing); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    L.pselinv_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.pselinv_default_opts.restype = None
    L.pselinv_analyze.argtypes = [ctypes.c_int64, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(vp)]
    L.pselinv_analyze_batch.argtypes = [ctypes.c_int32, vp, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(vp)]
    L.pselinv_factor.argtypes = [vp, vp, vp]
    L.pselinv_factor_unsym.argtypes = [vp, vp, vp, vp]
    L.pselinv_factor_bk.argtypes = [vp, vp, vp]
    L.pselinv_get_pivots.argtypes = [vp, vp, vp, vp]
    L.pselinv_selinv.argtypes = [vp, ctypes.c_int32, vp]
    L.pselinv_selinv_to_host.argtypes = [vp, vp, vp, vp]
    L.pselinv_get_panels.argtypes = [vp, ctypes.c_int32, vp, vp]
    L.pselinv_sync_status.argtypes = [vp, vp]
    L.pselinv_pole_sum.argtypes = [vp, vp, vp, vp]
    L.pselinv_selinv_pole_sum.argtypes = [vp, vp, vp, vp]
    L.pselinv_trace_sum.argtypes = [vp, vp, vp, vp]
    L.pselinv_set_debug.argtypes = [vp, ctypes.c_int32]
    L.pselinv_get_selected.argtypes = [vp, vp, vp]
    L.pselinv_get_selected_upper.argtypes = [vp, vp, vp]
    L.pselinv_logdet.argtypes = [vp, vp, vp]
    L.pselinv_logdet_grad.argtypes = [vp, vp, vp]
    L.pselinv_selinv_adjoint.argtypes = [vp, vp, ctypes.c_int32, vp, vp]
    L.pselinv_set_timing.argtypes = [vp, ctypes.c_int32]
    L.pselinv_get_timing.argtypes = [vp, vp, vp]
    L.pselinv_autotune.argtypes = [vp, vp, vp, vp]
    L.pselinv_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.pselinv_export_symbolic.argtypes = [vp, ctypes.POINTER(Symbolic)]
    L.pselinv_destroy.argtypes = [vp]
    L.pselinv_destroy.restype = None
    L.pselinv_last_error.argtypes = [vp]
    L.pselinv_last_error.restype = ctypes.c_char_p
    L.pselinv_block_inverse_static.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp]
    _lib = L
    return L


def default_opts(**kw) -> Opts:
    o = Opts()
    load_library().pselinv_default_opts(ctypes.byref(o))
    names = {f[0] for f in Opts._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class SelInv:
    """One analysed pattern (and its device state).

    ``SelInv(n, colptr, rowind, perm=None, **opts)`` runs pselinv_analyze on
    host numpy arrays.  ``factor(values)`` takes a CUDA tensor of
    batch x nnz values (user order), ``selinv(mode)`` enqueues the selected
    inversion, ``panels()`` / ``selected()`` return CUDA tensors.  With
    ``unsym=1`` the matrix is non-symmetric with a symmetric pattern:
    ``factor_unsym(lower, upper)`` and ``selected_upper()``.  With
    ``fp64_emulation=1`` steps 2 and 3 of an SPD
    matrix run on bf16 slices with exact integer sums (pselinv_opts in
    include/pselinv.h); call ``sync_status()`` after ``selinv`` to learn
    whether X was positive definite (PselinvError ERR_RANGE otherwise).  Option
    names are the fields of ``Opts``; an unknown name raises TypeError.
    """

    def __init__(self, n, colptr, rowind, perm=None, **opts):
        self._lib = load_library()
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        if isinstance(n, (list, tuple)):
            # uneven batch: lists of members -> pselinv_analyze_batch
            k = len(n)
            ns = np.ascontiguousarray(n, np.int64)
            cps = [np.ascontiguousarray(c, np.int64) for c in colptr]
            ris = [np.ascontiguousarray(r, np.int32) for r in rowind]
            pps = [None if (perm is None or perm[b] is None) else np.ascontiguousarray(perm[b], np.int32)
                   for b in range(k)]
            self._keep = (ns, cps, ris, pps)
            arr = lambda xs: (ctypes.c_void_p * k)(*[None if x is None else x.ctypes.data for x in xs])
            rc = self._lib.pselinv_analyze_batch(k, _ptr(ns), arr(cps), arr(ris), arr(pps),
                                                 ctypes.byref(self.opts), ctypes.byref(h))
            n = int(ns.sum())
        else:
            cp = np.ascontiguousarray(colptr, np.int64)
            ri = np.ascontiguousarray(rowind, np.int32)
            pp = None if perm is None else np.ascontiguousarray(perm, np.int32)
            rc = self._lib.pselinv_analyze(int(n), _ptr(cp), _ptr(ri), None if pp is None else _ptr(pp),
                                           ctypes.byref(self.opts), ctypes.byref(h))
        if rc != PSELINV_OK:
            raise PselinvError(rc, self._lib.pselinv_last_error(None).decode())
        self._h = h
        self.n = int(n)

    def _check(self, rc):
        if rc != PSELINV_OK:
            raise PselinvError(rc, self._lib.pselinv_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pselinv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- introspection ----
    @property
    def info(self) -> dict:
        inf = Info()
        self._check(self._lib.pselinv_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in Info._fields_}

    def symbolic(self) -> dict:
        v = Symbolic()
        self._check(self._lib.pselinv_export_symbolic(self._h, ctypes.byref(v)))
        n, nsn, nl = v.n, v.nsn, v.nlevels

        def arr(p, k):
            return np.ctypeslib.as_array(p, shape=(k,)).copy() if k > 0 else np.zeros(0, np.int64)

        rowptr = arr(v.rowptr, nsn + 1)
        relptr = arr(v.relptr, nsn + 1)
        return dict(n=n, nsn=nsn, nlevels=nl, perm=arr(v.perm, n), parent=arr(v.parent, n),
                    sn_start=arr(v.sn_start, nsn + 1), sn_parent=arr(v.sn_parent, nsn),
                    sigma=arr(v.sigma, nsn), rowptr=rowptr, rows=arr(v.rows, int(rowptr[-1])),
                    panel_off=arr(v.panel_off, nsn + 1), relptr=relptr, relidx=arr(v.relidx, int(relptr[-1])),
                    nblk=arr(v.nblk, nsn), level_ptr=arr(v.level_ptr, nl + 1), level_sn=arr(v.level_sn, nsn),
                    group_ptr=arr(v.group_ptr, nl + 1), group_sn_ptr=arr(v.group_sn_ptr, v.ngroups + 1),
                    group_sn=arr(v.group_sn, int(arr(v.group_sn_ptr, v.ngroups + 1)[-1])))

    # ---- numeric ----
    @property
    def torch_dtype(self):
        import torch
        return torch.complex128 if self.opts.dtype == C128 else torch.float64

    def factor(self, values, stream=None):
        assert values.is_cuda and values.dtype == self.torch_dtype and values.is_contiguous()
        assert values.numel() == self.opts.batch * self.info["nnz_a"]
        self._check(self._lib.pselinv_factor(self._h, ctypes.c_void_p(values.data_ptr()), _stream_ptr(stream)))

    def factor_bk(self, values, stream=None):
        """pselinv_factor_bk: LDL^T with Bunch-Kaufman 1x1/2x2 pivots inside supernodes."""
        assert values.is_cuda and values.dtype == self.torch_dtype and values.is_contiguous()
        assert values.numel() == self.opts.batch * self.info["nnz_a"]
        self._check(self._lib.pselinv_factor_bk(self._h, ctypes.c_void_p(values.data_ptr()), _stream_ptr(stream)))

    def pivots(self, stream=None):
        """(local pivot order, pivot type) of the last factor_bk, [batch, n] numpy arrays."""
        piv = np.zeros(self.opts.batch * self.n, np.int32)
        ty = np.zeros(self.opts.batch * self.n, np.int8)
        self._check(self._lib.pselinv_get_pivots(self._h, _ptr(piv), _ptr(ty), _stream_ptr(stream)))
        return piv.reshape(self.opts.batch, -1), ty.reshape(self.opts.batch, -1)

    def factor_unsym(self, lower, upper, stream=None):
        """pselinv_factor_unsym: A_ij (``lower``) and A_ji (``upper``) at the
        stored lower positions, CUDA tensors of batch x nnz values."""
        for v in (lower, upper):
            assert v.is_cuda and v.dtype == self.torch_dtype and v.is_contiguous()
            assert v.numel() == self.opts.batch * self.info["nnz_a"]
        self._check(self._lib.pselinv_factor_unsym(self._h, ctypes.c_void_p(lower.data_ptr()),
                                                   ctypes.c_void_p(upper.data_ptr()), _stream_ptr(stream)))

    def selinv(self, mode=LEVEL, stream=None):
        self._check(self._lib.pselinv_selinv(self._h, int(mode), _stream_ptr(stream)))

    def selinv_to_host(self, out, out_u=None, stream=None):
        """pselinv_selinv_to_host: LEVEL selinv with the X panels (and XU for
        non-symmetric handles) copied level by level into pinned CPU tensors
        of batch x panel_entries elements while the sweep runs."""
        n = self.opts.batch * self.info["panel_entries"]
        for o in (out, out_u):
            assert o is None or (o.device.type == "cpu" and o.numel() == n and o.dtype == self.torch_dtype
                                 and o.is_contiguous())
        self._check(self._lib.pselinv_selinv_to_host(
            self._h, ctypes.c_void_p(out.data_ptr()), None if out_u is None else ctypes.c_void_p(out_u.data_ptr()),
            _stream_ptr(stream)))
        return out.view(self.opts.batch, -1)

    def pole_sum(self, weights, out=None, stream=None):
        """pselinv_pole_sum: sum_b w_b X_b over the batch (X panel layout)."""
        import torch
        w = np.ascontiguousarray(weights, np.complex128 if self.opts.dtype == C128 else np.float64)
        assert w.size == self.opts.batch
        if out is None:
            out = torch.empty(self.info["panel_entries"], dtype=self.torch_dtype, device="cuda")
        self._check(self._lib.pselinv_pole_sum(self._h, ctypes.c_void_p(w.ctypes.data),
                                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def selinv_pole_sum(self, weights, out=None, stream=None):
        """pselinv_selinv_pole_sum: the batch's selected inversion (LEVEL) with
        sum_b w_b X_b accumulated in its write step (X panel layout)."""
        import torch
        w = np.ascontiguousarray(weights, np.complex128 if self.opts.dtype == C128 else np.float64)
        assert w.size == self.opts.batch
        if out is None:
            out = torch.empty(self.info["panel_entries"], dtype=self.torch_dtype, device="cuda")
        self._check(self._lib.pselinv_selinv_pole_sum(self._h, ctypes.c_void_p(w.ctypes.data),
                                                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def trace_error(self, values, stream=None):
        """E_b = |1 - (1/n) sum_{A_ij != 0} X_ij A_ji| per batch member (Eq. 16), from pselinv_trace_sum."""
        out = np.zeros(2 * self.opts.batch, np.float64)
        self._check(self._lib.pselinv_trace_sum(self._h, ctypes.c_void_p(values.data_ptr()), _ptr(out),
                                                _stream_ptr(stream)))
        s = out[0::2] + 1j * out[1::2]
        return np.abs(1.0 - s / self.n)

    def sync_status(self, stream=None):
        """Synchronise and raise PselinvError for a device-side failure of earlier
        work: a bad pivot of the last factorisation (ERR_ZERO_PIVOT /
        ERR_NONFINITE), a bounded wait that ran out (ERR_TIMEOUT)."""
        self._check(self._lib.pselinv_sync_status(self._h, _stream_ptr(stream)))

    def set_debug(self, flags):
        self._check(self._lib.pselinv_set_debug(self._h, int(flags)))

    def panels(self, which=0, out=None, stream=None):
        """X (which=0) or L (which=1) panels -- non-symmetric handles also XU (2)
        and U (3) -- as a [batch, panel_entries] tensor; ``out`` may be a CUDA
        tensor or a (pinned) CPU tensor."""
        import torch
        if out is None:
            out = torch.empty(self.opts.batch * self.info["panel_entries"], dtype=self.torch_dtype, device="cuda")
        assert out.numel() == self.opts.batch * self.info["panel_entries"] and out.dtype == self.torch_dtype
        self._check(self._lib.pselinv_get_panels(self._h, int(which), ctypes.c_void_p(out.data_ptr()),
                                                 _stream_ptr(stream)))
        return out.view(self.opts.batch, -1)

    def selected(self, out=None, stream=None):
        import torch
        nnz = self.info["nnz_a"]
        if out is None:
            out = torch.empty(self.opts.batch * nnz, dtype=self.torch_dtype, device="cuda")
        self._check(self._lib.pselinv_get_selected(self._h, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out.view(self.opts.batch, nnz)

    def selected_upper(self, out=None, stream=None):
        """Non-symmetric handles: X_ji at the stored lower positions (i, j)."""
        import torch
        nnz = self.info["nnz_a"]
        if out is None:
            out = torch.empty(self.opts.batch * nnz, dtype=self.torch_dtype, device="cuda")
        self._check(self._lib.pselinv_get_selected_upper(self._h, ctypes.c_void_p(out.data_ptr()),
                                                         _stream_ptr(stream)))
        return out.view(self.opts.batch, nnz)

    def logdet_grad(self, out=None, stream=None):
        """d log det A / d (stored lower values): X_jj on the diagonal, 2 X_ij off it."""
        import torch
        nnz = self.info["nnz_a"]
        if out is None:
            out = torch.empty(self.opts.batch * nnz, dtype=self.torch_dtype, device="cuda")
        self._check(self._lib.pselinv_logdet_grad(self._h, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out.view(self.opts.batch, nnz)

    def adjoint(self, G, g_kind=G_SYMMETRIC, out=None, stream=None):
        """pselinv_selinv_adjoint: dJ/d(stored lower values of A) for
        J = <G, X> (G symmetric on the selected pattern, panel layout) or,
        with g_kind=G_PANEL, for any J with dJ/d(X panels) = G."""
        import torch
        assert G.is_cuda and G.dtype == self.torch_dtype and G.is_contiguous()
        assert G.numel() == self.opts.batch * self.info["panel_entries"]
        nnz = self.info["nnz_a"]
        if out is None:
            out = torch.empty(self.opts.batch * nnz, dtype=self.torch_dtype, device="cuda")
        self._check(self._lib.pselinv_selinv_adjoint(self._h, ctypes.c_void_p(G.data_ptr()), int(g_kind),
                                                     ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out.view(self.opts.batch, nnz)

    def autotune(self, stream=None):
        """pselinv_autotune: returns {"split_k_rows", "small_cutoff", "level_tiles", "mode", "ms"}
        and keeps that schedule (pass "mode" to selinv)."""
        best = np.zeros(4, np.int32)
        ms = np.zeros(1, np.float64)
        self._check(self._lib.pselinv_autotune(self._h, _ptr(best), _ptr(ms), _stream_ptr(stream)))
        self.opts.split_k_rows, self.opts.small_cutoff, self.opts.level_tiles = (int(best[0]), int(best[1]),
                                                                                  int(best[2]))
        return {"split_k_rows": int(best[0]), "small_cutoff": int(best[1]), "level_tiles": int(best[2]),
                "mode": int(best[3]), "ms": float(ms[0])}

    def set_timing(self, enable=True):
        self._check(self._lib.pselinv_set_timing(self._h, 1 if enable else 0))

    def get_timing(self):
        """(ms per kernel class, launches per class) since the last call; classes:
        normalisation, step 2, step 3 partial products, step 3 finish."""
        ms = np.zeros(4, np.float64)
        ln = np.zeros(4, np.int64)
        self._check(self._lib.pselinv_get_timing(self._h, _ptr(ms), _ptr(ln)))
        return ms, ln

    def logdet(self, stream=None):
        out = np.zeros(2 * self.opts.batch, np.float64)
        self._check(self._lib.pselinv_logdet(self._h, _ptr(out), _stream_ptr(stream)))
        return out.reshape(self.opts.batch, 2)


def block_inverse_static(L, d, out=None, stream=None):
    """pselinv_block_inverse_static: M_b = L_b^{-T} D_b^{-1} L_b^{-1} for a
    batch of dense s x s blocks (CUDA float64 tensors, L: [count, s, s] or
    [count, s*s] column-major, d: [count, s]) without any allocation inside
    the library.  ``out`` (same shape as L) is allocated here by torch when
    not given."""
    import torch
    lib = load_library()
    count, s = d.shape
    assert L.is_cuda and d.is_cuda and L.dtype == torch.float64 and d.dtype == torch.float64
    assert L.is_contiguous() and d.is_contiguous() and L.numel() == count * s * s
    if out is None:
        out = torch.empty(count, s * s, dtype=torch.float64, device=L.device)
    rc = lib.pselinv_block_inverse_static(int(s), int(count), ctypes.c_void_p(L.data_ptr()),
                                          ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          _stream_ptr(stream))
    if rc != PSELINV_OK:
        raise PselinvError(rc, lib.pselinv_last_error(None).decode())
    return out


def _autograd():
    import torch

    class LogDet(torch.autograd.Function):
        """log det A(values) for real symmetric A (sum log|d_j| of the LDL^T
        pivots).  backward = the selected inverse at A's stored positions
        (pselinv_logdet_grad), scaled by the incoming gradient."""

        @staticmethod
        def forward(ctx, values, handle, mode):
            handle.factor(values.detach().contiguous())
            ld = handle.logdet()
            ctx.handle, ctx.mode = handle, mode
            return torch.tensor(ld[:, 0], dtype=torch.float64, device=values.device)

        @staticmethod
        def backward(ctx, g):
            h = ctx.handle
            h.selinv(ctx.mode)
            return h.logdet_grad() * g[:, None], None, None

    class SelectedInverse(torch.autograd.Function):
        """X panels (the selected inverse) of the batch of symmetric matrices
        with lower-CSC values ``values``; backward = the hand-written adjoint
        of the selected inversion and of the LDL^T (pselinv_selinv_adjoint)."""

        @staticmethod
        def forward(ctx, values, handle, mode):
            handle.factor(values.detach().contiguous())
            handle.selinv(mode)
            handle.sync_status()  # a bad pivot of the factorisation raises here
            ctx.handle = handle
            return handle.panels(0)

        @staticmethod
        def backward(ctx, g):
            return ctx.handle.adjoint(g.contiguous(), G_PANEL), None, None

    return LogDet, SelectedInverse


_LogDet = None
_SelInv = None


def logdet(values, handle, mode=LEVEL):
    """Differentiable log det of the batch of real symmetric matrices whose
    lower-CSC values are ``values`` ([batch, nnz] or [nnz]) on the pattern
    analysed by ``handle``; returns a [batch] tensor."""
    global _LogDet, _SelInv
    if _LogDet is None:
        _LogDet, _SelInv = _autograd()
    v = values if values.dim() == 2 else values.unsqueeze(0)
    out = _LogDet.apply(v, handle, mode)
    return out if values.dim() == 2 else out[0]


def selected_inverse(values, handle, mode=LEVEL):
    """Differentiable selected inverse: the X panels ([batch, panel_entries])
    of the matrices with lower-CSC values ``values`` ([batch, nnz]); the
    backward pass runs the library's adjoint kernels."""
    global _LogDet, _SelInv
    if _SelInv is None:
        _LogDet, _SelInv = _autograd()
    return _SelInv.apply(values, handle, mode)
