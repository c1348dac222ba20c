"""Python face of the deflated-CG library: torch tensors supply device memory
and the stream; every step of the solve runs in the library's CUDA kernels.

Method: Algorithm 1 (def-CG(k, ell)) with harmonic-Ritz recycling (Sec. 2.3,
Eq. 7) of de Roos & Hennig, arXiv 1706.00241.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _need_len(t: torch.Tensor, n: int, name: str) -> None:
    """The library reads or writes exactly n elements behind the pointer."""
    if t.numel() != n:
        raise ValueError(f"{name} must hold n = {n} elements, got {t.numel()}")


def _need_rows(t: torch.Tensor, rows: int, name: str, lda: int | None = None, min_cols: int = 0) -> int:
    """A row-major (rows, lda) matrix behind the pointer: t must be 2-D with
    that many rows and a row length equal to lda; returns lda."""
    if t.dim() != 2 or t.shape[0] != rows:
        raise ValueError(f"{name} must be a 2-D tensor with {rows} rows, got shape {tuple(t.shape)}")
    row = t.shape[1]
    lda = row if lda is None else int(lda)
    if lda != row:
        raise ValueError(f"lda = {lda} must equal the row length of {name} ({row})")
    if row < min_cols:
        raise ValueError(f"{name} needs at least {min_cols} columns, got {row}")
    return lda


class DefCG:
    """A def-CG(k, ell) solver context for systems of size n on the current GPU.

    Parameters follow ``dcg_config`` in include/dcg.h: ``window`` is "last" or
    "first" (which directions Algorithm 1 stores), ``select`` "largest" or "smallest"
    (Sec. 2.3), ``extraction`` "harmonic" (Eq. 7) or "ritz" (the orthogonal
    projection of Sec. 2.3), ``fg_form`` "explicit" (Gram products over Z and AZ)
    or "sparse" (Saad et al.'s forms from the scalars the solve records, Sec. 2.3;
    harmonic extraction only), ``refine_every`` the residual-replacement period (0 = only the
    final true-residual confirmation). ``reproject`` (default on) takes mu from
    (AW)^T (beta p + r), equal to (AW)^T r in exact arithmetic, which keeps the
    float32 directions A-conjugate to W.
    """

    def __init__(self, n: int, k: int, ell: int, tol: float, max_iter: int | None = None,
                 window: str = "last", select: str = "largest", refine_every: int = 0,
                 extraction: str = "harmonic", fg_form: str = "explicit",
                 warm_start: bool = False, reproject: bool = True,
                 record_history: bool = False, host_loop: bool = False, stream=None):
        self.lib = _lib.load()
        self.n, self.k, self.ell = int(n), int(k), int(ell)
        cfg = _lib.DcgConfig()
        cfg.n = self.n
        cfg.k = self.k
        cfg.ell = self.ell
        cfg.window = _lib.WINDOW[window]
        cfg.select = _lib.SELECT[select]
        cfg.extraction = _lib.EXTRACTION[extraction]
        cfg.fg_form = _lib.FG_FORM[fg_form]
        cfg.refine_every = int(refine_every)
        cfg.max_iter = int(max_iter if max_iter is not None else 10 * self.n)
        cfg.warm_start = int(bool(warm_start))
        cfg.reproject = int(bool(reproject))
        cfg.record_history = int(bool(record_history))
        cfg.host_loop = int(bool(host_loop))
        cfg.tol = float(tol)
        self.cfg = cfg
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ctx = ctypes.c_void_p()
        st = self.lib.dcg_create(ctypes.byref(cfg), ctypes.c_void_p(_stream_handle(self.stream)),
                                 ctypes.byref(self._ctx))
        _lib.check(st, None, "dcg_create")
        self._op_ref = None

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self.lib.dcg_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st, what):
        _lib.check(st, self._ctx, what)

    # -- operators ----------------------------------------------------------
    def set_operator_dense(self, A: torch.Tensor, lda: int | None = None, symmetric: bool = False):
        """Borrow a stored row-major float32 operator (n x n, or n x lda).
        ``symmetric``: A is exactly symmetric and the matvec reads only its
        upper triangle (dcg_set_operator_dense_sym), about half the bytes."""
        _dev_f32(A, "A")
        lda = _need_rows(A, self.n, "A", lda, min_cols=self.n)
        self._op_ref = A
        fn = self.lib.dcg_set_operator_dense_sym if symmetric else self.lib.dcg_set_operator_dense
        self._check(fn(self._ctx, ctypes.c_void_p(A.data_ptr()), lda),
                    "dcg_set_operator_dense_sym" if symmetric else "dcg_set_operator_dense")

    def set_operator_rbf(self, X: torch.Tensor, lengthscale: float, signal_var: float, noise: float,
                         xformat: str = "bf16"):
        """Matrix-free A = K + noise I over the rows of X (n x d float32, Sec. 3
        kernel). ``xformat`` "bf16" or "tf32": X is rounded to that format, which
        defines the operator, and Gram tiles run on the tensor cores."""
        _dev_f32(X, "X")
        n, d = X.shape
        if n != self.n:
            raise ValueError("X must have n rows")
        self._check(self.lib.dcg_set_operator_rbf(self._ctx, ctypes.c_void_p(X.data_ptr()), d,
                                                  _lib.XFORMAT[xformat], float(lengthscale),
                                                  float(signal_var), float(noise)), "dcg_set_operator_rbf")

    def set_rbf_params(self, lengthscale: float, signal_var: float, noise: float):
        """New hyperparameters for the current matrix-free operator (no re-copy of X)."""
        self._check(self.lib.dcg_set_rbf_params(self._ctx, float(lengthscale), float(signal_var), float(noise)),
                    "dcg_set_rbf_params")

    # -- solve --------------------------------------------------------------
    def solve(self, b: torch.Tensor, x: torch.Tensor | None = None, raise_on_error: bool = True):
        """Runs Algorithm 1 on (A, b); returns (x, info dict). b is float32,
        x float64 (the iterate accumulates in float64; see dcg_solve)."""
        _dev_f32(b, "b")
        _need_len(b, self.n, "b")
        if x is None:
            x = torch.zeros(b.shape, dtype=torch.float64, device=b.device)
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise TypeError("x must be a contiguous float64 CUDA tensor")
        _need_len(x, self.n, "x")
        info = _lib.DcgSolveInfo()
        st = self.lib.dcg_solve(self._ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                ctypes.byref(info))
        d = info.as_dict()
        d["status_name"] = _lib.STATUS_NAMES.get(st, str(st))
        if raise_on_error and st not in (_lib.DCG_OK,):
            self._check(st, "dcg_solve")
        return x, d

    def solve_multi(self, B: torch.Tensor, X: torch.Tensor | None = None, raise_on_error: bool = True):
        """Independent solves A x_c = b_c for the rows b_c of B (nrhs x n,
        float32), run in lockstep so that each operator pass serves every
        system still iterating (dcg_solve_multi); returns (X, list of info
        dicts), X float64 nrhs x n. Stores no directions: update_subspace
        needs a dcg_solve after it."""
        _dev_f32(B, "B")
        if B.dim() != 2 or B.shape[1] != self.n:
            raise ValueError(f"B must be (nrhs, {self.n}), got {tuple(B.shape)}")
        nrhs = B.shape[0]
        if not 1 <= nrhs <= _lib.DCG_MAX_RHS:
            raise ValueError(f"nrhs must lie in [1, {_lib.DCG_MAX_RHS}], got {nrhs}")
        if X is None:
            X = torch.zeros(B.shape, dtype=torch.float64, device=B.device)
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64 and X.is_contiguous()
                and tuple(X.shape) == tuple(B.shape)):
            raise TypeError("X must be a contiguous float64 CUDA tensor shaped like B")
        infos = (_lib.DcgSolveInfo * nrhs)()
        st = self.lib.dcg_solve_multi(self._ctx, nrhs, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                      infos)
        out = []
        for i in range(nrhs):
            d = infos[i].as_dict()
            d["status_name"] = _lib.STATUS_NAMES.get(d["status"], str(d["status"]))
            out.append(d)
        if raise_on_error and st != _lib.DCG_OK:
            self._check(st, "dcg_solve_multi")
        return X, out

    def update_subspace(self, wait: bool = True) -> int | None:
        """Harmonic-Ritz extraction of the next W (Sec. 2.3); returns its width.

        With ``wait=False`` the extraction is only enqueued on the solver's
        stream and None is returned; the next solve (or subspace query) waits
        for it and raises its error, if any. Work on other streams, such as
        forming the next operator, then overlaps it."""
        if not wait:
            self._check(self.lib.dcg_update_subspace_async(self._ctx), "dcg_update_subspace_async")
            return None
        k = ctypes.c_int32(0)
        self._check(self.lib.dcg_update_subspace(self._ctx, ctypes.byref(k)), "dcg_update_subspace")
        return k.value

    def ritz_values(self) -> np.ndarray:
        m = ctypes.c_int32(0)
        self._check(self.lib.dcg_get_ritz_values(self._ctx, None, 0, ctypes.byref(m)), "dcg_get_ritz_values")
        out = np.zeros(max(m.value, 1), dtype=np.float64)
        if m.value:
            self._check(self.lib.dcg_get_ritz_values(
                self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), m.value, ctypes.byref(m)),
                "dcg_get_ritz_values")
        return out[:m.value]

    def pencil(self):
        """(F, G) of the last extraction as float64 numpy arrays (m x m)."""
        m = ctypes.c_int32()
        self._check(self.lib.dcg_get_pencil(self._ctx, None, None, 0, ctypes.byref(m)), "dcg_get_pencil")
        F = np.zeros(m.value * m.value, dtype=np.float64)
        G = np.zeros_like(F)
        if m.value:
            pd = ctypes.POINTER(ctypes.c_double)
            self._check(self.lib.dcg_get_pencil(self._ctx, F.ctypes.data_as(pd), G.ctypes.data_as(pd), F.size,
                                                ctypes.byref(m)), "dcg_get_pencil")
        return F.reshape(m.value, m.value), G.reshape(m.value, m.value)

    def pencil_form(self) -> str:
        """How the last update formed F and G: "explicit" or "sparse"."""
        f = ctypes.c_int32()
        self._check(self.lib.dcg_get_pencil_form(self._ctx, ctypes.byref(f)), "dcg_get_pencil_form")
        return {v: k for k, v in _lib.FG_FORM.items()}[f.value]

    def get_subspace(self) -> torch.Tensor:
        """Current W as a (k_active, n) tensor (row j is column j of W)."""
        k = ctypes.c_int32(0)
        self._check(self.lib.dcg_get_subspace(self._ctx, None, ctypes.byref(k)), "dcg_get_subspace")
        W = torch.empty((max(k.value, 0), self.n), dtype=torch.float32, device="cuda")
        if k.value:
            self._check(self.lib.dcg_get_subspace(self._ctx, ctypes.c_void_p(W.data_ptr()), ctypes.byref(k)),
                        "dcg_get_subspace")
        return W

    def set_subspace(self, W: torch.Tensor):
        """Sets W from a (k, n) tensor (row j is column j of W)."""
        _dev_f32(W, "W")
        if W.numel() == 0:
            k = 0
        elif W.dim() != 2 or W.shape[1] != self.n:
            raise ValueError(f"W must be (k, n) with n = {self.n}, got shape {tuple(W.shape)}")
        else:
            k = W.shape[0]
        self._check(self.lib.dcg_set_subspace(self._ctx, ctypes.c_void_p(W.data_ptr() if k else 0), k),
                    "dcg_set_subspace")

    def history(self) -> np.ndarray:
        cnt = ctypes.c_int32(0)
        self._check(self.lib.dcg_get_history(self._ctx, None, 0, ctypes.byref(cnt)), "dcg_get_history")
        out = np.zeros(max(cnt.value, 1), dtype=np.float64)
        self._check(self.lib.dcg_get_history(self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             cnt.value, ctypes.byref(cnt)), "dcg_get_history")
        return out[:cnt.value]

    # -- single steps -------------------------------------------------------
    def matvec(self, p: torch.Tensor, q: torch.Tensor | None = None, want_pAp: bool = True):
        """q = A p with the fused p^T q (Algorithm 1)."""
        _dev_f32(p, "p")
        _need_len(p, self.n, "p")
        if q is None:
            q = torch.empty_like(p)
        _dev_f32(q, "q")
        _need_len(q, self.n, "q")
        d = ctypes.c_double(0.0)
        self._check(self.lib.dcg_matvec(self._ctx, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                        ctypes.byref(d) if want_pAp else None), "dcg_matvec")
        return q, (d.value if want_pAp else None)

    def rbf_dtheta(self, U: torch.Tensor, V: torch.Tensor) -> np.ndarray:
        """u_p^T (dA/dtheta) v_p for theta = (lengthscale, signal_var, noise) of
        the matrix-free operator; U, V are (P, n) float32 tensors (row p is the
        pair's vector). Returns a (P, 3) float64 array."""
        _dev_f32(U, "U")
        _dev_f32(V, "V")
        if U.dim() == 1:
            U, V = U[None], V[None]
        if U.shape != V.shape or U.shape[1] != self.n:
            raise ValueError("U and V must both be (P, n)")
        P = U.shape[0]
        out = (ctypes.c_double * (3 * P))()
        self._check(self.lib.dcg_rbf_dtheta(self._ctx, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                                            P, out), "dcg_rbf_dtheta")
        return np.array(out[:], dtype=np.float64).reshape(P, 3)

    def residual(self, b: torch.Tensor, x: torch.Tensor, r: torch.Tensor | None = None):
        """True residual r = b - A x (float32 r, float64 x); returns
        (r, |r|^2, entry-error estimate of |r|)."""
        _dev_f32(b, "b")
        _need_len(b, self.n, "b")
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise TypeError("x must be a contiguous float64 CUDA tensor")
        _need_len(x, self.n, "x")
        if r is None:
            r = torch.empty_like(b)
        _dev_f32(r, "r")
        _need_len(r, self.n, "r")
        rr, err = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.dcg_residual(self._ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(r.data_ptr()), ctypes.byref(rr), ctypes.byref(err)),
                    "dcg_residual")
        return r, rr.value, err.value

    def apply_block(self, V: torch.Tensor, Y: torch.Tensor | None = None) -> torch.Tensor:
        """Y = A V for a (c, n) tensor V (row j is column j), in one pass over A."""
        _dev_f32(V, "V")
        if V.dim() != 2 or V.shape[1] != self.n:
            raise ValueError(f"V must be (c, n) with n = {self.n}, got shape {tuple(V.shape)}")
        if Y is None:
            Y = torch.empty_like(V)
        _dev_f32(Y, "Y")
        if Y.shape != V.shape:
            raise ValueError(f"Y must have V's shape {tuple(V.shape)}, got {tuple(Y.shape)}")
        self._check(self.lib.dcg_apply_block(self._ctx, ctypes.c_void_p(V.data_ptr()), V.shape[0],
                                             ctypes.c_void_p(Y.data_ptr())), "dcg_apply_block")
        return Y

    def sync(self):
        self._check(self.lib.dcg_sync(self._ctx), "dcg_sync")

    def debug_arm_barrier_timeout(self, polls: int = 64):
        """Test hook: the next solve's grid barrier misses one arrival and its
        bounded wait gives up after ``polls`` polls (DCG_ERR_TIMEOUT)."""
        self._check(self.lib.dcg_debug_arm_barrier_timeout(self._ctx, int(polls)),
                    "dcg_debug_arm_barrier_timeout")

    def last_error(self) -> str:
        return self.lib.dcg_last_error(self._ctx).decode()


def form_rbf_dense(X: torch.Tensor, lengthscale: float, signal_var: float, noise: float,
                   out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """A = s^2 exp(-|x_i - x_j|^2 / (2 l^2)) + noise I as a dense float32 matrix (Sec. 3)."""
    lib = _lib.load()
    _dev_f32(X, "X")
    if X.dim() != 2:
        raise ValueError(f"X must be (n, d), got shape {tuple(X.shape)}")
    n, d = X.shape
    if out is None:
        out = torch.empty((n, n), dtype=torch.float32, device=X.device)
    _dev_f32(out, "out")
    _need_rows(out, n, "out", min_cols=n)
    st = lib.dcg_form_rbf_dense(ctypes.c_void_p(X.data_ptr()), n, d, float(lengthscale), float(signal_var),
                                float(noise), ctypes.c_void_p(out.data_ptr()), out.shape[1],
                                ctypes.c_void_p(_stream_handle(stream)))
    _lib.check(st, None, "dcg_form_rbf_dense")
    return out


def matvec_dense_noalloc(A: torch.Tensor, p: torch.Tensor, q: torch.Tensor, pAp: torch.Tensor | None = None,
                         lda: int | None = None, stream=None) -> None:
    """q = A p (and p^T q into the one-element float64 device tensor pAp) with
    no context and no device allocation: q and pAp are caller-owned. Calls on
    one device must not overlap in time (they share the library's scratch)."""
    lib = _lib.load()
    _dev_f32(A, "A")
    _dev_f32(p, "p")
    _dev_f32(q, "q")
    if pAp is not None and (not pAp.is_cuda or pAp.dtype != torch.float64 or pAp.numel() < 1):
        raise ValueError("pAp must be a float64 CUDA tensor with one element")
    n = p.numel()
    _need_len(q, n, "q")
    lda = _need_rows(A, n, "A", lda, min_cols=n)
    st = lib.dcg_matvec_dense_noalloc(ctypes.c_void_p(A.data_ptr()), n, lda, ctypes.c_void_p(p.data_ptr()),
                                      ctypes.c_void_p(q.data_ptr()),
                                      ctypes.c_void_p(pAp.data_ptr()) if pAp is not None else None,
                                      ctypes.c_void_p(_stream_handle(stream)))
    _lib.check(st, None, "dcg_matvec_dense_noalloc")
