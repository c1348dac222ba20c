"""Plain FP64 reference for def-CG(k, ell) and harmonic-Ritz recycling.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Paper: de Roos & Hennig, arXiv 1706.00241.
  * Eq. 1: the task, a sequence of SPD systems A^(i) x^(i) = b^(i).
  * Eq. 2: residual convention; Algorithm 1 uses r = b - A x, as here.
  * Sec. 2.2, Algorithm 1: Deflated-CG(k, ell)(A, b, x_{-1}, W, (AW), tol).
  * Sec. 2.3, Eq. 7: harmonic projection G u = theta F u with F = (AZ)^T Z,
    G = (AZ)^T (AZ), Z = [W, P_ell]; the next W is Z U for k chosen u.
  * Sec. 2.3, the equation before Eq. 7: orthogonal (Rayleigh-Ritz) projection
    Z^T A Z u = theta Z^T Z u, offered as the alternative extraction.
  * Sec. 2.3 (Saad et al.'s explicit forms): F and G of Eq. 7 built from the
    scalars of the run (E, G_W, d_j, alpha_j, |r_j|^2, (AW)^T r_j) instead of
    products over Z and AZ.
  * Sec. 3: the RBF kernel k(x_i, x_j) = theta^2 exp(-|x_i - x_j|^2 / (2 lambda^2)).

Readings where the paper is silent or ambiguous (each one is also listed in the
design notes of the repository):
  R1 mu_j is solved from (AW)^T r_j (Algorithm 1 writes W^T A r_j; equal for
     symmetric A).
  R2 stop when the recursive |r_j| <= tol |b| (relative, as in the Sec. 3
     experiments); then the true residual b - A x is formed; if it is above
     tol |b| it replaces r and the loop continues. b = 0 returns x = 0.
  R3 stored directions: window "first" keeps p_0..p_{ell-1}; "last" keeps the
     final ell directions whose A p was formed. A p_j is stored with p_j.
  R4 keep the k largest harmonic Ritz values (the experiment's choice, Sec. 2.2
     and the Fig. 1 caption); "smallest" is an option. Ties: lower index first.
  R5 each new W column is scaled to unit 2-norm, largest-magnitude entry positive.
  R6 if the Cholesky factorisation of E = W^T A W or of F fails, the matrix is
     eigendecomposed and directions with eigenvalue < 1e-12 * max are dropped.
  R13 residual replacement every m iterations: r <- b - A x, re-deflate
     (x += W g, r -= AW g, g = E^{-1} W^T r), and take mu from
     (AW)^T (beta p_j + r_{j+1}) so that p_{j+1} is re-projected against W.
     beta keeps the recursion's value |r_{j+1}|^2 / |r_j|^2 (before the
     replacement); rho is recomputed from the replaced residual. The two steps
     are the functions project_out and next_direction; defcg's A_true names
     the operator whose residual the replacements and checks form (iterative
     refinement when the loop operator only approximates it).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

F64 = np.float64

STATUS_OK = 0
STATUS_BREAKDOWN = 4
STATUS_MAXITER = 6


# ----------------------------------------------------------------------------
# Operator: RBF Gram matrix plus noise (Sec. 3)
# ----------------------------------------------------------------------------

def rbf_gram(X, lengthscale, signal_var=1.0, noise=0.0, rows=None):
    """Dense ``K + noise I`` with ``K_ij = s^2 exp(-|x_i - x_j|^2 / (2 l^2))`` (Sec. 3).

    The squared distance is taken in the difference form, sum_m (x_im - x_jm)^2,
    in float64. ``rows`` optionally selects a subset of rows (for sampled checks
    at sizes where the full matrix is too large); the noise is then added where
    the row index meets its own column.
    """
    X = np.asarray(X, dtype=F64)
    n, d = X.shape
    idx = np.arange(n) if rows is None else np.asarray(rows)
    out = np.empty((idx.size, n), dtype=F64)
    block = max(1, (1 << 23) // max(1, n * d))
    inv2l2 = 1.0 / (2.0 * lengthscale * lengthscale)
    for s in range(0, idx.size, block):
        sel = idx[s:s + block]
        diff = X[sel, None, :] - X[None, :, :]
        sq = np.einsum("ijm,ijm->ij", diff, diff)
        out[s:s + block] = signal_var * np.exp(-sq * inv2l2)
    out[np.arange(idx.size), idx] += noise
    return out


def rbf_matvec(X, lengthscale, signal_var=1.0, noise=0.0):
    """Matrix-free ``v -> (K + noise I) v`` by row blocks of the Sec. 3 kernel."""
    X = np.asarray(X, dtype=F64)
    n = X.shape[0]
    block = max(1, min(n, (1 << 22) // max(1, n * X.shape[1])))

    def apply(v):
        V = np.asarray(v, dtype=F64)
        out = np.empty_like(V)
        for s in range(0, n, block):
            rows = np.arange(s, min(n, s + block))
            out[s:s + rows.size] = rbf_gram(X, lengthscale, signal_var, noise, rows=rows) @ V
        return out

    return apply


def _mv(A, v):
    return A(v) if callable(A) else A @ v


def true_relres(A, b, x):
    """|b - A x| / |b| in float64 (the Sec. 3 stopping quantity)."""
    b = np.asarray(b, dtype=F64)
    nb = np.linalg.norm(b)
    r = b - _mv(A, np.asarray(x, dtype=F64))
    return np.linalg.norm(r) / nb if nb > 0 else np.linalg.norm(r)


# ----------------------------------------------------------------------------
# Small SPD solves with the rank-deficiency fallback (reading R6)
# ----------------------------------------------------------------------------

class _SPDSolver:
    """E^{-1} v through the Cholesky factor E = L L^T (float64)."""

    def __init__(self, E):
        self.L = np.linalg.cholesky(E)

    def __call__(self, v):
        y = sla.solve_triangular(self.L, v, lower=True)
        return sla.solve_triangular(self.L.T, y, lower=False)


def _galerkin(W, AW):
    """E = W^T A W, formed as W^T (AW) and symmetrised; returns (W, AW, solver)."""
    E = W.T @ AW
    E = 0.5 * (E + E.T)
    try:
        return W, AW, _SPDSolver(E)
    except np.linalg.LinAlgError:
        lam, Qe = np.linalg.eigh(E)
        keep = lam > 1e-12 * max(lam.max(), 0.0)
        W, AW = W @ Qe[:, keep], AW @ Qe[:, keep]
        E = W.T @ AW
        E = 0.5 * (E + E.T)
        return W, AW, _SPDSolver(E)


# ----------------------------------------------------------------------------
# Plain CG and def-CG (Algorithm 1)
# ----------------------------------------------------------------------------

@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    status: int
    relres_true: float
    history: list                 # recursive |r_j| / |b| for j = 0, 1, ...
    matvecs_loop: int = 0
    matvecs_setup: int = 0        # A x_{-1} (if nonzero) and A W
    matvecs_check: int = 0        # true-residual confirmations and replacements
    P: list = field(default_factory=list)   # stored p_j (window R3)
    Q: list = field(default_factory=list)   # stored A p_j
    d: list = field(default_factory=list)
    alpha: list = field(default_factory=list)
    beta: list = field(default_factory=list)
    mu: list = field(default_factory=list)
    k_used: int = 0
    W: np.ndarray | None = None   # W actually used (after R6)
    AW: np.ndarray | None = None
    p_history: list = field(default_factory=list)
    r_history: list = field(default_factory=list)
    x_history: list = field(default_factory=list)

    @property
    def matvecs(self):
        return self.matvecs_loop + self.matvecs_setup + self.matvecs_check


def cg(A, b, x_init=None, tol=1e-6, max_iter=None, keep_iterates=False):
    """Hestenes-Stiefel CG: the iteration of Algorithm 1 with no deflation (W empty).

    Stopping follows R2: relative recursive residual, confirmed by the true
    residual. Kept deliberately separate from ``defcg`` so that the k = 0 case
    of def-CG can be checked against it iterate by iterate.
    """
    b = np.asarray(b, dtype=F64)
    n = b.size
    max_iter = 10 * n if max_iter is None else max_iter
    x = np.zeros(n) if x_init is None else np.array(x_init, dtype=F64)
    bnorm = np.linalg.norm(b)
    res = SolveResult(x=x, iters=0, status=STATUS_OK, relres_true=0.0, history=[])
    if bnorm == 0.0:
        res.x = np.zeros(n)
        return res
    if x_init is not None and np.any(x):
        r = b - _mv(A, x)
        res.matvecs_setup += 1
    else:
        r = b.copy()
    p = r.copy()
    rho = r @ r
    thresh = tol * bnorm
    res.history.append(np.sqrt(rho) / bnorm)
    if keep_iterates:
        res.x_history.append(x.copy()); res.r_history.append(r.copy()); res.p_history.append(p.copy())
    converged = np.sqrt(rho) <= thresh
    if converged:
        r_true = b - _mv(A, x)
        res.matvecs_check += 1
        if np.linalg.norm(r_true) > thresh:
            r = r_true
            rho = r @ r
            converged = False
    j = 0
    while not converged:
        if j >= max_iter:
            res.status = STATUS_MAXITER
            break
        q = _mv(A, p)                       # A p_j, then d_j = p_j^T A p_j
        res.matvecs_loop += 1
        d = p @ q
        if not d > 0.0:
            res.status = STATUS_BREAKDOWN
            break
        alpha = rho / d                     # step length alpha_j = rho_j / d_j
        x = x + alpha * p                   # x_{j+1}
        r = r - alpha * q                   # r_{j+1}
        rho_new = r @ r
        j += 1
        res.history.append(np.sqrt(rho_new) / bnorm)
        if np.sqrt(rho_new) <= thresh:      # R2: confirm with the true residual
            r_true = b - _mv(A, x)
            res.matvecs_check += 1
            if np.linalg.norm(r_true) <= thresh:
                break
            r = r_true
            rho_new = r @ r
        beta = rho_new / rho                # beta_j = rho_{j+1} / rho_j
        p = beta * p + r                    # direction update with W empty
        rho = rho_new
        if keep_iterates:
            res.x_history.append(x.copy()); res.r_history.append(r.copy()); res.p_history.append(p.copy())
    res.x, res.iters = x, j
    res.relres_true = true_relres(A, b, x)
    return res


def project_out(x, r, W, AW, Esolve):
    """Deflation of an iterate (the initial projection of Algorithm 1, reused
    by R13 after a replacement): g = E^{-1} W^T r, x <- x + W g, r <- r - AW g.
    Afterwards W^T r = W^T r_in - (W^T AW) E^{-1} W^T r_in = 0, and x and r
    move together: x_out - x_in = W g and r_in - r_out = AW g."""
    g = Esolve(W.T @ r)
    return x + W @ g, r - AW @ g


def next_direction(r, p, beta, W, AW, Esolve, reproject):
    """Direction update of Algorithm 1: p <- beta p + r - W mu with
    E mu = (AW)^T r (R1). With ``reproject`` (R13, after a replacement) mu is
    taken from (AW)^T (beta p + r), so that (AW)^T p_out = 0 even when the
    incoming p is not A-conjugate to W; in exact arithmetic (AW)^T p = 0 and
    the two forms agree. Returns (mu, p_out)."""
    h = AW.T @ r
    if reproject:
        h = h + beta * (AW.T @ p)
    mu = Esolve(h)
    return mu, beta * p + r - W @ mu


def defcg(A, b, x_init=None, W=None, AW=None, tol=1e-6, max_iter=None, ell=0,
          window="last", refine_every=0, keep_iterates=False, A_true=None):
    """Deflated-CG(k, ell)(A, b, x_{-1}, W, (AW), tol): Algorithm 1, Sec. 2.2.

    ``A`` is a dense matrix or a callable v -> A v. ``W`` is n x k (k may be 0
    or None for plain CG behaviour). ``AW`` may be supplied (Algorithm 1 takes
    it optionally); otherwise it is formed with k products. Returns a
    ``SolveResult`` holding x, the iteration count, the recursive residual
    history and the stored directions p_j with A p_j (reading R3).

    ``A_true`` (default: ``A``) is the operator whose residual b - A_true x is
    formed by the true-residual steps (the warm-start r_{-1}, the R2
    confirmation, the R13 replacements and the reported residual), while the
    recursion, A W and the stored A p_j use ``A``. With an ``A`` that only
    approximates ``A_true`` this is iterative refinement: the GPU's
    mixed-precision operators iterate with rounded kernel entries and certify
    with accurate ones.
    """
    b = np.asarray(b, dtype=F64)
    n = b.size
    max_iter = 10 * n if max_iter is None else max_iter
    x = np.zeros(n) if x_init is None else np.array(x_init, dtype=F64)
    res = SolveResult(x=x, iters=0, status=STATUS_OK, relres_true=0.0, history=[])
    k = 0 if W is None else W.shape[1]
    if k:
        W = np.asarray(W, dtype=F64)
        if AW is None:
            AW = np.column_stack([_mv(A, W[:, i]) for i in range(k)])
            res.matvecs_setup += k
        AW = np.asarray(AW, dtype=F64)
        W, AW, Esolve = _galerkin(W, AW)
        k = W.shape[1]
    res.k_used, res.W, res.AW = k, W, AW
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        res.x = np.zeros(n)
        return res

    A_res = A if A_true is None else A_true

    def deflate(x, r):
        """Initial projection: x <- x + W E^{-1} W^T r, so that W^T r = 0 afterwards."""
        if not k:
            return x, r
        return project_out(x, r, W, AW, Esolve)

    if x_init is not None and np.any(x):
        r = b - _mv(A_res, x)               # r_{-1}
        res.matvecs_setup += 1
    else:
        r = b.copy()
    x, r = deflate(x, r)                    # initial projection: x_0, r_0
    if k:                                   # first direction: E mu_0 = W^T A r_0 (R1)
        mu = Esolve(AW.T @ r)
        p = r - W @ mu
    else:
        mu = np.zeros(0)
        p = r.copy()
    rho = r @ r
    thresh = tol * bnorm
    res.history.append(np.sqrt(rho) / bnorm)
    if keep_iterates:
        res.x_history.append(x.copy()); res.r_history.append(r.copy()); res.p_history.append(p.copy())

    def store(j, p, q, d, alpha):
        if ell <= 0:
            return
        if window == "first":
            if j < ell:
                res.P.append(p.copy()); res.Q.append(q.copy()); res.d.append(d); res.alpha.append(alpha)
        else:
            res.P.append(p.copy()); res.Q.append(q.copy()); res.d.append(d); res.alpha.append(alpha)
            if len(res.P) > ell:
                del res.P[0], res.Q[0], res.d[0], res.alpha[0]

    converged = np.sqrt(rho) <= thresh
    if converged:
        r_true = b - _mv(A_res, x)
        res.matvecs_check += 1
        if np.linalg.norm(r_true) > thresh:
            x, r = deflate(x, r_true)
            rho = r @ r
            converged = False
    j = 0
    while not converged:                     # while |r_j| > tol |b| (R2)
        if j >= max_iter:
            res.status = STATUS_MAXITER
            break
        q = _mv(A, p)
        res.matvecs_loop += 1
        d = p @ q                            # d_j = p_j^T A p_j
        if not d > 0.0:
            res.status = STATUS_BREAKDOWN
            break
        alpha = rho / d                      # step length alpha_j = rho_j / d_j
        x = x + alpha * p                    # x_{j+1}
        r = r - alpha * q                    # r_{j+1}
        store(j, p, q, d, alpha)             # direction store (R3)
        rho_new = r @ r
        j += 1
        res.history.append(np.sqrt(rho_new) / bnorm)
        rho_rec = rho_new                    # the recursion's own |r_{j+1}|^2
        replaced = False
        if np.sqrt(rho_new) <= thresh:       # R2
            r_true = b - _mv(A_res, x)
            res.matvecs_check += 1
            if np.linalg.norm(r_true) <= thresh:
                break
            x, r = deflate(x, r_true)
            rho_new = r @ r
            replaced = True
        elif refine_every and j % refine_every == 0:   # R13
            x, r = deflate(x, b - _mv(A_res, x))
            res.matvecs_check += 1
            rho_new = r @ r
            replaced = True
        beta = rho_rec / rho                 # beta_j (R13: from the recursion)
        if k:                                # mu step: E mu_{j+1} = (AW)^T r_{j+1} (R1; R13)
            mu, p = next_direction(r, p, beta, W, AW, Esolve, replaced)
        else:
            mu = np.zeros(0)
            p = beta * p + r
        res.beta.append(beta)
        res.mu.append(mu)
        rho = rho_new
        if keep_iterates:
            res.x_history.append(x.copy()); res.r_history.append(r.copy()); res.p_history.append(p.copy())
    res.x, res.iters = x, j
    res.relres_true = true_relres(A_res, b, x)
    return res


# ----------------------------------------------------------------------------
# Harmonic Ritz extraction (Sec. 2.3, Eq. 7)
# ----------------------------------------------------------------------------

@dataclass
class RitzResult:
    theta: np.ndarray        # all harmonic Ritz values, descending
    W: np.ndarray            # n x k_new, unit columns (R5)
    U: np.ndarray            # coefficients of the chosen vectors in Z (before R5 scaling)
    F: np.ndarray
    G: np.ndarray
    theta_selected: np.ndarray


def _whitener(F):
    """T with T^T F T = I: the Cholesky inverse, or the R6 eigen-truncation."""
    try:
        L = np.linalg.cholesky(F)
        return sla.solve_triangular(L, np.eye(F.shape[0]), lower=True).T
    except np.linalg.LinAlgError:
        lam, Qf = np.linalg.eigh(F)
        keep = lam > 1e-12 * max(lam.max(), 0.0)
        return Qf[:, keep] / np.sqrt(lam[keep])


def _pencil_extract(Z, F, G, k, select):
    """Solves G u = theta F u (F symmetric positive definite on span(Z)) by
    reducing with a factor T of F^{-1} (T^T F T = I, R6 when F is singular):
    C = T^T G T, C v = theta v, u = T v. Keeps k values per R4 and returns
    W = Z U scaled per R5, with the pencil's F and G."""
    T = _whitener(F)
    C = T.T @ G @ T
    C = 0.5 * (C + C.T)
    theta, V = np.linalg.eigh(C)            # ascending
    U_all = T @ V
    if select == "largest":
        order = np.argsort(-theta, kind="stable")
    elif select == "smallest":
        order = np.argsort(theta, kind="stable")
    else:
        raise ValueError(select)
    kk = min(k, theta.size)
    sel = order[:kk]
    U = U_all[:, sel]
    Wn = Z @ U
    Wn = Wn / np.linalg.norm(Wn, axis=0)
    piv = np.argmax(np.abs(Wn), axis=0)
    Wn = Wn * np.sign(Wn[piv, np.arange(kk)])
    return RitzResult(theta=np.sort(theta)[::-1], W=Wn, U=U, F=F, G=G,
                      theta_selected=theta[sel])


def harmonic_ritz(W, AW, P, Q, k, select="largest"):
    """k harmonic Ritz vectors from Z = [W, P_ell] and AZ = [AW, A P_ell] (Sec. 2.3).

    Forms F = (AZ)^T Z (symmetrised; it equals Z^T A Z for symmetric A) and
    G = (AZ)^T (AZ), solves G u = theta F u (Eq. 7) by reducing with a
    factor T of F^{-1} (T^T F T = I): C = T^T G T, C v = theta v, u = T v.
    Keeps k values per R4 and returns W = Z U scaled per R5.
    """
    cols = [np.asarray(W, dtype=F64)] if W is not None and W.shape[1] else []
    acols = [np.asarray(AW, dtype=F64)] if AW is not None and AW.shape[1] else []
    if len(P):
        cols.append(np.column_stack(P).astype(F64))
        acols.append(np.column_stack(Q).astype(F64))
    Z = np.hstack(cols)
    AZ = np.hstack(acols)
    F = AZ.T @ Z
    F = 0.5 * (F + F.T)
    G = AZ.T @ AZ
    G = 0.5 * (G + G.T)
    return _pencil_extract(Z, F, G, k, select)


def rayleigh_ritz(W, AW, P, Q, k, select="largest"):
    """k Ritz vectors by orthogonal projection onto Z = [W, P_ell] (Sec. 2.3).

    The Galerkin condition Z^T (A - theta I) Z u = 0 gives the pencil
    Z^T A Z u = theta Z^T Z u (the equation before Eq. 7). Z^T A Z is formed as
    Z^T [AW, A P_ell] and symmetrised; the pencil is reduced with a factor T of
    (Z^T Z)^{-1} (T^T Z^T Z T = I, R6 when Z is rank deficient): C = T^T (Z^T A Z) T,
    C v = theta v, u = T v. Keeps k values per R4 and returns W = Z U scaled
    per R5. The returned F and G are Z^T Z and Z^T A Z.
    """
    cols = [np.asarray(W, dtype=F64)] if W is not None and W.shape[1] else []
    acols = [np.asarray(AW, dtype=F64)] if AW is not None and AW.shape[1] else []
    if len(P):
        cols.append(np.column_stack(P).astype(F64))
        acols.append(np.column_stack(Q).astype(F64))
    Z = np.hstack(cols)
    AZ = np.hstack(acols)
    M = Z.T @ Z
    M = 0.5 * (M + M.T)
    K = Z.T @ AZ
    K = 0.5 * (K + K.T)
    return _pencil_extract(Z, M, K, k, select)


def sparse_FG(E, GW, d, alpha, rho, h):
    """F and G of Eq. 7 from the scalars of a def-CG run, without Z or AZ: the
    explicit sparse forms of Saad et al. that Sec. 2.3 mentions.

    For ell consecutive stored directions p_s .. p_{s+ell-1} with no residual
    replacement between r_s and r_{s+ell}:
      * A-conjugacy and (AW)^T p_j = 0 (Sec. 2.2) make F = (AZ)^T Z
        block diagonal: E = W^T A W, then diag(d_j), d_j = p_j^T A p_j;
      * A p_j = (r_j - r_{j+1}) / alpha_j with mutually orthogonal residuals
        makes (AP)^T (AP) tridiagonal: (rho_j + rho_{j+1}) / alpha_j^2 on the
        diagonal, -rho_{j+1} / (alpha_j alpha_{j+1}) beside it;
      * the same identity gives the coupling (AW)^T A p_j = (h_j - h_{j+1}) / alpha_j
        with h_j = (AW)^T r_j; the W block is G_W = (AW)^T (AW).

    E, GW: k x k. d, alpha: ell values. rho: ell + 1 values |r_j|^2,
    j = s .. s + ell. h: k x (ell + 1), columns (AW)^T r_j for the same j.
    """
    E = np.asarray(E, dtype=F64)
    k, ell = E.shape[0], len(d)
    d, alpha, rho = (np.asarray(v, dtype=F64) for v in (d, alpha, rho))
    m = k + ell
    F = np.zeros((m, m))
    G = np.zeros((m, m))
    if k:
        F[:k, :k] = 0.5 * (E + E.T)
        GW = np.asarray(GW, dtype=F64)
        G[:k, :k] = 0.5 * (GW + GW.T)
    for j in range(ell):
        F[k + j, k + j] = d[j]
        G[k + j, k + j] = (rho[j] + rho[j + 1]) / alpha[j] ** 2
        if j + 1 < ell:
            G[k + j, k + j + 1] = G[k + j + 1, k + j] = -rho[j + 1] / (alpha[j] * alpha[j + 1])
        if k:
            col = (np.asarray(h[:, j], dtype=F64) - np.asarray(h[:, j + 1], dtype=F64)) / alpha[j]
            G[:k, k + j] = col
            G[k + j, :k] = col
    return F, G


def harmonic_ritz_sparse(W, P, E, GW, d, alpha, rho, h, k, select="largest"):
    """Eq. 7 with F and G from ``sparse_FG`` (no pass over AZ); the rest as in
    ``harmonic_ritz``: the same pencil reduction, selection and W = Z U."""
    kw = W.shape[1] if W is not None else 0
    cols = [np.asarray(W, dtype=F64)] if kw else []
    if len(P):
        cols.append(np.column_stack(P).astype(F64))
    Z = np.hstack(cols)
    F, G = sparse_FG(E if kw else np.zeros((0, 0)), GW, d, alpha, rho, h)
    return _pencil_extract(Z, F, G, k, select)


# ----------------------------------------------------------------------------
# A sequence of systems (Eq. 1) with recycling between them (Fig. 1)
# ----------------------------------------------------------------------------

def run_sequence(operators, rhs, k, ell, tol, window="last", select="largest",
                 refine_every=0, max_iter=None, deflate=True, W0=None, extraction="harmonic"):
    """Solve A_t x_t = b_t in order, carrying W from one system to the next.

    The first system runs as plain CG unless ``W0`` is given (Fig. 1 caption);
    after each solve k new vectors are extracted by ``harmonic_ritz`` (Eq. 7),
    or by ``rayleigh_ritz`` with ``extraction="ritz"``.
    ``deflate=False`` runs plain CG on every system (the Sec. 3 comparison).
    Returns a list of per-system dicts.
    """
    out = []
    W = W0
    for A, b in zip(operators, rhs):
        if deflate:
            res = defcg(A, b, W=W, tol=tol, max_iter=max_iter, ell=ell, window=window,
                        refine_every=refine_every)
            extract = {"harmonic": harmonic_ritz, "ritz": rayleigh_ritz}[extraction]
            rr = extract(res.W, res.AW, res.P, res.Q, k, select=select)
            W = rr.W
            out.append({"result": res, "ritz": rr})
        else:
            res = cg(A, b, tol=tol, max_iter=max_iter)
            out.append({"result": res, "ritz": None})
    return out
