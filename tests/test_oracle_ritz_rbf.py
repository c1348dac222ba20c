"""Pins for harmonic-Ritz extraction (Sec. 2.3, Eq. 7), the RBF operator
(Sec. 3) and the sequence behaviour the paper reports qualitatively."""

import math

import numpy as np
import pytest
import scipy.linalg as sla

import dcg_synth as S
from oracle import dcg_oracle as O


def _split(Z, A, k):
    W = Z[:, :k]
    P = [Z[:, j] for j in range(k, Z.shape[1])]
    return W, A @ W, P, [A @ p for p in P]


def test_invariant_subspace_gives_exact_eigenpairs():
    # If span(Z) is invariant under A, Eq. 7 holds exactly on it: the harmonic
    # Ritz values are eigenvalues of A and the vectors are eigenvectors.
    n = 60
    eigs = np.linspace(1.0, 30.0, n)
    A, Q = S.spd_with_spectrum(eigs, seed=4)
    idx = np.array([3, 10, 17, 40, 41, 55, 58, 59])
    R = np.random.default_rng(2).standard_normal((idx.size, idx.size))
    Z = Q[:, idx] @ R                     # a non-orthogonal basis of the subspace
    W, AW, P, AP = _split(Z, A, 3)
    rr = O.harmonic_ritz(W, AW, P, AP, k=4, select="largest")
    np.testing.assert_allclose(rr.theta, np.sort(eigs[idx])[::-1], rtol=1e-10)
    np.testing.assert_allclose(rr.theta_selected, np.sort(eigs[idx])[::-1][:4], rtol=1e-10)
    for j in range(4):
        w = rr.W[:, j]
        assert abs(np.linalg.norm(w) - 1) < 1e-12
        assert np.linalg.norm(A @ w - rr.theta_selected[j] * w) <= 1e-9
    small = O.harmonic_ritz(W, AW, P, AP, k=2, select="smallest")
    np.testing.assert_allclose(small.theta_selected, np.sort(eigs[idx])[:2], rtol=1e-10)


def test_generalized_eigen_residual_and_scipy():
    n, m = 50, 9
    A, _ = S.spd_with_spectrum(np.geomspace(0.1, 100, n), seed=9)
    Z = np.random.default_rng(3).standard_normal((n, m))
    W, AW, P, AP = _split(Z, A, 4)
    rr = O.harmonic_ritz(W, AW, P, AP, k=m)
    AZ = A @ Z
    F, G = AZ.T @ Z, AZ.T @ AZ
    # G u = theta F u for every kept pair (Eq. 7)
    for j in range(m):
        u, th = rr.U[:, j], rr.theta_selected[j]
        assert np.linalg.norm(G @ u - th * F @ u) <= 1e-9 * np.linalg.norm(G) * np.linalg.norm(u)
    # harmonic Ritz values lie inside the spectrum of A
    ev = np.linalg.eigvalsh(A)
    assert rr.theta.max() <= ev[-1] * (1 + 1e-10) and rr.theta.min() >= ev[0] * (1 - 1e-10)
    # the general-pencil routine agrees on the values
    ref = sla.eigh(0.5 * (G + G.T), 0.5 * (F + F.T), eigvals_only=True)
    np.testing.assert_allclose(rr.theta, np.sort(ref)[::-1], rtol=1e-9)


def test_selection_count_sign_and_norm():
    n = 40
    A, _ = S.spd_with_spectrum(np.linspace(1, 9, n), seed=1)
    Z = np.random.default_rng(5).standard_normal((n, 5))
    W, AW, P, AP = _split(Z, A, 2)
    rr = O.harmonic_ritz(W, AW, P, AP, k=8)      # asks for more than m = 5
    assert rr.W.shape == (n, 5)
    np.testing.assert_allclose(np.linalg.norm(rr.W, axis=0), 1.0, rtol=1e-13)
    piv = np.argmax(np.abs(rr.W), axis=0)
    assert np.all(rr.W[piv, np.arange(5)] > 0)
    assert np.all(np.diff(rr.theta_selected) <= 0)


def test_rank_deficient_Z_falls_back():
    n = 30
    A, _ = S.spd_with_spectrum(np.linspace(1, 5, n), seed=2)
    Z = np.random.default_rng(6).standard_normal((n, 4))
    Z = np.column_stack([Z, Z[:, 1]])             # duplicated direction
    W, AW, P, AP = _split(Z, A, 2)
    rr = O.harmonic_ritz(W, AW, P, AP, k=3)
    assert np.all(np.isfinite(rr.W)) and rr.W.shape[1] == 3
    # the new vectors lie in span(Z)
    proj = Z @ np.linalg.lstsq(Z, rr.W, rcond=None)[0]
    assert np.linalg.norm(proj - rr.W) <= 1e-8


def test_first_system_uses_directions_only():
    # Fig. 1 caption: the first system is plain CG; W comes from P_ell alone.
    n = 80
    A, _ = S.spd_with_spectrum(np.geomspace(0.01, 50, n), seed=7)
    b = np.random.default_rng(1).standard_normal(n)
    res = O.defcg(A, b, W=None, tol=1e-8, ell=12, window="first")
    rr = O.harmonic_ritz(res.W, res.AW, res.P, res.Q, k=4)
    assert rr.W.shape == (n, 4)
    # the first ell directions span the Krylov space K_ell(A, r_0) (Eq. 3); its
    # largest harmonic Ritz value converges to lambda_max first
    assert abs(rr.theta_selected[0] - 50.0) / 50.0 < 1e-4


# ---------------------------------------------------------------------------
# RBF operator (Sec. 3)
# ---------------------------------------------------------------------------

def test_rbf_closed_form_points():
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0]])
    l, s2, sig2 = 0.7, 1.9, 0.05
    K = O.rbf_gram(X, l, s2, sig2)
    e = lambda sq: s2 * math.exp(-sq / (2 * l * l))
    expect = np.array([[s2 + sig2, e(1.0), e(4.0)],
                       [e(1.0), s2 + sig2, e(5.0)],
                       [e(4.0), e(5.0), s2 + sig2]])
    np.testing.assert_allclose(K, expect, rtol=1e-15, atol=0)


def test_rbf_spd_rows_and_matvec():
    X = np.random.default_rng(0).standard_normal((70, 3))
    K = O.rbf_gram(X, 1.3, 1.0, 1e-2)
    assert np.array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() > 0
    rows = np.array([0, 5, 69])
    np.testing.assert_array_equal(O.rbf_gram(X, 1.3, 1.0, 1e-2, rows=rows), K[rows])
    v = np.random.default_rng(1).standard_normal(70)
    np.testing.assert_allclose(O.rbf_matvec(X, 1.3, 1.0, 1e-2)(v), K @ v, rtol=1e-13, atol=1e-13)
    # the diagonal is s^2 + noise exactly
    np.testing.assert_array_equal(np.diag(K), np.full(70, 1.0 + 1e-2))


def test_sequence_recycling_saves_iterations():
    # Sec. 3 / Fig. 2: after the first system (plain CG), def-CG needs fewer
    # iterations than CG on each later system of a slowly changing sequence.
    cfg = S.SMALL_1024.scaled(256, T=4)
    X, bs = S.draw_sequence(cfg)
    ops = [O.rbf_gram(X, cfg.lengthscale(t), cfg.signal_var, cfg.noise) for t in range(cfg.T)]
    d = O.run_sequence(ops, bs, k=cfg.k, ell=cfg.ell, tol=cfg.tol)
    c = O.run_sequence(ops, bs, k=cfg.k, ell=cfg.ell, tol=cfg.tol, deflate=False)
    assert d[0]["result"].iters == c[0]["result"].iters
    for t in range(1, cfg.T):
        assert d[t]["result"].iters < c[t]["result"].iters
        assert d[t]["result"].relres_true <= cfg.tol


# ---------------------------------------------------------------------------
# Orthogonal (Rayleigh-Ritz) extraction: the equation before Eq. 7
# ---------------------------------------------------------------------------

def test_rayleigh_ritz_galerkin_condition_and_orthonormal_basis():
    # The definition: every returned pair (theta, v = Z u) leaves a residual
    # A v - theta v orthogonal to span(Z). And the values are those of the
    # standard symmetric problem Q^T A Q on an orthonormal basis Q of span(Z).
    n, k = 90, 4
    A, _ = S.spd_with_spectrum(np.geomspace(0.5, 80.0, 90), seed=17)
    Z = np.random.default_rng(5).standard_normal((n, 11))
    W, AW, P, AP = _split(Z, A, k)
    rr = O.rayleigh_ritz(W, AW, P, AP, k=6, select="largest")
    for j in range(6):
        v = Z @ rr.U[:, j]
        res = A @ v - rr.theta_selected[j] * v
        assert np.linalg.norm(Z.T @ res) <= 1e-10 * np.linalg.norm(Z) * np.linalg.norm(A @ v)
    Qz, _ = np.linalg.qr(Z)
    ref = np.sort(np.linalg.eigvalsh(Qz.T @ A @ Qz))[::-1]
    np.testing.assert_allclose(rr.theta, ref, rtol=1e-11)
    np.testing.assert_allclose(rr.theta_selected, ref[:6], rtol=1e-11)
    small = O.rayleigh_ritz(W, AW, P, AP, k=3, select="smallest")
    np.testing.assert_allclose(small.theta_selected, ref[::-1][:3], rtol=1e-11)
    # Cauchy interlacing: the i-th largest Ritz value lies between the i-th
    # largest and the (n - m + i)-th largest eigenvalue of A
    lam = np.sort(np.linalg.eigvalsh(A))[::-1]
    m = Z.shape[1]
    for i in range(m):
        assert lam[n - m + i] * (1 - 1e-12) <= rr.theta[i] <= lam[i] * (1 + 1e-12)
    for j in range(6):
        assert abs(np.linalg.norm(rr.W[:, j]) - 1) < 1e-12
        piv = np.argmax(np.abs(rr.W[:, j]))
        assert rr.W[piv, j] > 0


def test_rayleigh_ritz_on_cg_directions_is_the_lanczos_tridiagonal():
    # Plain CG from x = 0: p_0 .. p_{j-1} span K_j(A, b), so the Ritz values on
    # them are the eigenvalues of the Lanczos matrix that CG's own scalars
    # define (Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.7):
    # T_ii = 1/alpha_i + beta_{i-1}/alpha_{i-1}, T_{i,i+1} = sqrt(beta_i)/alpha_i.
    n, j = 120, 9
    A, _ = S.spd_with_spectrum(np.geomspace(1.0, 40.0, n), seed=23)
    b = np.random.default_rng(8).standard_normal(n)
    res = O.defcg(A, b, tol=1e-12, ell=j, window="first")
    assert len(res.P) == j and res.iters > j
    al, be = res.alpha[:j], res.beta[:j]
    T = np.zeros((j, j))
    for i in range(j):
        T[i, i] = 1.0 / al[i] + (be[i - 1] / al[i - 1] if i else 0.0)
        if i + 1 < j:
            T[i, i + 1] = T[i + 1, i] = math.sqrt(be[i]) / al[i]
    ref = np.sort(np.linalg.eigvalsh(T))[::-1]
    rr = O.rayleigh_ritz(None, None, res.P, res.Q, k=3)
    np.testing.assert_allclose(rr.theta, ref, rtol=1e-9)


def test_rayleigh_ritz_invariant_subspace_and_sequence():
    # On an invariant span(Z) the Ritz values are eigenvalues of A; a recycled
    # sequence with extraction="ritz" converges on every system.
    n = 60
    eigs = np.linspace(1.0, 30.0, n)
    A, Q = S.spd_with_spectrum(eigs, seed=4)
    idx = np.array([2, 9, 30, 50, 57, 59])
    Z = Q[:, idx] @ np.random.default_rng(3).standard_normal((idx.size, idx.size))
    W, AW, P, AP = _split(Z, A, 2)
    rr = O.rayleigh_ritz(W, AW, P, AP, k=3)
    np.testing.assert_allclose(rr.theta, np.sort(eigs[idx])[::-1], rtol=1e-10)
    for j in range(3):
        w = rr.W[:, j]
        assert np.linalg.norm(A @ w - rr.theta_selected[j] * w) <= 1e-9
    cfg = S.SMALL_1024.scaled(256, T=3)
    X, bs = S.draw_sequence(cfg, T=3)
    ops = [O.rbf_gram(X.astype(np.float64), cfg.lengthscale(t), cfg.signal_var, cfg.noise) for t in range(3)]
    out = O.run_sequence(ops, bs, cfg.k, cfg.ell, 1e-8, extraction="ritz")
    for o in out:
        assert o["result"].status == O.STATUS_OK and o["result"].relres_true <= 1e-8


# ---------------------------------------------------------------------------
# Sparse F and G from the scalars of the run (Saad et al., mentioned in Sec. 2.3)
# ---------------------------------------------------------------------------

def _sparse_inputs(res, s, ell):
    R = res.r_history
    W, AW = res.W, res.AW
    k = 0 if W is None else W.shape[1]
    E = W.T @ AW if k else np.zeros((0, 0))
    GW = AW.T @ AW if k else np.zeros((0, 0))
    rho = [R[j] @ R[j] for j in range(s, s + ell + 1)]
    h = np.column_stack([AW.T @ R[j] for j in range(s, s + ell + 1)]) if k else np.zeros((0, ell + 1))
    return E, GW, res.d, res.alpha, rho, h


@pytest.mark.parametrize("k,window", [(0, "first"), (4, "first"), (4, "last")])
def test_sparse_FG_equal_the_dense_products(k, window):
    # F = (AZ)^T Z and G = (AZ)^T (AZ) formed from Z and AZ must equal the
    # forms built only from E, G_W, d_j, alpha_j, |r_j|^2 and (AW)^T r_j; the
    # harmonic Ritz values and vectors then agree as well.
    n, ell = 150, 8
    A, _ = S.spd_with_spectrum(np.geomspace(1.0, 60.0, n), seed=31)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(n)
    W = rng.standard_normal((n, k)) if k else None
    if window == "first":
        res = O.defcg(A, b, W=W, tol=1e-12, ell=ell, window="first", keep_iterates=True)
        s = 0
    else:
        # stop by max_iter so that the residual after the last stored direction
        # is in the kept history
        res = O.defcg(A, b, W=W, tol=1e-14, max_iter=20, ell=ell, window="last", keep_iterates=True)
        assert res.status == O.STATUS_MAXITER and res.iters == 20
        s = res.iters - ell
    assert len(res.P) == ell and res.iters > ell
    dense = O.harmonic_ritz(res.W if k else None, res.AW if k else None, res.P, res.Q, 5)
    E, GW, d, alpha, rho, h = _sparse_inputs(res, s, ell)
    F, G = O.sparse_FG(E, GW, d, alpha, rho, h)
    np.testing.assert_allclose(F, dense.F, rtol=0, atol=1e-10 * np.abs(dense.F).max())
    np.testing.assert_allclose(G, dense.G, rtol=0, atol=1e-10 * np.abs(dense.G).max())
    sp = O.harmonic_ritz_sparse(res.W if k else None, res.P, E, GW, d, alpha, rho, h, 5)
    np.testing.assert_allclose(sp.theta, dense.theta, rtol=1e-9)
    for j in range(5):
        assert abs(sp.W[:, j] @ dense.W[:, j]) > 1 - 1e-9
