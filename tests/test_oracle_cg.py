"""Pins for the oracle's plain CG and def-CG (Algorithm 1, Sec. 2.2).

Each check compares the oracle with something other than itself: a dense
factorisation, a hand-derived exact run, a property CG must have in exact
arithmetic (finite termination, W^T r_j = 0, A-conjugacy, A-norm optimality of
each iterate over its search space), or CG on the reduced spectrum.
"""

import numpy as np
import pytest
import scipy.linalg as sla

import dcg_synth as S
from oracle import dcg_oracle as O


def _spd(n, seed, lo=1.0, hi=50.0):
    eigs = np.geomspace(lo, hi, n)
    return S.spd_with_spectrum(eigs, seed=seed)


def test_cg_two_by_two_exact_run():
    # A = [[4,1],[1,3]], b = [1,2], x_{-1} = 0. Worked by hand in exact fractions:
    # r0 = p0 = (1,2), A p0 = (6,7), d0 = 20, rho0 = 5, alpha0 = 1/4,
    # x1 = (1/4, 1/2), r1 = (-1/2, 1/4), rho1 = 5/16, beta0 = 1/16,
    # p1 = (-7/16, 3/8); CG ends after 2 steps at A^{-1} b = (1/11, 7/11).
    A = np.array([[4.0, 1.0], [1.0, 3.0]])
    b = np.array([1.0, 2.0])
    res = O.cg(A, b, tol=1e-14, keep_iterates=True)
    assert res.iters == 2
    np.testing.assert_allclose(res.x_history[1], [0.25, 0.5], rtol=0, atol=1e-15)
    np.testing.assert_allclose(res.r_history[1], [-0.5, 0.25], rtol=0, atol=1e-15)
    np.testing.assert_allclose(res.p_history[1], [-7 / 16, 3 / 8], rtol=0, atol=1e-15)
    np.testing.assert_allclose(res.x, [1 / 11, 7 / 11], rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 7, 64])
def test_cg_matches_cholesky(n):
    A, _ = _spd(n, seed=n)
    b = np.random.default_rng(n).standard_normal(n)
    x_ref = sla.cho_solve(sla.cho_factor(A), b)
    res = O.cg(A, b, tol=1e-14)
    assert res.status == O.STATUS_OK
    assert np.linalg.norm(res.x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)


def test_cg_terminates_in_distinct_eigenvalue_count():
    # A has 5 distinct eigenvalues (with multiplicity): exact CG stops after 5 steps.
    eigs = np.repeat([1.0, 2.0, 5.0, 11.0, 23.0], [10, 7, 9, 6, 8])
    A, _ = S.spd_with_spectrum(eigs, seed=3)
    b = np.random.default_rng(1).standard_normal(eigs.size)
    res = O.cg(A, b, tol=1e-11)
    assert res.iters <= 5
    assert O.true_relres(A, b, res.x) <= 1e-11


def test_cg_at_most_n_steps():
    # finite termination in n steps (exact arithmetic); a mild spectrum keeps
    # FP64 rounding from delaying it
    n = 24
    A, _ = _spd(n, seed=5, hi=8.0)
    b = np.random.default_rng(2).standard_normal(n)
    res = O.cg(A, b, tol=1e-10)
    assert res.iters <= n
    assert res.relres_true <= 1e-10


def test_zero_rhs_returns_zero():
    A, _ = _spd(8, seed=1)
    for fn in (O.cg, O.defcg):
        res = fn(A, np.zeros(8), tol=1e-8)
        assert res.iters == 0 and not np.any(res.x)


@pytest.mark.parametrize("n,k", [(5, 2), (40, 3), (64, 8)])
def test_defcg_matches_cholesky(n, k):
    A, _ = _spd(n, seed=10 + n)
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n)
    W = rng.standard_normal((n, k))
    x_ref = sla.cho_solve(sla.cho_factor(A), b)
    res = O.defcg(A, b, W=W, tol=1e-14)
    assert res.status == O.STATUS_OK
    assert np.linalg.norm(res.x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)


def test_defcg_warm_start_matches_cholesky():
    n, k = 50, 4
    A, _ = _spd(n, seed=77)
    rng = np.random.default_rng(3)
    b, x0, W = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal((n, k))
    res = O.defcg(A, b, x_init=x0, W=W, tol=1e-13)
    x_ref = sla.cho_solve(sla.cho_factor(A), b)
    assert np.linalg.norm(res.x - x_ref) <= 1e-11 * np.linalg.norm(x_ref)
    assert res.matvecs_setup == k + 1


def test_defcg_residuals_orthogonal_to_W_and_directions_conjugate():
    # Eq. 5 with conjugacy (Sec. 2.2): W^T r_j = 0 for all j, (AW)^T p_j = 0,
    # and successive directions are A-conjugate.
    n, k = 80, 5
    A, _ = _spd(n, seed=21, hi=200.0)
    rng = np.random.default_rng(4)
    b, W = rng.standard_normal(n), rng.standard_normal((n, k))
    res = O.defcg(A, b, W=W, tol=1e-10, keep_iterates=True)
    AW = A @ W
    # rounding leaves W^T r_j at the eps * |W| |b| level (absolute, not
    # relative to the shrinking |r_j|); a missing line-3 projection gives O(1)
    for r, p in zip(res.r_history, res.p_history):
        assert np.linalg.norm(W.T @ r) <= 1e-12 * np.linalg.norm(W) * np.linalg.norm(b)
        assert np.linalg.norm(AW.T @ p) <= 1e-9 * np.linalg.norm(AW) * np.linalg.norm(p)
    P = res.p_history
    for j in range(min(len(P) - 1, 12)):
        c = P[j] @ (A @ P[j + 1])
        assert abs(c) <= 1e-9 * np.sqrt((P[j] @ A @ P[j]) * (P[j + 1] @ A @ P[j + 1]))


def _a_norm_minimiser(A, b, x0, B):
    """argmin over x in x0 + span(B) of |x - A^{-1} b|_A, by least squares in
    the metric of the Cholesky factor (A = L L^T): min |L^T (x0 + B c - x*)|."""
    L = np.linalg.cholesky(A)
    xs = sla.cho_solve((L, True), b)
    c, *_ = np.linalg.lstsq(L.T @ B, L.T @ (xs - x0), rcond=None)
    return x0 + B @ c


@pytest.mark.parametrize("k,warm", [(0, False), (4, False), (4, True)])
def test_defcg_iterates_minimise_the_a_norm_error(k, warm):
    # Optimality of deflated CG (Saad, Yeung, Erhel and Guyomarc'h, SIAM J.
    # Sci. Comput. 21, 2000): the j-th iterate minimises |x - x*|_A over
    # x_{-1} + span(W) + K_j(H A, H r_0), H = I - W (W^T A W)^{-1} (AW)^T, with
    # r_0 the residual of the A-norm-best point of x_{-1} + span(W) (Sec. 2.2,
    # Eq. 5-6). k = 0 is the plain CG statement. The minimiser is computed here
    # by least squares on an orthonormal basis, not by a recursion.
    n = 60
    A, _ = _spd(n, seed=33, hi=30.0)
    rng = np.random.default_rng(12)
    b = rng.standard_normal(n)
    W = rng.standard_normal((n, k)) if k else None
    x_init = rng.standard_normal(n) if warm else None
    res = O.defcg(A, b, x_init=x_init, W=W, tol=1e-11, keep_iterates=True)
    xm1 = np.zeros(n) if x_init is None else x_init
    if k:
        x0 = _a_norm_minimiser(A, b, xm1, W)
        H = np.eye(n) - W @ np.linalg.solve(W.T @ A @ W, (A @ W).T)
    else:
        x0 = xm1
        H = np.eye(n)
    np.testing.assert_allclose(res.x_history[0], x0, rtol=0, atol=1e-11 * np.linalg.norm(x0))
    v = H @ (b - A @ x0)
    kry = []
    for j in range(1, min(9, len(res.x_history))):
        kry.append(v / np.linalg.norm(v))
        v = H @ (A @ kry[-1])
        Bj, _ = np.linalg.qr(np.column_stack(([W] if k else []) + kry))
        want = _a_norm_minimiser(A, b, xm1, Bj)
        got = res.x_history[j]
        assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want), j


def test_defcg_error_bounded_by_residual_in_the_a_norm():
    # |x - x*|_A^2 = r^T A^{-1} r <= |r|^2 / lambda_min, and |x*|_A^2 = b^T A^{-1} b
    # >= |b|^2 / lambda_max, so the relative A-norm error of the returned x is at
    # most sqrt(kappa) times its relative true residual; the residual meets tol.
    n, k = 200, 6
    eigs = np.geomspace(1e-2, 10.0, n)
    A, Q = S.spd_with_spectrum(eigs, seed=5)
    b = np.random.default_rng(6).standard_normal(n)
    res = O.defcg(A, b, W=Q[:, :k], tol=1e-8)
    xs = np.linalg.solve(A, b)
    e = res.x - xs
    rel_a = np.sqrt(e @ A @ e) / np.sqrt(xs @ A @ xs)
    relres = np.linalg.norm(b - A @ res.x) / np.linalg.norm(b)
    assert relres <= 1e-8
    assert rel_a <= np.sqrt(eigs[-1] / eigs[0]) * relres * (1 + 1e-8)


def test_defcg_k0_reproduces_cg_bitwise():
    # Algorithm 1 differs from CG only in the initial projection and the mu step (Sec. 2.2): with W
    # empty every iterate must be identical.
    n = 60
    A, _ = _spd(n, seed=8, hi=300.0)
    b = np.random.default_rng(9).standard_normal(n)
    a = O.cg(A, b, tol=1e-9, keep_iterates=True)
    d = O.defcg(A, b, W=None, tol=1e-9, keep_iterates=True)
    assert a.iters == d.iters
    for u, v in zip(a.x_history, d.x_history):
        assert np.array_equal(u, v)
    for u, v in zip(a.p_history, d.p_history):
        assert np.array_equal(u, v)
    assert np.array_equal(a.x, d.x)
    assert a.history == d.history


def test_exact_eigenvectors_reduce_to_cg_on_remaining_spectrum():
    # Deflating an exact invariant subspace W = Q_S leaves CG on diag(Lambda \ S)
    # with right-hand side Q_{S^c}^T b: same residual norms, same iteration count.
    # a mild bulk plus six large outliers (the shape of K + noise I); on a
    # mild bulk FP64 CG keeps orthogonality, so the identity holds to rounding
    n = 70
    eigs = np.concatenate([np.linspace(1.0, 6.0, n - 6), np.geomspace(50.0, 400.0, 6)])
    A, Q = S.spd_with_spectrum(eigs, seed=31)
    S_idx = np.arange(n - 6, n)           # the 6 largest, as the experiment deflates
    C_idx = np.arange(0, n - 6)
    b = np.random.default_rng(5).standard_normal(n)
    tau = 1e-9 * np.linalg.norm(b)
    res = O.defcg(A, b, W=Q[:, S_idx], tol=tau / np.linalg.norm(b))
    bp = Q[:, C_idx].T @ b
    red = O.cg(np.diag(eigs[C_idx]), bp, tol=tau / np.linalg.norm(bp))
    assert res.iters == red.iters
    h1 = np.array(res.history) * np.linalg.norm(b)
    h2 = np.array(red.history) * np.linalg.norm(bp)
    np.testing.assert_allclose(h1, h2, rtol=1e-7, atol=1e-12 * np.linalg.norm(b))
    # and the deflated run beats plain CG on the full spectrum
    full = O.cg(A, b, tol=tau / np.linalg.norm(b))
    assert res.iters < full.iters


def test_defcg_rank_deficient_W_drops_direction():
    # Reading R6: a duplicated column of W makes E singular; it is dropped.
    n = 30
    A, _ = _spd(n, seed=2)
    rng = np.random.default_rng(6)
    W = rng.standard_normal((n, 3))
    W = np.column_stack([W, W[:, 0]])
    b = rng.standard_normal(n)
    res = O.defcg(A, b, W=W, tol=1e-12)
    assert res.k_used == 3
    assert O.true_relres(A, b, res.x) <= 1e-12


def test_refinement_keeps_solution():
    n, k = 64, 4
    A, _ = _spd(n, seed=12, hi=1e4)
    rng = np.random.default_rng(7)
    b, W = rng.standard_normal(n), rng.standard_normal((n, k))
    res = O.defcg(A, b, W=W, tol=1e-11, refine_every=5)
    x_ref = sla.cho_solve(sla.cho_factor(A), b)
    assert res.relres_true <= 1e-11
    assert np.linalg.norm(res.x - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
    assert res.matvecs_check >= res.iters // 5


def test_window_first_and_last():
    n = 50
    A, _ = _spd(n, seed=13, hi=500.0)
    b = np.random.default_rng(8).standard_normal(n)
    first = O.defcg(A, b, tol=1e-10, ell=6, window="first", keep_iterates=True)
    last = O.defcg(A, b, tol=1e-10, ell=6, window="last", keep_iterates=True)
    assert len(first.P) == 6 and len(last.P) == 6
    for j in range(6):
        assert np.array_equal(first.P[j], first.p_history[j])
        np.testing.assert_allclose(first.Q[j], A @ first.p_history[j], rtol=1e-13, atol=1e-13)
    J = last.iters
    for j in range(6):
        assert np.array_equal(last.P[j], last.p_history[J - 6 + j])


def test_maxiter_status():
    A, _ = _spd(40, seed=3, hi=1e4)
    b = np.random.default_rng(1).standard_normal(40)
    res = O.defcg(A, b, tol=1e-12, max_iter=3)
    assert res.status == O.STATUS_MAXITER and res.iters == 3


def test_breakdown_on_indefinite():
    eigs = np.array([-1.0, 1.0, 2.0, 3.0])
    A, _ = S.spd_with_spectrum(eigs, seed=0)
    # b along the negative eigenvector gives d_0 = p^T A p < 0
    _, Q = S.spd_with_spectrum(eigs, seed=0)
    res = O.defcg(A, Q[:, 0], tol=1e-10)
    assert res.status == O.STATUS_BREAKDOWN


# ----------------------------------------------------------------------------
# Residual replacement (reading R13: r <- b - A x every m iterations, re-deflate,
# mu from (AW)^T (beta p + r), beta from the recursion; van der Vorst and Ye's
# residual replacement). In exact arithmetic with one operator a replacement
# changes nothing, so the branch is pinned three ways: its two steps as
# functions on arbitrary inputs, the no-op property with one operator, and its
# exact identities when the loop operator only approximates the certified one
# (iterative refinement, the GPU's mixed-precision setting).
# ----------------------------------------------------------------------------

def _galerkin_parts(n, k, seed):
    A, _ = _spd(n, seed=seed, hi=40.0)
    rng = np.random.default_rng(seed + 100)
    W = rng.standard_normal((n, k))
    AW = A @ W
    W, AW, Esolve = O._galerkin(W, AW)
    return A, W, AW, Esolve, rng


def test_project_out_deflates_and_moves_x_and_r_together():
    n, k = 40, 5
    A, W, AW, Esolve, rng = _galerkin_parts(n, k, seed=21)
    x, r = rng.standard_normal(n), rng.standard_normal(n)
    assert np.linalg.norm(W.T @ r) > 1.0          # the input is not deflated
    x2, r2 = O.project_out(x, r, W, AW, Esolve)
    # W^T r = 0 afterwards (the Galerkin condition of the initial projection)
    assert np.linalg.norm(W.T @ r2) <= 1e-12 * np.linalg.norm(W) * np.linalg.norm(r)
    # one coefficient vector g moves both: x2 - x = W g, r - r2 = AW g
    g, *_ = np.linalg.lstsq(W, x2 - x, rcond=None)
    np.testing.assert_allclose(W @ g, x2 - x, rtol=0, atol=1e-12 * np.linalg.norm(x2 - x))
    np.testing.assert_allclose(AW @ g, r - r2, rtol=0, atol=1e-12 * np.linalg.norm(AW @ g))
    # a residual consistent with x stays consistent: r = b - A x => r2 = b - A x2
    b = r + A @ x
    x3, r3 = O.project_out(x, b - A @ x, W, AW, Esolve)
    np.testing.assert_allclose(r3, b - A @ x3, rtol=0, atol=1e-12 * np.linalg.norm(b))


def test_next_direction_reprojects_an_arbitrary_direction():
    n, k = 40, 5
    A, W, AW, Esolve, rng = _galerkin_parts(n, k, seed=22)
    r, p, beta = rng.standard_normal(n), rng.standard_normal(n), 0.37
    assert np.linalg.norm(AW.T @ p) > 1.0         # p is not A-conjugate to W
    mu, p2 = O.next_direction(r, p, beta, W, AW, Esolve, reproject=True)
    # (AW)^T p2 = 0: the new direction is A-conjugate to W whatever p was
    assert np.linalg.norm(AW.T @ p2) <= 1e-12 * np.linalg.norm(AW) * np.linalg.norm(p)
    # p2 = beta p + r - W mu with mu solving E mu = (AW)^T (beta p + r)
    np.testing.assert_allclose(p2, beta * p + r - W @ mu, rtol=0, atol=1e-13 * np.linalg.norm(p2))
    E = W.T @ AW
    np.testing.assert_allclose(E @ mu, AW.T @ (beta * p + r), rtol=0,
                               atol=1e-11 * np.linalg.norm(AW.T @ (beta * p + r)))
    # the plain form (Algorithm 1's mu from (AW)^T r) leaves beta (AW)^T p behind
    _, p3 = O.next_direction(r, p, beta, W, AW, Esolve, reproject=False)
    np.testing.assert_allclose(AW.T @ p3, beta * (AW.T @ p), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("kappa,n,tol", [(10.0, 80, 1e-8), (20.0, 120, 1e-9)])
def test_replacement_is_a_noop_with_one_operator(kappa, n, tol):
    # Well-conditioned systems (kappa <= 20, measured: iterates of the two runs
    # agree to 5e-16 and 2e-13 of |b|); on harder ones FP64 CG's loss of
    # orthogonality makes the replaced and the recursive paths part visibly.
    k = 4
    A, _ = S.spd_with_spectrum(np.geomspace(1.0, kappa, n), seed=23)
    rng = np.random.default_rng(24)
    b, W = rng.standard_normal(n), rng.standard_normal((n, k))
    ref = O.defcg(A, b, W=W, tol=tol, keep_iterates=True)
    rep = O.defcg(A, b, W=W, tol=tol, refine_every=3, keep_iterates=True)
    assert rep.iters == ref.iters
    assert rep.matvecs_check >= ref.iters // 3
    bn = np.linalg.norm(b)
    for j in range(len(ref.x_history)):
        for a, c in ((rep.x_history[j], ref.x_history[j]), (rep.p_history[j], ref.p_history[j]),
                     (rep.r_history[j], ref.r_history[j])):
            assert np.linalg.norm(a - c) <= 1e-11 * bn, j
    np.testing.assert_allclose(rep.x, ref.x, rtol=0, atol=1e-11 * np.linalg.norm(ref.x))
    np.testing.assert_allclose(rep.beta, ref.beta, rtol=1e-6)


def _perturbed(A, rel, seed):
    rng = np.random.default_rng(seed)
    S_ = rng.standard_normal(A.shape)
    S_ = 0.5 * (S_ + S_.T)
    return A + rel * np.linalg.norm(A, 2) / np.linalg.norm(S_, 2) * S_


def test_replacement_identities_with_an_approximate_loop_operator():
    # The loop runs on A_loop = A + E (|E| = 1e-6 |A|), the replacements and
    # the final check on A: iterative refinement. Every replacement must
    # re-deflate (W^T r = 0 afterwards), keep p A_loop-conjugate to W, and take
    # beta from the recursion's |r_{j+1}|^2 over the current rho (recomputed
    # from the replaced residual); the solve must still certify tol on A.
    n, k, m = 120, 6, 5
    A, _ = _spd(n, seed=25, hi=200.0)
    A_loop = _perturbed(A, 1e-6, seed=26)
    rng = np.random.default_rng(27)
    b, W = rng.standard_normal(n), rng.standard_normal((n, k))
    tol = 1e-11
    res = O.defcg(A_loop, b, W=W, tol=tol, refine_every=m, keep_iterates=True, A_true=A)
    assert res.status == O.STATUS_OK
    assert O.true_relres(A, b, res.x) <= tol
    assert res.relres_true == O.true_relres(A, b, res.x)
    Wk, AWk = res.W, res.AW
    np.testing.assert_allclose(AWk, A_loop @ Wk, rtol=0, atol=1e-12 * np.linalg.norm(AWk))
    bn = np.linalg.norm(b)
    replaced_steps = [j for j in range(1, len(res.r_history)) if j % m == 0]
    assert len(replaced_steps) >= 3
    drift = 0.0
    for j in replaced_steps:
        r, p, x = res.r_history[j], res.p_history[j], res.x_history[j]
        assert np.linalg.norm(Wk.T @ r) <= 1e-12 * np.linalg.norm(Wk) * np.linalg.norm(r), j
        assert np.linalg.norm(AWk.T @ p) <= 1e-12 * np.linalg.norm(AWk) * np.linalg.norm(p), j
        # the replaced residual is the true one up to the re-deflation's
        # (A - A_loop) W g (|r - (b - A x)| <= 1.4e-11 |b| measured) and differs
        # from the recursion's (otherwise this test could not tell the choices
        # of beta apart)
        assert np.linalg.norm(r - (b - A @ x)) <= 1e-10 * bn, j
        drift = max(drift, abs(np.linalg.norm(r) - res.history[j] * bn) / np.linalg.norm(r))
    assert drift > 1e-9
    # beta_j = (recursion's |r_{j+1}|^2) / rho_j with rho_j = |r_j|^2 of the
    # residual the loop carries (the replaced one after a replacement), at
    # every step
    assert len(res.beta) == len(res.r_history) - 1
    for j in range(len(res.beta)):
        r = res.r_history[j]
        beta_expected = (res.history[j + 1] * bn) ** 2 / (r @ r)
        assert abs(res.beta[j] - beta_expected) <= 1e-12 * beta_expected, j


def test_refinement_reaches_the_certified_operator_solution():
    # With the approximate loop operator and no replacement other than the
    # final confirmation (R2), x still solves A x = b to tol: each failed
    # confirmation replaces r by b - A x and the recursion continues.
    n, k = 100, 4
    A, _ = _spd(n, seed=28, hi=300.0)
    A_loop = _perturbed(A, 1e-5, seed=29)
    rng = np.random.default_rng(30)
    b, W = rng.standard_normal(n), rng.standard_normal((n, k))
    for m in (0, 7):
        res = O.defcg(A_loop, b, W=W, tol=1e-11, refine_every=m, A_true=A)
        x_ref = sla.cho_solve(sla.cho_factor(A), b)
        assert O.true_relres(A, b, res.x) <= 1e-11
        assert np.linalg.norm(res.x - x_ref) <= 300.0 * 1e-11 * np.linalg.norm(x_ref)
        assert res.matvecs_check >= 2     # at least one failed confirmation
