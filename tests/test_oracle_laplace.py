"""Pins for the Laplace-approximation Newton loop of the Sec. 3 experiment
(oracle/laplace_oracle.py): closed forms against finite differences, the
restructured step against the plain Newton step, the mode's fixed-point
equation, the spectrum bound of the system, optimality against a generic
optimiser, and def-CG recycling along the Newton sequence."""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as sopt

import dcg_synth as S
from oracle import dcg_oracle as O
from oracle import laplace_oracle as L


def _problem(n=120, d=6, l=1.0, s2=9.0, seed=0):
    X, y = S.classification_data(n, d, seed=seed)
    return O.rbf_gram(X, l, s2, 0.0), y


def test_likelihood_derivatives_match_finite_differences():
    rng = np.random.default_rng(1)
    y = np.where(rng.random(7) < 0.5, -1.0, 1.0)
    f = 3.0 * rng.standard_normal(7)
    h = 1e-6
    for i in range(7):
        e = np.zeros(7)
        e[i] = h
        g_fd = (L.log_lik(y, f + e) - L.log_lik(y, f - e)) / (2 * h)
        assert abs(g_fd - L.grad_log_lik(y, f)[i]) <= 1e-8
        hess_fd = (L.grad_log_lik(y, f + e)[i] - L.grad_log_lik(y, f - e)[i]) / (2 * h)
        assert abs(-hess_fd - L.neg_hess_log_lik(f)[i]) <= 1e-8
    # large |f| stays finite and tends to the right limits
    assert L.log_lik([1.0], [-800.0]) == pytest.approx(-800.0)
    assert L.neg_hess_log_lik(np.array([60.0, -60.0])).max() < 1e-25


def test_restructured_step_equals_the_plain_newton_step():
    # Sec. 3 step (through A = I + H^1/2 K H^1/2) against the textbook form
    # f_new = (K^{-1} + H)^{-1} (H f + grad log p) with dense inverses
    K, y = _problem()
    f = np.random.default_rng(2).standard_normal(K.shape[0])
    A, b, c, s = L.newton_system(K, y, f)
    x = np.linalg.solve(A, b)
    f_new, a = L.newton_update(K, c, s, x)
    Kj = K + 1e-12 * np.eye(K.shape[0])
    h = L.neg_hess_log_lik(f)
    plain = np.linalg.solve(np.linalg.inv(Kj) + np.diag(h), h * f + L.grad_log_lik(y, f))
    assert np.linalg.norm(f_new - plain) <= 1e-7 * np.linalg.norm(plain)
    np.testing.assert_allclose(K @ a, f_new, rtol=1e-12, atol=1e-12)


def test_system_spectrum_is_bounded():
    # A - I = H^1/2 K H^1/2 is PSD and H <= 1/4, so 1 <= lambda(A) <= 1 + lambda_max(K)/4
    # <= 1 + n max K_ij / 4
    K, y = _problem()
    f = 2.0 * np.random.default_rng(3).standard_normal(K.shape[0])
    A, _, _, _ = L.newton_system(K, y, f)
    lam = np.linalg.eigvalsh(A)
    assert lam[0] >= 1 - 1e-12
    assert lam[-1] <= 1 + np.linalg.eigvalsh(K)[-1] / 4 + 1e-9
    assert lam[-1] <= 1 + K.shape[0] * K.max() / 4


def test_mode_satisfies_the_fixed_point_and_maximises_psi():
    # at the mode, grad Psi = grad log p - K^{-1} f = 0, i.e. f = K grad log p(y | f)
    # (Rasmussen and Williams 2006, Eq. 3.17); Psi rises at every Newton step;
    # a generic optimiser on -Psi (Cholesky for K^{-1}) finds no higher value
    K, y = _problem(n=60)
    f, a, hist, _ = L.laplace_mode(K, y, dpsi_tol=1e-12)
    assert np.linalg.norm(f - K @ L.grad_log_lik(y, f)) <= 1e-10 * np.linalg.norm(f)
    assert all(h1 > h0 for h0, h1 in zip(hist, hist[1:-1]))
    cf = sla.cho_factor(K + 1e-10 * np.eye(K.shape[0]))

    def neg_psi(v):
        kinv_v = sla.cho_solve(cf, v)
        return -(L.log_lik(y, v) - 0.5 * v @ kinv_v), -(L.grad_log_lik(y, v) - kinv_v)

    opt = sopt.minimize(neg_psi, np.zeros_like(f), jac=True, method="L-BFGS-B",
                        options={"gtol": 1e-10, "ftol": 1e-15, "maxiter": 5000})
    assert hist[-1] >= -opt.fun - 1e-6


def test_defcg_recycling_along_the_newton_sequence():
    # def-CG(8, 12) (the paper's setting) recycling W from one Newton system to
    # the next reaches the mode of the exact-solve loop and needs fewer CG
    # iterations than plain CG on every recycled system (the Sec. 3 finding,
    # here on synthetic data)
    K, y = _problem(n=400, d=10)
    state = {"W": None}

    def defcg_solve(A, b, t, deflate=True):
        r = O.defcg(A, b, W=state["W"] if deflate else None, tol=1e-8, ell=12)
        if deflate:
            state["W"] = O.harmonic_ritz(r.W, r.AW, r.P, r.Q, 8).W
        assert r.status == O.STATUS_OK and r.relres_true <= 1e-8
        return r.x, r.iters

    f_ref, _, h_ref, _ = L.laplace_mode(K, y, dpsi_tol=1.0)
    f_d, _, h_d, it_d = L.laplace_mode(K, y, solve=defcg_solve, dpsi_tol=1.0)
    f_c, _, h_c, it_c = L.laplace_mode(K, y, solve=lambda A, b, t: defcg_solve(A, b, t, False), dpsi_tol=1.0)
    assert len(h_d) == len(h_ref) == len(h_c)
    # solves to 1e-8 with kappa(A) <= 1 + lambda_max(K)/4: the Newton iterates
    # stay within ~1e-6 of the exact-solve ones
    assert np.linalg.norm(f_d - f_ref) <= 1e-5 * np.linalg.norm(f_ref)
    assert np.linalg.norm(f_c - f_ref) <= 1e-5 * np.linalg.norm(f_ref)
    assert it_d[0] == it_c[0]
    assert all(d < c for d, c in zip(it_d[1:], it_c[1:])), (it_d, it_c)
