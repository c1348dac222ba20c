"""Plain FP64 reference for the paper's own experiment (Sec. 3): the Newton
loop of the Laplace approximation for binary GP classification, whose linear
systems (the system pair of Sec. 3) form the sequence def-CG recycles across.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Model (Sec. 3): latent f ~ GP(0, K) with the RBF kernel, logistic likelihood
p(y_i | f_i) = sigma(y_i f_i), labels y_i in {-1, +1}. Newton maximises
Psi(f) = log p(y | f) - 1/2 f^T K^{-1} f (the terms of Sec. 3's objective that
depend on f). With H = -grad grad log p(y | f) = diag(pi (1 - pi)),
pi = sigma(f), one step (the restructured form of Sec. 3, Rasmussen and
Williams 2006, Algorithm 3.1) is

    c = H f + grad log p(y | f)
    A = I + H^{1/2} K H^{1/2},   b = H^{1/2} K c      (the system of Sec. 3)
    x = A^{-1} b
    a = c - H^{1/2} x,           f_new = K a,   Psi(f_new) = log p(y | f_new) - 1/2 f_new^T a.

The loop stops when Psi rises by less than ``dpsi_tol`` (Sec. 3 uses 1).
The eigenvalues of A lie in [1, 1 + lambda_max(K) / 4]; the paper states the
bound as [1, n max K / 4] (reading: lambda_max(K) <= n max K_ij, and the
leading 1 belongs to the upper end too).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

F64 = np.float64


def log_lik(y, f):
    """log p(y | f) = sum_i log sigma(y_i f_i), evaluated as -log(1 + exp(-y f))."""
    return float(-np.sum(np.logaddexp(0.0, -np.asarray(y, F64) * np.asarray(f, F64))))


def grad_log_lik(y, f):
    """d/df log p(y | f) = t - pi with t = (y + 1) / 2, pi = sigma(f)."""
    pi = 0.5 * (1.0 + np.tanh(0.5 * np.asarray(f, F64)))
    return 0.5 * (np.asarray(y, F64) + 1.0) - pi


def neg_hess_log_lik(f):
    """Diagonal of H = -grad grad log p(y | f) = pi (1 - pi)."""
    pi = 0.5 * (1.0 + np.tanh(0.5 * np.asarray(f, F64)))
    return pi * (1.0 - pi)


def newton_system(K, y, f):
    """The Sec. 3 system of one Newton step at f: returns A, b and the
    quantities the update needs (c, the square root of H)."""
    K = np.asarray(K, F64)
    h = neg_hess_log_lik(f)
    s = np.sqrt(h)
    c = h * f + grad_log_lik(y, f)
    A = np.eye(K.shape[0]) + s[:, None] * K * s[None, :]
    b = s * (K @ c)
    return A, b, c, s


def newton_update(K, c, s, x):
    """a = c - H^{1/2} x, f = K a: the new iterate from the system's solution."""
    a = c - s * x
    return np.asarray(K, F64) @ a, a


def psi(y, f, a):
    """log p(y | f) - 1/2 f^T K^{-1} f with K^{-1} f = a (f = K a)."""
    return log_lik(y, f) - 0.5 * float(np.asarray(f, F64) @ np.asarray(a, F64))


def cholesky_solver(A, b, t):
    """Exact solve of the Newton system (the Cholesky column of the Sec. 3 table)."""
    return sla.cho_solve(sla.cho_factor(A), b), None


def laplace_mode(K, y, solve=cholesky_solver, dpsi_tol=1.0, max_newton=50):
    """Newton's method for the mode of the Laplace approximation (Sec. 3).

    ``solve(A, b, t) -> (x, info)`` solves the t-th Newton system; a def-CG
    solver that recycles W from one call to the next is the method under
    study. Starts from f = 0 and stops when Psi rises by less than
    ``dpsi_tol``. Returns f, a, the Psi history and the per-step infos.
    """
    K = np.asarray(K, F64)
    n = K.shape[0]
    f = np.zeros(n)
    a = np.zeros(n)
    hist = [psi(y, f, a)]
    infos = []
    for t in range(max_newton):
        A, b, c, s = newton_system(K, y, f)
        x, info = solve(A, b, t)
        f, a = newton_update(K, c, s, x)
        hist.append(psi(y, f, a))
        infos.append(info)
        if hist[-1] - hist[-2] < dpsi_tol:
            break
    return f, a, hist, infos
