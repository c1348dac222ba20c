"""Plain FP64 reference for the hyperparameter gradient of a GP whose solves
run through def-CG (the differentiation form built on the paper's method).

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

The paper motivates sequences of systems by hyperparameter search (Sec. 1)
and uses the RBF kernel of Sec. 3; it does not differentiate. What is computed
here is the textbook Gaussian-process negative log marginal likelihood

    L(theta) = 1/2 y^T A^{-1} y + 1/2 log det A + n/2 log 2 pi,
    A = K + noise I,  K_ij = s2 exp(-D_ij / (2 l^2)),  D_ij = |x_i - x_j|^2,

and its gradient (Rasmussen & Williams 2006, Eq. 5.9)

    dL/dtheta = -1/2 alpha^T (dA/dtheta) alpha + 1/2 tr(A^{-1} dA/dtheta),
    alpha = A^{-1} y,

with dA/dl = K * D / l^3 (elementwise), dA/ds2 = K / s2, dA/dnoise = I. The
trace term is also given in its stochastic form (Hutchinson 1990):
tr(A^{-1} M) ~ mean_p (A^{-1} z_p)^T M z_p over Rademacher probes z_p.
Parameters are (lengthscale l, signal variance s2, noise variance noise);
gradients are with respect to these (log-space gradients are theta * grad).

Every dense factorisation is numpy/scipy FP64 (Cholesky, triangular solves).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .dcg_oracle import rbf_gram

F64 = np.float64
NAMES = ("lengthscale", "signal_var", "noise")


def sq_dist(X):
    """D_ij = sum_m (x_im - x_jm)^2 in the difference form, float64."""
    X = np.asarray(X, dtype=F64)
    diff = X[:, None, :] - X[None, :, :]
    return np.einsum("ijm,ijm->ij", diff, diff)


def dA_dtheta(X, lengthscale, signal_var):
    """The three derivative matrices (dA/dl, dA/ds2, dA/dnoise) as dense float64."""
    D = sq_dist(X)
    l = float(lengthscale)
    E = np.exp(-D / (2.0 * l * l))           # K / s2
    K = signal_var * E
    return K * D / l ** 3, E, np.eye(X.shape[0])


def dtheta_forms(X, lengthscale, signal_var, U, V):
    """Bilinear forms u_p^T (dA/dtheta) v_p for each column pair (u_p, v_p).

    Returns an array of shape (P, 3): columns are theta = l, s2, noise.
    """
    U = np.atleast_2d(np.asarray(U, dtype=F64).T).T
    V = np.atleast_2d(np.asarray(V, dtype=F64).T).T
    mats = dA_dtheta(X, lengthscale, signal_var)
    out = np.empty((U.shape[1], 3))
    for p in range(U.shape[1]):
        for t, M in enumerate(mats):
            out[p, t] = U[:, p] @ (M @ V[:, p])
    return out


def _chol(A):
    return sla.cho_factor(A, lower=True)


def gp_nll(X, y, lengthscale, signal_var, noise):
    """L(theta) by Cholesky: 1/2 y^T A^{-1} y + sum log diag(L) + n/2 log 2 pi."""
    A = rbf_gram(X, lengthscale, signal_var, noise)
    c = _chol(A)
    y = np.asarray(y, dtype=F64)
    alpha = sla.cho_solve(c, y)
    logdet = 2.0 * np.sum(np.log(np.diag(c[0])))
    return 0.5 * y @ alpha + 0.5 * logdet + 0.5 * y.size * np.log(2.0 * np.pi)


def gp_nll_grad(X, y, lengthscale, signal_var, noise):
    """Exact dL/d(l, s2, noise): -1/2 alpha^T M alpha + 1/2 tr(A^{-1} M)."""
    A = rbf_gram(X, lengthscale, signal_var, noise)
    c = _chol(A)
    y = np.asarray(y, dtype=F64)
    alpha = sla.cho_solve(c, y)
    Ainv = sla.cho_solve(c, np.eye(A.shape[0]))
    g = np.empty(3)
    for t, M in enumerate(dA_dtheta(X, lengthscale, signal_var)):
        g[t] = -0.5 * alpha @ (M @ alpha) + 0.5 * np.sum(Ainv * M)
    return g


def datafit_grad(X, y, lengthscale, signal_var, noise):
    """Gradient of the data-fit term 1/2 y^T A^{-1} y alone: -1/2 alpha^T M alpha."""
    A = rbf_gram(X, lengthscale, signal_var, noise)
    alpha = sla.cho_solve(_chol(A), np.asarray(y, dtype=F64))
    return np.array([-0.5 * alpha @ (M @ alpha) for M in dA_dtheta(X, lengthscale, signal_var)])


def hutchinson(Ainv_Z, M, Z):
    """mean_p (A^{-1} z_p)^T M z_p: the probe estimate of tr(A^{-1} M)."""
    Ainv_Z = np.asarray(Ainv_Z, dtype=F64)
    Z = np.asarray(Z, dtype=F64)
    return float(np.mean(np.einsum("ip,ip->p", Ainv_Z, M @ Z)))


def logdet_grad_probes(X, lengthscale, signal_var, noise, Z):
    """1/2 tr(A^{-1} dA/dtheta) by Hutchinson with the given probes (columns of Z),
    the probe solves A u_p = z_p done by Cholesky."""
    A = rbf_gram(X, lengthscale, signal_var, noise)
    U = sla.cho_solve(_chol(A), np.asarray(Z, dtype=F64))
    return np.array([0.5 * hutchinson(U, M, Z) for M in dA_dtheta(X, lengthscale, signal_var)])


def gp_nll_grad_probes(X, y, lengthscale, signal_var, noise, Z):
    """dL/dtheta with the trace term estimated from the fixed probes Z."""
    return (datafit_grad(X, y, lengthscale, signal_var, noise)
            + logdet_grad_probes(X, lengthscale, signal_var, noise, Z))


def adam_path(grad_fn, log_theta0, steps, lr=0.05, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015) on phi = log theta with dL/dphi = theta * dL/dtheta.

    grad_fn(step, theta) returns dL/dtheta at theta (3 values). Returns the list
    of log-parameters after each step (the first entry is log_theta0).
    """
    phi = np.asarray(log_theta0, dtype=F64).copy()
    m = np.zeros_like(phi)
    v = np.zeros_like(phi)
    path = [phi.copy()]
    for t in range(1, steps + 1):
        theta = np.exp(phi)
        g = theta * np.asarray(grad_fn(t - 1, theta), dtype=F64)
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        phi = phi - lr * mhat / (np.sqrt(vhat) + eps)
        path.append(phi.copy())
    return path
