"""Pins for the GP gradient oracle (oracle/gp_oracle.py), each independent of
the formula it checks: finite differences of the likelihood and of the
operator itself, a closed form in the limit of a vanishing lengthscale,
exactness of Rademacher probes on diagonal matrices, unbiasedness, and the
closed-form first steps of Adam."""

import numpy as np
import pytest

import dcg_synth as S
from oracle import dcg_oracle as O
from oracle import gp_oracle as G


def _data(n=40, d=3, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.random((n, d))
    y = np.sin(6 * X[:, 0]) + 0.1 * rng.standard_normal(n)
    return X, y


@pytest.mark.parametrize("theta", [(0.5, 1.0, 0.1), (0.9, 2.3, 0.03), (0.3, 0.7, 0.5)])
def test_nll_grad_matches_central_differences_in_log_space(theta):
    X, y = _data()
    g = G.gp_nll_grad(X, y, *theta)
    h = 1e-5
    for t in range(3):
        up = np.array(theta, dtype=float)
        dn = np.array(theta, dtype=float)
        up[t] *= np.exp(h)
        dn[t] *= np.exp(-h)
        fd = (G.gp_nll(X, y, *up) - G.gp_nll(X, y, *dn)) / (2 * h)     # dL/dlog(theta_t)
        assert abs(fd - theta[t] * g[t]) <= 1e-6 * max(1.0, abs(fd)), (t, fd, theta[t] * g[t])


def test_dtheta_forms_match_operator_differences():
    # u^T (A(theta + h) - A(theta - h)) v / 2h with A from the Sec. 3 kernel
    X, _ = _data(n=30, d=4, seed=2)
    rng = np.random.default_rng(5)
    U = rng.standard_normal((30, 3))
    V = rng.standard_normal((30, 3))
    l, s2, noise = 0.7, 1.3, 0.2
    forms = G.dtheta_forms(X, l, s2, U, V)
    h = 1e-6
    params = np.array([l, s2, noise])
    for t in range(3):
        up, dn = params.copy(), params.copy()
        up[t] += h
        dn[t] -= h
        dA = (O.rbf_gram(X, *up) - O.rbf_gram(X, *dn)) / (2 * h)
        for p in range(3):
            fd = U[:, p] @ dA @ V[:, p]
            assert abs(fd - forms[p, t]) <= 1e-7 * max(1.0, abs(fd)), (t, p, fd, forms[p, t])


def test_nll_grad_closed_form_for_vanishing_lengthscale():
    # Distinct points and l -> 0: K -> s2 I, so A = (s2 + noise) I and
    # L = |y|^2 / (2c) + n/2 log c + n/2 log 2pi with c = s2 + noise;
    # dL/ds2 = dL/dnoise = -|y|^2 / (2c^2) + n / (2c), dL/dl -> 0.
    X, y = _data(n=25, d=2, seed=3)
    l, s2, noise = 1e-4, 1.7, 0.3
    c = s2 + noise
    n = y.size
    L = y @ y / (2 * c) + 0.5 * n * np.log(c) + 0.5 * n * np.log(2 * np.pi)
    assert abs(G.gp_nll(X, y, l, s2, noise) - L) <= 1e-10 * abs(L)
    g = G.gp_nll_grad(X, y, l, s2, noise)
    ref = -(y @ y) / (2 * c * c) + n / (2 * c)
    assert abs(g[0]) <= 1e-12
    assert abs(g[1] - ref) <= 1e-10 * abs(ref)
    assert abs(g[2] - ref) <= 1e-10 * abs(ref)


def test_hutchinson_is_exact_for_diagonal_matrices():
    # z_i^2 = 1 for Rademacher entries, so sum_i (a_i^{-1} z_i) m_i z_i = tr exactly
    rng = np.random.default_rng(1)
    a = rng.random(50) + 0.5
    m = rng.standard_normal(50)
    Z = S.rademacher(50, 3, seed=11)
    est = G.hutchinson(Z / a[:, None], np.diag(m), Z)
    assert abs(est - np.sum(m / a)) <= 1e-12 * np.sum(np.abs(m / a))


def test_probe_gradient_is_unbiased():
    # Mean over many probes approaches the exact trace term within 5 standard errors.
    X, y = _data(n=24, d=2, seed=4)
    theta = (0.6, 1.1, 0.15)
    exact = G.gp_nll_grad(X, y, *theta) - G.datafit_grad(X, y, *theta)
    Z = S.rademacher(24, 20000, seed=7)
    A = O.rbf_gram(X, *theta)
    U = np.linalg.solve(A, Z)
    for t, M in enumerate(G.dA_dtheta(X, theta[0], theta[1])):
        samples = 0.5 * np.einsum("ip,ip->p", U, M @ Z)
        se = samples.std(ddof=1) / np.sqrt(samples.size)
        assert abs(samples.mean() - exact[t]) <= 5 * se + 1e-12, (t, samples.mean(), exact[t], se)
    # and the probe gradient with these probes is the data-fit part plus that mean
    gp = G.gp_nll_grad_probes(X, y, *theta, Z[:, :16])
    df = G.datafit_grad(X, y, *theta)
    for t, M in enumerate(G.dA_dtheta(X, theta[0], theta[1])):
        assert abs(gp[t] - df[t] - 0.5 * np.mean(np.einsum("ip,ip->p", U[:, :16], M @ Z[:, :16]))) <= 1e-10


def test_adam_closed_form_steps():
    # Constant gradient g: bias-corrected moments are exactly g and g^2, so
    # every step moves phi by -lr * g / (|g| + eps).
    g = np.array([0.3, -2.0, 1e-3])
    phi0 = np.log(np.array([0.5, 1.0, 0.1]))
    path = G.adam_path(lambda t, th: g / th, phi0, steps=4, lr=0.05)
    step = -0.05 * g / (np.abs(g) + 1e-8)
    for t in range(1, 5):
        assert np.allclose(path[t] - path[t - 1], step, rtol=1e-12, atol=1e-15)
