"""GPU parity of the differentiation form (hyperparameter gradient through
def-CG solves of the matrix-free RBF operator) against the FP64 oracle in
oracle/gp_oracle.py: the derivative-form kernel, the adjoint-solve gradient of
the data-fit term (also against central finite differences), the probe
gradient of the log-determinant with the same fixed probes, and Adam paths.

The operator is defined by X rounded to BF16; the oracle reads the same
rounded points. Solves run to the relative residual 1e-9 (exact-form
refinement), which bounds the solution error by ~3e-6 at kappa ~ 3e3; the
exact-form residual of this operator can certify down to ~1e-10, so 1e-9
keeps clear of that floor.
"""

import numpy as np
import pytest

import dcg_synth as S
from oracle import dcg_oracle as O
from oracle import gp_oracle as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA = (0.5, 1.0, 0.1)      # lengthscale, signal variance, noise of the gradient workload


@pytest.fixture(scope="module")
def dcg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_00241_gb300 import build
    build.build()
    import paper_1706_00241_gb300 as P
    return P


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


@pytest.mark.parametrize("n,d,P", [(1, 3, 1), (130, 8, 1), (1000, 8, 5), (2100, 20, 17), (777, 33, 40)])
def test_dtheta_forms_match_oracle(dcg, n, d, P):
    rng = np.random.default_rng(n + d + P)
    X = rng.random((n, d)).astype(np.float32)
    Xr = S.round_to_bf16(X).astype(np.float64)
    U = rng.standard_normal((P, n)).astype(np.float32)
    V = rng.standard_normal((P, n)).astype(np.float32)
    l, s2, noise = 0.4 + 0.05 * d ** 0.5, 1.3, 0.07
    with dcg.DefCG(n, 0, 0, 1e-6) as s:
        s.set_operator_rbf(dev(X), l, s2, noise, xformat="bf16")
        got = s.rbf_dtheta(dev(U), dev(V))
    ref = G.dtheta_forms(Xr, l, s2, U.T.astype(np.float64), V.T.astype(np.float64))
    # scale: |u|^T |M| |v| per pair and parameter; float32 entries (ex2.approx,
    # float32 distances) and float32 sums over 64-point tiles
    mats = G.dA_dtheta(Xr, l, s2)
    Ua, Va = np.abs(U.astype(np.float64)), np.abs(V.astype(np.float64))
    for t, M in enumerate(mats):
        scale = np.einsum("pi,pi->p", Ua, (np.abs(M) @ Va.T).T)
        assert np.all(np.abs(got[:, t] - ref[:, t]) <= 2e-5 * scale + 1e-12), (t, got[:, t], ref[:, t])


def _grad_problem(n):
    cfg = S.GRAD_32768.scaled(n, T=1)
    X, _ = S.draw_sequence(cfg)
    y = S.gp_targets(X).astype(np.float32)
    Xr = S.round_to_bf16(X.astype(np.float32)).astype(np.float64)
    return cfg, X.astype(np.float32), Xr, y


def _solver(dcg, cfg, X, n):
    s = dcg.DefCG(n, cfg.k, cfg.ell, 1e-9, refine_every=50, max_iter=6000)
    s.set_operator_rbf(dev(X), *THETA, xformat="bf16")
    return s


def test_gradient_matches_cholesky_and_finite_differences(dcg):
    n = 2048
    cfg, X, Xr, y = _grad_problem(n)
    y64 = y.astype(np.float64)
    yd = dev(y)
    Zn = S.rademacher(n, 16, seed=1000)                   # (n, 16)
    Zd = dev(Zn.T)
    with _solver(dcg, cfg, X, n) as s:
        # data-fit term through the adjoint solve
        th = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
        fit = dcg.gp_objective(th, yd, s)
        fit.backward()
        g_fit = th.grad.numpy().copy()
        assert s.last_forward_info["status"] == 0 and s.last_adjoint_info["status"] == 0
        A = O.rbf_gram(Xr, *THETA)
        alpha = np.linalg.solve(A, y64)
        assert abs(fit.item() - 0.5 * y64 @ alpha) <= 1e-8 * abs(0.5 * y64 @ alpha)
        ref_fit = G.datafit_grad(Xr, y64, *THETA)
        assert np.all(np.abs(g_fit - ref_fit) <= 1e-4 * np.abs(ref_fit)), (g_fit, ref_fit)
        # central differences of the data-fit value in log space
        h = 1e-5
        for t in range(3):
            up, dn = np.array(THETA), np.array(THETA)
            up[t] *= np.exp(h)
            dn[t] *= np.exp(-h)
            fu = 0.5 * y64 @ np.linalg.solve(O.rbf_gram(Xr, *up), y64)
            fd_ = 0.5 * y64 @ np.linalg.solve(O.rbf_gram(Xr, *dn), y64)
            fd = (fu - fd_) / (2 * h)
            assert abs(fd - THETA[t] * g_fit[t]) <= 1e-4 * abs(fd), (t, fd, THETA[t] * g_fit[t])
        # full objective: data fit + probe estimate of the log-determinant term
        th2 = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
        obj = dcg.gp_objective(th2, yd, s, Zd)
        obj.backward()
        g_all = th2.grad.numpy().copy()
        assert all(i["status"] == 0 for i in s.last_probe_infos)
    ref_all = G.gp_nll_grad_probes(Xr, y64, *THETA, Zn)
    ref_ld = G.logdet_grad_probes(Xr, *THETA, Zn)
    assert np.all(np.abs((g_all - g_fit) - ref_ld) <= 1e-4 * np.abs(ref_ld)), (g_all - g_fit, ref_ld)
    assert np.all(np.abs(g_all - ref_all) <= 1e-4 * np.abs(ref_all)), (g_all, ref_all)


def test_adam_path_matches_oracle(dcg):
    n, steps, P = 1024, 3, 4
    cfg, X, Xr, y = _grad_problem(n)
    y64 = y.astype(np.float64)
    probes = [S.rademacher(n, P, seed=1000 + t) for t in range(steps)]
    with _solver(dcg, cfg, X, n) as s:
        path, grads = dcg.fit_gp(s, dev(y), THETA, steps=steps, lr=0.05, probes=lambda t: dev(probes[t].T))
    ref = G.adam_path(lambda t, th: G.gp_nll_grad_probes(Xr, y64, *th, probes[t]), np.log(THETA), steps, lr=0.05)
    for t in range(steps + 1):
        assert np.allclose(np.log(path[t]), ref[t], rtol=0, atol=1e-6), (t, np.log(path[t]), ref[t])


def test_lockstep_probes_match_one_by_one(dcg):
    # The probe solves of the log-determinant term in lockstep (one operator
    # pass per iteration for all of them) and one after another are the same
    # solves up to the rounding of the block product: the probe gradients
    # agree to the solves' accuracy (tol 1e-9, kappa ~ 3e3: ~3e-6 relative
    # in each u_p, averaged over the probes).
    n, P = 1500, 12
    cfg, X, Xr, y = _grad_problem(n)
    Zd = dev(S.rademacher(n, P, seed=7).T)
    grads = []
    for block in (True, False):
        with _solver(dcg, cfg, X, n) as s:
            th = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
            dcg.gp_objective(th, dev(y), s, Zd, block_probes=block).backward()
            assert len(s.last_probe_infos) == P and all(i["status"] == 0 for i in s.last_probe_infos)
            grads.append(th.grad.numpy().copy())
    assert np.all(np.abs(grads[0] - grads[1]) <= 1e-5 * np.abs(grads[1])), grads
