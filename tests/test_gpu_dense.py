"""GPU parity of the stored-operator path against the FP64 oracle.

Every test calls the CUDA path through the C ABI (paper_1706_00241_gb300 is a
ctypes binding) and compares with ``oracle/`` on the same seeded inputs from
``dcg_synth``. Tolerances are stated per test with the arithmetic behind them.
"""

import json
import os

import numpy as np
import pytest

import dcg_synth as S
from oracle import dcg_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


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


def padded(A32, lda):
    n = A32.shape[0]
    out = np.zeros((n, lda), dtype=np.float32)
    out[:, :n] = A32
    return out


def rbf_problem(n, d, l, noise, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    return X


# ---------------------------------------------------------------------------
# A1: forming the RBF operator
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,d", [(1, 3), (67, 5), (1000, 8), (1030, 16)])
def test_form_rbf_matches_oracle(dcg, n, d):
    X = rbf_problem(n, d, 1.0, 1e-2)
    l, s2, noise = 1.3, 0.9, 1e-2
    lda = (n + 3) // 4 * 4
    A = torch.zeros((n, lda), dtype=torch.float32, device="cuda")
    dcg.form_rbf_dense(dev(X), l, s2, noise, out=A)
    torch.cuda.synchronize()
    got = A.cpu().numpy()[:, :n].astype(np.float64)
    ref = O.rbf_gram(X.astype(np.float64), l, s2, noise)
    # float32 distances (d terms) and expf: a few ulp of the entry plus the
    # float32 rounding of |x_i - x_j|^2 amplified by |dK/d(sq)| = K / (2 l^2)
    sq_scale = 4.0 * np.max(np.sum(X.astype(np.float64) ** 2, axis=1))
    tol = 1e-6 * np.abs(ref) + 4e-7 * sq_scale / (2 * l * l) * np.abs(ref) + 1e-7
    assert np.all(np.abs(got - ref) <= tol)


# ---------------------------------------------------------------------------
# A5: the matvec q = A p with the fused p^T A p
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 5, 257, 1001, 2049, 4099, 9000])
def test_matvec_matches_oracle(dcg, n):
    rng = np.random.default_rng(n)
    lda = (n + 3) // 4 * 4
    A32 = rng.standard_normal((n, n)).astype(np.float32)
    A32 = (A32 + A32.T) * 0.5
    p = rng.standard_normal(n).astype(np.float32)
    Ad = dev(padded(A32, lda))
    with dcg.DefCG(n, 0, 0, 1e-6) as s:
        s.set_operator_dense(Ad, lda)
        q, pAp = s.matvec(dev(p))
        q = q.cpu().numpy().astype(np.float64)
    A64, p64 = A32.astype(np.float64), p.astype(np.float64)
    ref = A64 @ p64
    # float32 products summed in float32 over <= n/512 + 8 terms per thread,
    # then a 256-way tree: error <= (n/512 + 16) * eps32 * sum_j |a_ij p_j|
    bound = (n / 512 + 16) * 6e-8 * (np.abs(A64) @ np.abs(p64))
    assert np.all(np.abs(q - ref) <= bound + 1e-30)
    # p^T q is summed in float64 from the float32 q the kernel stored
    assert abs(pAp - p64 @ q) <= 1e-12 * (np.abs(p64) @ np.abs(q))


def test_matvec_full_size_sampled_rows(dcg):
    # The stored workload at n = 16384 in the bench launch configuration; rows sampled so the
    # float64 reference is cheap.
    cfg = S.DENSE_16384
    X, bs = S.draw_sequence(cfg, T=1)
    X32 = X.astype(np.float32)
    n = cfg.n
    A = dcg.form_rbf_dense(dev(X32), cfg.lengthscale(19), 1.0, cfg.noise)
    p = bs[0].astype(np.float32)
    with dcg.DefCG(n, cfg.k, cfg.ell, cfg.tol) as s:
        s.set_operator_dense(A)
        q, pAp = s.matvec(dev(p))
    rows = np.random.default_rng(1).choice(n, 96, replace=False)
    Arows = A[torch.tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    ref = Arows @ p.astype(np.float64)
    got = q.cpu().numpy()[rows].astype(np.float64)
    bound = (n / 512 + 16) * 6e-8 * (np.abs(Arows) @ np.abs(p.astype(np.float64)))
    assert np.all(np.abs(got - ref) <= bound)
    qq = q.cpu().numpy().astype(np.float64)
    assert abs(pAp - p.astype(np.float64) @ qq) <= 1e-12 * (np.abs(p) @ np.abs(qq))


@pytest.mark.parametrize("n", [1, 5, 63, 64, 65, 256, 257, 511, 513, 1000, 2047, 2049, 4100, 9000])
def test_symmetric_matvec_matches_oracle(dcg, n):
    # dcg_set_operator_dense_sym: only the upper triangle is read. The strictly
    # lower triangle and the padding columns hold NaN, so any read of them
    # would show in q (sizes around the 256-row bands and 512-column chunks of
    # the work items). All sums are float32: a row's part of a stage over 2
    # products per lane, a 32-lane tree and 8 warps; the transposed
    # contributions over the <= 256 rows of a band in four interleaved chains;
    # then <= n / 256 + n / 512 + 1 partials. The worst case is about
    # 130 eps32 sum_j |a_ij p_j|; with random signs the errors grow like the
    # square root of the terms, and the test takes 100 eps32.
    rng = np.random.default_rng(10 + n)
    lda = (n + 3) // 4 * 4 + 4
    A32 = rng.standard_normal((n, n)).astype(np.float32)
    A32 = (A32 + A32.T) * np.float32(0.5)
    assert np.array_equal(A32, A32.T)
    p = rng.standard_normal(n).astype(np.float32)
    stored = np.full((n, lda), np.nan, dtype=np.float32)
    stored[:, :n] = np.triu(A32) + np.tril(np.full((n, n), np.nan, dtype=np.float32), -1)
    with dcg.DefCG(n, 0, 0, 1e-6) as s:
        s.set_operator_dense(dev(stored), lda, symmetric=True)
        for _ in range(2):   # the partial-sum buffers are reused
            q, pAp = s.matvec(dev(p))
            qh = q.cpu().numpy().astype(np.float64)
            A64, p64 = A32.astype(np.float64), p.astype(np.float64)
            ref = A64 @ p64
            bound = 100 * 6e-8 * (np.abs(A64) @ np.abs(p64))
            assert np.all(np.isfinite(qh))
            assert np.all(np.abs(qh - ref) <= bound + 1e-30), np.max(np.abs(qh - ref) / (bound + 1e-30))
            assert abs(pAp - p64 @ qh) <= 1e-12 * (np.abs(p64) @ np.abs(qh))


def test_symmetric_operator_solves_like_the_full_one(dcg):
    # The n = 16384 stored workload at its last lengthscale, plain CG and
    # def-CG with a recycled subspace, once with the full-matrix matvec and
    # once with the upper-triangle one: both certify tol (the true residual
    # reads the full matrix) and take the same number of iterations within
    # what the float32 recursion makes of the two summation orders (measured:
    # 210 and 200 at kappa ~1e6): 10 % + 2.
    cfg = S.DENSE_16384
    X, bs = S.draw_sequence(cfg, T=2)
    X32 = X.astype(np.float32)
    A = dcg.form_rbf_dense(dev(X32), cfg.lengthscale(19), 1.0, cfg.noise)
    res = {}
    for sym in (False, True):
        with dcg.DefCG(cfg.n, cfg.k, cfg.ell, cfg.tol) as s:
            s.set_operator_dense(A, symmetric=sym)
            _, i0 = s.solve(dev(bs[0]))
            s.update_subspace()
            x, i1 = s.solve(dev(bs[1]))
            res[sym] = (i0, i1)
            assert i0["status"] == 0 and i1["status"] == 0
            assert i0["relres_true"] <= cfg.tol and i1["relres_true"] <= cfg.tol
    for a, b in zip(res[False], res[True]):
        assert abs(a["iters"] - b["iters"]) <= 2 + 0.1 * a["iters"], (a["iters"], b["iters"])


def test_symmetric_matvec_full_size_sampled_rows(dcg):
    cfg = S.DENSE_16384
    X, bs = S.draw_sequence(cfg, T=1)
    n = cfg.n
    A = dcg.form_rbf_dense(dev(X.astype(np.float32)), cfg.lengthscale(19), 1.0, cfg.noise)
    p = bs[0].astype(np.float32)
    with dcg.DefCG(n, cfg.k, cfg.ell, cfg.tol) as s:
        s.set_operator_dense(A, symmetric=True)
        q, pAp = s.matvec(dev(p))
    rows = np.random.default_rng(2).choice(n, 96, replace=False)
    Arows = A[torch.tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    ref = Arows @ p.astype(np.float64)
    got = q.cpu().numpy()[rows].astype(np.float64)
    bound = 100 * 6e-8 * (np.abs(Arows) @ np.abs(p.astype(np.float64)))
    assert np.all(np.abs(got - ref) <= bound)


# ---------------------------------------------------------------------------
# A2: multi-vector product Y = A V
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,c", [(5, 1), (1001, 7), (2048, 33), (3001, 65), (700, 129), (1024, 32), (4100, 96),
                                 (2000, 1), (516, 129), (16384, 32), (3001, 8), (1999, 16), (2047, 12), (4097, 9),
                                 (36551, 8)])
def test_apply_block_matches_oracle(dcg, n, c):
    # n % 4 == 0 with more than 16 columns runs on the tensor cores (split
    # TF32, one TMEM accumulator per 32-wide K stage added into float32
    # registers: per product ~3 2^-22 from the split, accumulation within a
    # stage, then float32 sums of n / 32 stage results), otherwise on the FP32
    # pipe (float32 chains, 8-, 16- or 32-column blocks); both within
    # (n / 32 + 32) eps32 sum |v_j a_ij|.
    rng = np.random.default_rng(c)
    lda = (n + 3) // 4 * 4
    A32 = rng.standard_normal((n, n)).astype(np.float32)
    V = rng.standard_normal((c, n)).astype(np.float32)    # row j = column j of V
    with dcg.DefCG(n, 0, 0, 1e-6) as s:
        s.set_operator_dense(dev(padded(A32, lda)), lda)
        Y = s.apply_block(dev(V)).cpu().numpy().astype(np.float64)
    ref = V.astype(np.float64) @ A32.astype(np.float64).T
    bound = (n / 32 + 32) * 6e-8 * (np.abs(V.astype(np.float64)) @ np.abs(A32.astype(np.float64)).T)
    assert np.all(np.abs(Y - ref) <= bound)


# ---------------------------------------------------------------------------
# A3-A8: solves
# ---------------------------------------------------------------------------
def _spd32(n, eigs_lo, eigs_hi, seed):
    eigs = np.geomspace(eigs_lo, eigs_hi, n)
    A, Q = S.spd_with_spectrum(eigs, seed=seed)
    return A.astype(np.float32), Q, eigs


@pytest.mark.parametrize("n,k", [(1001, 0), (1001, 8), (2050, 16)])
def test_solve_well_conditioned_matches_oracle(dcg, n, k):
    # kappa = 10: |x - x*| / |x*| <= kappa * relres, so relres <= 1e-6 on both
    # sides bounds the solution difference by ~2e-5; tol = 1e-7 gives margin
    # for the 1e-5 solution-error target.
    A32, _, _ = _spd32(n, 1.0, 10.0, seed=n + k)
    A64 = A32.astype(np.float64)
    rng = np.random.default_rng(k)
    b = rng.standard_normal(n).astype(np.float32)
    W = rng.standard_normal((k, n)).astype(np.float32)
    lda = (n + 3) // 4 * 4
    tol = 1e-6
    with dcg.DefCG(n, max(k, 1), 16, tol, record_history=True) as s:
        s.set_operator_dense(dev(padded(A32, lda)), lda)
        if k:
            s.set_subspace(dev(W))
        x, info = s.solve(dev(b))
        hist = s.history()
    x = x.cpu().numpy().astype(np.float64)
    ref = O.defcg(A64, b.astype(np.float64), W=W.T.astype(np.float64) if k else None, tol=tol)
    assert info["status"] == 0
    relres = np.linalg.norm(b - A64 @ x) / np.linalg.norm(b)
    assert relres <= tol * 1.001
    assert abs(info["relres_true"] - relres) <= 1e-3 * relres + 1e-12
    assert abs(info["iters"] - ref.iters) <= 2
    assert np.linalg.norm(x - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    assert info["matvecs_setup"] == k
    # the recursive residual history follows the oracle's while rounding is small
    m = min(len(hist), len(ref.history), 8)
    np.testing.assert_allclose(hist[:m], ref.history[:m], rtol=1e-4)


def test_exact_eigenvectors_deflate(dcg):
    # W = exact eigenvectors of the 8 largest eigenvalues: the iteration count is
    # that of CG on the remaining spectrum (pinned in the oracle), within 2.
    n = 1500
    eigs = np.concatenate([np.linspace(1.0, 5.0, n - 8), np.geomspace(100.0, 1000.0, 8)])
    A, Q = S.spd_with_spectrum(eigs, seed=4)
    A32 = A.astype(np.float32)
    b = np.random.default_rng(3).standard_normal(n).astype(np.float32)
    W = Q[:, -8:].T.astype(np.float32)
    with dcg.DefCG(n, 8, 0, 1e-6) as s:
        s.set_operator_dense(dev(A32))
        s.set_subspace(dev(W))
        x, info = s.solve(dev(b))
    ref = O.defcg(A32.astype(np.float64), b.astype(np.float64), W=W.T.astype(np.float64), tol=1e-6)
    plain = O.cg(A32.astype(np.float64), b.astype(np.float64), tol=1e-6)
    assert abs(info["iters"] - ref.iters) <= 2
    assert info["iters"] < plain.iters


def test_zero_rhs(dcg):
    n = 300
    A32, _, _ = _spd32(n, 1, 10, 1)
    with dcg.DefCG(n, 4, 8, 1e-6, warm_start=True) as s:
        s.set_operator_dense(dev(A32))
        x0 = torch.ones(n, device="cuda", dtype=torch.float64)
        x, info = s.solve(torch.zeros(n, device="cuda"), x0)
    assert info["status"] == 0 and info["iters"] == 0
    assert torch.count_nonzero(x).item() == 0


def test_breakdown_on_indefinite(dcg):
    n = 64
    eigs = np.concatenate([[-1.0], np.linspace(1, 3, n - 1)])
    A, Q = S.spd_with_spectrum(eigs, seed=2)
    with dcg.DefCG(n, 0, 0, 1e-8) as s:
        s.set_operator_dense(dev(A.astype(np.float32)))
        x, info = s.solve(dev(Q[:, 0]), raise_on_error=False)
    assert info["status"] == 4


def test_maxiter_reports_true_residual(dcg):
    n = 800
    A32, _, _ = _spd32(n, 1e-3, 10, 5)
    b = np.random.default_rng(0).standard_normal(n).astype(np.float32)
    with dcg.DefCG(n, 0, 0, 1e-10, max_iter=5) as s:
        s.set_operator_dense(dev(A32))
        x, info = s.solve(dev(b), raise_on_error=False)
    assert info["status"] == 6 and info["iters"] == 5
    x = x.cpu().numpy().astype(np.float64)
    rr = np.linalg.norm(b - A32.astype(np.float64) @ x) / np.linalg.norm(b)
    assert abs(info["relres_true"] - rr) <= 1e-4 * rr


def test_warm_start_matches_oracle(dcg):
    n = 1200
    A32, _, _ = _spd32(n, 1, 10, 9)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(n).astype(np.float32)
    x0 = rng.standard_normal(n).astype(np.float32)
    W = rng.standard_normal((4, n)).astype(np.float32)
    with dcg.DefCG(n, 4, 0, 1e-6, warm_start=True) as s:
        s.set_operator_dense(dev(A32))
        s.set_subspace(dev(W))
        x, info = s.solve(dev(b), torch.tensor(x0.astype(np.float64), device="cuda"))
    ref = O.defcg(A32.astype(np.float64), b.astype(np.float64), x_init=x0.astype(np.float64),
                  W=W.T.astype(np.float64), tol=1e-6)
    assert info["matvecs_setup"] == 5
    assert abs(info["iters"] - ref.iters) <= 2
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)


def test_refinement_every_m(dcg):
    n = 1000
    A32, _, _ = _spd32(n, 1e-2, 10, 11)
    b = np.random.default_rng(2).standard_normal(n).astype(np.float32)
    rng = np.random.default_rng(5)
    W = rng.standard_normal((6, n)).astype(np.float32)
    with dcg.DefCG(n, 6, 0, 1e-6, refine_every=10) as s:
        s.set_operator_dense(dev(A32))
        s.set_subspace(dev(W))
        x, info = s.solve(dev(b))
    ref = O.defcg(A32.astype(np.float64), b.astype(np.float64), W=W.T.astype(np.float64), tol=1e-6,
                  refine_every=10)
    assert info["status"] == 0
    assert info["matvecs_check"] >= info["iters"] // 10
    # kappa = 1e3: float32 CG runs a few steps longer than float64 (5 % + 2)
    assert abs(info["iters"] - ref.iters) <= 2 + 0.05 * ref.iters
    xx = x.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(b - A32.astype(np.float64) @ xx) / np.linalg.norm(b) <= 1e-6


# ---------------------------------------------------------------------------
# A9: harmonic Ritz extraction
# ---------------------------------------------------------------------------
def test_ritz_keeps_exact_invariant_subspace(dcg):
    # W spans the top-6 eigenvectors; the extraction from Z = [W, P] must return
    # those eigenvalues as the largest harmonic Ritz values (Eq. 7 is exact on
    # an invariant subspace) and the same span.
    n = 1024
    eigs = np.concatenate([np.linspace(1.0, 4.0, n - 6), np.geomspace(50.0, 500.0, 6)])
    A, Q = S.spd_with_spectrum(eigs, seed=8)
    A32 = A.astype(np.float32)
    b = np.random.default_rng(1).standard_normal(n).astype(np.float32)
    R = np.random.default_rng(2).standard_normal((6, 6))
    W = (Q[:, -6:] @ R).T.astype(np.float32)
    with dcg.DefCG(n, 6, 12, 1e-6) as s:
        s.set_operator_dense(dev(A32))
        s.set_subspace(dev(W))
        s.solve(dev(b))
        k_new = s.update_subspace()
        theta = s.ritz_values()
        Wn = s.get_subspace().cpu().numpy().astype(np.float64)
    assert k_new == 6
    np.testing.assert_allclose(theta[:6], np.sort(eigs[-6:])[::-1], rtol=2e-5)
    # span check: the principal angles between span(W_new) and span(Q_S)
    qn, _ = np.linalg.qr(Wn.T)
    s_vals = np.linalg.svd(Q[:, -6:].T @ qn, compute_uv=False)
    assert s_vals.min() > 1 - 1e-6
    np.testing.assert_allclose(np.linalg.norm(Wn, axis=1), 1.0, rtol=1e-5)
    piv = np.argmax(np.abs(Wn), axis=1)
    assert np.all(Wn[np.arange(6), piv] > 0)


def test_ritz_smallest_keeps_exact_invariant_subspace(dcg):
    # select="smallest" (Sec. 2.3): W spans the 6 smallest eigenvectors, well
    # separated from a bulk in [1, 4]. Eq. 7 is exact on an invariant subspace
    # and the directions of P are A-conjugate to it, so the 6 smallest harmonic
    # Ritz values are those eigenvalues and the new W spans the same space.
    n = 1024
    small = np.linspace(0.1, 0.35, 6)
    eigs = np.concatenate([small, np.linspace(1.0, 4.0, n - 6)])
    A, Q = S.spd_with_spectrum(eigs, seed=9)
    A32 = A.astype(np.float32)
    b = np.random.default_rng(3).standard_normal(n).astype(np.float32)
    R = np.random.default_rng(4).standard_normal((6, 6))
    W = (Q[:, :6] @ R).T.astype(np.float32)
    with dcg.DefCG(n, 6, 12, 1e-6, select="smallest") as s:
        s.set_operator_dense(dev(A32))
        s.set_subspace(dev(W))
        s.solve(dev(b))
        k_new = s.update_subspace()
        theta = s.ritz_values()
        Wn = s.get_subspace().cpu().numpy().astype(np.float64)
    assert k_new == 6
    # the values come back descending over all of Z; the selected ones are last
    np.testing.assert_allclose(np.sort(theta)[:6], small, rtol=1e-4)
    assert np.sort(theta)[6] > 0.9
    qn, _ = np.linalg.qr(Wn.T)
    s_vals = np.linalg.svd(Q[:, :6].T @ qn, compute_uv=False)
    assert s_vals.min() > 1 - 1e-6
    np.testing.assert_allclose(np.linalg.norm(Wn, axis=1), 1.0, rtol=1e-5)
    piv = np.argmax(np.abs(Wn), axis=1)
    assert np.all(Wn[np.arange(6), piv] > 0)


def test_ritz_first_window_matches_oracle(dcg):
    # First system (plain CG) with window FIRST: the first ell directions span
    # a Krylov space on which float32 and float64 agree closely.
    n = 2000
    A32, _, eigs = _spd32(n, 0.5, 200.0, 13)
    b = np.random.default_rng(4).standard_normal(n).astype(np.float32)
    with dcg.DefCG(n, 4, 10, 1e-6, window="first") as s:
        s.set_operator_dense(dev(A32))
        s.solve(dev(b))
        s.update_subspace()
        theta = s.ritz_values()
    ref = O.defcg(A32.astype(np.float64), b.astype(np.float64), tol=1e-6, ell=10, window="first")
    rr = O.harmonic_ritz(None, None, ref.P, ref.Q, 4)
    np.testing.assert_allclose(theta, rr.theta, rtol=1e-3)


def test_rayleigh_ritz_first_window_matches_oracle(dcg):
    # extraction="ritz" (the orthogonal projection of Sec. 2.3) on the first
    # ell CG directions: the same float32 Krylov space as the harmonic test
    # above, so the Ritz values agree with the oracle's to the same 1e-3.
    n = 2000
    A32, _, eigs = _spd32(n, 0.5, 200.0, 13)
    b = np.random.default_rng(4).standard_normal(n).astype(np.float32)
    with dcg.DefCG(n, 4, 10, 1e-6, window="first", extraction="ritz") as s:
        s.set_operator_dense(dev(A32))
        s.solve(dev(b))
        k_new = s.update_subspace()
        theta = s.ritz_values()
        Wn = s.get_subspace().cpu().numpy().astype(np.float64)
    ref = O.defcg(A32.astype(np.float64), b.astype(np.float64), tol=1e-6, ell=10, window="first")
    rr = O.rayleigh_ritz(None, None, ref.P, ref.Q, 4)
    assert k_new == 4
    np.testing.assert_allclose(theta, rr.theta, rtol=1e-3)
    # the Ritz vectors are unit and agree with the oracle's up to float32
    # rounding of the directions (largest values: well separated)
    np.testing.assert_allclose(np.linalg.norm(Wn, axis=1), 1.0, rtol=1e-5)
    for j in range(2):
        assert np.abs(Wn @ rr.W[:, j]).max() > 1 - 1e-3


def test_rayleigh_ritz_keeps_exact_invariant_subspace(dcg):
    # W spans the top-6 eigenvectors. W^T A P = 0 then forces W^T P = 0, so the
    # orthogonal projection is exact on span(W) and its 6 largest Ritz values
    # are those eigenvalues; the new W spans the same space.
    n = 1024
    eigs = np.concatenate([np.linspace(1.0, 4.0, n - 6), np.geomspace(50.0, 500.0, 6)])
    A, Q = S.spd_with_spectrum(eigs, seed=8)
    A32 = A.astype(np.float32)
    b = np.random.default_rng(1).standard_normal(n).astype(np.float32)
    R = np.random.default_rng(2).standard_normal((6, 6))
    W = (Q[:, -6:] @ R).T.astype(np.float32)
    with dcg.DefCG(n, 6, 12, 1e-6, extraction="ritz") as s:
        s.set_operator_dense(dev(A32))
        s.set_subspace(dev(W))
        s.solve(dev(b))
        k_new = s.update_subspace()
        theta = s.ritz_values()
        Wn = s.get_subspace().cpu().numpy().astype(np.float64)
    assert k_new == 6
    np.testing.assert_allclose(theta[:6], np.sort(eigs[-6:])[::-1], rtol=2e-5)
    assert theta[6] < 4.0 * (1 + 1e-4)
    qn, _ = np.linalg.qr(Wn.T)
    s_vals = np.linalg.svd(Q[:, -6:].T @ qn, compute_uv=False)
    assert s_vals.min() > 1 - 1e-6


def test_rayleigh_ritz_sequence_small_matches_oracle(dcg):
    # The n = 1024 sequence with extraction="ritz" against the float64 oracle
    # running the same extraction: every solve meets tol, the recycled solves
    # take fewer iterations than plain CG on the GPU, and the counts follow
    # the oracle's within the float32 excess measured for the harmonic pencil
    # on this sequence (8 % .. 26 %): 35 % + 2 per system, 25 % in total.
    # The top Ritz value is a lower bound on lambda_max (Cauchy interlacing);
    # from t = 1 on the oracle's sits 0.3 % .. 1.4 % below it, on a window of
    # directions that the float32 solve does not reproduce, so the GPU's value
    # is checked against that bound and its distance to lambda_max against
    # the oracle's (at most twice it, plus 1e-3).
    cfg = S.RBFSequence(**{**S.SMALL_1024.__dict__, "tol": 1e-6})
    got = _sequence_gpu(dcg, cfg, cfg.T, 1e-6, extraction="ritz")
    X, bs = S.draw_sequence(cfg, T=cfg.T)
    X64 = X.astype(np.float32).astype(np.float64)
    ops = [O.rbf_gram(X64, cfg.lengthscale(t), cfg.signal_var, cfg.noise) for t in range(cfg.T)]
    ref = O.run_sequence(ops, [b.astype(np.float64) for b in bs], cfg.k, cfg.ell, 1e-6, extraction="ritz")
    counts = [(info["iters"], r["result"].iters) for info, r in zip(got, ref)]
    for (gi, oi), info, r in zip(counts, got, ref):
        assert info["status"] == 0 and info["relres_true"] <= 1e-6
        assert abs(gi - oi) <= 2 + 0.35 * oi, counts
    for t, (info, r) in enumerate(zip(got, ref)):
        lam_max = np.linalg.eigvalsh(ops[t])[-1]
        gap_o = (lam_max - r["ritz"].theta[0]) / lam_max
        th = info["theta"][0]
        assert th <= lam_max * (1 + 1e-5), (t, th, lam_max)
        assert (lam_max - th) / lam_max <= 2 * gap_o + 1e-3, (t, th, r["ritz"].theta[0], lam_max)
    tot_g, tot_o = sum(c[0] for c in counts), sum(c[1] for c in counts)
    assert abs(tot_g - tot_o) <= 0.25 * tot_o, counts
    plain = _sequence_gpu(dcg, cfg, cfg.T, 1e-6, deflate=False)
    for t in range(1, cfg.T):
        assert got[t]["iters"] < plain[t]["iters"], (t, got[t]["iters"], plain[t]["iters"])


def _sequence_gpu(dcg, cfg, T, tol, deflate=True, refine_every=0, host_loop=False, keep_A=False,
                  extraction="harmonic", symmetric=False):
    X, bs = S.draw_sequence(cfg, T=T)
    Xd = dev(X.astype(np.float32))
    n = cfg.n
    out = []
    with dcg.DefCG(n, cfg.k if deflate else 0, cfg.ell if deflate else 0, tol, refine_every=refine_every,
                   host_loop=host_loop, extraction=extraction) as s:
        A = torch.empty((n, n), dtype=torch.float32, device="cuda")
        for t in range(T):
            dcg.form_rbf_dense(Xd, cfg.lengthscale(t), cfg.signal_var, cfg.noise, out=A)
            s.set_operator_dense(A, symmetric=symmetric)
            x, info = s.solve(dev(bs[t]))
            if deflate:
                s.update_subspace()
                info["theta"] = s.ritz_values()[:8]
            info["x"] = x.cpu().numpy()
            if keep_A:
                info["A"] = A.cpu().numpy()
            out.append(info)
    return out


def test_sequence_small_matches_oracle_golden(dcg):
    # n = 1024 sequence (5 systems, kappa 391 .. 5.9e3), tol 1e-6, k = 8,
    # ell = 32, window last, against the float64 oracle (tests/golden).
    # Iteration counts: float32 CG loses orthogonality at eps32 instead of
    # eps64 and needs more steps on these ill-conditioned systems, and the
    # recycled W comes from float32 directions; the measured excess grows from
    # 8 % to 26 % along the sequence. Bound: 30 % + 2 per system, 22 % in total.
    g = json.load(open(os.path.join(HERE, "golden", "small_1024_tol1e-6_oracle.json")))
    cfg = S.RBFSequence(**{**S.SMALL_1024.__dict__, "tol": 1e-6})
    got = _sequence_gpu(dcg, cfg, cfg.T, 1e-6)
    counts = [(info["iters"], ref["defcg_iters"]) for info, ref in zip(got, g["systems"])]
    for (gi, oi), info, ref in zip(counts, got, g["systems"]):
        assert info["status"] == 0
        assert info["relres_true"] <= 1e-6
        assert abs(gi - oi) <= 2 + 0.30 * oi, counts
        np.testing.assert_allclose(info["theta"][0], ref["theta_top"][0], rtol=1e-3)
    tot_g, tot_o = sum(c[0] for c in counts), sum(c[1] for c in counts)
    assert abs(tot_g - tot_o) <= 0.22 * tot_o, counts
    plain = _sequence_gpu(dcg, cfg, cfg.T, 1e-6, deflate=False)
    for t in range(1, cfg.T):
        assert got[t]["iters"] < plain[t]["iters"]


def test_sequence_small_error_against_cholesky(dcg):
    # Besides following the oracle, each solution of the n = 1024 sequence is
    # compared with the exact solution x* of the float32 operator the GPU formed
    # (float64 Cholesky here). The relative residual, formed here in float64,
    # meets tol and agrees with the library's compensated true residual; the
    # relative A-norm error is at most sqrt(kappa) times it, since
    # |e|_A^2 = r^T A^{-1} r <= |r|^2 / lambda_min and |x*|_A^2 >= |b|^2 / lambda_max.
    import scipy.linalg as sla
    cfg = S.RBFSequence(**{**S.SMALL_1024.__dict__, "tol": 1e-6})
    got = _sequence_gpu(dcg, cfg, cfg.T, 1e-6, keep_A=True)
    _, bs = S.draw_sequence(cfg, T=cfg.T)
    for t, info in enumerate(got):
        A = info["A"].astype(np.float64)
        b = bs[t].astype(np.float32).astype(np.float64)
        x = np.asarray(info["x"], dtype=np.float64)
        relres = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert info["status"] == 0 and relres <= 1e-6 * (1 + 1e-6), (t, relres)
        np.testing.assert_allclose(info["relres_true"], relres, rtol=1e-6)
        lam = np.linalg.eigvalsh(A)
        xs = sla.cho_solve(sla.cho_factor(A), b)
        e = x - xs
        rel_a = np.sqrt(e @ A @ e) / np.sqrt(xs @ A @ xs)
        assert rel_a <= np.sqrt(lam[-1] / lam[0]) * relres * (1 + 1e-6), (t, rel_a, lam[-1] / lam[0])


@pytest.mark.parametrize("symmetric", [False, True])
def test_sequence_dense_16384_full_size(dcg, symmetric):
    # The benchmark workload at full size, all 20 systems (n = 16384, k = 32,
    # ell = 64), with the full-matrix and with the upper-triangle matvec
    # (the benchmark's): each solve reaches the true relative residual 1e-6;
    # per-system iteration counts follow the float64 oracle's
    # (tests/golden, written by tests/golden/make_golden.py) within 10 % + 2
    # (float32 recursion, reading G8); for systems 0, 10 and 19 the solution
    # error against the oracle's x is within kappa (2 tol + 5e-7), with kappa
    # the oracle's Lanczos estimate and 5e-7 the float32 operator's entry
    # error (float32 distances, the 2-ulp exponential): 6e-6 at t = 0 (kappa
    # 2.5, inside the 1e-5 float32 target), 4e-4 at t = 10 (kappa 164),
    # 1.2e-2 at t = 19 (kappa 4.8e3). Measured: 1.1e-7, 4.2e-7 and 3.4e-6,
    # so the 1e-5 float32 target holds on all three and is asserted too.
    g = json.load(open(os.path.join(HERE, "golden", "dense_16384_oracle.json")))
    gx = np.load(os.path.join(HERE, "golden", "dense_16384_oracle_x.npz"))
    got = _sequence_gpu(dcg, S.DENSE_16384, 20, 1e-6, symmetric=symmetric)
    for info, ref in zip(got, g["systems"]):
        assert info["status"] == 0 and info["relres_true"] <= 1e-6, (ref["t"], info)
        assert abs(info["iters"] - ref["defcg_iters"]) <= 2 + 0.1 * ref["defcg_iters"], (info["iters"], ref)
        key = f"x_{ref['t']}"
        if key in gx:
            xo = gx[key]
            err = np.linalg.norm(info["x"] - xo) / np.linalg.norm(xo)
            bound = ref["kappa_lanczos"] * (2e-6 + 5e-7)
            print("t=%d kappa=%.3g err=%.2e bound=%.2e" % (ref["t"], ref["kappa_lanczos"], err, bound))
            assert err <= bound and err <= 1e-5, (ref["t"], err, bound)


@pytest.mark.parametrize("refine_every", [0, 7])
def test_host_loop_matches_graph(dcg, refine_every):
    # The host-driven loop launches the graph's kernels in the same order with
    # the same arguments; every reduction has a fixed order, so iterates,
    # counts and Ritz values are bit-identical.
    cfg = S.SMALL_1024
    g = _sequence_gpu(dcg, cfg, 3, 1e-6, refine_every=refine_every)
    h = _sequence_gpu(dcg, cfg, 3, 1e-6, refine_every=refine_every, host_loop=True)
    for a, b in zip(g, h):
        assert a["iters"] == b["iters"] and a["matvecs_check"] == b["matvecs_check"]
        assert a["status"] == b["status"] == 0
        assert np.array_equal(a["x"], b["x"])
        assert np.array_equal(a["theta"], b["theta"])


def test_async_update_overlapped_with_forming_matches_sync(dcg):
    # dcg_update_subspace_async, with the next operator formed on a second
    # stream while the extraction runs, gives bit-identical solves to the
    # synchronous update: the extraction reads W, AW and the stored
    # directions, never A, and the next solve waits for both.
    cfg = S.DENSE_16384.scaled(3000, T=5)
    X, bs = S.draw_sequence(cfg, T=cfg.T)
    Xd = dev(X.astype(np.float32))
    n = cfg.n
    lda = (n + 3) // 4 * 4
    runs = []
    for overlap in (False, True):
        side = torch.cuda.Stream()
        A = torch.empty((n, lda), dtype=torch.float32, device="cuda")
        xs, its = [], []
        with dcg.DefCG(n, cfg.k, cfg.ell, 1e-6) as s:
            main = s.stream
            dcg.form_rbf_dense(Xd, cfg.lengthscale(0), cfg.signal_var, cfg.noise, out=A)
            for t in range(cfg.T):
                s.set_operator_dense(A, lda)
                x, info = s.solve(dev(bs[t]))
                assert info["status"] == 0 and info["relres_true"] <= 1e-6
                xs.append(x.cpu().numpy())
                its.append(info["iters"])
                if not overlap:
                    s.update_subspace()
                    if t + 1 < cfg.T:
                        dcg.form_rbf_dense(Xd, cfg.lengthscale(t + 1), cfg.signal_var, cfg.noise, out=A)
                else:
                    side.wait_stream(main)  # the solve is complete; the update below is not waited for
                    assert s.update_subspace(wait=False) is None
                    if t + 1 < cfg.T:
                        dcg.form_rbf_dense(Xd, cfg.lengthscale(t + 1), cfg.signal_var, cfg.noise, out=A,
                                           stream=side)
                        main.wait_stream(side)
            s.sync()
            k_final = s.get_subspace().shape[0]
        runs.append((xs, its, k_final))
    (xs0, it0, k0), (xs1, it1, k1) = runs
    assert it0 == it1 and k0 == k1 == cfg.k
    for a, b in zip(xs0, xs1):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("extraction,select", [("harmonic", "largest"), ("harmonic", "smallest"),
                                               ("ritz", "largest")])
def test_kept_ritz_values_are_float64_on_the_gpu_pencil(dcg, extraction, select):
    # The eigen-solve of Eq. 7 runs in float32 on the scaled pencil; the kept
    # values are then the pencil's float64 Rayleigh quotients at the float32
    # eigenvectors. Reference: the very pencil the GPU formed (dcg_get_pencil),
    # reduced in float64 by the same rule (unit-diagonal scaling, diagonally
    # pivoted Cholesky of F that stops below 1e-4, reading G5), then solved in
    # float64 (scipy.linalg.eigh). Compared on the first extraction of a
    # sequence (Z = P, nearly A-conjugate directions: a well-conditioned
    # pencil): the kept values agree to 1e-8 relative when the largest are
    # kept (measured 5.6e-9 harmonic, 2.1e-9 Ritz; the quotient's error is
    # quadratic in the float32 vector's); the smallest harmonic values
    # cluster near the noise level, where the float32 vectors' error grows as
    # 1 / gap: 3e-6 (measured 1.1e-6). Once W joins Z the pencil has
    # near-degenerate values and nearly dependent columns, which the float32
    # and a float64 pivoted reduction need not drop alike, so later
    # extractions are not compared value by value. The oracle's own pencil
    # comes from float64 directions, so it is not the comparison here.
    import scipy.linalg as sla

    def reduced(F, G):
        d = 1.0 / np.sqrt(np.diag(F))
        Fs, Gs = F * d[:, None] * d[None, :], G * d[:, None] * d[None, :]
        R, keep = Fs.copy(), []
        rest = list(range(len(d)))
        while rest:
            j = max(rest, key=lambda i: R[i, i])
            if R[j, j] < 1e-4:
                break
            keep.append(j)
            rest.remove(j)
            col = R[:, j] / np.sqrt(R[j, j])
            R = R - np.outer(col, col)
        keep = sorted(keep)
        return Fs[np.ix_(keep, keep)], Gs[np.ix_(keep, keep)]
    cfg = S.SMALL_1024
    X, bs = S.draw_sequence(cfg, T=3)
    with dcg.DefCG(cfg.n, cfg.k, cfg.ell, 1e-6, extraction=extraction, select=select) as s:
        A = torch.empty((cfg.n, cfg.n), dtype=torch.float32, device="cuda")
        worst, compared = 0.0, 0
        for t in range(3):
            dcg.form_rbf_dense(dev(X.astype(np.float32)), cfg.lengthscale(t), cfg.signal_var, cfg.noise, out=A)
            s.set_operator_dense(A)
            s.solve(dev(bs[t]))
            k_new = s.update_subspace()
            F, G = s.pencil()
            Fr, Gr = reduced(0.5 * (F + F.T), 0.5 * (G + G.T))
            ev = np.sort(sla.eigh(Gr, Fr, eigvals_only=True))[::-1]
            th = s.ritz_values()
            kept = th[:k_new] if select == "largest" else th[len(th) - k_new:]
            ref = ev[:k_new] if select == "largest" else ev[len(ev) - k_new:]
            if t == 0 and len(th) == len(ev):   # first extraction, same number of directions kept
                rel = np.max(np.abs(kept - ref) / np.abs(ref))
                worst = max(worst, rel)
                compared += 1
                assert rel <= (1e-8 if select == "largest" else 3e-6), (t, rel)
        print(extraction, select, "worst relative error of the kept values %.2e" % worst)
        assert compared == 1
