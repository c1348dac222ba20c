"""GPU parity of the sparse F, G of the harmonic pencil (Sec. 2.3, the forms of
Saad et al.): fg_form="sparse" builds F and G from the scalars the solve
records per stored direction (d_j, alpha_j, |r_j|^2, (AW)^T r_j) instead of
the Gram products over Z and AZ.

Checks: (1) on a well-conditioned system, where float32 keeps the
A-conjugacy and residual orthogonality the forms rest on, the sparse pencil
equals the explicit one entry by entry up to float32 rounding, and the kept
harmonic Ritz values agree (a wrong slot, a wrong residual index or a dropped
coupling term moves entries by O(1)); (2) the kept values follow the float64
oracle's own sparse extraction (oracle.harmonic_ritz_sparse on the oracle's
run); (3) on the n = 1024 kernel sequence the recycled subspaces it gives
serve as well as the explicit ones (iteration counts).
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
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _problem(n, k, seed):
    A, _ = S.spd_with_spectrum(np.geomspace(1.0, 20.0, n), seed=seed)
    A32 = A.astype(np.float32)
    rng = np.random.default_rng(seed + 1)
    b = rng.standard_normal(n).astype(np.float32)
    W = rng.standard_normal((k, n)).astype(np.float32)
    return A32, b, W


def _gpu_pencil(dcg, A32, b, W, ell, window, fg_form, tol):
    # the context keeps max(k, 4) vectors: with an empty W (k = 0) the first
    # solve is plain CG and the extraction still draws 4 from its directions
    n = A32.shape[0]
    with dcg.DefCG(n, max(W.shape[0], 4), ell, tol, window=window, fg_form=fg_form) as s:
        s.set_operator_dense(dev(A32))
        if W.shape[0]:
            s.set_subspace(dev(W))
        x, info = s.solve(dev(b))
        assert info["status"] == 0, info
        s.update_subspace()
        assert s.pencil_form() == fg_form
        F, G = s.pencil()
        theta = s.ritz_values()
    return F, G, theta, info


@pytest.mark.parametrize("k,window", [(4, "first"), (4, "last"), (8, "last")])
def test_sparse_pencil_equals_explicit(dcg, k, window):
    # kappa = 20, tol 1e-5 (no replacement inside the window; ~30 iterations,
    # so the last-window ring has wrapped). Entry differences: float32
    # rounding of the recursion and of the recorded scalars against float64
    # Gram sums of the float32 vectors, well under 1e-4 of the largest entry.
    n, ell = 2000, 10
    A32, b, W = _problem(n, k, 7 + k)
    Fe, Ge, te, ie = _gpu_pencil(dcg, A32, b, W, ell, window, "explicit", 1e-5)
    Fs, Gs, ts, is_ = _gpu_pencil(dcg, A32, b, W, ell, window, "sparse", 1e-5)
    assert ie["iters"] == is_["iters"] and ie["iters"] > ell   # the solve does not depend on fg_form
    assert Fe.shape == Fs.shape == (k + ell, k + ell)
    np.testing.assert_allclose(Fs, Fe, rtol=0, atol=1e-4 * np.abs(Fe).max())
    np.testing.assert_allclose(Gs, Ge, rtol=0, atol=1e-4 * np.abs(Ge).max())
    # the structure itself: F block diagonal; in the P block of G each
    # direction couples only to its neighbours (tridiagonal in iteration
    # order; the slots of the last-window ring are in ring order, so the
    # pair that straddles the ring's seam sits off the band)
    P = Gs[k:, k:]
    assert np.count_nonzero(Fs[:k, k:]) == 0 and np.count_nonzero(Fs[k:, k:] - np.diag(np.diag(Fs[k:, k:]))) == 0
    assert np.count_nonzero(P - np.diag(np.diag(P))) == 2 * (ell - 1)
    assert np.all(np.count_nonzero(P, axis=1) <= 3)
    np.testing.assert_allclose(ts, te, rtol=1e-4)


@pytest.mark.parametrize("k,window", [(4, "first"), (4, "last"), (8, "last")])
def test_sparse_extraction_matches_oracle(dcg, k, window):
    # The oracle's own run (float64, the same float32 operator, b and W) and
    # its sparse extraction: the kept harmonic Ritz values agree to the 1e-3
    # that the explicit extraction's test allows (float32 Krylov space).
    n, ell = 2000, 10
    A32, b, W = _problem(n, k, 7 + k)
    _, _, theta, info = _gpu_pencil(dcg, A32, b, W, ell, window, "sparse", 1e-5)
    W64 = W.T.astype(np.float64) if k else None
    # with the last window the oracle runs the GPU's iteration count (stopped
    # by max_iter, so that the residual after the last stored direction is in
    # its history): the same window of the Krylov sequence
    ref = O.defcg(A32.astype(np.float64), b.astype(np.float64), W=W64, ell=ell, window=window, keep_iterates=True,
                  tol=1e-5 if window == "first" else 1e-14, max_iter=None if window == "first" else info["iters"])
    s = 0 if window == "first" else ref.iters - ell
    R = ref.r_history
    E = W64.T @ ref.AW if k else np.zeros((0, 0))
    GW = ref.AW.T @ ref.AW if k else np.zeros((0, 0))
    rho = [R[j] @ R[j] for j in range(s, s + ell + 1)]
    h = np.column_stack([ref.AW.T @ R[j] for j in range(s, s + ell + 1)]) if k else np.zeros((0, ell + 1))
    rr = O.harmonic_ritz_sparse(W64, ref.P, E, GW, ref.d, ref.alpha, rho, h, max(k, 4))
    np.testing.assert_allclose(theta, rr.theta, rtol=1e-3)


def test_without_w_the_update_takes_the_gram_products(dcg):
    # A solve without W is plain CG: its first-window directions of a
    # well-conditioned system still give the oracle's values, but the library
    # does not trust the tridiagonal model there (ghost values once a Ritz
    # value converges in float32) and takes the Gram products.
    n, ell = 2000, 10
    A32, b, W = _problem(n, 0, 7)
    with dcg.DefCG(n, 4, ell, 1e-5, window="first", fg_form="sparse") as s:
        s.set_operator_dense(dev(A32))
        s.solve(dev(b))
        s.update_subspace()
        assert s.pencil_form() == "explicit"


def test_sparse_sequence_recycles_like_explicit(dcg):
    # The n = 1024 kernel sequence (5 systems, kappa 391 .. 5.9e3, k = 8,
    # ell = 32, window last, tol 1e-6). The first system has no W and every
    # system whose last window holds a residual replacement falls back to the
    # Gram products; the others take the sparse forms (measured: pencils equal
    # to 2e-8 of the largest entry there). The subspaces recycled cut the
    # iterations as the explicit ones do: per system within 10 % + 2 of the
    # explicit extraction's, and below plain CG from the second system on.
    cfg = S.RBFSequence(**{**S.SMALL_1024.__dict__, "tol": 1e-6})
    X, bs = S.draw_sequence(cfg, T=cfg.T)
    Xd = dev(X.astype(np.float32))
    iters = {}
    for form in ("explicit", "sparse"):
        with dcg.DefCG(cfg.n, cfg.k, cfg.ell, 1e-6, fg_form=form) as s:
            A = torch.empty((cfg.n, cfg.n), dtype=torch.float32, device="cuda")
            out = []
            for t in range(cfg.T):
                dcg.form_rbf_dense(Xd, cfg.lengthscale(t), cfg.signal_var, cfg.noise, out=A)
                s.set_operator_dense(A)
                _, info = s.solve(dev(bs[t].astype(np.float32)))
                assert info["status"] == 0 and info["relres_true"] <= 1e-6
                s.update_subspace()
                out.append((info["iters"], s.pencil_form()))
            iters[form] = out
    g = json.load(open(os.path.join(HERE, "golden", "small_1024_tol1e-6_oracle.json")))
    plain = [ref["cg_iters"] for ref in g["systems"]]
    print("iterations explicit", iters["explicit"], "sparse", iters["sparse"], "oracle plain CG", plain)
    assert all(f == "explicit" for _, f in iters["explicit"])
    assert sum(f == "sparse" for _, f in iters["sparse"]) >= 1
    for (e, _), (sp, _) in zip(iters["explicit"], iters["sparse"]):
        assert abs(sp - e) <= 2 + 0.1 * e, iters
    for t in range(1, cfg.T):
        assert iters["sparse"][t][0] < plain[t], (iters, plain)
