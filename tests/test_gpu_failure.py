"""Failure handling on the GPU without a fault: a bounded device-side wait is
made to run out through the library's test hook (one CTA withholds its
arrival at the fused iteration kernel's grid barrier, and the wait gives up
after a few polls). The solve must end with DCG_ERR_TIMEOUT, name the wait,
and leave the context usable: the next solve of the same system reproduces,
bit for bit, the solve made before the failure.
"""

import numpy as np
import pytest

import dcg_synth as S
from oracle import dcg_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DCG_ERR_TIMEOUT = 7
DCG_ERR_INVALID_ARG = 1


@pytest.fixture(scope="module")
def dcg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_00241_gb300 import build
    build.build()
    import paper_1706_00241_gb300 as P
    return P


@pytest.mark.parametrize("host_loop", [False, True])
def test_barrier_timeout_is_reported_and_the_context_recovers(dcg, host_loop):
    cfg = S.SMALL_1024.scaled(2048, T=2)
    X, bs = S.draw_sequence(cfg)
    X32 = X.astype(np.float32)
    A32 = O.rbf_gram(X32.astype(np.float64), cfg.lengthscale(0), cfg.signal_var, cfg.noise).astype(np.float32)
    A = torch.tensor(A32, device="cuda")
    b0 = torch.tensor(bs[0].astype(np.float32), device="cuda")
    b1 = torch.tensor(bs[1].astype(np.float32), device="cuda")
    tol = 1e-6
    with dcg.DefCG(cfg.n, cfg.k, cfg.ell, tol, host_loop=host_loop) as s:
        s.set_operator_dense(A)
        s.solve(b0)
        assert s.update_subspace() == cfg.k        # W active: the k x k matrices are staged
        x_ref, info_ref = s.solve(b1)
        x_ref = x_ref.clone()
        assert info_ref["status"] == 0 and info_ref["k_used"] == cfg.k
        s.debug_arm_barrier_timeout(polls=64)
        x_bad, info_bad = s.solve(b1, raise_on_error=False)
        assert info_bad["status"] == DCG_ERR_TIMEOUT, info_bad
        assert "site 4" in s.last_error() and "grid barrier" in s.last_error()
        assert info_bad["iters"] <= 1
        assert torch.isfinite(x_bad).all()
        # the hook is one-shot: the same solve again equals the one before
        x_again, info_again = s.solve(b1)
        assert info_again["status"] == 0
        assert info_again["iters"] == info_ref["iters"]
        assert torch.equal(x_again, x_ref)
        b64 = bs[1].astype(np.float32).astype(np.float64)
        A64 = A32.astype(np.float64)
        relres = np.linalg.norm(b64 - A64 @ x_again.cpu().numpy()) / np.linalg.norm(b64)
        assert relres <= tol
    torch.cuda.synchronize()


def test_barrier_timeout_hook_rejects_bad_arguments(dcg):
    n = 256
    A = torch.eye(n, device="cuda")
    with dcg.DefCG(n, 0, 0, 1e-6) as s:
        with pytest.raises(Exception):
            s.debug_arm_barrier_timeout(polls=0)       # no operator yet: STATE, then bad polls
        s.set_operator_dense(A)
        lib = dcg.load()
        assert lib.dcg_debug_arm_barrier_timeout(s._ctx, 0) == DCG_ERR_INVALID_ARG
        assert lib.dcg_debug_arm_barrier_timeout(s._ctx, (1 << 22) + 1) == DCG_ERR_INVALID_ARG
