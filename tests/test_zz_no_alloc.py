"""Context-free stored-operator matvec on the library's fixed scratch
(dcg_matvec_dense_noalloc) against the context entry point dcg_matvec, both
called through the C ABI. The two run the same kernel with the same grid and
reduction order, so q and p^T q must be bit-identical. Two calls in a row
check that the scratch (the arrival counter, the timeout word and the per-CTA
partials) is left ready for the next call.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DCG_ERR_INVALID_ARG = 1


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_00241_gb300 import build
    build.build()
    import paper_1706_00241_gb300 as P
    return P


def _operator(n, lda, seed):
    rng = np.random.default_rng(seed)
    A = np.zeros((n, lda), dtype=np.float32)
    A[:, :n] = rng.standard_normal((n, n)).astype(np.float32)
    p = rng.standard_normal(n).astype(np.float32)
    return A, p


@pytest.mark.parametrize("n", [1, 37, 1000, 4099, 16384])
def test_noalloc_matvec_matches_context_matvec(P, n):
    lda = (n + 3) // 4 * 4 + 4
    A, p = _operator(n, lda, 100 + n)
    Ad = torch.tensor(A, device="cuda")
    pd = torch.tensor(p, device="cuda")
    with P.DefCG(n, 0, 0, 1e-6) as s:
        s.set_operator_dense(Ad, lda)
        q_ref_d, pAp_ref = s.matvec(pd)
        q_ref_d = q_ref_d.clone()
        q_ref = q_ref_d.cpu().numpy().astype(np.float64)
    lib = P.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    q = torch.empty(n, dtype=torch.float32, device="cuda")
    pAp = torch.empty(1, dtype=torch.float64, device="cuda")
    scale = np.abs(A[:, :n]).astype(np.float64) @ np.abs(p).astype(np.float64)
    for _ in range(2):
        q.fill_(float("nan"))
        pAp.fill_(float("nan"))
        st = lib.dcg_matvec_dense_noalloc(ctypes.c_void_p(Ad.data_ptr()), n, lda, ctypes.c_void_p(pd.data_ptr()),
                                          ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(pAp.data_ptr()), stream)
        assert st == 0, lib.dcg_last_error(None)
        torch.cuda.synchronize()
        qh = q.cpu().numpy().astype(np.float64)
        got = float(pAp.cpu().item())
        # same kernel, grid and reduction order as the context matvec
        assert torch.equal(q, q_ref_d), np.max(np.abs(qh - q_ref))
        assert got == pAp_ref, (got, pAp_ref)
    # and both against the float64 product (float32 accumulation over n terms)
    ref = A[:, :n].astype(np.float64) @ p.astype(np.float64)
    assert np.all(np.abs(qh - ref) <= 2e-7 * np.sqrt(n) * 8 * scale + 1e-30)


def test_noalloc_matvec_without_pAp(P):
    n = 2048
    A, p = _operator(n, n, 5)
    Ad = torch.tensor(A, device="cuda")
    pd = torch.tensor(p, device="cuda")
    q = torch.empty(n, dtype=torch.float32, device="cuda")
    P.matvec_dense_noalloc(Ad, pd, q)
    torch.cuda.synchronize()
    ref = A.astype(np.float64) @ p.astype(np.float64)
    scale = np.abs(A).astype(np.float64) @ np.abs(p).astype(np.float64)
    assert np.all(np.abs(q.cpu().numpy() - ref) <= 1e-5 * scale)


def test_noalloc_matvec_rejects_bad_arguments(P):
    n = 64
    A, p = _operator(n, n, 6)
    Ad = torch.tensor(A, device="cuda")
    pd = torch.tensor(np.concatenate([p, [0.0]]).astype(np.float32), device="cuda")
    q = torch.empty(n, dtype=torch.float32, device="cuda")
    lib = P.load()
    vp = ctypes.c_void_p
    st = lib.dcg_matvec_dense_noalloc(vp(Ad.data_ptr()), n, n + 2, vp(pd.data_ptr()), vp(q.data_ptr()), None, None)
    assert st == DCG_ERR_INVALID_ARG and b"lda" in lib.dcg_last_error(None)
    st = lib.dcg_matvec_dense_noalloc(vp(Ad.data_ptr()), n, n, vp(pd.data_ptr() + 4), vp(q.data_ptr()), None, None)
    assert st == DCG_ERR_INVALID_ARG and b"aligned" in lib.dcg_last_error(None)
    st = lib.dcg_matvec_dense_noalloc(vp(Ad.data_ptr()), 0, n, vp(pd.data_ptr()), vp(q.data_ptr()), None, None)
    assert st == DCG_ERR_INVALID_ARG
