"""CPU checks of the Python binding's argument checks: every tensor whose
pointer goes to the library must hold exactly the elements the library reads
or writes, so a mis-sized tensor is rejected in Python before any call."""

import pytest
import torch

from paper_1706_00241_gb300 import solver as SV


def test_need_len():
    SV._need_len(torch.zeros(6), 6, "b")
    SV._need_len(torch.zeros(2, 3), 6, "b")        # any shape with n elements
    with pytest.raises(ValueError, match="n = 6"):
        SV._need_len(torch.zeros(5), 6, "b")


def test_need_rows():
    assert SV._need_rows(torch.zeros(4, 8), 4, "A", min_cols=4) == 8
    assert SV._need_rows(torch.zeros(4, 8), 4, "A", 8, min_cols=4) == 8
    with pytest.raises(ValueError, match="lda = 12"):
        SV._need_rows(torch.zeros(4, 8), 4, "A", 12)           # lda beyond the tensor's rows
    with pytest.raises(ValueError, match="4 rows"):
        SV._need_rows(torch.zeros(3, 8), 4, "A")
    with pytest.raises(ValueError, match="at least 4 columns"):
        SV._need_rows(torch.zeros(4, 3), 4, "A", min_cols=4)
    with pytest.raises(ValueError, match="2-D"):
        SV._need_rows(torch.zeros(16), 4, "A")


@pytest.fixture
def bare(monkeypatch):
    # a DefCG of size 6 with no library behind it: the CUDA-tensor check is
    # stubbed so that CPU tensors reach the size checks, which must raise
    # before the (absent) library is touched
    monkeypatch.setattr(SV, "_dev_f32", lambda t, name: t)
    s = object.__new__(SV.DefCG)
    s.n, s.k, s.ell = 6, 2, 4
    s.lib = None
    s._ctx = None
    return s


def test_methods_reject_mis_sized_tensors(bare):
    s = bare
    with pytest.raises(ValueError, match="b must hold"):
        s.solve(torch.zeros(5))
    with pytest.raises(ValueError, match="A must be a 2-D tensor with 6 rows"):
        s.set_operator_dense(torch.zeros(5, 8))
    with pytest.raises(ValueError, match="lda = 12"):
        s.set_operator_dense(torch.zeros(6, 8), 12)
    with pytest.raises(ValueError, match="W must be"):
        s.set_subspace(torch.zeros(2, 5))
    with pytest.raises(ValueError, match="p must hold"):
        s.matvec(torch.zeros(5))
    with pytest.raises(ValueError, match="q must hold"):
        s.matvec(torch.zeros(6), torch.zeros(4))
    with pytest.raises(ValueError, match="V must be"):
        s.apply_block(torch.zeros(3, 5))
    with pytest.raises(ValueError, match="Y must have"):
        s.apply_block(torch.zeros(3, 6), torch.zeros(2, 6))


def test_solve_multi_rejects_bad_blocks(bare):
    # lockstep solves: B is (nrhs, n) with 1 <= nrhs <= DCG_MAX_RHS, X float64
    # on the device and shaped like B; all checked before the library is called
    s = bare
    with pytest.raises(ValueError, match=r"B must be \(nrhs, 6\)"):
        s.solve_multi(torch.zeros(3, 5))
    with pytest.raises(ValueError, match=r"B must be \(nrhs, 6\)"):
        s.solve_multi(torch.zeros(18))
    with pytest.raises(ValueError, match="nrhs must lie in"):
        s.solve_multi(torch.zeros(0, 6))
    with pytest.raises(ValueError, match="nrhs must lie in"):
        s.solve_multi(torch.zeros(33, 6))
    with pytest.raises(TypeError, match="X must be"):
        s.solve_multi(torch.zeros(3, 6), torch.zeros(3, 6, dtype=torch.float64))   # not on the device
    with pytest.raises(TypeError, match="X must be"):
        s.solve_multi(torch.zeros(3, 6), torch.zeros(2, 6, dtype=torch.float64))


def test_free_functions_reject_mis_sized_tensors(monkeypatch):
    monkeypatch.setattr(SV, "_dev_f32", lambda t, name: t)
    monkeypatch.setattr(SV._lib, "load", lambda: None)
    with pytest.raises(ValueError, match="out must be a 2-D tensor with 6 rows"):
        SV.form_rbf_dense(torch.zeros(6, 3), 1.0, 1.0, 0.1, out=torch.zeros(5, 6))
    with pytest.raises(ValueError, match="at least 6 columns"):
        SV.form_rbf_dense(torch.zeros(6, 3), 1.0, 1.0, 0.1, out=torch.zeros(6, 4))
    with pytest.raises(ValueError, match="q must hold"):
        SV.matvec_dense_noalloc(torch.zeros(6, 8), torch.zeros(6), torch.zeros(5))
    with pytest.raises(ValueError, match="lda = 9"):
        SV.matvec_dense_noalloc(torch.zeros(6, 8), torch.zeros(6), torch.zeros(6), lda=9)
