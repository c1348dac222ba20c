"""The paper's experiment (Sec. 3): Newton's method for the mode of the
Laplace approximation in binary GP classification, each Newton system
A = I + H^{1/2} K H^{1/2}, b = H^{1/2} K (H f + grad log p(y | f)) solved by
def-CG with the subspace recycled from one Newton step to the next.

Every numerical step runs in the library: dcg_laplace_system forms A, b (and
the step's c, s), dcg_solve solves, dcg_update_subspace extracts the next W,
dcg_laplace_update forms a, f = K a and Psi. This module only sequences the
calls and keeps the buffers.
"""

from __future__ import annotations

import ctypes

import torch

from . import _lib


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def laplace_mode(solver, K: torch.Tensor, y: torch.Tensor, dpsi_tol: float = 1.0, max_newton: int = 50,
                 recycle: bool = True, on_step=None):
    """Runs the Newton loop from f = 0 until Psi rises by less than
    ``dpsi_tol`` (Sec. 3 uses 1). ``solver`` is a DefCG context of size n
    (its k and ell give def-CG(k, ell); k = 0 is plain CG). K: row-major
    float32 (n, ldk) CUDA tensor, exactly symmetric; y: float32 labels +-1.
    ``on_step(solver, t, info)`` runs after each Newton system is solved (and
    its subspace extracted). Returns (f, a, psi history, per-step solve
    infos)."""
    n = solver.n
    if K.dim() != 2 or K.shape[0] != n or K.shape[1] < n or K.shape[1] % 4 or K.dtype != torch.float32:
        raise ValueError("K must be a float32 (n, ldk) tensor with ldk >= n, ldk % 4 == 0")
    if y.numel() != n or y.dtype != torch.float32 or not y.is_cuda:
        raise ValueError("y must hold n float32 labels on the GPU")
    ldk = K.shape[1]
    dev = K.device
    lib = solver.lib
    A = torch.empty((n, ldk), dtype=torch.float32, device=dev)
    b = torch.empty(n, dtype=torch.float32, device=dev)
    c = torch.zeros(n, dtype=torch.float64, device=dev)
    s = torch.zeros(n, dtype=torch.float32, device=dev)
    f = torch.zeros(n, dtype=torch.float64, device=dev)
    a = torch.zeros(n, dtype=torch.float64, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    psi = ctypes.c_double()

    def update():
        solver._check(lib.dcg_laplace_update(solver._ctx, _ptr(K), ldk, _ptr(y), _ptr(c), _ptr(s), _ptr(x),
                                             _ptr(f), _ptr(a), ctypes.byref(psi)), "dcg_laplace_update")
        return psi.value

    hist = [update()]            # f = K 0 = 0, a = 0: Psi(0) = n log(1/2)
    infos = []
    for _ in range(max_newton):
        solver._check(lib.dcg_laplace_system(solver._ctx, _ptr(K), ldk, _ptr(y), _ptr(f), _ptr(A), ldk, _ptr(b),
                                             _ptr(c), _ptr(s)), "dcg_laplace_system")
        solver.set_operator_dense(A, ldk, symmetric=True)
        _, info = solver.solve(b, x)
        infos.append(info)
        if recycle and solver.k > 0:
            solver.update_subspace()
        if on_step is not None:
            on_step(solver, len(infos) - 1, info)
        hist.append(update())
        if hist[-1] - hist[-2] < dpsi_tol:
            break
    return f, a, hist, infos


__all__ = ["laplace_mode"]
