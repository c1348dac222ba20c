"""CPU FP64 oracle for deflated CG with harmonic-Ritz recycling.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code with the CUDA path; both take their inputs from ``dcg_synth``.

Every function follows the paper (de Roos & Hennig, "Krylov Subspace Recycling
for Fast Iterative Least-Squares in Machine Learning", arXiv 1706.00241) and
cites the passage it implements. All arithmetic is float64 numpy; matrix
products, Cholesky and the symmetric eigensolver are library primitives used
as single steps, with no blocking or reordering beyond the algorithm.

Parity status per function (what pins it; tests in ``tests/test_oracle_*.py``):
  rbf_gram, rbf_matvec   pinned: closed form at hand-computed points, symmetry, SPD
  cg                     pinned: dense solve on tiny N, finite termination in
                         (#distinct eigenvalues) steps, exact rational 2x2 run
  defcg                  pinned: dense solve, W^T r_j = 0, A-conjugacy, k = 0
                         reproduces cg bitwise, exact eigenvectors give CG on
                         the reduced spectrum; the replacement branch (R13):
                         project_out / next_direction identities on arbitrary
                         inputs, no-op with one operator, W^T r = 0,
                         (AW)^T p = 0 and the recursion's beta under an
                         approximate loop operator (A_true)
  harmonic_ritz          pinned: invariant subspace gives exact eigenvalues and
                         eigenvectors; generalized-eigen residual
  rayleigh_ritz          pinned: Galerkin condition, orthonormal-basis eigenvalues,
                         the CG-Lanczos tridiagonal, Cauchy interlacing
  sparse_FG, harmonic_ritz_sparse
                         pinned: equal to the products over Z and AZ
  laplace_oracle         pinned: finite differences of the likelihood, the plain
                         Newton step, the mode's fixed-point equation, the
                         system's spectrum bound, a generic optimiser
  gp_oracle.gp_nll, gp_nll_grad
                         pinned: central finite differences in log space, the
                         closed form for a vanishing lengthscale
  gp_oracle.dtheta_forms pinned: finite differences of the operator
  gp_oracle.hutchinson, logdet_grad_probes, gp_nll_grad_probes
                         pinned: exact on diagonal matrices, unbiased over
                         20000 probes (5 standard errors)
  gp_oracle.adam_path    pinned: closed-form steps under a constant gradient
"""

from .dcg_oracle import (  # noqa: F401
    SolveResult,
    cg,
    defcg,
    harmonic_ritz,
    rbf_gram,
    rbf_matvec,
    run_sequence,
    true_relres,
)
