"""GB300 deflated conjugate gradients with harmonic-Ritz subspace recycling.

Implements the hot path of de Roos & Hennig, "Krylov Subspace Recycling for
Fast Iterative Least-Squares in Machine Learning" (arXiv 1706.00241):
Algorithm 1 (def-CG(k, ell)) over a sequence of SPD systems (Eq. 1) with the
harmonic projection of Sec. 2.3 (Eq. 7) between solves, as hand-written
sm_103a CUDA behind the C ABI in include/dcg.h. This package is the thin
Python binding (torch supplies device memory and streams).
"""

from ._lib import DcgError, load  # noqa: F401
from .solver import DefCG, form_rbf_dense, matvec_dense_noalloc  # noqa: F401
from .autograd import DefCGSolve, LogDetProbes, fit_gp, gp_objective, rademacher_probes  # noqa: F401
from .laplace import laplace_mode  # noqa: F401
