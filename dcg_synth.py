"""Seeded synthetic inputs for deflated-CG sequences.

This module only draws random numbers and lays out workload descriptions. It
holds none of the solver's arithmetic: no kernel evaluation, no CG step, no
eigen-extraction. Both the CPU oracle (``oracle/``) and the CUDA path
(``paper_1706_00241_gb300``) take their inputs from here, so neither depends on
a random generator implemented twice.

The workloads are Gaussian-process style sequences of SPD systems
``A_t x_t = b_t`` (Eq. 1 of the paper) with ``A_t = K_t + noise * I`` where
``K_t`` is an RBF Gram matrix (Sec. 3) whose lengthscale moves along a path
``l_t``. The paper's own data set (infinite-MNIST digits 3 vs 5, Sec. 3) is
not available; these seeded draws stand in for it.

Draw order for a sequence (PCG64 via ``numpy.random.default_rng(seed)``):
X first (n x d, float64), then ``b_0 .. b_{T-1}`` in order. Values are drawn
in float64 and cast by the consumer.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class RBFSequence:
    """A sequence of RBF systems ``(K_t + noise I) x_t = b_t``.

    ``lengthscale(t) = l0 * (1 + growth * t)``; ``signal_var`` is the RBF
    amplitude theta^2 of Sec. 3; ``noise`` the diagonal shift.
    """

    name: str
    n: int
    d: int
    T: int
    l0: float
    growth: float
    noise: float
    signal_var: float = 1.0
    k: int = 8
    ell: int = 32
    tol: float = 1e-6
    x_dist: str = "normal"  # "normal": N(0,1); "uniform": U[0,1]
    seed: int = 0
    storage: str = "dense"  # "dense" (stored FP32 A) or "rbf" (matrix-free)
    x_dtype: str = "fp32"  # element type of X for the matrix-free operator
    refine_every: int = 0
    extra: dict = field(default_factory=dict, compare=False)

    def lengthscale(self, t: int) -> float:
        return self.l0 * (1.0 + self.growth * t)

    def scaled(self, n: int, T: int | None = None, name: str | None = None) -> "RBFSequence":
        """Same generator parameters at a smaller size (downscaled parity cases)."""
        return RBFSequence(
            name=name or f"{self.name}@n{n}", n=n, d=self.d, T=self.T if T is None else T,
            l0=self.l0, growth=self.growth, noise=self.noise, signal_var=self.signal_var,
            k=self.k, ell=self.ell, tol=self.tol, x_dist=self.x_dist, seed=self.seed,
            storage=self.storage, x_dtype=self.x_dtype, refine_every=self.refine_every,
            extra=dict(self.extra))


# The five workloads. Sizes, lengthscale paths and noise levels are the ones the
# benchmark configurations name; parameters they leave open (signal variance,
# ell for the larger cases) take the values listed in the design notes.
SMALL_1024 = RBFSequence(name="rbf_n1024_d8_T5", n=1024, d=8, T=5, l0=1.0, growth=0.1,
                         noise=1e-2, k=8, ell=32, tol=1e-8)
DENSE_16384 = RBFSequence(name="dense_fp32_n16384_d16_T20", n=16384, d=16, T=20, l0=0.8,
                          growth=0.05, noise=1e-3, k=32, ell=64, tol=1e-6)
MF_131072 = RBFSequence(name="rbf_bf16_n131072_d32_T30", n=131072, d=32, T=30, l0=2.0,
                        growth=0.03, noise=1e-2, k=64, ell=128, tol=1e-6, storage="rbf",
                        x_dtype="bf16", refine_every=50)
GRAD_32768 = RBFSequence(name="gp_grad_n32768_d8", n=32768, d=8, T=30, l0=0.5, growth=0.0,
                         noise=0.1, k=32, ell=64, tol=1e-6, x_dist="uniform", storage="rbf",
                         extra={"probes": 16, "adam_lr": 0.05})
MF_262144 = RBFSequence(name="rbf_fp32_n262144_d4_T40", n=262144, d=4, T=40, l0=0.5,
                        growth=0.02, noise=1e-2, k=64, ell=128, tol=1e-6, storage="rbf",
                        x_dtype="fp32", refine_every=50)

WORKLOADS = {w.name: w for w in (SMALL_1024, DENSE_16384, MF_131072, GRAD_32768, MF_262144)}


def draw_sequence(cfg: RBFSequence, T: int | None = None):
    """Return ``(X, [b_0, ..., b_{T-1}])`` in float64, drawn in the fixed order."""
    T = cfg.T if T is None else T
    rng = np.random.default_rng(cfg.seed)
    if cfg.x_dist == "normal":
        X = rng.standard_normal((cfg.n, cfg.d))
    elif cfg.x_dist == "uniform":
        X = rng.random((cfg.n, cfg.d))
    else:
        raise ValueError(cfg.x_dist)
    bs = [rng.standard_normal(cfg.n) for _ in range(T)]
    return X, bs


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even); returns float32.

    Used to produce the BF16-stored copy of X that both sides read; it is a
    storage format conversion, not solver arithmetic.
    """
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def round_to_tf32(a: np.ndarray) -> np.ndarray:
    """Round float values to TF32 (10 explicit mantissa bits, ties to even)."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 13) & 1
    u = (u + 0xFFF + lsb) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def random_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian with sign fix)."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))


def spd_with_spectrum(eigs, seed: int = 0):
    """Return ``(A, Q)`` with ``A = Q diag(eigs) Q^T`` for a random orthogonal Q.

    A test-matrix generator: the spectrum is prescribed so that properties of
    the solver (termination, deflation of known eigenvectors) can be checked.
    """
    eigs = np.asarray(eigs, dtype=np.float64)
    rng = np.random.default_rng(seed)
    Q = random_orthogonal(eigs.size, rng)
    A = (Q * eigs) @ Q.T
    A = 0.5 * (A + A.T)
    return A, Q


def rademacher(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` Rademacher probe vectors (entries +-1) as an (n, count) float64 array."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random((n, count)) < 0.5, -1.0, 1.0)


def gp_targets(X: np.ndarray, seed: int = 0) -> np.ndarray:
    """Regression targets ``y = sin(6 x_0) + 0.1 eps`` for the gradient workload."""
    rng = np.random.default_rng(seed + 1)
    return np.sin(6.0 * X[:, 0]) + 0.1 * rng.standard_normal(X.shape[0])


def classification_data(n: int, d: int, seed: int = 0, spread: float = 0.15, latent: int = 0,
                        latent_spread: float = 0.15):
    """Binary classification inputs in the shape of the Sec. 3 experiment
    (images of two digits, pixel values in [0, 1], labels +-1): two classes
    around seeded centres in [0.3, 0.7]^d with Gaussian spread, clipped to
    [0, 1], labels alternating +1, -1. A synthetic stand-in for the infinite
    MNIST threes and fives, which are not available here.

    With ``latent`` > 0 each class also varies along its own ``latent``
    seeded directions (coordinates N(0, latent_spread^2) per direction after
    a 1/sqrt(latent) scaling of the directions), with ``spread`` then the
    isotropic noise: images of a digit lie near a low-dimensional manifold,
    which spreads the kernel's spectrum the way real digits do (isotropic
    noise alone in many dimensions makes all distances nearly equal).
    The draws with latent = 0 are unchanged. Returns X (n, d) float64 and y
    (n,) float64."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.3, 0.7, size=(2, d))
    y = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    cls = (y < 0).astype(int)
    X = centres[cls] + spread * rng.standard_normal((n, d))
    if latent > 0:
        dirs = rng.standard_normal((2, latent, d)) / np.sqrt(latent)
        z = latent_spread * rng.standard_normal((n, latent))
        X = X + np.einsum("nl,nld->nd", z, dirs[cls])
    return np.clip(X, 0.0, 1.0), y
