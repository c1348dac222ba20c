"""Writes stored oracle results used by the GPU parity tests and bench.py.

Calls only ``oracle/`` and ``dcg_synth`` (never the CUDA path). Each golden file
records the workload, the oracle settings and per-system results of def-CG
(Algorithm 1 with harmonic-Ritz recycling, Sec. 2.3) and plain CG.

    python tests/golden/make_golden.py dense_16384     # ~15 min, 1 core-heavy
    (also writes dense_16384_oracle_x.npz: the oracle's x for systems 0, 10
    and 19, with a Lanczos condition estimate of each in the JSON)
"""

from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import dcg_synth as S  # noqa: E402
from oracle import dcg_oracle as O  # noqa: E402


def lanczos_kappa(alpha, beta):
    """Condition estimate of A from a plain CG run: the extreme eigenvalues of
    the Lanczos tridiagonal that CG's step lengths and beta build (T_jj =
    1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j);
    at convergence they approximate A's extreme eigenvalues."""
    m = len(alpha)
    Tm = np.zeros((m, m))
    for j in range(m):
        Tm[j, j] = 1.0 / alpha[j] + (beta[j - 1] / alpha[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            Tm[j, j + 1] = Tm[j + 1, j] = np.sqrt(beta[j]) / alpha[j]
    ev = np.linalg.eigvalsh(Tm)
    return float(ev[-1] / ev[0]), float(ev[0]), float(ev[-1])


def sequence_golden(cfg: S.RBFSequence, T: int, out_name: str, keep_x=()):
    X, bs = S.draw_sequence(cfg, T=T)
    X32 = X.astype(np.float32).astype(np.float64)   # the operator both sides see
    W = None
    rows = []
    xs = {}
    t_solve = 0.0
    t_cg = 0.0
    for t in range(T):
        A = O.rbf_gram(X32, cfg.lengthscale(t), cfg.signal_var, cfg.noise)
        b = bs[t].astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        res = O.defcg(A, b, W=W, tol=cfg.tol, ell=cfg.ell, window="last")
        rr = O.harmonic_ritz(res.W, res.AW, res.P, res.Q, cfg.k, select="largest")
        t1 = time.perf_counter()
        cg = O.cg(A, b, tol=cfg.tol)
        t2 = time.perf_counter()
        extra = {}
        if t in keep_x:
            # plain CG through defcg (k = 0 reproduces cg iterate by iterate)
            # keeping every step length, for the Lanczos condition estimate
            full = O.defcg(A, b, tol=cfg.tol, ell=10 ** 9, window="first")
            kappa, lmin, lmax = lanczos_kappa(full.alpha, full.beta)
            extra = {"kappa_lanczos": kappa, "lambda_min_lanczos": lmin, "lambda_max_lanczos": lmax}
            xs[f"x_{t}"] = res.x
        t_solve += t1 - t0
        t_cg += t2 - t1
        W = rr.W
        rows.append({
            "t": t,
            "lengthscale": cfg.lengthscale(t),
            "defcg_iters": res.iters,
            "defcg_matvecs": res.matvecs,
            "defcg_relres_true": res.relres_true,
            "cg_iters": cg.iters,
            "cg_matvecs": cg.matvecs,
            "theta_top": [float(v) for v in rr.theta_selected[:8]],
            "defcg_seconds": t1 - t0,
            "cg_seconds": t2 - t1,
            **extra,
        })
        print(json.dumps(rows[-1]), flush=True)
    out = {
        "workload": cfg.name,
        "n": cfg.n, "d": cfg.d, "T": T, "k": cfg.k, "ell": cfg.ell, "tol": cfg.tol,
        "window": "last", "select": "largest",
        "x": "X ~ N(0,1) drawn by dcg_synth.draw_sequence(seed 0), rounded to float32",
        "oracle": "oracle.dcg_oracle.defcg / harmonic_ritz / cg, float64 numpy",
        "systems": rows,
        "total_defcg_matvecs": int(sum(r["defcg_matvecs"] for r in rows)),
        "total_cg_matvecs": int(sum(r["cg_matvecs"] for r in rows)),
        "defcg_seconds": t_solve,
        "cg_seconds": t_cg,
    }
    with open(os.path.join(HERE, out_name), "w") as f:
        json.dump(out, f, indent=1)
    if xs:
        np.savez_compressed(os.path.join(HERE, out_name.replace(".json", "_x.npz")), **xs)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "dense_16384"
    if which == "dense_16384":
        sequence_golden(S.DENSE_16384, S.DENSE_16384.T, "dense_16384_oracle.json", keep_x=(0, 10, 19))
    elif which == "small_1024":
        cfg = S.SMALL_1024
        small = S.RBFSequence(**{**cfg.__dict__, "tol": 1e-6})
        sequence_golden(small, cfg.T, "small_1024_tol1e-6_oracle.json")
    else:
        raise SystemExit(f"unknown golden {which}")
