"""Writes stored oracle results used by the GPU parity tests and bench.py.

Calls only ``oracle/`` and ``dcg_synth`` (never the CUDA path). Each golden file
records the workload, the oracle settings and per-system results of def-CG
(Algorithm 1 with harmonic-Ritz recycling, Sec. 2.3) and plain CG.

    python tests/golden/make_golden.py dense_16384     # ~10 min, 1 core-heavy
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


def sequence_golden(cfg: S.RBFSequence, T: int, out_name: str):
    X, bs = S.draw_sequence(cfg, T=T)
    X32 = X.astype(np.float32).astype(np.float64)   # the operator both sides see
    W = None
    rows = []
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


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "dense_16384"
    if which == "dense_16384":
        sequence_golden(S.DENSE_16384, S.DENSE_16384.T, "dense_16384_oracle.json")
    elif which == "small_1024":
        cfg = S.SMALL_1024
        small = S.RBFSequence(**{**cfg.__dict__, "tol": 1e-6})
        sequence_golden(small, cfg.T, "small_1024_tol1e-6_oracle.json")
    else:
        raise SystemExit(f"unknown golden {which}")
