"""Benchmark: time-to-1e-6-residual per sequence of def-CG (k = 32 recycled
harmonic Ritz vectors from the last 64 directions) vs plain CG on the stored
dense FP32 workload: 20 RBF systems A_t = K_t + 1e-3 I, n = 16384, X ~ N(0,1)
in R^{16384 x 16}, lengthscale l_t = 0.8 (1 + 0.05 t), b_t ~ N(0,1).

A step is one whole sequence (A1-A9 of the hot path): per system, form A_t on
the GPU, solve with def-CG (start-of-solve product, projection, the
graph-captured loop, true-residual confirmation) and extract the next W by
harmonic Ritz (overlapped with forming the next operator). The metric is the
whole step; the solve-only time is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: replicas only (independent sequences per rank, no collective).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import dcg_synth as S  # noqa: E402

METRIC = "time-to-1e-6-residual per sequence and matvecs/sec, def-CG vs plain CG, % of roofline"
CFG = S.DENSE_16384
FALLBACK_HBM_GBS = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of floats over the ranks of the default process
    group (the values unchanged on one rank or without a group)."""
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def per_replica(seq_s, world):
    """Seconds per sequence for N replicas: N sequences finish per timed step."""
    return seq_s / world


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_sequence(P, torch, solver, Xd, bs_dev, A, T, deflate, ev_pool, side=None, forms=None):
    """One sequence; returns per-system infos and device-timed (form, solve) ms.

    With a side stream and deflation, A_{t+1} is formed on the side stream
    while the harmonic-Ritz update of system t runs on the solver's stream
    (dcg_update_subspace_async: the update reads W, AW and the stored
    directions, never A; the next solve waits for both). The solve times then
    include the update, and the form times overlap them."""
    infos = []
    stream = torch.cuda.current_stream()
    fs, fe, ss, se = (ev_pool[i * T:(i + 1) * T] for i in range(4))
    overlap = side is not None and deflate
    fs[0].record(stream)
    P.form_rbf_dense(Xd, CFG.lengthscale(0), CFG.signal_var, CFG.noise, out=A)
    fe[0].record(stream)
    for t in range(T):
        solver.set_operator_dense(A, symmetric=True)   # k_form_rbf writes A exactly symmetric
        ss[t].record(stream)
        x, info = solver.solve(bs_dev[t])
        infos.append(info)
        if overlap:
            side.wait_stream(stream)      # the solve is complete (A free); the update is not waited for
            solver.update_subspace(wait=False)
            if forms is not None:         # waits for the update (untimed passes only)
                forms.append(solver.pencil_form())
            se[t].record(stream)
            if t + 1 < T:
                fs[t + 1].record(side)
                P.form_rbf_dense(Xd, CFG.lengthscale(t + 1), CFG.signal_var, CFG.noise, out=A, stream=side)
                fe[t + 1].record(side)
                stream.wait_stream(side)
        else:
            if deflate:
                solver.update_subspace()
            se[t].record(stream)
            if t + 1 < T:
                fs[t + 1].record(stream)
                P.form_rbf_dense(Xd, CFG.lengthscale(t + 1), CFG.signal_var, CFG.noise, out=A)
                fe[t + 1].record(stream)
    solver.sync()                          # a pending update of the last system
    torch.cuda.synchronize()
    form_ms = sum(fs[t].elapsed_time(fe[t]) for t in range(T))
    solve_ms = sum(ss[t].elapsed_time(se[t]) for t in range(T))
    return infos, form_ms, solve_ms


def launches_of(infos, deflate):
    total = 0
    for i in infos:
        checks = i["matvecs_check"] - (1 if i["status"] != 0 else 0)
        fin = 1 if i["status"] != 0 else 0
        total += 1                       # form A_t
        total += 8 + 1                   # start of solve + loop gate
        total += 4 * i["iters"] + 3 * checks   # symmetric matvec (2 launches), fused kernel, gate
        total += 2 + fin                 # final gate, final residual, finalize
        if deflate:
            total += 9                   # harmonic Ritz extraction (with the float64 refinement)
    return total


def gpu_arm(args):
    import torch

    import paper_1706_00241_gb300 as P
    from paper_1706_00241_gb300 import build as B

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    # solver stream at high priority, so that the one-CTA eigen-solve of an
    # overlapped update gets an SM ahead of the next operator's formation,
    # which runs on the (default-priority) side stream
    main = torch.cuda.Stream(priority=-1)
    torch.cuda.set_stream(main)
    side = torch.cuda.Stream()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()
    n, T = CFG.n, (args.systems if args.systems else CFG.T)
    X, bs = S.draw_sequence(CFG, T=T)
    X32 = X.astype(np.float32)
    b32 = [b.astype(np.float32) for b in bs]
    Xd = torch.tensor(X32, device="cuda")
    bs_dev = [torch.tensor(b, device="cuda") for b in b32]
    A = torch.empty((n, n), dtype=torch.float32, device="cuda")
    ev_pool = [torch.cuda.Event(enable_timing=True) for _ in range(4 * T)]

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def make(deflate, fg_form="explicit"):
        return P.DefCG(n, CFG.k if deflate else 0, CFG.ell if deflate else 0, CFG.tol,
                       max_iter=20000, window="last", select="largest", host_loop=args.host_loop, fg_form=fg_form)

    # warm-up (builds the graph, first-touch of buffers)
    solver = make(True)
    for _ in range(args.warmup):
        solver.set_subspace(torch.zeros((0, n), device="cuda"))
        run_sequence(P, torch, solver, Xd, bs_dev, A, T, True, ev_pool, side)

    # timed region: K whole sequences
    seq_solve_ms, seq_form_ms, all_infos = [], [], []
    with ClockSampler(local) as clk:
        barrier()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record()
        for _ in range(args.steps):
            solver.set_subspace(torch.zeros((0, n), device="cuda"))
            infos, fm, sm = run_sequence(P, torch, solver, Xd, bs_dev, A, T, True, ev_pool, side)
            seq_solve_ms.append(sm)
            seq_form_ms.append(fm)
            all_infos.append(infos)
        t_end.record()
        barrier()
    step_ms = t_start.elapsed_time(t_end) / args.steps
    solve_ms_mean = float(np.mean(seq_solve_ms))
    solve_ms_mean, step_ms = max_over_ranks([solve_ms_mean, step_ms], device="cuda")
    infos = all_infos[-1]
    loop_mv = sum(i["iters"] for i in infos)
    check_mv = sum(i["matvecs_check"] for i in infos)
    setup_cols = sum(i["matvecs_setup"] for i in infos)
    ok = all(i["status"] == 0 and i["relres_true"] <= CFG.tol for i in infos)

    # plain CG on the same sequence (same GPU, same kernels, k = 0)
    plain = make(False)
    run_sequence(P, torch, plain, Xd, bs_dev, A, T, False, ev_pool)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record()
    pinfos, _, plain_solve_ms = run_sequence(P, torch, plain, Xd, bs_dev, A, T, False, ev_pool)
    pe1.record()
    torch.cuda.synchronize()
    plain_ms = pe0.elapsed_time(pe1)   # whole sequence: forming A_t and solving
    plain_mv = sum(i["iters"] + i["matvecs_check"] for i in pinfos)
    plain.close()

    # def-CG with the sparse F, G of Sec. 2.3 on the same sequence: one
    # untimed pass that also records which form each update took, one timed
    sparse = make(True, "sparse")
    forms = []
    run_sequence(P, torch, sparse, Xd, bs_dev, A, T, True, ev_pool, side, forms=forms)
    sparse.set_subspace(torch.zeros((0, n), device="cuda"))
    se0, se1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    se0.record()
    sinfos, _, _ = run_sequence(P, torch, sparse, Xd, bs_dev, A, T, True, ev_pool, side)
    se1.record()
    torch.cuda.synchronize()
    sparse_ms = se0.elapsed_time(se1)
    sparse.close()

    # roofline of the dominant kernel: the symmetric TMA matvec q = A p (two
    # launches, k_symv_tma and k_symv_fin, timed together), CUDA events on the
    # solver's stream, same launch configuration as in the loop
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    p = bs_dev[0].clone()
    q = torch.empty_like(p)
    P.form_rbf_dense(Xd, CFG.lengthscale(T - 1), CFG.signal_var, CFG.noise, out=A)
    solver.set_operator_dense(A, symmetric=True)
    for _ in range(3):
        solver.matvec(p, q, want_pAp=False)
    reps = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        solver.matvec(p, q, want_pAp=False)
    e1.record(stream)
    torch.cuda.synchronize()
    gemv_ms = e0.elapsed_time(e1) / reps
    gemv_bytes = 2.0 * n * (n + 1) + 8.0 * n  # the upper triangle once, p read and q written
    achieved = gemv_bytes / (gemv_ms * 1e-3) / 1e9

    # end to end through the public API with host buffers: X and b_t from
    # pinned host memory, x_t back to pinned host memory, inside the timing
    Xh = torch.tensor(X32).pin_memory()
    bh = [torch.tensor(b).pin_memory() for b in b32]
    xh = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(T)]
    solver.set_subspace(torch.zeros((0, n), device="cuda"))
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    Xd2 = Xh.to("cuda", non_blocking=True)
    e2e_infos = []
    cur = torch.cuda.current_stream()
    P.form_rbf_dense(Xd2, CFG.lengthscale(0), CFG.signal_var, CFG.noise, out=A)
    for t in range(T):
        solver.set_operator_dense(A, symmetric=True)
        bd = bh[t].to("cuda", non_blocking=True)
        x, info = solver.solve(bd)
        xh[t].copy_(x, non_blocking=True)
        side.wait_stream(cur)
        solver.update_subspace(wait=False)
        if t + 1 < T:
            P.form_rbf_dense(Xd2, CFG.lengthscale(t + 1), CFG.signal_var, CFG.noise, out=A, stream=side)
            cur.wait_stream(side)
        e2e_infos.append(info)
    solver.sync()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - w0
    solver.close()

    traffic = None
    tf = os.path.join(ROOT, "profiles", "symv_dense_n16384.md")
    if os.path.exists(tf):
        for line in open(tf):
            if line.startswith("dram_bytes_per_launch:"):
                try:
                    traffic = float(line.split(":")[1])
                except ValueError:
                    traffic = None

    # the timed step is one whole sequence: forming each A_t and solving it
    seq_s = step_ms / 1e3
    solve_s = solve_ms_mean / 1e3
    value = per_replica(seq_s, world)
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "s/sequence",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded dcg_synth draws standing in for the paper's MNIST workload)",
        "config": {
            "workload": CFG.name, "n": n, "d": CFG.d, "systems": T, "k": CFG.k, "ell": CFG.ell,
            "window": "last", "tol": CFG.tol, "operator": "stored dense fp32 (1 GiB > L2)",
            "l2": "inputs larger than L2 (A is 1 GiB per system)", "parallelism": f"replicas x{world}",
            "launch": "host loop (profiling mode)" if args.host_loop else "one CUDA graph per solve",
            **({"systems_override": T} if args.systems else {}),
        },
        "defcg": {
            "s_per_sequence": seq_s, "solve_s_per_sequence": solve_s, "iters": loop_mv,
            "check_matvecs": check_mv, "setup_columns": setup_cols,
            "matvecs_per_s": (loop_mv + check_mv) / solve_s,
            "all_converged": ok, "iters_per_system": [i["iters"] for i in infos],
            "form_ms_per_sequence": float(np.mean(seq_form_ms)),
        },
        "plain_cg": {
            "s_per_sequence": plain_ms / 1e3, "solve_s_per_sequence": plain_solve_ms / 1e3,
            "iters": sum(i["iters"] for i in pinfos), "matvecs_per_s": plain_mv / (plain_solve_ms / 1e3),
            "iters_per_system": [i["iters"] for i in pinfos],
        },
        "speedup_vs_plain_cg": (plain_ms / 1e3) / seq_s,
        "defcg_sparse_fg": {
            "what": "def-CG with F, G of Eq. 7 from the recorded scalars (Sec. 2.3, fg_form sparse); "
                    "one timed sequence",
            "s_per_sequence": sparse_ms / 1e3, "iters": sum(i["iters"] for i in sinfos),
            "iters_per_system": [i["iters"] for i in sinfos],
            "all_converged": all(i["status"] == 0 and i["relres_true"] <= CFG.tol for i in sinfos),
            "updates_sparse": sum(f == "sparse" for f in forms), "updates": len(forms),
        },
        "roofline": {
            "kernel": "k_symv_tma + k_symv_fin (q = A p from the upper triangle, fused p^T q)",
            "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "peak_kind": peak_kind, "traffic": traffic,
            "algorithmic_bytes_per_launch": gemv_bytes, "launch_ms": gemv_ms,
        },
        "e2e": {
            "value": e2e_s, "unit": "s/sequence",
            "h2d_bytes_per_step": int(X32.nbytes + T * n * 4),
            "d2h_bytes_per_step": int(T * n * 8),
        },
        "gpu_launches": launches_of(infos, True) * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and args.matrix_free != "none":
        out["matrix_free"] = matrix_free_block(P, torch, args.matrix_free)
    if rank == 0 and world == 1 and not args.no_paper:
        out["paper_experiment"] = paper_block(P, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(samples=2)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# ---------------------------------------------------------------------------
# Matrix-free workloads (BF16 n = 131072 sequence; TF32 n = 262144 kernels)
# ---------------------------------------------------------------------------
def ex2_peak(P):
    """Exponentials per second of the special-function units, measured now by
    the library's probe (dcg_measure_ex2_rate)."""
    import ctypes
    lib = P.load()
    ps, pc = ctypes.c_double(), ctypes.c_double()
    st = lib.dcg_measure_ex2_rate(None, ctypes.byref(ps), ctypes.byref(pc))
    if st != 0:
        return None, None
    return ps.value, pc.value


def mf_kernels(P, torch, cfg, fmt, ex2_ps):
    """The matvec and the exact-form true residual of a matrix-free workload at
    full size, CUDA events over repeated launches on the current stream."""
    X, bs = S.draw_sequence(cfg, T=2)
    n = cfg.n
    stream = torch.cuda.current_stream()
    with P.DefCG(n, 0, 0, cfg.tol) as s:
        s.set_operator_rbf(torch.tensor(X.astype(np.float32), device="cuda"), cfg.lengthscale(0), cfg.signal_var,
                           cfg.noise, xformat=fmt)
        p = torch.tensor(bs[0].astype(np.float32), device="cuda")
        q = torch.empty_like(p)
        x = torch.tensor(bs[1], device="cuda")

        def timed(fn, reps):
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        mv_ms = timed(lambda: s.matvec(p, q, want_pAp=False), 10)
        res_ms = timed(lambda: s.residual(p, x), 3)
    entries = float(n) * n
    dk = cfg.d * (3 if fmt == "fp32" else 1) + 3     # coordinates of a tile row (with -|x|^2/2)
    kpad = (dk + 15) // 16 * 16 if fmt == "bf16" else (dk + 7) // 8 * 8
    tflops = 2.0 * entries * kpad / (mv_ms * 1e-3) / 1e12
    tpeak, _ = tensor_peak(fmt)
    # the symmetric kernel forms each tile pair (I, J >= I) once: the
    # exponentials it needs are the tiles on and above the diagonal
    nt = (n + 127) // 128
    exps = 128.0 * 128.0 * nt * (nt + 1) / 2
    tflops *= exps / entries
    out = {"n": n, "d": cfg.d, "x_format": fmt,
           "matvec": {"kernel": "k_rbf_mv_sym + k_rbf_mv_fin (tcgen05 Gram tiles of the pairs J >= I, exp on "
                                "the SFU, row and column contractions)",
                      "launch_ms": mv_ms, "entries_per_s": entries / (mv_ms * 1e-3),
                      "exponentials_per_launch": exps,
                      "tensor_tflops": tflops, "tensor_frac": tflops / tpeak},
           "true_residual": {"kernel": "k_rbf_resid + k_rbf_resid_fin (exact-form entries, Dot2 sums)",
                             "launch_ms": res_ms, "matvec_equivalents": res_ms / mv_ms}}
    if ex2_ps:
        achieved = exps / (mv_ms * 1e-3)
        out["matvec"]["roofline"] = {"bound": "sfu", "achieved": achieved, "peak": ex2_ps, "unit": "exp2/s",
                                     "frac": achieved / ex2_ps,
                                     "peak_kind": "measured now (dcg_measure_ex2_rate)"}
    return out


def mf_sequence(P, torch, cfg, deflate):
    """One whole matrix-free sequence (set the lengthscale l_t, solve, extract
    the next W asynchronously), CUDA events around the sequence."""
    X, bs = S.draw_sequence(cfg)
    n = cfg.n
    bd = [torch.tensor(b.astype(np.float32), device="cuda") for b in bs]
    solver = P.DefCG(n, cfg.k if deflate else 0, cfg.ell if deflate else 0, cfg.tol, max_iter=20000,
                     refine_every=cfg.refine_every)
    solver.set_operator_rbf(torch.tensor(X.astype(np.float32), device="cuda"), cfg.lengthscale(0),
                            cfg.signal_var, cfg.noise, xformat=cfg.x_dtype)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    torch.cuda.synchronize()
    e0.record(stream)
    for t in range(cfg.T):
        solver.set_rbf_params(cfg.lengthscale(t), cfg.signal_var, cfg.noise)
        _, info = solver.solve(bd[t], raise_on_error=False)
        infos.append(info)
        if deflate:
            solver.update_subspace(wait=False)
    solver.sync()
    e1.record(stream)
    torch.cuda.synchronize()
    solver.close()
    secs = e0.elapsed_time(e1) / 1e3
    return {"s_per_sequence": secs, "iters": sum(i["iters"] for i in infos),
            "check_matvecs": sum(i["matvecs_check"] for i in infos),
            "setup_columns": sum(i["matvecs_setup"] for i in infos),
            "all_converged": all(i["status"] == 0 and i["relres_true"] <= cfg.tol for i in infos),
            "iters_per_system": [i["iters"] for i in infos],
            "checks_per_system": [i["matvecs_check"] for i in infos]}


# The paper's experiment at its size (Sec. 3): n = 36551 images of d = 784
# pixels, Newton for the Laplace mode with def-CG(8, 12) or CG on every
# system, relative residual 1e-5, stop when Psi rises by less than 1. The
# infinite-MNIST threes and fives are not available: the stand-in draws two
# classes near 4-dimensional manifolds (dcg_synth.classification_data with
# latent = 4); the paper does not state its kernel hyperparameters, the
# stand-in uses l = 3, theta^2 = 9 (first system: ~30 CG iterations).
PAPER_N, PAPER_D = 36551, 784
PAPER_DATA = {"spread": 0.03, "latent": 4, "latent_spread": 0.15}
PAPER_L, PAPER_S2 = 3.0, 9.0
PAPER_TABLE1 = {"cholesky_s": 4317.0, "cg_s": 1821.0, "defcg_s": 1571.0,
                "hardware": "CPU, unspecified (paper, Table 1: cumulative after 9 Newton systems)"}


def paper_block(P, torch):
    X, y = S.classification_data(PAPER_N, PAPER_D, seed=0, **PAPER_DATA)
    n = PAPER_N
    ldk = (n + 3) // 4 * 4
    Xd = torch.tensor(X.astype(np.float32), device="cuda")
    yd = torch.tensor(y.astype(np.float32), device="cuda")
    K = torch.empty((n, ldk), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    P.form_rbf_dense(Xd, PAPER_L, PAPER_S2, 0.0, out=K)
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"n": n, "d": PAPER_D, "lengthscale": PAPER_L, "signal_var": PAPER_S2, "tol": 1e-5,
           "data": "two seeded classes near 4-dimensional manifolds in [0,1]^784 (stand-in for infinite MNIST 3 vs 5)",
           "form_K_ms": e0.elapsed_time(e1), "paper_table1_context": PAPER_TABLE1}
    for name, k, ell in (("defcg", 8, 12), ("cg", 0, 0)):
        with P.DefCG(n, k, ell, 1e-5, max_iter=5000) as s:
            P.laplace_mode(s, K, yd, dpsi_tol=1.0)          # warm-up: graph, scratch, first launches
            s.set_subspace(torch.zeros((0, n), device="cuda"))
            e0.record(stream)
            f, a, h, infos = P.laplace_mode(s, K, yd, dpsi_tol=1.0)
            e1.record(stream)
            torch.cuda.synchronize()
            out[name] = {"s_total": e0.elapsed_time(e1) / 1e3, "newton_steps": len(infos),
                         "iters_per_system": [i["iters"] for i in infos], "psi_final": h[-1],
                         "all_converged": all(i["status"] == 0 and i["relres_true"] <= 1e-5 for i in infos)}
    out["speedup_vs_cg"] = out["cg"]["s_total"] / out["defcg"]["s_total"]
    return out


def matrix_free_block(P, torch, mode):
    ex2_ps, ex2_pc = ex2_peak(P)
    out = {"ex2_peak": {"per_s": ex2_ps, "per_clock_per_sm": ex2_pc, "kind": "measured now (dcg_measure_ex2_rate)"}}
    c3, c5 = S.MF_131072, S.MF_262144
    out[c3.name] = mf_kernels(P, torch, c3, c3.x_dtype, ex2_ps)
    out[c5.name] = mf_kernels(P, torch, c5, c5.x_dtype, ex2_ps)
    if mode == "all":
        d = mf_sequence(P, torch, c3, True)
        pl = mf_sequence(P, torch, c3, False)
        out[c3.name].update({"defcg": d, "plain_cg": pl,
                             "speedup_vs_plain_cg": pl["s_per_sequence"] / d["s_per_sequence"],
                             "sequence": f"{c3.T} systems, k = {c3.k}, ell = {c3.ell}, refinement every "
                                         f"{c3.refine_every}, tol {c3.tol}"})
    return out


# ---------------------------------------------------------------------------
# Gradient workload (opt-in): Adam on the GP hyperparameters through def-CG
# solves of the matrix-free operator, n = 32768, d = 8, 16 probes per step
# ---------------------------------------------------------------------------
def gradient_arm(args):
    import torch

    import paper_1706_00241_gb300 as P
    from paper_1706_00241_gb300 import build as B

    torch.cuda.set_device(0)
    B.build()
    cfg = S.GRAD_32768
    n = args.n if args.n else cfg.n
    X, bs = S.draw_sequence(cfg, T=1)
    Xd = torch.tensor(X[:n].astype(np.float32), device="cuda")
    y = torch.tensor(bs[0][:n].astype(np.float32), device="cuda")
    theta0 = (cfg.l0, cfg.signal_var, cfg.noise)
    out = {"workload": cfg.name, "n": n, "d": cfg.d, "adam_steps": args.gradient_steps,
           "probes": cfg.extra["probes"], "tol": cfg.tol, "refine_every": 50, "x_format": "bf16",
           "per_step": "1 forward + 1 adjoint + 16 probe solves (in lockstep: one operator pass per iteration "
                       "for all probes still iterating), one derivative-form pass each"}
    short = max(1, args.gradient_steps // 10)
    # probes in lockstep (dcg_solve_multi) unless the run's name says otherwise
    runs = (("defcg", cfg.k, cfg.ell, args.gradient_steps, True),
            ("defcg_first_steps", cfg.k, cfg.ell, short, True),
            ("defcg_first_steps_probes_one_by_one", cfg.k, cfg.ell, short, False),
            ("plain_cg", 0, 0, short, True))
    for name, k, ell, steps, block in runs:
        s = P.DefCG(n, k, ell, cfg.tol, refine_every=50, max_iter=20000)
        s.set_operator_rbf(Xd, *theta0, xformat="bf16")
        iters = []
        orig_solve, orig_multi = s.solve, s.solve_multi

        def counted(b, x=None, _f=orig_solve):
            r = _f(b, x) if x is not None else _f(b)
            iters.append(r[1]["iters"] + r[1]["matvecs_check"])
            return r

        def counted_multi(B, X=None, _f=orig_multi):
            r = _f(B, X) if X is not None else _f(B)
            iters.extend(i["iters"] + i["matvecs_check"] for i in r[1])
            return r
        s.solve, s.solve_multi = counted, counted_multi
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        path, grads = P.fit_gp(s, y, theta0, steps=steps, lr=cfg.extra["adam_lr"], probes=cfg.extra["probes"],
                               block_probes=block)
        torch.cuda.synchronize()
        dt = time.perf_counter() - w0
        s.close()
        out[name] = {"steps": steps, "s_total": dt, "s_per_step": dt / steps, "solves": len(iters),
                     "matvecs": int(sum(iters)), "matvecs_per_step": sum(iters) / steps,
                     "theta_final": [float(v) for v in path[-1]]}
    # the same first steps of the Adam path (the systems change along it)
    out["speedup_first_steps_vs_plain_cg"] = out["plain_cg"]["s_total"] / out["defcg_first_steps"]["s_total"]
    out["speedup_lockstep_probes"] = (out["defcg_first_steps_probes_one_by_one"]["s_total"]
                                      / out["defcg_first_steps"]["s_total"])
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# Kernel-only mode: one hot kernel on its own (for ncu captures of a small case)
# ---------------------------------------------------------------------------
def kernel_arm(args):
    import torch

    import paper_1706_00241_gb300 as P
    from paper_1706_00241_gb300 import build as B

    torch.cuda.set_device(0)
    B.build()
    stream = torch.cuda.current_stream()
    if args.kernel in ("gemv", "symv"):
        n = args.n or CFG.n
        X, bs = S.draw_sequence(CFG.scaled(n, T=1) if n != CFG.n else CFG, T=1)
        Xd = torch.tensor(X.astype(np.float32), device="cuda")
        A = torch.empty((n, n), dtype=torch.float32, device="cuda")
        P.form_rbf_dense(Xd, CFG.lengthscale(0), CFG.signal_var, CFG.noise, out=A)
        solver = P.DefCG(n, 0, 0, CFG.tol)
        sym = args.kernel == "symv"
        solver.set_operator_dense(A, symmetric=sym)
        if sym:   # the upper triangle with its diagonal, p read, q written
            algo = 2.0 * n * (n + 1) + 8.0 * n
            name = "k_symv_tma + k_symv_fin (q = A p from the upper triangle, fused p^T q)"
        else:
            algo = 4.0 * n * n + 8.0 * n
            name = "k_rowop_tma<false> (q = A p, fused p^T q)"
        unit, bound = "GB/s", "hbm"
        peak, kind = peaks()
        workload = f"stored dense fp32 n={n}"
    elif args.kernel in ("apply_block", "form", "iter"):
        return kernel_arm_dense(args, P, torch, stream)
    elif args.kernel == "multi":
        return kernel_arm_multi(args, P, torch)
    elif args.kernel == "resid":
        # the exact-form true residual of the matrix-free operator (k_rbf_resid
        # + k_rbf_resid_fin), on the bf16 n = 131072 workload's generator
        cfg = S.MF_131072 if args.xformat == "bf16" else S.MF_262144
        n = args.n or cfg.n
        X, bs = S.draw_sequence(cfg.scaled(n, T=2) if n != cfg.n else cfg, T=2)
        solver = P.DefCG(n, 0, 0, cfg.tol)
        solver.set_operator_rbf(torch.tensor(X.astype(np.float32), device="cuda"), cfg.lengthscale(0),
                                cfg.signal_var, cfg.noise, xformat=args.xformat)
        b = torch.tensor(bs[1].astype(np.float32), device="cuda")
        x = torch.tensor(bs[0], device="cuda")
        for _ in range(args.warmup):
            solver.residual(b, x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            solver.residual(b, x)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        solver.close()
        print(json.dumps({"kernel": "k_rbf_resid + k_rbf_resid_fin (exact-form true residual)",
                          "workload": f"matrix-free rbf n={n} d={cfg.d} {args.xformat}", "launch_ms": ms,
                          "launches": args.steps, "entries_per_s": float(n) * n / (ms * 1e-3)}))
        return
    else:
        cfg = S.MF_131072 if args.xformat == "bf16" else S.MF_262144
        n = args.n or cfg.n
        rng = np.random.default_rng(0)
        X = rng.standard_normal((n, cfg.d)).astype(np.float32)
        Xd = torch.tensor(X, device="cuda")
        solver = P.DefCG(n, 0, 0, cfg.tol)
        solver.set_operator_rbf(Xd, cfg.lengthscale(0), cfg.signal_var, cfg.noise, xformat=args.xformat)
        dk = cfg.d * (3 if args.xformat == "fp32" else 1) + 3   # tile-row coordinates (with -|x|^2/2)
        dpad = (dk + 15) // 16 * 16 if args.xformat == "bf16" else (dk + 7) // 8 * 8
        nt = (n + 127) // 128
        algo = 2.0 * (128.0 * 128.0 * nt * (nt + 1) / 2) * dpad   # Gram FLOPs of the tile pairs J >= I
        name = "k_rbf_mv_sym + k_rbf_mv_fin (tcgen05 Gram tiles of the pairs J >= I, fused exp and contractions)"
        unit, bound = "TFLOP/s", "tensor"
        peak, kind = tensor_peak(args.xformat)
        workload = f"matrix-free rbf n={n} d={cfg.d} {args.xformat}"
    p = torch.tensor(np.random.default_rng(1).standard_normal(n).astype(np.float32), device="cuda")
    q = torch.empty_like(p)
    for _ in range(args.warmup):
        solver.matvec(p, q, want_pAp=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        solver.matvec(p, q, want_pAp=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    scale = 1e9 if unit == "GB/s" else 1e12
    achieved = algo / (ms * 1e-3) / scale
    solver.close()
    print(json.dumps({"kernel": name, "workload": workload, "launch_ms": ms, "launches": args.steps,
                      "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                                   "frac": achieved / peak, "peak_kind": kind,
                                   "algorithmic_per_launch": algo}}))


def kernel_arm_multi(args, P, torch):
    """One lockstep solve (dcg_solve_multi) of the gradient workload's probes:
    n = 32768, d = 8, BF16 points, k = 32, refinement every 50, W from one
    solve of the targets and its update; --cols probes (default 16). Times
    the lockstep solve (median of --steps after --warmup, wall clock: the
    loop is driven from the host) and the same probes solved one after
    another, for profiling captures of its kernels (k_rbf_mv_tc,
    k_rbf_resid_multi)."""
    cfg = S.GRAD_32768
    n = args.n or cfg.n
    X, _ = S.draw_sequence(cfg.scaled(n, T=1) if n != cfg.n else cfg, T=1)
    nprobe = args.cols or cfg.extra["probes"]
    Xd = torch.tensor(X.astype(np.float32), device="cuda")
    y = torch.tensor(S.gp_targets(X).astype(np.float32), device="cuda")
    Z = torch.tensor(np.ascontiguousarray(S.rademacher(n, nprobe, seed=1000).T.astype(np.float32)), device="cuda")
    with P.DefCG(n, cfg.k, cfg.ell, cfg.tol, refine_every=50, max_iter=20000) as s:
        s.set_operator_rbf(Xd, cfg.l0, cfg.signal_var, cfg.noise, xformat="bf16")
        s.solve(y)
        s.update_subspace()
        for _ in range(args.warmup):          # also allocates the per-system buffers
            s.solve_multi(Z)
        times = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            _, infos = s.solve_multi(Z)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - w0)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        single = [s.solve(Z[c].contiguous())[1] for c in range(nprobe)]
        torch.cuda.synchronize()
        t_single = time.perf_counter() - w0
    t_multi = statistics.median(times)
    its = [i["iters"] for i in infos]
    print(json.dumps({"kernel": "dcg_solve_multi (lockstep: k_rbf_mv_tc block product, k_iter_fused per system, "
                                "k_rbf_resid_multi checks)",
                      "workload": f"{cfg.name}: {nprobe} Rademacher probes, n={n}, d={cfg.d}, bf16, k={cfg.k}",
                      "s_lockstep": t_multi, "s_one_by_one": t_single, "speedup": t_single / t_multi,
                      "iters_max": max(its), "ms_per_lockstep_iteration": 1e3 * t_multi / max(its),
                      "iters": its, "iters_one_by_one": [i["iters"] for i in single],
                      "all_converged": all(i["status"] == 0 for i in infos)}))


def kernel_arm_dense(args, P, torch, stream):
    """Single-kernel timing on the stored workload, for profiling:
    apply_block: Y = A W with 32 columns (k_apply_block); form: A = K + sigma^2 I
    (k_form_rbf); iter: system 1 of the sequence solved in host-loop mode
    after system 0 and its update (its k_iter_fused launches are the ones a
    profiler captures; the line reports the solve)."""
    n = args.n or CFG.n
    X, bs = S.draw_sequence(CFG.scaled(n, T=2) if n != CFG.n else CFG, T=2)
    Xd = torch.tensor(X.astype(np.float32), device="cuda")
    A = torch.empty((n, n), dtype=torch.float32, device="cuda")
    P.form_rbf_dense(Xd, CFG.lengthscale(0), CFG.signal_var, CFG.noise, out=A)
    hz = 2.07e9
    if args.kernel == "iter":
        solver = P.DefCG(n, CFG.k, CFG.ell, CFG.tol, window="last", select="largest", host_loop=True)
        solver.set_operator_dense(A)
        solver.solve(torch.tensor(bs[0].astype(np.float32), device="cuda"))
        solver.update_subspace()
        P.form_rbf_dense(Xd, CFG.lengthscale(1), CFG.signal_var, CFG.noise, out=A)
        solver.set_operator_dense(A)
        b1 = torch.tensor(bs[1].astype(np.float32), device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = solver.solve(b1)
        e1.record(stream)
        torch.cuda.synchronize()
        solver.close()
        print(json.dumps({"kernel": "k_iter_fused (inside a host-loop solve)", "workload": f"stored dense fp32 n={n}, "
                          f"system 1, k={CFG.k}", "solve_ms": e0.elapsed_time(e1), "iters": info["iters"],
                          "status": info["status"]}))
        return
    if args.kernel == "apply_block":
        solver = P.DefCG(n, 0, 0, CFG.tol)
        lda = (n + 3) // 4 * 4    # rows start on 16-byte boundaries (TMA)
        if lda != n:
            Ap = torch.zeros((n, lda), dtype=torch.float32, device="cuda")
            Ap[:, :n] = A
            A = Ap
        solver.set_operator_dense(A, lda)
        cols = args.cols or CFG.k
        V = torch.tensor(np.random.default_rng(1).standard_normal((cols, n)).astype(np.float32), device="cuda")
        fn = lambda: solver.apply_block(V)
        if cols >= 32:
            algo, unit, bound = 2.0 * n * n * cols, "TFLOP/s", "alu"
            peak, kind = 152 * 128 * 2 * hz / 1e12, "nominal FP32 FMA (152 SMs x 128 lanes x 2070 MHz)"
        else:
            # a few columns: A read once bounds it
            algo, unit, bound = 4.0 * n * n, "GB/s", "hbm"
            peak, kind = peaks()
        name = f"Y = A W, {cols} columns (k_apply_tc where n % 4 == 0, else k_apply_block)"
    else:
        solver = None
        fn = lambda: P.form_rbf_dense(Xd, CFG.lengthscale(0), CFG.signal_var, CFG.noise, out=A)
        algo, unit, bound = 4.0 * n * n, "GB/s", "hbm"
        peak, kind = peaks()
        name = "k_form_rbf (A = K + sigma^2 I, written once)"
    for _ in range(args.warmup):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    achieved = algo / (ms * 1e-3) / (1e9 if unit == "GB/s" else 1e12)
    if solver is not None:
        solver.close()
    print(json.dumps({"kernel": name, "workload": f"stored dense fp32 n={n}", "launch_ms": ms, "launches": args.steps,
                      "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                                   "frac": achieved / peak, "peak_kind": kind, "algorithmic_per_launch": algo}}))


def tensor_peak(xformat):
    """Dense tensor peak for the operand type: the measured bf16 figure; TF32
    at the nominal tf32/bf16 ratio (1.1 / 2.25) of it."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        bf16 = float(json.load(open(p))["bf16_tflops"])
        kind = "measured"
    else:
        bf16, kind = 1900.0, "fallback"
    if xformat == "bf16":
        return bf16, kind
    return bf16 * 1.1 / 2.25, kind + " (bf16 x nominal tf32/bf16)"


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def _golden_total_matvecs():
    """The oracle's matvec total over the whole sequence, when a stored oracle
    run of this exact workload exists (written by tests/golden/make_golden.py)."""
    gdir = os.path.join(ROOT, "tests", "golden")
    for name in sorted(os.listdir(gdir)) if os.path.isdir(gdir) else []:
        if not name.endswith("_oracle.json"):
            continue
        d = json.load(open(os.path.join(gdir, name)))
        if (d.get("workload") == CFG.name and d.get("tol") == CFG.tol
                and "total_defcg_matvecs" in d):
            return d["total_defcg_matvecs"], f"tests/golden/{name}"
    return None, None


class OracleSample:
    """Oracle inputs for the first systems of the sequence, formed once; the
    formation of each A_t is timed here and added per system to the
    extrapolated sequence time (the GPU step also forms every A_t)."""

    def __init__(self, systems=2):
        from oracle import dcg_oracle as O
        self.O = O
        X, bs = S.draw_sequence(CFG, T=systems)
        X64 = X.astype(np.float32).astype(np.float64)
        self.A, form = [], []
        for t in range(systems):
            w0 = time.perf_counter()
            self.A.append(O.rbf_gram(X64, CFG.lengthscale(t), CFG.signal_var, CFG.noise))
            form.append(time.perf_counter() - w0)
        self.form_s = float(np.mean(form))   # oracle formation of one A_t
        self.b = [b.astype(np.float32).astype(np.float64) for b in bs]
        self.W = [None]
        for t in range(systems - 1):   # the W each sampled system starts from
            res = O.defcg(self.A[t], self.b[t], W=self.W[-1], tol=CFG.tol, ell=CFG.ell, window="last")
            self.W.append(O.harmonic_ritz(res.W, res.AW, res.P, res.Q, CFG.k).W)

    def time_system(self, t):
        O = self.O
        w0 = time.perf_counter()
        res = O.defcg(self.A[t], self.b[t], W=self.W[t], tol=CFG.tol, ell=CFG.ell, window="last")
        O.harmonic_ritz(res.W, res.AW, res.P, res.Q, CFG.k)
        return time.perf_counter() - w0, res.matvecs


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def extrapolate(solve_s, mv, sampled):
    total, src = _golden_total_matvecs()
    if total:
        return solve_s / mv * total, (f"extrapolated by matvec count to the oracle's full-sequence total "
                                      f"{total} ({src})")
    return solve_s * CFG.T / sampled, "extrapolated by system count (no golden)"


def cpu_baseline(samples=2, min_seconds=10.0):
    """Oracle def-CG + harmonic Ritz on systems 0 .. samples-1 of the sequence,
    repeated until at least min_seconds of oracle work is timed, extrapolated
    to the whole sequence by matvec count."""
    smp = OracleSample(samples)
    solve_s, mv, reps = 0.0, 0, 0
    while solve_s < min_seconds:
        for t in range(samples):
            dt, m = smp.time_system(t)
            solve_s += dt
            mv += m
        reps += 1
    est, how = extrapolate(solve_s, mv, samples * reps)
    est += CFG.T * smp.form_s
    return {"value": est, "unit": "s/sequence", "cores": _cores(), "kind": "oracle",
            "sample": f"systems 0..{samples - 1} of the n={CFG.n} sequence, FP64 numpy def-CG + harmonic "
                      f"Ritz, repeated {reps}x ({solve_s:.2f} s, {mv} matvecs), {how}; plus {CFG.T} x the "
                      f"oracle's formation of one A_t ({smp.form_s:.2f} s)"}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    smp = OracleSample(2)
    vals = []
    for s in range(args.warmup + args.steps):
        dt, mv = smp.time_system(1)
        if s >= args.warmup:
            vals.append(extrapolate(dt, mv, 1)[0] + CFG.T * smp.form_s)
    value = float(np.mean(vals))
    how = extrapolate(1.0, 1, 1)[1]
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s/sequence", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": CFG.name, "n": CFG.n, "systems": CFG.T, "k": CFG.k, "ell": CFG.ell},
        "cpu_baseline": {"value": value, "unit": "s/sequence", "cores": _cores(), "kind": "oracle",
                         "sample": f"per step: FP64 numpy def-CG + harmonic Ritz on system 1 of the n={CFG.n} "
                                   "sequence (W recycled from system 0), " + how
                                   + f"; plus {CFG.T} x the oracle's formation of one A_t ({smp.form_s:.2f} s)"},
        "e2e": {"value": value, "unit": "s/sequence", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paper", action="store_true",
                    help="skip the Sec. 3 Laplace-approximation Newton loop at the paper's size (n = 36551, d = 784)")
    ap.add_argument("--matrix-free", choices=["all", "kernels", "none"], default="all",
                    help="after the stored headline: the matrix-free kernels at full size and (all) one whole "
                         "BF16 n = 131072 sequence with def-CG and with plain CG")
    ap.add_argument("--host-loop", action="store_true",
                    help="launch the solve's kernels from the host instead of one CUDA graph "
                         "(profiling mode: ncu cannot list kernels inside conditional graphs)")
    ap.add_argument("--kernel", choices=["gemv", "symv", "rbf_mv", "resid", "apply_block", "form", "iter", "multi"],
                    default=None,
                    help="time one hot kernel alone (q = A p) instead of the sequence")
    ap.add_argument("--cols", type=int, default=None,
                    help="columns of W for --kernel apply_block (default k); probes for --kernel multi (default 16)")
    ap.add_argument("--n", type=int, default=0, help="system size for --kernel (default: the workload's)")
    ap.add_argument("--systems", type=int, default=0,
                    help="solve only the first T systems of the sequence (small profiling captures; "
                         "not a benchmark line)")
    ap.add_argument("--xformat", choices=["bf16", "tf32", "fp32"], default="bf16", help="X format for --kernel rbf_mv")
    ap.add_argument("--gradient", action="store_true",
                    help="instead of the sequence: Adam on the GP hyperparameters through def-CG solves "
                         "(matrix-free, n = 32768, 16 probes per step); def-CG and plain CG also over the "
                         "first tenth of the steps")
    ap.add_argument("--gradient-steps", type=int, default=30)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.kernel:
        kernel_arm(args)
    elif args.gradient:
        gradient_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
