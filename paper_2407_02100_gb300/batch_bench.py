"""Benchmark of batched solves: many independent 3D Poisson problems of
different sizes solved together (one sweep launch per colour over all
problems, CUDA-graph V-cycle, per-problem FP64 CG) against the same problems
solved one after another with the single-problem API.

Default workload: 64 problems, Q3, n drawn per problem uniformly from
{16, 24, ..., 96} (seed 0), independent N(0,1) right-hand sides, FP32
smoother / V-cycle inside FP64 CG to 1e-10.

    python -m paper_2407_02100_gb300.batch_bench [--problems 64] [--precision fp32]
"""
import argparse
import json
import time

import numpy as np
import torch

from . import build, gmg, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=64)
    ap.add_argument("--degree", type=int, default=3)
    ap.add_argument("--nmin", type=int, default=16)
    ap.add_argument("--nmax", type=int, default=96)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--no-sequential", action="store_true")
    a = ap.parse_args()
    build.build()
    prec = gmg.GMG_FP32 if a.precision == "fp32" else gmg.GMG_FP64
    rng = np.random.default_rng(a.seed)
    choices = np.arange(a.nmin, a.nmax + 1, 8)
    ns = [int(x) for x in rng.choice(choices, size=a.problems)]
    nodes = sum((n * a.degree + 1) ** 3 for n in ns)
    B = gmg.Batch(3, a.degree, ns, precision=prec)
    rhs = [inputs.random_nodal(3, a.degree, n, a.seed * 1000 + i) for i, n in enumerate(ns)]
    b = B.pack(rhs, dtype=torch.float64)
    del rhs
    u = B.zeros(dtype=torch.float64)
    ppc = gmg.gmg_batch_autotune(B.h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    u.zero_()
    gmg.gmg_batch_cg_solve(B.h, len(ns), u, b, 1e-10, 100)      # warm-up (captures the graph)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.reps):
        u.zero_()
        st, its, res = gmg.gmg_batch_cg_solve(B.h, len(ns), u, b, 1e-10, 100)
    e1.record()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / a.reps * 1e-3
    out = {"problems": len(ns), "degree": a.degree, "n_cells": ns, "nodes": nodes,
           "precision": a.precision, "ppc": ppc, "batched_s": t_batch,
           "batched_mdofs": nodes / t_batch / 1e6, "iterations_max": max(its),
           "iterations_min": min(its), "rel_residual_max": max(res)}
    if not a.no_sequential:
        # the same problems one after another through the single-problem API
        probs = []
        for i, n in enumerate(ns):
            off, ne, _ = B.layouts[i][0], B.layouts[i][1], None
            probs.append(gmg.Problem(3, a.degree, n, precision=prec))
        sols = [P.zeros(dtype=torch.float64) for P in probs]
        rhs_views = [b[B.layouts[i][0]:B.layouts[i][0] + B.layouts[i][1]] for i in range(len(ns))]
        for P, x, r in zip(probs, sols, rhs_views):
            gmg.cg_gmg_solve(P.h, x, r, 1e-10, 100)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for P, x, r in zip(probs, sols, rhs_views):
            x.zero_()
            gmg.cg_gmg_solve(P.h, x, r, 1e-10, 100)
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        diff = max(float(torch.linalg.vector_norm(x - u[B.layouts[i][0]:B.layouts[i][0] + B.layouts[i][1]])
                         / torch.linalg.vector_norm(x)) for i, x in enumerate(sols))
        out.update({"sequential_s": t_seq, "sequential_mdofs": nodes / t_seq / 1e6,
                    "speedup": t_seq / t_batch, "max_rel_diff_vs_sequential": diff})
        for P in probs:
            P.close()
    print(json.dumps(out))
    B.close()


if __name__ == "__main__":
    main()
