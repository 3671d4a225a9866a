"""GMG-PCG time to solution for one problem, FP64 smoother against the FP32
smoother / V-cycle (FFMA kernels, and with the tensor-core TF32 sweep)
inside the same FP64 CG (the outer residual, dot products
and coarse data stay FP64), with iteration counts and the difference between
the two solutions.

    python -m paper_2407_02100_gb300.solve_bench --dim 3 --degree 7 --n 48 --dist normal
"""
import argparse
import json

import torch

from . import build, gmg, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=3)
    ap.add_argument("--degree", type=int, default=7)
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--dist", choices=["normal", "uniform"], default="normal")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--rtol", type=float, default=1e-10)
    a = ap.parse_args()
    build.build()
    rhs = inputs.random_nodal(a.dim, a.degree, a.n, a.seed, a.dist)
    nodes = (a.n * a.degree + 1) ** a.dim
    out = {"dim": a.dim, "degree": a.degree, "n_cells": a.n, "nodes": nodes, "rtol": a.rtol}
    sols = {}
    for name, prec in (("fp64", gmg.GMG_FP64), ("fp64_closure", gmg.GMG_FP64), ("fp32_mixed", gmg.GMG_FP32),
                       ("fp32_tc_mixed", gmg.GMG_FP32_TC), ("fp32_tf32_mixed", gmg.GMG_FP32_TF32)):
        P = gmg.Problem(a.dim, a.degree, a.n, precision=prec)
        # fp64: shared-face sweep where it applies (3D, k >= 3); fp64_closure:
        # every patch residual on its own closure
        gmg.gmg_set_shared_faces(P.h, name != "fp64_closure")
        b = P.to_device(rhs, dtype=torch.float64)
        u = P.zeros(dtype=torch.float64)
        gmg.cg_gmg_solve(P.h, u, b, a.rtol, 200)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            u.zero_()
            _, st = gmg.cg_gmg_solve(P.h, u, b, a.rtol, 200)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        r = P.zeros(dtype=torch.float64)
        gmg.gmg_apply_operator_f64(P.h, P.finest, u, r)
        res = float(torch.linalg.vector_norm(b - r) / torch.linalg.vector_norm(b))
        sols[name] = u
        out[name] = {"time_to_solution_ms": ms, "mdofs": nodes / ms * 1e3 / 1e6,
                     "iterations": st.iterations, "final_rel_residual": res, "levels": P.n_levels}
        del P
    for name in ("fp64_closure", "fp32_mixed", "fp32_tc_mixed", "fp32_tf32_mixed"):
        out[name]["rel_diff_vs_fp64_solution"] = float(
            torch.linalg.vector_norm(sols[name] - sols["fp64"]) / torch.linalg.vector_norm(sols["fp64"]))
        out["speedup_" + name] = out["fp64"]["time_to_solution_ms"] / out[name]["time_to_solution_ms"]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
