"""Variable-coefficient benchmark: -div(a grad u) = f on the unit cube, Q3,
a = exp(g) with g a Gaussian random field (sigma 1, correlation length 0.1,
one value per cell), seeded N(0,1) right-hand side, FP32 smoother / V-cycle
inside FP64 CG to 1e-10.  Compares the plain mean-coefficient FD local
solver with the learned correction (trained on exact patch solves of the
problem's own patches of every level), over a range of dampings.

    python -m paper_2407_02100_gb300.learned_bench --n 64 --samples 200000
"""
import argparse
import json
import time

import numpy as np
import torch

from . import build, gmg, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=3)
    ap.add_argument("--degree", type=int, default=3)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--sigma", type=float, default=1.0)
    ap.add_argument("--corr", type=float, default=0.1)
    ap.add_argument("--samples", type=int, default=200000)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--omegas", default="1.0,0.8,0.6")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fd-only", action="store_true",
                    help="only the damped-FD solves (no training), with per-phase times")
    a = ap.parse_args()
    build.build()
    prec = gmg.GMG_FP32 if a.precision == "fp32" else gmg.GMG_FP64
    dim, k, n = a.dim, a.degree, a.n
    coef = inputs.lognormal_coefficient(dim, n, a.seed, a.sigma, a.corr)
    rhs = inputs.random_nodal(dim, k, n, a.seed + 1)
    nint = (2 * k - 1) ** dim
    # every patch of the coarser levels (where the coefficient varies most
    # inside a patch) plus a random share of the finest level, shuffled
    n_levels = gmg.Problem(dim, k, n, precision=prec).n_levels
    nfine = (n - 1) ** dim
    total = gmg.learned_patch_count(dim, n, n_levels)
    rng = np.random.default_rng(a.seed + 2)
    nf = max(0, min(nfine, a.samples - (total - nfine)))
    verts = rng.permutation(np.concatenate([rng.permutation(nfine)[:nf], np.arange(nfine, total)]))
    ns = len(verts)
    res = None if a.fd_only else torch.tensor(np.random.default_rng(a.seed + 3).standard_normal((ns, nint)),
                                              device="cuda")
    out = {"dim": dim, "degree": k, "n_cells": n, "sigma": a.sigma, "corr_len": a.corr,
           "coef_contrast": float(coef.max() / coef.min()), "samples": ns, "precision": a.precision,
           "runs": []}
    for om in [float(x) for x in a.omegas.split(",")]:
        for mode in ("fd_mean",) if a.fd_only else ("fd_mean", "learned"):
            P = gmg.Problem(dim, k, n, precision=prec, damping=om)
            gmg.gmg_set_coefficient(P.h, coef)
            rec = {"omega": om, "local_solver": mode}
            if mode == "learned":
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                hist, kept = gmg.gmg_learned_train(P.h, verts, res, steps=a.steps, batch=4096, lr=3e-3,
                                                   seed=a.seed)
                torch.cuda.synchronize()
                rec.update({"train_s": time.perf_counter() - t0, "loss_first": hist[0], "loss_last": hist[-1],
                            "kept_patches": kept, "levels_kept_mask": gmg.gmg_learned_levels(P.h)})
            b = P.to_device(rhs, dtype=torch.float64)
            u = P.zeros(dtype=torch.float64)
            st, s = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 300, raise_on_error=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            u.zero_()
            st, s = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 300, raise_on_error=False)
            torch.cuda.synchronize()
            rec.update({"status": gmg.STATUS.get(st, st), "iterations": s.iterations,
                        "rel_residual": s.relative_residual,
                        "time_to_solution_ms": (time.perf_counter() - t0) * 1e3})
            if a.fd_only:  # a third solve with per-phase GPU times
                gmg.gmg_set_phase_timing(P.h, True)
                u.zero_()
                _, s = gmg.cg_gmg_solve(P.h, u, b, 1e-10, 300, raise_on_error=False)
                rec["phase_ms"] = gmg.phase_times(s)
            out["runs"].append(rec)
            del P
    print(json.dumps(out))


if __name__ == "__main__":
    main()
