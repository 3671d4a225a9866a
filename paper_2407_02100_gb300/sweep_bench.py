"""Smoother and operator micro-benchmark (CUDA events on the problem's stream).

Times finest-level multiplicative patch sweeps (all colours, gmg_smooth) and
matrix-free operator applications on one uniform level, for a chosen
dimension, degree, mesh and precision, and prints the rates:

    python -m paper_2407_02100_gb300.sweep_bench --dim 3 --degree 4 --n 64 --precision fp64

It is also the driver used for ncu captures of the patch kernel (a few
launches on a workload whose vectors exceed L2).
"""
import argparse
import json

import torch

from . import build, gmg, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=3)
    ap.add_argument("--degree", type=int, default=4)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp32_tc", "fp32_tf32"], default="fp64")
    ap.add_argument("--sweeps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--variant", choices=["combined", "separated", "batched"], default="combined",
                    help="Algorithm 4, 3 or 5 of the paper")
    ap.add_argument("--batch", type=int, default=32768, help="n_B of Algorithm 5")
    ap.add_argument("--no-apply", action="store_true",
                    help="time the sweep only (for captures of the sweep's kernels alone)")
    ap.add_argument("--slab", type=int, default=0,
                    help="skewed-slab width in vertex rows (0: one launch per colour, -1: fit L2)")
    ap.add_argument("--closure", action="store_true",
                    help="FP64 3D: evaluate every patch residual on its own closure (no shared faces)")
    ap.add_argument("--tile-operator", action="store_true",
                    help="FP64 3D: time the tile kernel instead of the three-pass operator")
    ap.add_argument("--graph", action="store_true",
                    help="capture one sweep (one operator application) as a CUDA graph and time its replays")
    ap.add_argument("--transfers", action="store_true",
                    help="time the restriction to and prolongation from the next coarser level instead")
    a = ap.parse_args()
    build.build()
    if a.transfers:
        return time_transfers(a)
    prec = {"fp64": gmg.GMG_FP64, "fp32": gmg.GMG_FP32, "fp32_tc": gmg.GMG_FP32_TC,
            "fp32_tf32": gmg.GMG_FP32_TF32}[a.precision]
    # a side stream of our own: graph capture needs one (the legacy default
    # stream cannot be captured)
    side = torch.cuda.Stream() if a.graph else torch.cuda.current_stream()
    with torch.cuda.stream(side):
        P = gmg.Problem(a.dim, a.degree, a.n, n_levels=1, precision=prec)
    gmg.gmg_set_slab_width(P.h, a.slab)
    gmg.gmg_set_shared_faces(P.h, not a.closure)
    gmg.gmg_set_three_pass_operator(P.h, not a.tile_operator)
    u = P.to_device(inputs.random_nodal(a.dim, a.degree, a.n, 1))
    b = P.to_device(inputs.random_nodal(a.dim, a.degree, a.n, 2))
    y = P.zeros()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        with torch.cuda.stream(side):
            for _ in range(a.warmup):
                fn()
            torch.cuda.synchronize()
            if a.graph:  # replay one captured call; the launches then cost what they cost in a solve
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=side):
                    fn()
                g.replay()
                torch.cuda.synchronize()
                run = g.replay
            else:
                run = fn
            e0.record(side)
            for _ in range(reps):
                run()
            e1.record(side)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e-3

    variant = {"combined": gmg.GMG_SWEEP_COMBINED, "separated": gmg.GMG_SWEEP_SEPARATED,
               "batched": gmg.GMG_SWEEP_BATCHED}[a.variant]
    t_sweep = timed(lambda: gmg.gmg_smooth_variant(P.h, 0, u, b, variant, a.batch, False), a.sweeps)
    t_apply = float("nan") if a.no_apply else timed(lambda: gmg.gmg_apply_operator(P.h, 0, u, y), a.sweeps)
    nodes = (a.n * a.degree + 1) ** a.dim
    print(json.dumps({"dim": a.dim, "degree": a.degree, "n_cells": a.n, "precision": a.precision,
                      "variant": a.variant, "batch": a.batch if a.variant == "batched" else None,
                      "slab_width": gmg.gmg_slab_width(P.h, 0), "shared_faces": gmg.gmg_shared_faces(P.h),
                      "three_pass_operator": gmg.gmg_three_pass_operator(P.h),
                      "graph": a.graph, "nodes": nodes, "sweep_ms": t_sweep * 1e3, "sweep_mdofs": nodes / t_sweep / 1e6,
                      "apply_ms": t_apply * 1e3, "apply_mdofs": nodes / t_apply / 1e6}))
    P.close()


def time_transfers(a):
    """Restriction of a fine-level vector to the next coarser level and
    prolongation back (added to the fine vector), timed over a.sweeps calls
    each after a.warmup."""
    prec = {"fp64": gmg.GMG_FP64, "fp32": gmg.GMG_FP32}[a.precision]
    P = gmg.Problem(a.dim, a.degree, a.n, n_levels=2, precision=prec)
    f = P.to_device(inputs.random_nodal(a.dim, a.degree, a.n, 1))
    c = P.zeros(0)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    for _ in range(a.warmup):
        gmg.gmg_restrict(P.h, 1, f, c)
        gmg.gmg_prolongate_add(P.h, 0, c, f)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.sweeps):
        gmg.gmg_restrict(P.h, 1, f, c)
    e1.record()
    for _ in range(a.sweeps):
        gmg.gmg_prolongate_add(P.h, 0, c, f)
    e2.record()
    torch.cuda.synchronize()
    print(json.dumps({"dim": a.dim, "degree": a.degree, "n_cells": a.n, "precision": a.precision,
                      "restrict_ms": e0.elapsed_time(e1) / a.sweeps,
                      "prolongate_ms": e1.elapsed_time(e2) / a.sweeps}))
    P.close()


if __name__ == "__main__":
    main()
