#!/usr/bin/env python
"""Benchmark of the GB300 vertex-patch smoother inside GMG-preconditioned CG.

Workload (one step): 3D Poisson, continuous Q4 hex elements, uniform 64^3
cell mesh (257^3 = 16,974,593 nodes, 16,581,375 interior DoFs), zero Dirichlet
data, seeded U[-1,1] right-hand side on the interior nodes; plain FP64
GMG(V(1,1), 8-colour multiplicative vertex-patch smoother, exact coarse
solve by fast diagonalisation on 2^3 cells, levels 64-32-16-8-4-2)
preconditioned CG from u = 0 to ||r|| <= 1e-10 ||b||.

Reported: whole-job solve throughput (all nodes / time to 1e-10) as
`value`; the finest-level smoother sweep rate and its roofline against the
FP64 arithmetic peak; the same solve end to end through the C ABI with
host buffers (`e2e`); the FP64 oracle timed on the host cores on a bounded
sample (`cpu_baseline`).  `--impl reference` times the oracle alone.

Multi-GPU (torchrun, one rank per GPU): the problem does not shard, so
every rank solves an independent replica with its own seed (replicas only,
weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "smoother MDoF/s & HBM GB/s; GMG-CG time to 1e-10, FP32/learned vs FP64 plain"
DIM, DEGREE, N_CELLS = 3, 4, 64
RTOL = 1e-10
# method's operation count per vertex patch, 3D Q4: 2^3 cells x 7 sum-
# factorised 1D contractions of (k+1)^4 multiply-adds + 6 FD contractions of
# (2k-1)^4 multiply-adds, 2 flops per multiply-add (98,812)
FLOP_PER_PATCH = 8 * 7 * 625 * 2 + 6 * 2401 * 2
# minimum HBM traffic of a sweep: read b, read u, write u (8 bytes each) per node
BYTES_PER_NODE = 24
# FP64 peak derived from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# The FP64 sweep runs each colour as two launches, the face kernel and the
# patch kernel (shared-face form); "per launch" figures below are per colour
# step (both kernels).  DRAM bytes of one average colour step at this
# workload, from ncu over every launch of 5 sweeps of the current kernels
# (dram__bytes_read.sum + dram__bytes_write.sum: 18,627.3 MB / 40 colour steps)
TRAFFIC_PER_LAUNCH = (6166.0e6 + 685.0e6 + 8954.5e6 + 2821.8e6) / 40
# FP64 operations the kernels execute per patch (ncu SASS thread-instruction
# counts of the 29,791-patch colour 0, per patch: face kernel 3,925.7 DFMA;
# patch kernel 9,506 DFMA, 1,960 DADD, 686 DMUL)
EXECUTED_FLOP_PER_PATCH = 2 * (3925.7 + 9506) + 1960 + 686
# FP64 pipe activity of the two kernels (ncu, one colour step each, current
# kernels)
FP64_PIPE_ACTIVE = {"face_kernel": 0.805, "patch_face_kernel": 0.811}
CPU_SAMPLE = dict(dim=3, degree=4, n_cells=8, n_levels=3)
WORKLOAD = ("3D Poisson Q4, 64^3 cells, FP64 GMG(V(1,1), 8-colour vertex-patch smoother) "
            "preconditioned CG to 1e-10")


def max_over_ranks(value, dist=None, device="cpu"):
    """Largest value over all ranks (the job time is the slowest rank's)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(nodes_per_rank, world_size, steps, max_ms):
    """Whole-job throughput in MDoF/s: nodes solved by all ranks / job time."""
    return nodes_per_rank * world_size * steps / (max_ms * 1e-3) / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


_ORACLE = {}


def time_oracle_solve(repeats=1):
    """Oracle PCG (FP64, assembled matrices, dense LU patch solves) on the
    bounded sample mesh; returns (MDoF/s, seconds per solve, iterations).
    The oracle's set-up (assembly) is built once and not timed."""
    from oracle.multigrid import Multigrid
    from paper_2407_02100_gb300 import inputs
    s = CPU_SAMPLE
    if "mg" not in _ORACLE:
        _ORACLE["mg"] = Multigrid(s["dim"], s["degree"], s["n_cells"], s["n_levels"])
    mg = _ORACLE["mg"]
    b = inputs.random_nodal(s["dim"], s["degree"], s["n_cells"], 0, "uniform")
    nodes = (s["n_cells"] * s["degree"] + 1) ** s["dim"]
    best = None
    its = 0
    for _ in range(repeats):
        t0 = time.perf_counter()
        _, its, _ = mg.pcg(b, rtol=RTOL)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return nodes / best / 1e6, best, its


def cpu_sample_text():
    s = CPU_SAMPLE
    return (f"oracle PCG to 1e-10, 3D Q{s['degree']} {s['n_cells']}^3 cells "
            f"({(s['n_cells'] * s['degree'] + 1) ** 3} nodes), {s['n_levels']} levels, "
            "same V(1,1) 8-colour patch smoother (dense LU patch solves), seed 0 U[-1,1]")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        time_oracle_solve(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, dt, its = time_oracle_solve(1)
        vals.append(dt)
    total = time.perf_counter() - t0
    s = CPU_SAMPLE
    nodes = (s["n_cells"] * s["degree"] + 1) ** s["dim"]
    value = nodes * args.steps / sum(vals) / 1e6
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "MDoF/s (all nodes / GMG-CG time to 1e-10)", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(vals) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded U[-1,1] RHS)",
        "config": {"workload": WORKLOAD, "sample": cpu_sample_text()},
        "cpu_baseline": {"value": value, "unit": "MDoF/s", "cores": cores, "kind": "oracle",
                         "sample": cpu_sample_text()},
        "e2e": {"value": value, "unit": "MDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": total,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_2407_02100_gb300 import build as pbuild
    from paper_2407_02100_gb300 import gmg, inputs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pbuild.build()
    if dist is not None:
        dist.barrier()

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()
    P = gmg.Problem(DIM, DEGREE, N_CELLS, n_levels=0, precision=gmg.GMG_FP64)
    n_elems, N, py, pz = P.layout()
    nodes = N ** DIM
    b_dense = inputs.random_nodal(DIM, DEGREE, N_CELLS, args.seed + rank, "uniform")
    b = P.to_device(b_dense, dtype=torch.float64)
    u = P.zeros(dtype=torch.float64)

    def solve():
        u.zero_()
        status, st = gmg.cg_gmg_solve(P.h, u, b, RTOL, 100)
        return st

    for _ in range(args.warmup):
        st = solve()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    launches0 = gmg.gmg_kernel_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    with ClockSampler(local) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            st = solve()
            iters.append(st.iterations)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = gmg.gmg_kernel_launch_count() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    ms_per_step = ms / args.steps
    value = whole_job_rate(nodes, ws, args.steps, ms)

    # ---- dominant kernel: the finest-level patch sweep (8 colour launches) ----
    us = P.zeros(dtype=torch.float64)
    us.copy_(u)
    n_sweeps = args.sweeps
    for _ in range(2):
        gmg.gmg_smooth(P.h, P.finest, us, b, 1, False)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(n_sweeps):
        gmg.gmg_smooth(P.h, P.finest, us, b, 1, False)
    s1.record(stream)
    torch.cuda.synchronize()
    sweep_s = s0.elapsed_time(s1) * 1e-3 / n_sweeps
    patches = (N_CELLS - 1) ** DIM
    flops_sweep = FLOP_PER_PATCH * patches
    achieved_tflops = flops_sweep / sweep_s / 1e12
    executed_tflops = EXECUTED_FLOP_PER_PATCH * patches / sweep_s / 1e12
    hbm_gbs = BYTES_PER_NODE * nodes / sweep_s / 1e9

    # ---- end to end through the C ABI with host buffers ----
    b_pin = torch.empty(n_elems, dtype=torch.float64, pin_memory=True)
    b_pin.copy_(b.cpu())
    u_pin = torch.empty(n_elems, dtype=torch.float64, pin_memory=True)
    b_e2e = torch.empty_like(b)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        b_e2e.copy_(b_pin, non_blocking=True)
        u.zero_()
        gmg.cg_gmg_solve(P.h, u, b_e2e, RTOL, 100)
        u_pin.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, "cuda")
    e2e_value = whole_job_rate(nodes, ws, 1, e2e_s * 1e3)

    # ---- parity of the final solution (residual computed on the device by the
    # library's FP64 operator, norm by torch) ----
    r = P.zeros(dtype=torch.float64)
    gmg.gmg_apply_operator_f64(P.h, P.finest, u, r)
    rel_res = float(torch.linalg.vector_norm(b - r) / torch.linalg.vector_norm(b))

    # ---- mixed precision: FP32 smoother / V-cycle inside the FP64 CG, same
    # workload, same accuracy target ----
    P32 = gmg.Problem(DIM, DEGREE, N_CELLS, n_levels=0, precision=gmg.GMG_FP32)
    u32 = P32.zeros(dtype=torch.float64)
    st32 = None
    for _ in range(args.warmup):
        u32.zero_()
        _, st32 = gmg.cg_gmg_solve(P32.h, u32, b, RTOL, 100)
    torch.cuda.synchronize()
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(args.steps):
        u32.zero_()
        _, st32 = gmg.cg_gmg_solve(P32.h, u32, b, RTOL, 100)
    m1.record(stream)
    torch.cuda.synchronize()
    ms32 = m0.elapsed_time(m1) / args.steps
    diff32 = float(torch.linalg.vector_norm(u32 - u) / torch.linalg.vector_norm(u))
    gmg.gmg_apply_operator_f64(P32.h, P32.finest, u32, r)
    res32 = float(torch.linalg.vector_norm(b - r) / torch.linalg.vector_norm(b))
    us32 = P32.zeros()
    bs32 = b.to(torch.float32)
    for _ in range(2):
        gmg.gmg_smooth(P32.h, P32.finest, us32, bs32, 1, False)
    torch.cuda.synchronize()
    s0.record(stream)
    for _ in range(n_sweeps):
        gmg.gmg_smooth(P32.h, P32.finest, us32, bs32, 1, False)
    s1.record(stream)
    torch.cuda.synchronize()
    sweep32_s = s0.elapsed_time(s1) * 1e-3 / n_sweeps
    P32.close()

    if rank != 0:
        P.close()
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        v, dt, its = time_oracle_solve(1)
        cpu = {"value": v, "unit": "MDoF/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": cpu_sample_text() + f"; {dt:.2f} s per solve, {its} iterations"}

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "MDoF/s (all nodes / GMG-CG time to 1e-10)",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded U[-1,1] RHS on interior nodes)",
        "config": {"workload": WORKLOAD,
                   "nodes": nodes, "interior_dofs": (N_CELLS * DEGREE - 1) ** DIM,
                   "levels": P.n_levels, "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (u, b: 136 MB each)",
                   "cg_iterations": iters[-1], "final_rel_residual": rel_res},
        "time_to_solution_ms": ms_per_step,
        "smoother": {"ms_per_sweep": sweep_s * 1e3, "mdofs": nodes / sweep_s / 1e6,
                     "hbm_gbs_algorithmic": hbm_gbs, "patches": patches,
                     "flop_per_patch": FLOP_PER_PATCH},
        "fp32_mixed": {"time_to_solution_ms": ms32, "mdofs": nodes / (ms32 * 1e-3) / 1e6,
                       "cg_iterations": st32.iterations, "final_rel_residual": res32,
                       "rel_diff_vs_fp64_solution": diff32,
                       "speedup_vs_fp64": ms_per_step / ms32,
                       "smoother_ms_per_sweep": sweep32_s * 1e3,
                       "smoother_mdofs": nodes / sweep32_s / 1e6,
                       "smoother_hbm_gbs_algorithmic": 12 * nodes / sweep32_s / 1e9},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved_tflops / FP64_PEAK_TFLOPS,
                     "traffic": TRAFFIC_PER_LAUNCH,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum over every "
                                       "launch of 5 sweeps, per colour step (face kernel + patch kernel)",
                     "algorithmic_bytes_per_launch": BYTES_PER_NODE * nodes / 8,
                     "executed_flop_per_patch": EXECUTED_FLOP_PER_PATCH,
                     "executed_tflops": executed_tflops,
                     "executed_frac": executed_tflops / FP64_PEAK_TFLOPS,
                     "fp64_pipe_active_ncu": FP64_PIPE_ACTIVE,
                     "kernel": "face_kernel<4,128> + patch_face_kernel<4,256,5,2> (FP64 shared-face "
                               "sweep), one pair of launches per colour; timed as whole sweeps",
                     "peak_source": "derived: 152 SM x 4 FP64 flop/clk x 2.07 GHz",
                     "note": "achieved and frac count the method's operation count (98,812 flop per "
                             "patch); the kernels execute 29,510 FP64 flop per patch (banded two-cell "
                             "matrices, even/odd FD, residual from the closure faces, each face "
                             "evaluated once per colour), so frac > 1; executed_frac and the FP64 "
                             "pipe activity are the utilisation of the hardware"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "MDoF/s", "h2d_bytes_per_step": n_elems * 8,
                "d2h_bytes_per_step": n_elems * 8},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    P.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--sweeps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
