#!/usr/bin/env python
"""Benchmark of the GB300 vertex-patch smoother inside GMG-preconditioned CG.

Workload (one step): 3D Poisson, continuous Q4 hex elements, uniform 64^3
cell mesh (257^3 = 16,974,593 nodes, 16,581,375 interior DoFs), zero Dirichlet
data, seeded U[-1,1] right-hand side on the interior nodes; plain FP64
GMG(V(1,1), 8-colour multiplicative vertex-patch smoother, exact coarse
solve by fast diagonalisation on 2^3 cells, levels 64-32-16-8-4-2)
preconditioned CG from u = 0 to ||r|| <= 1e-10 ||b||.

Reported: whole-job solve throughput (all nodes / time to 1e-10) as
`value`; the finest-level smoother sweep rate and its roofline (the FP64
sweep runs in double-float arithmetic on the FP32 pipe and is bound by
instruction issue: executed warp instructions per second against the issue
slots of the GPU at the sampled clock, and beside it the method's FP64
operation count per second against the FP64 FMA peak measured in the same
run); the same solve end to end through
the C ABI with host buffers (`e2e`); the FP32-mixed solve of the same
workload; the FP64 oracle's sweep of the full 64^3 grid timed on the host
cores at one core and at all cores (`cpu_baseline`); and two further
workloads of the paper's method, each timed once after a warm-up:
`c3` (3D Q7 48^3, FP64 against FP32 and tensor-core smoothers inside FP64
CG), `c4` (64 independent Q3 problems, batched against one after another)
and `c5` (3D Q3 64^3 variable coefficient, damped mean-coefficient FD
against the learned correction, FP64 and FP32).  `--impl reference` times
the oracle's PCG alone on a bounded sample.

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
# FP64 peak from unit counts and clock (152 SMs x 2 DFMA/clk x 2 flop x
# 2.07 GHz), used only if the in-run measurement (gmg_fma_peak) fails
FP64_PEAK_DERIVED_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# The FP64 sweep runs each colour as two launches, the face kernel and the
# patch kernel (shared-face form), both in double-float arithmetic on the
# FP32 pipe; "per launch" figures below are per colour step (both kernels).
# From ncu over every launch of 7 sweeps of the current kernels at this
# workload (profiles/face_sweep_fp64_q4_64.md), per average colour step of
# 31,256 patches: DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum)
# and warp instructions issued (smsp__inst_executed.sum), face + patch kernel.
TRAFFIC_PER_LAUNCH = (151.86e6 + 16.79e6) + (221.64e6 + 69.60e6)
WARP_INST_PER_PATCH = (90.91e6 + 212.46e6) / (250047 / 8)
EXECUTED_SOURCE = ("profiles/face_sweep_fp64_q4_64.md: ncu smsp__inst_executed.sum over every launch of 7 sweeps "
                   "(face_kernel_df + patch_face_kernel), per patch")
# issue slots of GB300: 152 SMs x 4 schedulers, one warp instruction each per clock
ISSUE_SLOTS_PER_CLOCK = 152 * 4
# FP32 pipe activity of the two kernels (ncu --set full, one colour step each)
PIPE_ACTIVE = {"face_kernel_df": {"fma": 0.468, "alu": 0.283, "issue": 0.697},
               "patch_face_kernel": {"fma": 0.457, "alu": 0.232, "issue": 0.672}}
CPU_SAMPLE = dict(dim=3, degree=4, n_cells=8, n_levels=3)
BLAS_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")
# further workloads of the method, measured in the same run (one timed solve each)
C3 = dict(dim=3, degree=7, n_cells=48, seed=0, dist="normal")
C5 = dict(dim=3, degree=3, n_cells=64, seed=0, sigma=1.0, corr_len=0.1, samples=200000, steps=400)
C4 = dict(problems=64, degree=3, nmin=16, nmax=96, seed=0)
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


def oracle_sweep_child(threads):
    """One oracle sweep (Algorithm 4, dense LU patch solves, patch-local
    blocks) of the full benchmark grid, 3D Q4 64^3, from u = 0 with the
    bench's right-hand side; run in a fresh process whose BLAS thread count
    the parent fixed.  Prints seconds per colour and per sweep as JSON."""
    import numpy as np
    from oracle.mesh import Mesh
    from oracle.smoother import PatchSmoother
    from paper_2407_02100_gb300 import inputs
    m = Mesh(DIM, DEGREE, N_CELLS)
    sm = PatchSmoother(m)
    b = inputs.random_nodal(DIM, DEGREE, N_CELLS, 0, "uniform")
    u = np.zeros_like(b)
    per = []
    t_all = time.perf_counter()
    for c in sm.colour_order(False):
        t0 = time.perf_counter()
        sm.colour_step(u, b, c)
        per.append(time.perf_counter() - t0)
    total = time.perf_counter() - t_all
    print(json.dumps({"threads": threads, "seconds_per_sweep": total, "seconds_per_colour": per,
                      "nodes": m.n_nodes}), flush=True)
    return 0


def time_oracle_sweep(threads):
    """Runs oracle_sweep_child in a fresh interpreter with `threads` BLAS
    threads (set before numpy loads); returns its JSON record or None."""
    env = dict(os.environ)
    for v in BLAS_THREAD_VARS:
        env[v] = str(threads)
    try:
        res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sweep-child",
                              "--threads", str(threads)], env=env, capture_output=True, text=True,
                             timeout=600)
    except subprocess.TimeoutExpired:
        return None
    for ln in res.stdout.splitlines()[::-1]:
        if ln.startswith("{"):
            return json.loads(ln)
    return None


def cpu_baseline_record(gpu_sweep_mdofs):
    """The oracle's sweep of the full benchmark grid at one core and at all
    cores (BLAS threads; the gather is plain NumPy indexing), and the oracle
    PCG on the bounded 8^3 sample for the solve metric."""
    nproc = os.cpu_count() or 1
    one = time_oracle_sweep(1)
    allc = time_oracle_sweep(nproc)
    rec = {"kind": "oracle", "unit": "MDoF/s (one smoother sweep, all nodes)"}
    if allc:
        rec.update({"value": allc["nodes"] / allc["seconds_per_sweep"] / 1e6, "cores": nproc,
                    "seconds_per_sweep": allc["seconds_per_sweep"]})
    if one:
        rec["single_core"] = {"value": one["nodes"] / one["seconds_per_sweep"] / 1e6, "cores": 1,
                              "seconds_per_sweep": one["seconds_per_sweep"]}
    rec["sample"] = ("oracle smoother sweep (Algorithm 4, ascending colours, dense LU patch solves "
                     "from patch-local blocks) of the full 3D Q4 64^3 grid (16,974,593 nodes, "
                     "250,047 patches), u = 0, the bench's seed-0 U[-1,1] right-hand side; "
                     f"nproc = {nproc}; cores = BLAS threads allowed")
    if "value" in rec and gpu_sweep_mdofs:
        rec["gpu_sweep_over_oracle"] = gpu_sweep_mdofs / rec["value"]
    v, dt, its = time_oracle_solve(1)
    rec["pcg_sample"] = {"value": v, "unit": "MDoF/s (all nodes / GMG-CG time to 1e-10)", "cores": nproc,
                         "sample": cpu_sample_text() + f"; {dt:.2f} s per solve, {its} iterations"}
    return rec


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
    with ClockSampler(local) as sweep_clocks:
        s0.record(stream)
        for _ in range(n_sweeps):
            gmg.gmg_smooth(P.h, P.finest, us, b, 1, False)
        s1.record(stream)
        torch.cuda.synchronize()
    sweep_s = s0.elapsed_time(s1) * 1e-3 / n_sweeps
    patches = (N_CELLS - 1) ** DIM
    flops_sweep = FLOP_PER_PATCH * patches
    method_tflops = flops_sweep / sweep_s / 1e12
    inst_rate = WARP_INST_PER_PATCH * patches / sweep_s / 1e12        # T warp instructions / s
    sweep_clk = sweep_clocks.summary()
    sm_hz = (sweep_clk.get("sm_mhz") or 2070.0) * 1e6
    issue_peak = ISSUE_SLOTS_PER_CLOCK * sm_hz / 1e12
    hbm_gbs = BYTES_PER_NODE * nodes / sweep_s / 1e9

    # ---- measured FMA peaks of this GPU (roofline denominators) ----
    try:
        peak64, peak64_src = gmg.gmg_fma_peak(gmg.GMG_FP64), "measured in this run: gmg_fma_peak(GMG_FP64)"
    except gmg.GmgError:
        peak64, peak64_src = FP64_PEAK_DERIVED_TFLOPS, "derived: 152 SM x 4 FP64 flop/clk x 2.07 GHz"
    try:
        peak32 = gmg.gmg_fma_peak(gmg.GMG_FP32)
    except gmg.GmgError:
        peak32 = None

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

    # ---- per-phase times of one FP64 solve (events per phase, no graph) ----
    gmg.gmg_set_phase_timing(P.h, True)
    up = P.zeros(dtype=torch.float64)
    _, st_ph = gmg.cg_gmg_solve(P.h, up, b, RTOL, 100)
    gmg.gmg_set_phase_timing(P.h, False)
    phases = gmg.phase_times(st_ph)
    del up

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
    with ClockSampler(local) as clocks32:
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
    del us32, bs32, u32

    extra = {}
    if not args.no_extra and ws == 1:
        P.close()
        del us, r, b_e2e
        torch.cuda.empty_cache()
        extra["c3"] = c3_leg(gmg, inputs, torch, local)
        torch.cuda.empty_cache()
        extra["c5"] = c5_leg(gmg, inputs, torch, local)
        torch.cuda.empty_cache()
        extra["c4"] = c4_leg(gmg, inputs, torch, local)
        torch.cuda.empty_cache()
    else:
        P.close()

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_record(nodes / sweep_s / 1e6)

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
        "arithmetic": "FP64 vectors, CG scalars, dot products, transfers and coarse solve; the patch sweep "
                      "and the level operator in double-float (pairs of f32, about 48 significant bits, "
                      "Dot2 accumulation), parity with the FP64 oracle within 1e-12",
        "data": "synthetic (seeded U[-1,1] RHS on interior nodes)",
        "config": {"workload": WORKLOAD,
                   "nodes": nodes, "interior_dofs": (N_CELLS * DEGREE - 1) ** DIM,
                   "levels": P.n_levels, "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (u, b: 136 MB each)",
                   "cg_iterations": iters[-1], "final_rel_residual": rel_res},
        "time_to_solution_ms": ms_per_step,
        "phase_ms": phases,
        "smoother": {"ms_per_sweep": sweep_s * 1e3, "mdofs": nodes / sweep_s / 1e6,
                     "hbm_gbs_algorithmic": hbm_gbs, "patches": patches,
                     "flop_per_patch": FLOP_PER_PATCH, "clocks": sweep_clk},
        "fp32_mixed": {"time_to_solution_ms": ms32, "mdofs": nodes / (ms32 * 1e-3) / 1e6,
                       "cg_iterations": st32.iterations, "final_rel_residual": res32,
                       "rel_diff_vs_fp64_solution": diff32,
                       "speedup_vs_fp64": ms_per_step / ms32,
                       "smoother_ms_per_sweep": sweep32_s * 1e3,
                       "smoother_mdofs": nodes / sweep32_s / 1e6,
                       "smoother_hbm_gbs_algorithmic": 12 * nodes / sweep32_s / 1e9,
                       "smoother_work_equivalent_tflops": flops_sweep / sweep32_s / 1e12,
                       "smoother_work_equivalent_frac_of_fp32_peak":
                           (flops_sweep / sweep32_s / 1e12 / peak32) if peak32 else None,
                       "fp32_fma_peak_tflops": peak32,
                       "clocks": clocks32.summary()},
        "roofline": {"bound": "alu", "achieved": inst_rate, "peak": issue_peak, "unit": "Twarp-inst/s",
                     "frac": inst_rate / issue_peak,
                     "peak_source": "derived: 152 SMs x 4 schedulers x 1 warp instruction per clock x the SM "
                                    f"clock sampled during the sweeps ({sm_hz / 1e6:.0f} MHz); no issue-rate "
                                    "peak is measured by the driver",
                     "traffic": TRAFFIC_PER_LAUNCH,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum over every launch of 7 "
                                       "sweeps, per colour step (face kernel + patch kernel); "
                                       "profiles/face_sweep_fp64_q4_64.md",
                     "algorithmic_bytes_per_launch": BYTES_PER_NODE * nodes / 8,
                     "executed_warp_inst_per_patch": WARP_INST_PER_PATCH,
                     "executed_source": EXECUTED_SOURCE,
                     "pipe_active_ncu": PIPE_ACTIVE,
                     "fp64_equivalent": {"achieved": method_tflops, "unit": "TFLOP/s", "peak": peak64,
                                         "frac": method_tflops / peak64, "peak_source": peak64_src,
                                         "flop_per_patch": FLOP_PER_PATCH,
                                         "note": "the method's FP64 operation count (2^3 cells x 7 contractions of "
                                                 "(k+1)^4 + 6 FD contractions of (2k-1)^4 multiply-adds) per second, "
                                                 "against the measured FP64 FMA peak; the kernels compute the sweep "
                                                 "in double-float arithmetic on the FP32 pipe with a regrouped "
                                                 "(banded, even/odd, shared-face) operation count"},
                     "kernel": "face_kernel_df<4,128> + patch_face_kernel<4,256,5,1> (FP64 shared-face sweep in "
                               "double-float arithmetic), one pair of launches per colour; timed as whole sweeps"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "MDoF/s", "h2d_bytes_per_step": n_elems * 8,
                "d2h_bytes_per_step": n_elems * 8},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def timed_solve(gmg, torch, P, u, b, local, max_it=300, repeats=3):
    """One warm-up solve, then `repeats` timed solves (CUDA events on the
    current stream, clocks sampled around them); returns (median ms, stats,
    status, clocks) of the last solve.  The median keeps one solve slowed by
    the host (a launch gap) from standing for the leg."""
    u.zero_()
    gmg.cg_gmg_solve(P.h, u, b, RTOL, max_it, raise_on_error=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    with ClockSampler(local) as ck:
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            u.zero_()
            e0.record(stream)
            status, st = gmg.cg_gmg_solve(P.h, u, b, RTOL, max_it, raise_on_error=False)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    return sorted(times)[len(times) // 2], st, status, ck.summary()


def rel_diff(torch, a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def c3_leg(gmg, inputs, torch, local):
    """3D Poisson Q7 48^3 (38,272,753 nodes), N(0,1) RHS: the FP64 solve
    against FP32 (FFMA) and 3xTF32 tensor-core smoothers inside the same FP64
    CG, time to 1e-10 and the difference to the FP64 solution."""
    c = C3
    rhs = inputs.random_nodal(c["dim"], c["degree"], c["n_cells"], c["seed"], c["dist"])
    nodes = (c["n_cells"] * c["degree"] + 1) ** c["dim"]
    out = {"workload": "3D Poisson Q7, 48^3 cells, N(0,1) RHS, GMG(V(1,1))-PCG to 1e-10",
           "nodes": nodes}
    ref = None
    for name, prec in (("fp64", gmg.GMG_FP64), ("fp32_mixed", gmg.GMG_FP32),
                       ("fp32_tc_mixed", gmg.GMG_FP32_TC)):
        P = gmg.Problem(c["dim"], c["degree"], c["n_cells"], precision=prec)
        b = P.to_device(rhs, dtype=torch.float64)
        u = P.zeros(dtype=torch.float64)
        ms, st, status, ck = timed_solve(gmg, torch, P, u, b, local)
        rec = {"time_to_solution_ms": ms, "mdofs": nodes / ms * 1e3 / 1e6, "iterations": st.iterations,
               "rel_residual": st.relative_residual, "status": gmg.STATUS.get(status, status), "clocks": ck}
        if ref is None:
            ref = u.clone()
        else:
            rec["rel_diff_vs_fp64_solution"] = rel_diff(torch, u, ref)
        out[name] = rec
        P.close()
        del u, b
    for name in ("fp32_mixed", "fp32_tc_mixed"):
        out[name]["speedup_vs_fp64"] = out["fp64"]["time_to_solution_ms"] / out[name]["time_to_solution_ms"]
    return out


def c4_leg(gmg, inputs, torch, local):
    """64 independent 3D Poisson problems, Q3, n drawn from {16, 24, ..., 96}
    (seeded), N(0,1) right-hand sides: one batched FP32-smoother PCG (one
    sweep launch per colour over all problems, CUDA-graph V-cycle, FP64 CG
    per problem, autotuned patches per CTA) against the same problems solved
    one after another through the single-problem API."""
    import numpy as np
    c = C4
    rng = np.random.default_rng(c["seed"])
    ns = [int(x) for x in rng.choice(np.arange(c["nmin"], c["nmax"] + 1, 8), size=c["problems"])]
    nodes = sum((n * c["degree"] + 1) ** 3 for n in ns)
    B = gmg.Batch(3, c["degree"], ns, precision=gmg.GMG_FP32)
    rhs = [inputs.random_nodal(3, c["degree"], n, c["seed"] * 1000 + i) for i, n in enumerate(ns)]
    b = B.pack(rhs, dtype=torch.float64)
    del rhs
    u = B.zeros(dtype=torch.float64)
    ppc = gmg.gmg_batch_autotune(B.h)
    u.zero_()
    gmg.gmg_batch_cg_solve(B.h, len(ns), u, b, RTOL, 100)      # warm-up (captures the graph)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    with ClockSampler(local) as ck:
        u.zero_()
        e0.record(stream)
        _, its, res = gmg.gmg_batch_cg_solve(B.h, len(ns), u, b, RTOL, 100)
        e1.record(stream)
        torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1)
    probs = [gmg.Problem(3, c["degree"], n, precision=gmg.GMG_FP32) for n in ns]
    sols = [P.zeros(dtype=torch.float64) for P in probs]
    views = [b[B.layouts[i][0]:B.layouts[i][0] + B.layouts[i][1]] for i in range(len(ns))]
    for P, x, r in zip(probs, sols, views):
        gmg.cg_gmg_solve(P.h, x, r, RTOL, 100)
    torch.cuda.synchronize()
    e0.record(stream)
    for P, x, r in zip(probs, sols, views):
        x.zero_()
        gmg.cg_gmg_solve(P.h, x, r, RTOL, 100)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1)
    diff = max(float(torch.linalg.vector_norm(x - u[B.layouts[i][0]:B.layouts[i][0] + B.layouts[i][1]])
                     / torch.linalg.vector_norm(x)) for i, x in enumerate(sols))
    for P in probs:
        P.close()
    B.close()
    return {"workload": "64 independent 3D Poisson problems, Q3, n in {16..96} step 8, N(0,1) RHS, "
                        "FP32 smoother in FP64 PCG to 1e-10 per problem",
            "nodes": nodes, "batched_ms": t_batch, "batched_mdofs": nodes / t_batch * 1e3 / 1e6,
            "sequential_ms": t_seq, "speedup_vs_sequential": t_seq / t_batch, "ppc": ppc,
            "iterations_min": min(its), "iterations_max": max(its), "rel_residual_max": max(res),
            "max_rel_diff_vs_sequential": diff, "clocks": ck.summary()}


def c5_leg(gmg, inputs, torch, local):
    """3D variable coefficient -div(a grad u) = f, Q3 64^3, a = exp(g), g a
    Gaussian random field (sigma 1, correlation length 0.1): damped
    mean-coefficient FD against the learned correction (trained in this run
    on exact patch solves), FP64 and FP32 smoothers inside FP64 CG."""
    import numpy as np
    c = C5
    dim, k, n = c["dim"], c["degree"], c["n_cells"]
    coef = inputs.lognormal_coefficient(dim, n, c["seed"], c["sigma"], c["corr_len"])
    rhs = inputs.random_nodal(dim, k, n, c["seed"] + 1)
    nodes = (n * k + 1) ** dim
    nint = (2 * k - 1) ** dim
    out = {"workload": "3D -div(a grad u) = f, Q3, 64^3 cells, a = exp(GRF sigma 1, l 0.1), N(0,1) RHS, "
                       "GMG(V(1,1))-PCG to 1e-10",
           "nodes": nodes, "coef_contrast": float(coef.max() / coef.min()), "samples": None}
    ref = None
    for pname, prec in (("fp64", gmg.GMG_FP64), ("fp32", gmg.GMG_FP32)):
        for mode in ("fd_mean", "learned"):
            P = gmg.Problem(dim, k, n, precision=prec)
            gmg.gmg_set_coefficient(P.h, coef)
            rec = {}
            if mode == "learned":
                nfine = (n - 1) ** dim
                total = gmg.learned_patch_count(dim, n, P.n_levels)
                rng = np.random.default_rng(c["seed"] + 2)
                nf = max(0, min(nfine, c["samples"] - (total - nfine)))
                verts = rng.permutation(np.concatenate([rng.permutation(nfine)[:nf], np.arange(nfine, total)]))
                res = torch.tensor(np.random.default_rng(c["seed"] + 3).standard_normal((len(verts), nint)),
                                   device="cuda")
                out["samples"] = len(verts)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                hist, kept = gmg.gmg_learned_train(P.h, verts, res, steps=c["steps"], batch=4096, lr=3e-3,
                                                   seed=c["seed"])
                torch.cuda.synchronize()
                rec.update({"train_s": time.perf_counter() - t0, "loss_first": hist[0], "loss_last": hist[-1],
                            "kept_patches": kept, "levels_kept_mask": gmg.gmg_learned_levels(P.h),
                            "levels": P.n_levels})
                del res
            b = P.to_device(rhs, dtype=torch.float64)
            u = P.zeros(dtype=torch.float64)
            ms, st, status, ck = timed_solve(gmg, torch, P, u, b, local)
            rec.update({"time_to_solution_ms": ms, "iterations": st.iterations,
                        "rel_residual": st.relative_residual, "status": gmg.STATUS.get(status, status),
                        "clocks": ck})
            if ref is None:
                ref = u.clone()
            else:
                rec["rel_diff_vs_fp64_fd_mean_solution"] = rel_diff(torch, u, ref)
            out[f"{pname}_{mode}"] = rec
            P.close()
            del u, b
    base = out["fp64_fd_mean"]["time_to_solution_ms"]
    for key in ("fp64_learned", "fp32_fd_mean", "fp32_learned"):
        out[key]["speedup_vs_fp64_fd_mean"] = base / out[key]["time_to_solution_ms"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--sweeps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the C3 and C5 legs")
    ap.add_argument("--oracle-sweep-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--threads", type=int, default=1, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sweep_child:
        return oracle_sweep_child(args.threads)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
