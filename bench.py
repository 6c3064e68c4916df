"""Benchmark: branch-MPC solves per second to KKT <= 1e-5 (FP32) on one or more GPUs.

One step = one batch of seeded synthetic scenario-tree problems solved to
convergence by the whole hot path (RK4 linearisation, tree Riccati recursion,
forward rollout, merit line search, BCL update) in one persistent kernel
launch per dynamics model, replayed from a captured CUDA graph.  The default
workload is the mixed batch: 4,096 problems with 2-64 scenarios, horizons
20-60, 1-5 obstacles, kinematic and dynamic bicycles.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload config1..config4] [--batch B]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores
  python bench.py --single ...           # single-problem latency against its critical path

Under torchrun every rank solves its own shard of B problems (weak scaling, no
data-path collective); rank 0 prints one JSON line.

Roofs.  The solver's work per problem is a chain of dependent steps (the tree
sweeps walk the depth N + 1 twice per iteration), so the roof that binds is
latency: a problem's iteration cannot be shorter than that of a single-path
tree of the same depth and model run with one node per thread (its critical
path, measured here on the same kernel).  The FP32 ALU roof uses the FP32 FMA
peak measured by the library's own microbenchmark; the HBM roof the measured
copy bandwidth (MEASURED_PEAKS.json).
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

import scenes  # noqa: E402

METRIC = "BMPC solves/sec at KKT<=1e-5 (FP32)"
DEFAULT_WORKLOAD, DEFAULT_BATCH = "config4", 4096
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 148, 128, 2032.0


def workload(name: str, batch: int, rank: int = 0):
    """Seeded problems of the named configuration; each rank gets its own seeds."""
    if name == "config1":
        return [scenes.config1(rank * batch + i) for i in range(batch)]
    if name == "config2":
        return [scenes.config2(rank * batch + i) for i in range(batch)]
    if name == "config4":
        return [scenes.config4_problem(4 + rank, i) for i in range(batch)]
    if name == "config3":
        return [scenes.config3(rank * batch + i) for i in range(batch)]
    if name == "unicycle":
        return [scenes.unicycle(rank * batch + i) for i in range(batch)]
    if name.startswith("mass_spring"):   # mass_spring or mass_springNr: per-branch spring constants
        nr = int(name[len("mass_spring"):] or 5)
        return [scenes.mass_spring(rank * batch + i, N=30, Nr=nr, constrained=True) for i in range(batch)]
    raise ValueError(name)


# ----------------------------------------------------------------- algorithmic flop model
def flops_model(p) -> dict:
    """Algorithmic FP32 flops per node of one inner iteration, by phase (FMA = 2 flops).

    Counted from the arithmetic the method needs, not from instructions: RK4 with forward-mode
    tangents, the tree Riccati step, the rollout, one line-search evaluation per step size.
    """
    nx, model, nsub = int(p["nx"]), int(p["model"]), max(1, int(p["params"][9]))
    nz = nx + 2
    ns = nx * (nx + 1) // 2
    rhs = {0: 20, 1: 70, 2: 2 * nx * nz, 3: 16}[model]
    nnz = {0: 7, 1: 18, 2: nx * nz, 3: 6}[model]
    n_obs = int(p["n_obs"])
    if model == 2:
        lin_dyn = 2 * nx * nz
        ls_dyn = 2 * nx * nz
    else:
        per_stage = rhs + 2 * nnz * nz + 2 * nx * nz + 4 * nx * nz
        lin_dyn = nsub * (4 * per_stage + 2 * nx * nz + 2 * nx)
        ls_dyn = nsub * 4 * (rhs + 6 * nx)
    con = 8 * nx + 30 * n_obs + 20
    return dict(
        lin_dyn=lin_dyn,                         # f, A, B: only where the point has moved
        linearise=con + 2 * nx * nx + 8 * nx,    # cost, penalty terms, defects, KKT: at every check
        riccati=(2 * nx ** 3 + 4 * nx * nx + 2 * ns * nx + 4 * nx * nx + 2 * nx * nx + ns * (2 * nx + 4)
                 + 12 * nx + 60 + ns + 2 * nx * nx),
        forward=4 * nx * nx + 8 * nx + 8 * nx,
        ls_eval=ls_dyn + con + 6 * nx + 6 * nx,
        update=6 * nx,
        outer=con,
    )


def algorithmic_bytes_per_node_iter(p) -> float:
    """Minimum DRAM bytes per node and inner iteration: read and write x, u, lambda, y; read the
    obstacle data (5 values each); write and read the feedback law K, k between the two sweeps."""
    nx, nc, n_obs = int(p["nx"]), 2 * 2 * int(p["box_on"]) + int(p["n_obs"]) + 2 * int(p["lane_on"]), int(p["n_obs"])
    state = 2 * nx + 2 + nc
    return 4.0 * (2 * state + 5 * n_obs + 2 * (2 * nx + 2))


def algorithmic_flops(problems, results) -> float:
    tot = 0.0
    for p, r in zip(problems, results):
        m = flops_model(p)
        n = int(p["n"])
        it = r["inner_iters"]
        checks = it + r["outer_iters"]            # linearisation + KKT check per inner step and per outer exit
        moved = it + 1                            # dynamics linearised at the start and after every step
        tot += n * (moved * m["lin_dyn"] + checks * m["linearise"] + it * (m["riccati"] + m["forward"] + m["update"])
                    + r["ls_evals"] * m["ls_eval"] + r["outer_iters"] * m["outer"])
    return tot


# ----------------------------------------------------------------- clocks sampling
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=smax, reasons=sorted(reasons),
                    samples=len(sm))


# ----------------------------------------------------------------- CPU oracle leg
def oracle_rate(name: str, seconds: float, max_problems: int, rank: int = 0):
    """The FP64 oracle as it stands, one thread, on a bounded sample of the workload."""
    import oracle
    oracle.build()
    probs = workload(name, max_problems, rank)
    t0 = time.perf_counter()
    solved = done = 0
    for p in probs:
        r = oracle.solve(p, **oracle.PRODUCT_RULE)
        done += 1
        solved += int(r["status"] == oracle.OK)
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return dict(value=solved / dt, attempted_per_s=done / dt, unit="solves/s", cores=1, kind="oracle",
                sample=f"{done} {name} problems solved sequentially with the FP64 oracle ({dt:.1f} s), "
                       f"the library's failed-outer-step rule (oracle.PRODUCT_RULE)")


def _oracle_converged(p):
    import oracle
    return int(oracle.solve(p, **oracle.PRODUCT_RULE)["status"] == oracle.OK)


def run_reference(args):
    """The FP64 oracle, unchanged, on the host cores: each step solves a bounded sample of the
    workload (ref_sample problems per worker process) and counts the converged solves."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp

    import oracle
    oracle.build()
    workers = max(1, args.ref_workers or (os.cpu_count() or 1))
    pool = mp.get_context("spawn").Pool(workers) if workers > 1 else None
    steps = []
    for s in range(args.warmup + args.steps):
        probs = workload(args.workload, args.ref_sample * workers, rank=1000 + s)
        tsolve = time.perf_counter()
        flags = pool.map(_oracle_converged, probs, chunksize=1) if pool else [_oracle_converged(p) for p in probs]
        dt = time.perf_counter() - tsolve
        if s >= args.warmup:
            steps.append((sum(flags), dt))
    if pool:
        pool.close()
    tot_s = sum(d for _, d in steps)
    value = sum(n for n, _ in steps) / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / len(steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "batch": args.ref_sample * workers},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": workers, "kind": "oracle",
                             "sample": f"{args.ref_sample * workers} {args.workload} problems per step, FP64 oracle, "
                                       f"one problem per process on {workers} processes"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- ncu traffic
PROFILES = {"config2": "bmpc_solve_kernel_config2.md", "config4": "bmpc_solve_kernel_config4.md"}
KERNEL_SOURCES = ("paper_2506_13624_b300/csrc/bmpc_kernel.cu", "paper_2506_13624_b300/csrc/bmpc_layout.h")


def kernel_sha():
    import hashlib
    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for f in KERNEL_SOURCES:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload_name, node_iters):
    """DRAM bytes (read + write) of one step's solve launches, scaled from the committed ncu capture
    of the same workload on a reduced batch by node-iterations (a problem's traffic is its scratch
    rows, written and read once or twice per node and iteration); None when there is no capture of
    this workload or the kernel sources changed since it was taken."""
    name = PROFILES.get(workload_name)
    path = os.path.join(ROOT, "profiles", name) if name else None
    if not path or not os.path.exists(path):
        return None
    kv = {}
    with open(path) as fh:
        for line in fh:
            k, _, v = line.partition(":")
            if k in ("kernel_sha256", "dram_bytes_per_node_iteration"):
                kv[k] = v.strip()
    if kv.get("kernel_sha256") != kernel_sha() or "dram_bytes_per_node_iteration" not in kv:
        return None
    return float(kv["dram_bytes_per_node_iteration"]) * node_iters


# ----------------------------------------------------------------- latency floor (critical path)
CHAIN_N = (20, 40, 60)


def chain_floor(bmpc, models, seeds=3):
    """Cycles per inner iteration of single-path trees (one scenario) of depth N in CHAIN_N, per model,
    solved one at a time with one node per thread (64 threads, per-path sweeps), and a straight-line
    fit T(N) = a + b (N + 1): b is the per-stage latency of the two sweeps (t_bwd + t_fwd), a the
    rest of an iteration (the node-parallel phases at one node per thread and their block
    reductions).  Also the sweeps alone: backward and forward cycles per stage."""
    fits = {}
    for m in models:
        xs, ys, bw, fw = [], [], [], []
        for N in CHAIN_N:
            ps = [scenes.chain_problem(s, m, N) for s in range(seeds)]
            for p in ps:
                b = bmpc.Batch([p])
                b.set_problems()
                o = bmpc.default_opts(block_threads=64, variant=2)
                b.solve(o)
                b.solve(o)
                r = b.get_solutions(want_arrays=False)[0]
                b.close()
                it = max(1, r["inner_iters"])
                c = r["cycles"]
                per = (c["linearise"] + c["backward"] + c["forward"] + c["linesearch"]) / it
                xs.append(N + 1)
                ys.append(per)
                bw.append(c["backward"] / it / (N + 1))
                fw.append(c["forward"] / it / (N + 1))
        slope, icpt = np.polyfit(np.asarray(xs, float), np.asarray(ys, float), 1)
        fits[int(m)] = dict(a_cycles=float(icpt), b_cycles_per_stage=float(slope),
                            t_bwd_cycles=float(np.median(bw)), t_fwd_cycles=float(np.median(fw)))
    return fits


def depth(p):
    return int(np.max(p["stage"]))


def crit_cycles_per_iter(p, fits):
    f = fits[int(p["model"])]
    return f["a_cycles"] + f["b_cycles_per_stage"] * (depth(p) + 1)


# ----------------------------------------------------------------- weak scaling over ranks
def reduce_over_ranks(ms, e2e_s, n_conv, dist=None, device="cpu"):
    """The slowest rank's step times and the converged solves of all ranks: every rank solves its
    own shard of independent problems, so the whole job's rate is their sum over the max time."""
    import torch
    t = torch.tensor([ms, e2e_s], dtype=torch.float64, device=device)
    c = torch.tensor([float(n_conv)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(c[0])


# ----------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)

    # CPU baseline first (rank 0, N = 1 only), before the GPU is busy
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_rate(args.workload, args.cpu_seconds, 256)

    from paper_2506_13624_b300 import bmpc
    problems = workload(args.workload, args.batch, rank)
    stream = torch.cuda.Stream()
    b = bmpc.Batch(problems, stream=stream)
    b.set_problems()
    opts = bmpc.default_opts(block_threads=args.block_threads, blocks_per_sm=args.blocks_per_sm,
                             ls_chunk=args.ls_chunk, variant=args.variant, queue_order=args.queue_order,
                             hessian=args.hessian)
    if args.max_iters > 0:
        opts.max_iters = args.max_iters
    if args.block_threads_model:
        per_model = [int(v) for v in args.block_threads_model.split(",")]
        opts.block_threads_model = (type(opts.block_threads_model))(*(per_model + [0] * 4)[:4])
    tuned = None
    if args.autotune:
        opts, us = b.autotune(opts)
        tuned = dict(block_threads=opts.block_threads, variant=opts.variant, ls_chunk=opts.ls_chunk,
                     us_per_problem=us)
    for _ in range(args.warmup):
        b.solve(opts, graph=True)
    res = b.get_solutions(want_arrays=False)
    conv = np.array([r["status"] == 0 for r in res])

    # roof denominators measured on this device before the timed region: the FP32 FMA peak of the
    # library's microbenchmark and the critical path of single-path trees of every model present
    with torch.cuda.stream(stream):
        fp32_peak = bmpc.fp32_peak_tflops()
    fits = chain_floor(bmpc, sorted({int(p["model"]) for p in problems}))

    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        b.solve(opts, graph=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = sampler.stop() if rank == 0 else None
    res = b.get_solutions(want_arrays=False)
    n_conv = int(sum(r["status"] == 0 for r in res))

    # end to end through the C ABI with host buffers, every step: the batch's node-major inputs
    # (pinned host arrays a control loop overwrites in place) copied host to device and laid out
    # on the device, the solve, and the node-major solutions copied back into pinned host arrays.
    # Two handles on two streams take the steps in turn, so that one step's copies overlap the
    # other handle's solve; a handle waits for its previous step before it is reused.
    b2 = bmpc.Batch(problems, stream=torch.cuda.Stream())
    b2.set_problems()
    pipe = (b, b2)
    fin = b.flat_inputs()
    fouts = (b.flat_outputs(), b2.flat_outputs())
    for j, bb in enumerate(pipe):
        bb.set_problems_flat(*fin)
        bb.solve(opts, graph=True)
        bb.get_solutions_flat(fouts[j])
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        bb = pipe[k % 2]
        if k >= 2:
            bb.wait_solutions(want_stats=False)
        bb.set_problems_flat(*fin)
        bb.solve(opts, graph=True)
        bb.get_solutions_flat_async(fouts[k % 2])
    e2e_stats = [bb.wait_solutions() for bb in pipe]
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_conv = [int(sum(st[i].status == 0 for i in range(bb.n))) for bb, st in zip(pipe, e2e_stats)]
    h2d, d2h = b.transfer_bytes_flat()
    b2.close()

    ms_max, e2e_max, total_conv = reduce_over_ranks(ms, e2e_s, n_conv, dist if world > 1 else None, "cuda")
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    ms, e2e_s = ms_max, e2e_max
    value = total_conv / (ms / 1e3)
    flops = algorithmic_flops(problems, res)
    n_models = len({int(p["model"]) for p in problems})   # one solve (+ one queue-order) kernel per model
    achieved = flops / (ms / 1e3) / 1e12
    iters = np.array([r["inner_iters"] for r in res])
    # latency roof: every problem's iterations against its critical path (same cycle counter)
    meas_cyc = np.array([sum(r["cycles"][k] for k in ("linearise", "backward", "forward", "linesearch"))
                         for r in res], dtype=np.float64)
    crit_cyc = np.array([crit_cycles_per_iter(p, fits) * r["inner_iters"] for p, r in zip(problems, res)])
    lat_frac = float(crit_cyc.sum() / max(meas_cyc.sum(), 1.0))
    clk_hz = ((clocks or {}).get("sm_mhz") or SM_MAX_MHZ) * 1e6
    lat_achieved = float(iters.sum() / (meas_cyc.sum() / clk_hz))
    lat_peak = float(iters.sum() / (crit_cyc.sum() / clk_hz))
    node_iters = float(sum(int(p["n"]) * r["inner_iters"] for p, r in zip(problems, res)))
    alg_bytes = float(sum(int(p["n"]) * r["inner_iters"] * algorithmic_bytes_per_node_iter(p)
                          for p, r in zip(problems, res)))
    hbm_peak = None
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as fh:
            hbm_peak = json.load(fh).get("hbm_gbs")
    hbm_achieved = alg_bytes / (ms / 1e3) / 1e9
    clk = (clocks or {}).get("sm_mhz") or SM_MAX_MHZ
    bwd_us = np.array([r["cycles"]["backward"] for r in res]) / (clk * 1e6) * 1e6
    ric_us_iter = float(np.sum(bwd_us) / max(1, iters.sum()))
    tot_us = np.array([r["cycles"]["total"] for r in res]) / (clk * 1e6) * 1e6
    phases = {}
    for ph in ("linearise", "backward", "forward", "linesearch", "total"):
        cyc = np.array([r["cycles"][ph] for r in res], dtype=np.float64)
        phases[ph] = float(cyc.sum() / max(1, iters.sum()) / clk)   # microseconds per problem-iteration
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "batch_per_gpu": args.batch,
                   "nodes_per_gpu": int(sum(int(p["n"]) for p in problems)),
                   "l2": f"working set {(b.data_bytes + b.scratch_bytes) / 1e9:.2f} GB > 126 MB L2, no flush",
                   "launch": "one persistent kernel per model per step, CUDA graph replay",
                   "opts": {"block_threads": opts.block_threads,
                            "block_threads_model": list(opts.block_threads_model),
                            "variant": opts.variant, "ls_chunk": opts.ls_chunk,
                            "max_iters": opts.max_iters, "autotuned": tuned is not None,
                            "hessian": "exact, eigenvalue-modified" if opts.hessian else "Gauss-Newton",
                            "queue_order": "longest predicted first (previous step's iterations)"
                            if opts.queue_order == 1 else "largest tree first"}},
        "converged_fraction": float(conv.mean()),
        "node_iterations_per_step": node_iters,
        "tree_riccati_us_per_iter": ric_us_iter,
        "phase_us_per_iter": phases,
        "solve_latency_us": {"mean": float(tot_us.mean()), "max": float(tot_us.max())},
        "inner_iters": {"mean": float(iters.mean()), "max": int(iters.max()),
                        "outer_mean": float(np.mean([r["outer_iters"] for r in res])),
                        "ls_evals_per_iter": float(sum(r["ls_evals"] for r in res) / max(1, iters.sum()))},
        "gpu_launches": args.steps * n_models * (2 if opts.queue_order == 1 else 1),
        "roofline": {"bound": "latency", "achieved": lat_achieved, "peak": lat_peak,
                     "unit": "inner iterations/s per problem in flight", "frac": lat_frac,
                     "traffic": profiled_traffic(args.workload, node_iters),
                     "traffic_unit": "bytes per step (ncu dram read + write of the solve launches, scaled by "
                                     "node-iterations from a reduced-batch capture)",
                     "peak_source": "critical path per iteration: single-path trees of the same depth and model, "
                                    "one node per thread, alone on the GPU (measured before the timed region)",
                     "chain_fit_cycles": fits,
                     "alu": {"achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                             "peak_source": "measured: the library's FP32 FMA microbenchmark (bmpc_selftest_fma)"},
                     "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                             "frac": (hbm_achieved / hbm_peak) if hbm_peak else None,
                             "algorithmic_bytes_per_step": alg_bytes,
                             "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"}},
        "e2e": {"value": total_conv / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
                "converged_per_step": e2e_conv,
                "pipeline": "two handles on two streams in turn: one step's copies overlap the other's solve"},
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_single(args):
    """Single-problem latency: each of the first P problems of the workload solved alone (a batch of
    one, 512 threads per problem), timed with CUDA events over `steps` solves after `warmup`, against
    the critical path of its depth and model (the chain floor)."""
    import torch
    from paper_2506_13624_b300 import bmpc
    torch.cuda.set_device(0)
    problems = workload(args.workload, args.single)
    fits = chain_floor(bmpc, sorted({int(p["model"]) for p in problems}))
    rows = []
    for p in problems:
        s = torch.cuda.Stream()
        b = bmpc.Batch([p], stream=s)
        b.set_problems()
        o = bmpc.default_opts(block_threads=args.block_threads or 512, variant=args.variant, hessian=args.hessian)
        for _ in range(args.warmup):
            b.solve(o, graph=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            b.solve(o, graph=True)
        e1.record(s)
        e1.synchronize()
        r = b.get_solutions(want_arrays=False)[0]
        b.close()
        ms = e0.elapsed_time(e1) / args.steps
        it = max(1, r["inner_iters"])
        c = r["cycles"]
        per_cyc = (c["linearise"] + c["backward"] + c["forward"] + c["linesearch"]) / it
        clk = 2032.0   # cycles -> microseconds at the maximum SM clock (single solves: the GPU is otherwise idle)
        phases = {k: c[k] / it / clk for k in ("linearise", "backward", "forward", "linesearch")}
        rows.append(dict(nodes=int(p["n"]), depth=depth(p), model=int(p["model"]), iters=r["inner_iters"],
                         status=r["status"], ms=ms, us_per_iter=1e3 * ms / it, phase_us_per_iter=phases,
                         latency_frac=crit_cycles_per_iter(p, fits) / per_cyc,
                         bwd_fwd_share=(c["backward"] + c["forward"]) / max(1, c["total"])))
    out = {"workload": args.workload, "mode": "single problem per launch", "hessian": args.hessian,
           "chain_fit_cycles": fits,
           "mean_ms": float(np.mean([r["ms"] for r in rows])),
           "mean_us_per_iter": float(np.mean([r["us_per_iter"] for r in rows])),
           "mean_latency_frac": float(np.mean([r["latency_frac"] for r in rows])),
           "mean_phase_us_per_iter": {k: float(np.mean([r["phase_us_per_iter"][k] for r in rows]))
                                      for k in ("linearise", "backward", "forward", "linesearch")},
           "problems": rows}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- general-size tree LQR (Sec. V-A)
def lqr_work(parent, nx, nu, batch):
    """Algorithmic FP32 flops and minimum DRAM bytes of one tree LQR solve (include/bmpc_lqr.h):
    per edge T1 = PA, T2 = PB, A'T1, A'T2, B'T2, g and its products; per non-leaf node the Cholesky
    of H, the n_x + 1 solves, P and p; the forward sweep.  Bytes: every input read once, every
    output written once, and P, p, K, k read once more by the parent's step or the forward sweep."""
    n = len(parent)
    leaves = n - len(set(int(v) for v in parent[1:]))
    edges, inner = n - 1, n - leaves
    f_edge = 4 * nx ** 3 + 4 * nx * nx * nu + 2 * nx * nu * nu + 4 * nx * nx + 2 * nx * nu
    f_node = nu ** 3 / 3 + 2 * nu * nu * (nx + 1) + 2 * nx * nx * nu + 2 * nx * nu
    f_fwd = 2 * nx * nx + 2 * nx * nu
    flops = batch * (edges * (f_edge + f_fwd) + inner * (f_node + 2 * nu * nx) + n * 2 * nx * nx)
    words_in = n * (nx * nx + nx * nu + nx + nx * nx + nx) + inner * (nu * nu + nu)
    words_out = n * (nx * nx + 2 * nx + nu * nx + nu + 2 * nx + nu)
    words_reread = n * (nx * nx + nx) + inner * (nu * nx + nu)
    return float(flops), 4.0 * batch * (words_in + words_out + words_reread)


def run_lqr(args):
    """Tree LQR timings at the sizes of Sec. V-A: tree LQR against the number of scenario paths
    (n_x = 30, n_d = 2), batch LQR against the batch size (n_x = 10, N = 80) and single LQR against
    the horizon (n_x = 30).  One JSON line per case; each solve is a CUDA graph of its launches,
    timed with CUDA events over `steps` replays after `warmup`."""
    import torch
    from paper_2506_13624_b300 import bmpc, lqr
    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fp32_peak = bmpc.fp32_peak_tflops()
    hbm_peak = None
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as fh:
            hbm_peak = json.load(fh).get("hbm_gbs")
    cases = ([("tree", 15, 40, nr, 1) for nr in (1, 3, 5, 7, 9)]
             + [("batch", 5, 80, 0, b) for b in (1, 16, 64, 256, 1024)]
             + [("single", 15, N, 0, 1) for N in (20, 40, 60, 80, 100)])
    if args.lqr_only:   # e.g. "single:100" (horizon), "tree:9" (N_r), "batch:1024" (batch size)
        kind, val = args.lqr_only.split(":")
        key = {"single": 2, "tree": 3, "batch": 4}[kind]
        cases = [c for c in cases if c[0] == kind and c[key] == int(val)]
    for kind, M, N, Nr, batch in cases:
        d = scenes.mass_spring_chain(0, M=M, N=N, Nr=Nr, batch=batch)
        dev = lambda a: torch.tensor(np.ascontiguousarray(a, np.float32), device="cuda")
        ins = [dev(d[k]) for k in ("Q", "R", "q", "r", "A", "B", "c", "x0")]
        h = lqr.TreeLQR(d["parent"], d["nx"], d["nu"], batch=batch, stream=s, schedule=args.lqr_schedule)
        with torch.cuda.stream(s):
            h.solve(*ins)                                  # eager run: checks H
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                h.solve(*ins, check=False)
            for _ in range(args.warmup):
                g.replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(s)
            for _ in range(args.steps):
                g.replay()
            e1.record(s)
        e1.synchronize()
        h.status()
        us = 1e3 * e0.elapsed_time(e1) / args.steps
        flops, byts = lqr_work(d["parent"], d["nx"], d["nu"], batch)
        tf, gbs = flops / (us * 1e-6) / 1e12, byts / (us * 1e-6) / 1e9
        line = {"metric": "tree LQR solve time (Sec. V-A)", "value": us, "unit": "us/solve", "higher_is_better": False,
                "dtype": "f32", "data": "synthetic",
                "config": {"case": kind, "masses": M, "nx": d["nx"], "nu": d["nu"], "N": N, "Nr": Nr, "nd": 2 if Nr else 1,
                           "paths": 2 ** Nr, "nodes": int(len(d["parent"])), "batch": batch,
                           "schedule": "one block per problem" if h.fused else "a launch per stage and sweep",
                           "launches_per_solve": 1 if h.fused else 2 * h.stages, "steps": args.steps,
                           "warmup": args.warmup},
                "roofline": {"alu": {"achieved": tf, "peak": fp32_peak, "unit": "TFLOP/s", "frac": tf / fp32_peak,
                                     "flops_per_solve": flops},
                             "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                     "frac": gbs / hbm_peak if hbm_peak else None, "bytes_per_solve": byts},
                             "launch": {"us_per_launch": us / (1 if h.fused else 2 * h.stages)}}}
        print(json.dumps(line), flush=True)
        h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=["config1", "config2", "config3", "config4", "unicycle", "mass_spring1",
                                                            "mass_spring3", "mass_spring5", "mass_spring7", "mass_spring9"])
    ap.add_argument("--batch", type=int, default=DEFAULT_BATCH)
    ap.add_argument("--single", type=int, default=0, metavar="P",
                    help="single-problem latency of the first P problems of the workload (one per launch)")
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--block-threads-model", default="", metavar="K,D,L,U",
                    help="threads per problem for the kinematic, dynamic, linear and unicycle launches")
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--ls-chunk", type=int, default=2)
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--hessian", type=int, default=0, choices=[0, 1],
                    help="1: exact Hessian of the Lagrangian with eigenvalue modification (Sec. IV-A)")
    ap.add_argument("--queue-order", type=int, default=1, choices=[0, 1])
    ap.add_argument("--max-iters", type=int, default=0)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--lqr", action="store_true",
                    help="the general-size tree LQR at the sizes of Sec. V-A (one JSON line per case)")
    ap.add_argument("--lqr-only", default="", metavar="CASE:VALUE",
                    help="one tree LQR case: single:N, tree:N_r or batch:B")
    ap.add_argument("--lqr-schedule", type=int, default=0, choices=[0, 1, 2],
                    help="tree LQR launch schedule: 0 cost model, 1 per stage, 2 one block per problem")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=4, help="oracle problems per worker per reference step")
    ap.add_argument("--ref-workers", type=int, default=0, help="oracle worker processes (0: all host cores)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "b300":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.single:
        run_single(args)
    elif args.lqr:
        run_lqr(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
