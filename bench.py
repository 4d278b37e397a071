#!/usr/bin/env python
"""Benchmark of the end-to-end electrochemical solve on one GB300 (or N replicas).

One step = bgs_create (from device-resident CSR blocks) + bgs_setup + bgs_solve to a true
relative residual of 1e-8 on the 3D 128^3 five-field layered system (10.5M DOFs, seed 1).
`value` is the plain-method FP64 setup+solve seconds per step; the mixed-precision form
(FP32 hierarchy, BF16 coupling values, FP64 Krylov) is timed the same way and reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 the driver launches one rank per GPU with torchrun; every rank solves its own copy
(replicas: the solve has no data-parallel split on one node here), rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "setup+solve sec to rtol 1e-8 at 10.5M DOFs, mixed vs FP64 on same GB300; SpMV HBM GB/s"
# DRAM bytes (read + write) of one finest-level FP64 Chebyshev-step launch on the 128^3 phi_s block,
# per SpMV variant the autotuner can pick for it (-1 = SELL-32 with diagonal offsets, 0 = SELL-32,
# k = CSR with k threads per row), from
# the ncu captures named beside each; a variant without a capture of its current code (SELL-32's
# FP64 loop changed after its capture) reports null
CHEB_FINE_TRAFFIC = {
    -1: (206.510592e6, "profiles/k_dia_cheb_phi_s_128cubed.md"),
    1: (275.055616e6, "profiles/k_spmv1_cheb_phi_s_128cubed.md"),
}
WORKLOAD = "C4"
# FP64 peak of one GB300 from its unit counts and clock: 152 SMs x 2 FMA/clock x 2 FLOP x 2.07 GHz
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--config", default=WORKLOAD)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-c5", action="store_true", help="skip the 160x160x400 (51.2M DOFs) measurement")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-profile", action="store_true")
    p.add_argument("--no-clocks", action="store_true", help="skip the nvidia-smi clock sampler")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the block-Jacobi, DD(0)-ILU(0) species and numeric re-setup measurements")
    p.add_argument("--arms", default="both", choices=["both", "fp64", "mixed"])
    p.add_argument("--graph", type=int, default=None, help="override the library default (CUDA graph sweep)")
    p.add_argument("--reorth-eta", type=float, default=None, help="override the re-orthogonalisation threshold")
    p.add_argument("--theta-grid", default=None,
                   help="comma-separated drop tolerances: solve the phi_s block alone by FGMRES(30) with one "
                        "V-cycle per iteration for each, print one JSON line per value and exit")
    p.add_argument("--rtol", type=float, default=1e-8, help="relative tolerance for --theta-grid")
    p.add_argument("--sigma-means", default=None,
                   help="anode,separator,cathode conductivity means for --theta-grid (default: the workload's)")
    p.add_argument("--profile-case", default=None,
                   choices=["vcycle", "arnoldi", "spmv", "krylov", "setup", "gram_schmidt"],
                   help="run one small kernel case for an ncu capture and exit")
    p.add_argument("--profile-precision", type=int, default=0, choices=[0, 1],
                   help="hierarchy precision of --profile-case vcycle (0 FP64, 1 FP32)")
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------------------------
# ranks: replicas only (no data-path collective); barrier + MAX of the per-rank step time
# --------------------------------------------------------------------------------------------
def rank_barrier(dist):
    if dist is not None and dist.is_initialized():
        dist.barrier()


def rank_max(value, dist, device="cpu"):
    """MAX over ranks of a per-rank scalar (the slowest replica sets the time)."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_sum(value, dist, device="cpu"):
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): bounded sample
# --------------------------------------------------------------------------------------------
def workload_dofs(name):
    from battery_system import spec
    c = spec.CONFIGS[name]
    return 5 * c["nx"] * c["ny"] * c["nz"]


def workload_desc(name):
    from battery_system import spec
    c = spec.CONFIGS[name]
    dims = f"{c['nx']}x{c['ny']}" + (f"x{c['nz']}" if c["dim"] == 3 else "")
    kind = "layered pellet stack (20 repeats along z)" if c["stack"] else "layered system (thirds along x)"
    return f"{name}: {c['dim']}D {dims} {kind}, 5 fields (phi_s, phi_e, p, c1, c2)"


def workload_line(name, system, seed):
    return workload_desc(name) + f", {system.ndof} DOFs, {system.nnz} nnz, seed {seed}"


def oracle_threads():
    import oracle
    return oracle.set_threads(0)


def oracle_step(system):
    """One complete FP64 oracle create + setup + solve of the system on the host's threads (the
    oracle's row loops run in parallel; its results do not depend on the thread count).  Returns
    (seconds, x, info)."""
    import oracle
    t0 = time.perf_counter()
    o = oracle.bgs_for_system(system)
    x, info = o.solve(system.b)
    dt = time.perf_counter() - t0
    del o
    return dt, x, info


def reference_arm(args, rank, world):
    """The oracle on the same workload, metric and unit as the GPU arm: every step (warm-up or
    timed) is one complete create + setup + solve of the 128^3 system on the host's threads."""
    if rank != 0:
        return
    import battery_system as bs
    import oracle
    oracle.build()
    system = bs.assemble(args.config, seed=args.seed)
    threads = oracle_threads()
    for _ in range(args.warmup):
        oracle_step(system)
    times, iters = [], None
    for _ in range(args.steps):
        dt, x, info = oracle_step(system)
        times.append(dt)
        iters = info.iters
    v = statistics.mean(times)
    sample = (f"one complete oracle create+setup+solve of the {args.config} system per step on {threads} host "
              f"threads ({iters} iterations, rtol 1e-8); mean of {args.steps} steps")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded layered battery system)",
            "config": {"workload": workload_line(args.config, system, args.seed), "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------------
class _Blk:
    pass


def device_blocks(system, torch, pinned=False):
    blocks = []
    nbytes = 0
    for r in range(5):
        row = []
        for c in range(5):
            B = system.blocks.get((r, c))
            if B is None:
                row.append(None)
                continue
            o = _Blk()
            if pinned:
                o.rowptr = torch.from_numpy(B.rowptr).pin_memory()
                o.col = torch.from_numpy(B.col).pin_memory()
                o.val = torch.from_numpy(B.val).pin_memory()
                last = int(B.rowptr[-1])
            else:
                o.rowptr = torch.from_numpy(B.rowptr).cuda()
                o.col = torch.from_numpy(B.col).cuda()
                o.val = torch.from_numpy(B.val).cuda()
                last = int(B.rowptr[-1])
            nbytes += B.rowptr.nbytes + B.col.nbytes + B.val.nbytes
            from paper_2602_13079_gb300 import _Rowptr
            o.rowptr = _Rowptr(o.rowptr, last)
            row.append(o)
        blocks.append(row)
    return blocks, nbytes


def gpu_arm(args, rank, world):
    import torch
    import battery_system as bs
    from battery_system import spec
    import paper_2602_13079_gb300 as bgs
    from paper_2602_13079_gb300 import _build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    _build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        rank_barrier(dist)

    def allmax(v):
        return rank_max(v, dist, "cuda")

    tg = time.perf_counter()
    system = bs.assemble(args.config, seed=args.seed)
    t_gen = time.perf_counter() - tg
    sizes = system.field_sizes
    order = list(spec.WORKLOAD_ORDER)
    # the end-to-end inputs are staged in pinned host memory up front, before the run's other
    # large host arrays, as a caller would stage them
    if not args.no_e2e:
        hblocks, hbytes = device_blocks(system, torch, pinned=True)
        bh = torch.from_numpy(system.b).pin_memory()
        xh = torch.zeros_like(bh).pin_memory()
    blocks, mat_bytes = device_blocks(system, torch)
    b = torch.from_numpy(system.b).cuda()
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    extra = {} if args.graph is None else {"graph": args.graph}
    if args.reorth_eta is not None:
        extra["reorth_eta"] = args.reorth_eta

    def step(precision, prof=False):
        s = bgs.Solver(blocks, sizes, order, precision=precision, **extra)
        s.setup()
        if prof:
            s.bgs_set_profiling(True)
        info = s.bgs_solve(b, x)
        stats = {k: s.bgs_kernel_stats(v) for k, v in bgs.KERNEL_CLASSES.items()} if prof else None
        if prof:
            stats["_fine_format"] = s.bgs_level_format(spec.PHI_S, 0, 0)
            # FP64 operations of the finest-level Chebyshev steps of one iteration: per step 2 nnz
            # (row sum) + 5 per row (D^-1 r, e' = alpha e + D^-1 r, x' = x + c2 e'); steps per
            # V-cycle 2 deg - 1 (the first pre-smoothing step from x = 0 has no SpMV)
            flops = 0.0
            for k in range(5):
                li = s.bgs_level_info(k, 0)
                deg = s.options.cheb_degree[k]
                flops += (2 * deg - 1) * (2.0 * li["nnz"] + 5.0 * li["rows"])
            stats["_fine_flops"] = flops * info.iters
        s.close()
        return info, stats

    def timed(precision):
        for _ in range(args.warmup):
            step(precision)
        barrier()
        torch.cuda.synchronize()
        l0 = bgs.bgs_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(step(precision)[0])
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / args.steps
        launches = bgs.bgs_launch_count() - l0
        return allmax(ms), infos, launches

    clk = None if args.no_clocks else Clocks(local)
    ms64, inf64, launches64, x64 = None, None, 0, None
    msmx, infmx, xmx = None, None, None
    if args.arms in ("both", "fp64"):
        ms64, inf64, launches64 = timed(0)
        x64 = x.cpu().numpy()
    if args.arms in ("both", "mixed"):
        msmx, infmx, launchesmx = timed(1)
        xmx = x.cpu().numpy()
        if ms64 is None:
            ms64, inf64, launches64, x64 = msmx, infmx, launchesmx, xmx
    clocks = clk.stop() if clk else {"sm_mhz": None, "reasons": ["not sampled"]}

    def summary(ms, infos, xs):
        i = infos[-1]
        rel = float(np.linalg.norm(system.b - system.matvec(xs)) / np.linalg.norm(system.b))
        return {"s_per_step": ms / 1e3, "setup_s": statistics.mean(k.t_setup_ms for k in infos) / 1e3,
                "solve_s": statistics.mean(k.t_solve_ms for k in infos) / 1e3, "iters": i.iters,
                "reorth_steps": i.reorth,
                "converged": bool(i.converged), "rel_true_resid_host_check": rel}

    arm64 = summary(ms64, inf64, x64)
    armmx = summary(msmx, infmx, xmx) if msmx is not None else None
    if armmx is not None:
        armmx["rel_diff_vs_fp64"] = float(np.linalg.norm(xmx - x64) / np.linalg.norm(x64))

    # the other sweeps and block solvers, and the numeric re-setup, on the same system (FP64;
    # one warm-up and `steps` timed steps each, CUDA events on the same stream)
    variants = None
    if not args.no_variants:
        def timed_variant(fn):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = [fn() for _ in range(args.steps)]
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / args.steps, res[-1]

        def step_opts(**kw):
            def fn():
                g = bgs.Solver(blocks, sizes, order, precision=0, **kw)
                g.setup()
                info = g.bgs_solve(b, x)
                g.close()
                return info
            return fn

        variants = {}
        for name, kw in (("jacobi", dict(jacobi=1)),
                         ("dd_ilu_species", dict(subsolver=[0, 0, 0, 1, 1]))):
            ms, info = timed_variant(step_opts(**kw))
            rel = float(np.linalg.norm(system.b - system.matvec(x.cpu().numpy())) / np.linalg.norm(system.b))
            variants[name] = {"s_per_step": ms / 1e3, "setup_s": info.t_setup_ms / 1e3,
                              "solve_s": info.t_solve_ms / 1e3, "iters": info.iters,
                              "converged": bool(info.converged), "rel_true_resid_host_check": rel}
        # numeric re-setup: same handle, new values (every value x (1 + 1e-3 u)), then a solve
        g = bgs.Solver(blocks, sizes, order, precision=0)
        g.setup()
        rng = np.random.default_rng(5)
        newvals = [[None if B is None else B.val * torch.from_numpy(
            1.0 + 1e-3 * rng.uniform(0, 1, int(B.val.numel()))).cuda() for B in row] for row in blocks]

        def upd():
            g.bgs_update_values(newvals)
            return g.bgs_solve(b, x)
        ms, info = timed_variant(upd)
        variants["update_values"] = {"s_per_step": ms / 1e3, "update_s": info.t_setup_ms / 1e3,
                                     "solve_s": info.t_solve_ms / 1e3, "iters": info.iters,
                                     "converged": bool(info.converged),
                                     "note": "bgs_update_values + solve on one handle (aggregation kept)"}
        g.close()
        del newvals

    # per-kernel-class timing inside a solve (CUDA events on the library stream)
    prof = prof_mx = None
    if not args.no_profile:
        _, prof = step(0, prof=True)
        _, prof_mx = step(1, prof=True)

    # FP64 SpMV of the full operator (L2 flushed before every launch): the standalone CSR entry
    # point and the solver's own operator (SELL-32); algorithmic bytes count stored entries only
    A = system.full_csr()
    rp, ci, va = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.col, A.val))
    xs = torch.rand(A.nrows, dtype=torch.float64, device="cuda")
    ys = torch.zeros_like(xs)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    op = bgs.Solver(blocks, sizes, order, precision=0)

    def time_spmv(fn):
        out = []
        for it in range(13):
            flush.fill_(float(it))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= 3:
                out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    spmv_csr_ms = time_spmv(lambda: bgs.bgs_csr_spmv(A.nrows, A.nnz, rp, ci, va, xs, ys, 0, stream))
    spmv_lib_ms = time_spmv(lambda: op.bgs_full_spmv(xs, ys))
    spmv_layout = op.bgs_level_format(0, 0, 3, with_block=True)
    op.close()
    # bytes every layout moves (values, x, y) and the CSR layout's (plus its column and row indices)
    spmv_bytes = A.nnz * 8 + 8 * A.nrows * 2
    spmv_bytes_csr = spmv_bytes + A.nnz * 4 + 4 * (A.nrows + 1)
    spmv_gbs = spmv_bytes / (spmv_lib_ms * 1e-3) / 1e9
    spmv_ms = [spmv_lib_ms]
    del rp, ci, va, xs, ys, flush

    # end to end through the C ABI from pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        phases = []

        def hstep():
            # each library call returns after its stream work (create, setup and solve synchronise),
            # so the host clock between them splits the step without adding synchronisation
            t = [time.perf_counter()]
            s = bgs.Solver(hblocks, sizes, order, precision=0, **extra)
            t.append(time.perf_counter())
            s.setup()
            t.append(time.perf_counter())
            s.bgs_solve(bh, xh)
            t.append(time.perf_counter())
            s.close()
            t.append(time.perf_counter())
            phases.append([b - a for a, b in zip(t, t[1:])])

        hstep()
        phases.clear()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        torch.cuda.synchronize()
        barrier()
        e2e_s = allmax((time.perf_counter() - t0) / args.steps)
        split = [statistics.median(p[k] for p in phases) * 1e3 for k in range(4)]
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(hbytes + bh.numel() * 8),
               "d2h_bytes_per_step": int(xh.numel() * 8), "precision": "fp64",
               "median_ms": dict(zip(("create", "setup", "solve", "close"), (round(v, 2) for v in split))),
               "steps_ms": [[round(v * 1e3, 2) for v in p] for p in phases]}

    # the largest workload (160x160x400 pellet stack, 51.2M DOFs): FP64 and mixed, one warm-up and
    # two timed steps each (CUDA events), clocks sampled over its own timed region
    c5 = None
    if not args.no_c5 and args.config == WORKLOAD:
        del blocks, b, x
        if not args.no_e2e:
            del hblocks, bh, xh
        torch.cuda.synchronize()
        sys5 = bs.assemble("C5", seed=args.seed)
        blocks5, _ = device_blocks(sys5, torch)
        b5 = torch.from_numpy(sys5.b).cuda()
        x5 = torch.zeros_like(b5)
        torch.cuda.synchronize()

        def step5(precision):
            g5 = bgs.Solver(blocks5, sys5.field_sizes, order, precision=precision, **extra)
            g5.setup()
            info = g5.bgs_solve(b5, x5)
            g5.close()
            return info

        clk5 = None if args.no_clocks else Clocks(local)
        c5 = {"workload": workload_line("C5", sys5, args.seed), "steps": 2, "warmup": 1}
        for name, precision in (("fp64", 0), ("mixed", 1)):
            step5(precision)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos = [step5(precision) for _ in range(2)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms = allmax(e0.elapsed_time(e1) / 2)
            xs5 = x5.cpu().numpy()
            rel = float(np.linalg.norm(sys5.b - sys5.matvec(xs5)) / np.linalg.norm(sys5.b))
            c5[name] = {"s_per_step": ms / 1e3, "setup_s": statistics.mean(k.t_setup_ms for k in infos) / 1e3,
                        "solve_s": statistics.mean(k.t_solve_ms for k in infos) / 1e3, "iters": infos[-1].iters,
                        "converged": bool(infos[-1].converged), "rel_true_resid_host_check": rel}
        c5["mixed_speedup_vs_fp64"] = c5["fp64"]["s_per_step"] / c5["mixed"]["s_per_step"]
        c5["clocks"] = clk5.stop() if clk5 else None
        del blocks5, b5, x5, sys5

    peak, peak_kind = measured_peaks()
    roof = None
    if prof:
        # Dominant kernel: the fused Chebyshev step on the finest level (top share of the ncu launch
        # list, profiles/launch_list_c4_fp64_step.md), in the SpMV variant the autotuner chose for the
        # 128^3 diagonal blocks in this process
        fmt = prof.pop("_fine_format")
        kname = ("k_dia<double,double,double,ECheb>" if fmt == -1 else
                 "k_sell<double,double,double,ECheb>" if fmt == 0 else f"k_spmv<{fmt},double,double,double,ECheb>")
        traffic, tsrc = CHEB_FINE_TRAFFIC.get(fmt, (None, "no ncu capture of this variant"))
        fine_flops = prof.pop("_fine_flops")
        d = prof["chebyshev_fine"]
        ach = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
        roof = {"bound": "hbm", "kernel": kname + " (Chebyshev step, finest level, FP64)",
                "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_kind": peak_kind,
                "traffic": traffic, "traffic_source": tsrc,
                "launches": d["launches"], "avg_launch_ms": d["ms"] / max(d["launches"], 1),
                "bytes_per_launch": d["bytes"] / max(d["launches"], 1),
                # the same kernel against the FP64 pipe, the other limit of the FP64 step: 152 SMs x
                # 2 FP64 FMA per clock x 2.07 GHz = 1.26 TFLOP/s nominal
                "fp64_pipe": {"bound": "alu", "achieved": fine_flops / (d["ms"] * 1e-3) / 1e12,
                              "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                              "frac": fine_flops / (d["ms"] * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS},
                "classes": {k: {"launches": v["launches"], "ms": v["ms"],
                                "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                            for k, v in prof.items()}}
        if prof_mx:
            fmx = prof_mx.pop("_fine_format")
            prof_mx.pop("_fine_flops")
            roof["fine_kernel_mixed"] = ("k_dia<float,float,float,ECheb>" if fmx == -1 else
                                         "k_sell<float,float,float,ECheb>" if fmx == 0 else
                                         f"k_spmv<{fmx},float,float,float,ECheb>")
            roof["classes_mixed"] = {k: {"launches": v["launches"], "ms": v["ms"],
                                         "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                                     for k, v in prof_mx.items()}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # one complete oracle run of the same system on the host's threads; its solution also gives
        # the error of both GPU forms against the FP64 oracle
        threads = oracle_threads()
        dt, xo, io = oracle_step(system)
        cpu = {"value": dt, "unit": "s", "cores": threads, "kind": "oracle",
               "sample": f"one complete oracle create+setup+solve of the same {args.config} system "
                         f"({io.iters} iterations) on {threads} host threads"}
        on = np.linalg.norm(xo)
        arm64["rel_err_vs_oracle"] = float(np.linalg.norm(x64 - xo) / on)
        if armmx is not None:
            armmx["rel_err_vs_oracle"] = float(np.linalg.norm(xmx - xo) / on)
        del xo

    if rank == 0:
        v = ms64 / 1e3
        line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded layered battery system)",
                "config": {"workload": workload_line(args.config, system, args.seed),
                           "order": "[phi_s, phi_e] -> p -> [c1, c2]", "rtol": 1e-8, "restart": 50,
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": f"inputs larger than L2 (matrix {system.nnz * 12 / 1e9:.1f} GB)",
                           "generation_s": t_gen,
                           "graph": int(bgs.bgs_default_options(**extra).graph)},
                "fp64": arm64, "mixed": armmx, "variants": variants,
                "mixed_speedup_vs_fp64": (ms64 / msmx) if msmx else None,
                "spmv_full_fp64": {"layout": {-2: "node blocks", -1: "diagonal-offset SELL-32",
                                              0: "SELL-32"}.get(spmv_layout[0], f"CSR, {spmv_layout[0]} lanes"),
                                   "threads_per_block": spmv_layout[1],
                                   "ms": statistics.median(spmv_ms), "bytes": spmv_bytes, "GBps": spmv_gbs,
                                   "frac_of_measured_peak": spmv_gbs / peak,
                                   "bytes_note": "values + x + y, the bytes every layout moves",
                                   "csr_ms": spmv_csr_ms,
                                   "csr_GBps": spmv_bytes_csr / (spmv_csr_ms * 1e-3) / 1e9},
                "solves_per_s": world / (ms64 / 1e3),
                "gpu_launches": int(launches64 // max(args.steps, 1)) * args.steps,
                "gpu_launches_per_step": int(launches64 // max(args.steps, 1)),
                "clocks": clocks, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "c5": c5}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def profile_case(args):
    """Small, self-contained cases for single-kernel ncu captures (inputs larger than L2, a few
    GB on the device): one V-cycle on the 128^3 phi_s block alone; one Arnoldi dot pass over 16
    basis vectors of 10.5M entries; one SpMV with the 128^3 full operator; one FP64 solve of the
    64^3 system launched step by step (the Arnoldi update kernels); and, not for ncu, the set-up's
    phase timeline at 128^3 (stderr)."""
    import torch
    import battery_system as bs
    import paper_2602_13079_gb300 as bgs
    from paper_2602_13079_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    if args.profile_case == "arnoldi":
        n, cnt = 5 * 128 ** 3, 16
        V = torch.rand((cnt, n), dtype=torch.float64, device="cuda")
        w = torch.rand(n, dtype=torch.float64, device="cuda")
        h = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
        for _ in range(2):
            assert bgs.bgs_arnoldi_dots(V, n, cnt, w, n, h) == 0
        torch.cuda.synchronize()
        print("arnoldi case done", float(h[-1]))
        return
    if args.profile_case == "gram_schmidt":
        # the FGMRES Gram-Schmidt pass (dots and update, FP64 / fixed-point split) at 128^3 rows with
        # 16 unit basis vectors, as in a mid-cycle Arnoldi step
        n, cnt = 5 * 128 ** 3, 16
        V = torch.randn((cnt, n), dtype=torch.float64, device="cuda")
        V /= V.norm(dim=1, keepdim=True)
        w0 = torch.randn(n, dtype=torch.float64, device="cuda")
        h = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
        nw = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(2):
            w = w0.clone()
            assert bgs.bgs_gram_schmidt_pass(V, n, cnt, w, n, h, nw) == 0
        torch.cuda.synchronize()
        print("gram_schmidt case done", float(nw[0]))
        return
    if args.profile_case == "krylov":
        # one FP64 solve of the 3D 64^3 system (1.31M DOFs): the Arnoldi kernels of its later
        # iterations read more basis than L2 holds (20 vectors of 10.5 MB)
        system = bs.assemble("C2", seed=args.seed)
        g = bgs.solver_for_system(system, graph=0)
        g.setup()
        x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
        info = g.bgs_solve(torch.from_numpy(system.b).cuda(), x)
        torch.cuda.synchronize()
        print("krylov case done", info.iters)
        return
    system = bs.assemble(args.config, seed=args.seed)
    if args.profile_case == "setup":
        # the set-up's timeline (BGS_TRACE=async: host clock and stream of every phase mark, to
        # stderr) for one set-up per precision after three untraced ones
        blocks, _ = device_blocks(system, torch)
        for precision in (0, 1):
            for rep in range(4):
                if rep == 3:
                    os.environ["BGS_TRACE"] = "async"
                    print(f"=== precision {precision}", file=sys.stderr, flush=True)
                s = bgs.Solver(blocks, system.field_sizes, list(range(5)), precision=precision)
                s.setup()
                torch.cuda.synchronize()
                sys.stderr.flush()
                os.environ.pop("BGS_TRACE", None)
                s.close()
        print("setup case done")
        return
    if args.profile_case == "vcycle":
        B = system.blocks[(0, 0)]

        class _B:
            pass
        o = _B()
        o.rowptr, o.col, o.val = B.rowptr, B.col, B.val
        s = bgs.Solver([[o]], [B.nrows], [0], precision=args.profile_precision)
        s.setup()
        b = torch.from_numpy(system.b[:B.nrows].copy()).cuda()
        x = torch.zeros_like(b)
        for _ in range(2):
            s.bgs_apply_vcycle(0, b, x)
        torch.cuda.synchronize()
        print("vcycle case done", float(x.norm()))
    else:
        blocks, _ = device_blocks(system, torch)
        s = bgs.Solver(blocks, system.field_sizes, list(range(5)))
        xs = torch.rand(system.ndof, dtype=torch.float64, device="cuda")
        ys = torch.zeros_like(xs)
        for _ in range(2):
            s.bgs_full_spmv(xs, ys)
        torch.cuda.synchronize()
        print("spmv case done", float(ys.norm()))


def theta_grid(args):
    """The drop-tolerance grid search of Sec. 3.1.4 on the phi_s block of the workload: for each
    theta, set-up and FGMRES(30) solve to 1e-8 with one V-cycle per iteration (CUDA events), the
    level sizes and the iteration count."""
    import torch
    import battery_system as bs
    import paper_2602_13079_gb300 as bgs
    from paper_2602_13079_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    sig = tuple(float(v) for v in args.sigma_means.split(",")) if args.sigma_means else None
    system = bs.assemble(args.config, seed=args.seed, sigma_means=sig)
    B = system.blocks[(0, 0)]

    class _B:
        pass
    o = _B()
    o.rowptr, o.col, o.val = B.rowptr, B.col, B.val
    b = torch.from_numpy(system.b[:B.nrows].copy()).cuda()
    for th in (float(t) for t in args.theta_grid.split(",")):
        line = {"theta": th, "workload": workload_desc(args.config) + " phi_s block", "rows": B.nrows,
                "sigma_means": list(sig) if sig else "workload"}
        try:
            times = []
            for rep in range(3):
                x = torch.zeros_like(b)
                g = bgs.Solver([[o]], [B.nrows], [0], restart=30, theta=[th], rtol=args.rtol)
                t0 = time.perf_counter()
                g.setup()
                info = g.bgs_solve(b, x, check=False)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
                levels = [g.bgs_level_info(0, l)["rows"] for l in range(g.bgs_num_levels(0))]
                g.close()
            line.update({"rtol": args.rtol, "iters": info.iters, "converged": bool(info.converged),
                         "rel_true_resid": info.rel_true_resid, "setup_s": info.t_setup_ms / 1e3,
                         "solve_s": info.t_solve_ms / 1e3, "setup_plus_solve_s": min(times[1:]),
                         "levels": levels})
        except bgs.BGSError as e:
            line.update({"error": str(e)})
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
    if args.theta_grid:
        theta_grid(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    gpu_arm(args, rank, world)


if __name__ == "__main__":
    main()
