#!/usr/bin/env python
"""Benchmark: implicit steps/s of the 1,024-fiber x 64-point curved-fiber cloud
(65,536 points in [0,40]^3, N(0,1) external force per node), mixed precision
(FP32 far field inside GMRES, FP64 refinement to 1e-8), one GPU per rank.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Each rank solves an independent replica (seed = rank): weak scaling, no
collective on the data path; the barrier and the max-over-ranks timing use
torch.distributed.  Prints ONE JSON line on rank 0.

--impl reference times the CPU oracle (the plain FP64 implementation in
oracle/) on a bounded sample of the same workload on this host's cores.
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

import workloads as wl  # noqa: E402

# algorithmic flops per pair: the Stokeslet formula (27), the stresslet (31)
# and the float-float evaluations of the Stokeslet (218) and the stresslet
# (235), FMA = 2, counted from the float-float formulas; the rsqrt seed is on
# the SFU and not counted
FLOPS_PER_PAIR = {"stokeslet": 27.0, "stresslet": 31.0, "stokeslet_ff": 218.0, "stresslet_ff": 235.0}
KS_NAMES = ["stokeslet_fp32", "stokeslet_fp64", "stresslet_fp32", "stresslet_fp64", "stokeslet_ff",
            "stokeslet_fp32_plain", "stresslet_ff"]
WORKLOAD = "cloud-1024x64: 1,024 curved fibers x 64 Chebyshev points (65,536 points), [0,40]^3"


# the library's default inner tolerance of the mixed solve (fs_options_default);
# both arms name it in their config
DEFAULT_INNER_TOL = 1e-6


def workload_config(s, ws: int, inner_tol: float, relax: int) -> dict:
    """The headline workload as both arms report it: the cloud, its physical
    parameters, the solve's tolerances and how it is run."""
    return {"workload": WORKLOAD, "fibers": s.n_fibers, "points_per_fiber": 64,
            "precision": "mixed", "tol": 1e-8, "inner_tol": inner_tol, "relax": relax,
            "eps": s.eps, "mu": s.mu, "E": s.E, "dt": s.dt,
            "state": "every step from the initial cloud (device-to-device reset timed)",
            "l2": "inputs larger than L2 (per-step fiber blocks 537 MB, Krylov basis 128 MB)",
            "parallelism": "replicas" if ws > 1 else "1 GPU"}


def job_time(x: float, dist, device) -> float:
    """A per-rank time as the job's: the maximum over ranks (the job ends
    with its slowest rank); unchanged on one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed (replicas, weak
    scaling) over the job's time."""
    return units_per_rank * ws / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 9 for k in range(4)
                          if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), with the
    architecture."""
    import platform
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return "%s (%s)" % (name or "unknown model", platform.machine())


def oracle_baseline(s, gpu_fp64_iters: int, budget_fibers: int = 512, budget_targets: int = 32768):
    """Time the CPU oracle on a bounded sample of the workload and scale to one
    step: per-fiber setup (geometry, self block, LU) for `budget_fibers` fibers
    scaled to all fibers, plus (1 + iters) far-field sums, each timed on
    `budget_targets` targets x all sources and scaled to all targets."""
    from oracle import kernels as ok
    from oracle import system
    ok.build()
    M, N = s.n_fibers, int(s.n_per_fiber[0])
    sub = wl.Suspension(s.n_per_fiber[:budget_fibers], s.X[:budget_fibers * N], s.L[:budget_fibers],
                        s.f_ext[:budget_fibers * N], s.mu, s.eps, s.E, s.dt)
    t0 = time.perf_counter()
    system.from_suspension(sub)
    t_setup = (time.perf_counter() - t0) * M / budget_fibers
    fid = s.fiber_id()
    W = np.repeat(s.L / 2.0, N)[:, None] * 0.02 * s.f_ext
    idx = np.linspace(0, s.n_points - 1, budget_targets).astype(np.int64)
    t0 = time.perf_counter()
    ok.stokeslet(s.X[idx], s.X, W, s.mu, fid[idx], fid)
    t_ff = (time.perf_counter() - t0) * s.n_points / budget_targets
    n_ff = 1 + gpu_fp64_iters
    t_step = t_setup + n_ff * t_ff
    sample = ("oracle setup of %d of %d fibers (x%.0f) + far-field sum on %d of %d targets "
              "(x%.0f), times %d far fields (right-hand side + %d GMRES iterations of the FP64 "
              "path on the same step); %.1f s measured" % (
                  budget_fibers, M, M / budget_fibers, budget_targets, s.n_points,
                  s.n_points / budget_targets, n_ff, gpu_fp64_iters,
                  t_setup * budget_fibers / M + t_ff * budget_targets / s.n_points))
    return {"value": 1.0 / t_step, "unit": "steps/s", "cores": ok.threads(), "cpu": cpu_model(),
            "kind": "oracle", "sample": sample, "seconds_per_step_extrapolated": t_step}


def traffic_for(kernel_class: str, name: str = "traffic.txt"):
    """A per-launch ncu figure of a direct-sum kernel class from a committed
    summary under profiles/ (DRAM bytes per launch, dram__bytes_read.sum +
    dram__bytes_write.sum, in traffic.txt; the FMA-pipe active fraction in
    pipe_util.txt), if it was taken on the current source of the direct-sum
    kernels (else None).  Lines: <kernel class> <value> <sha1 of
    csrc/pairsum.cu>."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    try:
        import hashlib
        src = open(os.path.join(ROOT, "paper_1602_05650_gb300", "csrc", "pairsum.cu"), "rb").read()
        sha = hashlib.sha1(src).hexdigest()
        for line in open(p):
            f = line.split()
            if len(f) == 3 and not line.startswith("#") and f[0] == kernel_class and f[2] == sha:
                return float(f[1])
    except Exception:
        return None
    return None


def run_reference(args, ws, rank):
    if rank != 0:
        return
    s = wl.cfg_cloud_mixed(0)
    vals = []
    base = None
    for k in range(args.warmup + args.steps):
        base = oracle_baseline(s, gpu_fp64_iters=args.ref_iters, budget_fibers=128, budget_targets=8192)
        if k >= args.warmup:
            vals.append(base["seconds_per_step_extrapolated"])
    t = float(np.mean(vals))
    line = {"metric": "implicit steps/s (%s; mixed FP32/FP64, GMRES 1e-8)" % WORKLOAD,
            "value": 1.0 / t, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(s, ws, args.inner_tol if args.inner_tol > 0 else DEFAULT_INNER_TOL,
                                      0 if args.no_relax else 1),
            "cpu_baseline": {"kind": "oracle", "cores": base["cores"], "cpu": base["cpu"],
                             "sample": base["sample"], "value": 1.0 / t, "unit": "steps/s"},
            "e2e": {"value": 1.0 / t, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_kernel(args, ws, rank, local, fs, torch, dist):
    """Direct-sum kernel alone: the cloud's far field with same-fiber exclusion."""
    dev = torch.device("cuda", local)
    s = wl.cfg_cloud_mixed(seed=rank)
    P = args.points or s.n_points
    prec = {"stokeslet_fp32": fs.FS_SUM_FP32, "stokeslet_fp64": fs.FS_SUM_FP64, "stokeslet_ff": fs.FS_SUM_FF,
            "stokeslet_fp32_plain": fs.FS_SUM_FP32_PLAIN}[args.kernel]
    opt = fs.fs_options_default()
    opt.profile = 1
    opt.tile_override = args.tile
    stream = torch.cuda.Stream(device=dev)
    h = fs.fs_create([], s.mu, s.eps, s.E, s.dt, options=opt, stream=stream)
    X = torch.tensor(s.X[:P], dtype=torch.float64, device=dev)
    Wf = torch.tensor(s.f_ext[:P] * 0.02, dtype=torch.float64, device=dev)
    fid = torch.tensor(s.fiber_id()[:P], dtype=torch.int32, device=dev)
    out = torch.empty_like(X)
    for _ in range(args.warmup):
        fs.fs_stokeslet_apply(h, X, Wf, X, out, fid, fid, prec)
    torch.cuda.synchronize()
    fs.fs_kernel_stats(h, reset=True)
    for _ in range(args.steps):
        fs.fs_stokeslet_apply(h, X, Wf, X, out, fid, fid, prec)
    st = fs.fs_kernel_stats(h, reset=True)[{fs.FS_SUM_FP32: 0, fs.FS_SUM_FP64: 1, fs.FS_SUM_FF: 4,
                                            fs.FS_SUM_FP32_PLAIN: 5}[prec]]
    fs.fs_destroy(h)
    if rank == 0:
        pairs_s = st[2] / (st[1] * 1e-3)
        fpp = FLOPS_PER_PAIR["stokeslet_ff" if args.kernel == "stokeslet_ff" else "stokeslet"]
        print(json.dumps({"kernel": args.kernel, "tile": args.tile, "points": P, "launches": st[0],
                          "ms_per_launch": st[1] / st[0], "pairs_per_s": pairs_s,
                          "tflops": fpp * pairs_s / 1e12}), flush=True)


def _timed_steps(fs, torch, h, stream, X, L, F, steps, warmup):
    """Every step from the same state; CUDA events on the context's stream."""
    for _ in range(warmup):
        fs.fs_set_state(h, X, L, F)
        fs.fs_step(h, info=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(steps):
        fs.fs_set_state(h, X, L, F)
        infos.append(fs.fs_step(h, info=True))
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, infos


def run_workload(args, ws, rank, local, fs, torch):
    """Secondary workloads (one JSON line each, not the headline):
    confined  2,000 x 32 fibers in a radius-20 sphere with 12,288 surface nodes,
              mixed and FP64 steps/s;
    batched   256 independent systems (fibers log-uniform in [8, 512], N in
              {16, 32, 64}) in one context, mixed steps/s and systems/s:
              host-driven cycles, graph cycles, and autotuned launch shapes;
    large     the 1,048,576-point Stokeslet sum (8,192 x 128 fibers in
              [0,80]^3, own-fiber exclusion): direct in FP32 hi/lo, FP32 plain
              and float-float over all targets, FP64 over 16,384 sampled
              targets; the treecode at orders 6 and 8 with its error on the
              sampled targets;
    sediment  the four sedimenting clouds of Sec. 4.3 (1,024 x 16 each) in
              one batch, advanced --steps steps: steps/s and the settling
              speeds relative to V_c;
    kinetics  1,024 growing and shrinking microtubules (dynamic instability
              with the paper's rates), advanced --steps steps;
    tree-step one implicit step of 1,048,576 points (32,768 fibers x 32) with
              the treecode far field and with the direct one;
    tree-case one treecode sum of 262,144 points (4,096 fibers x 64 in
              [0,50]^3, own-fiber exclusion) at --tree-order / --tree-theta,
              timed after one untimed call: the small case for profiling the
              treecode's kernels;
    aster     the confined aster of Table 2 (32, 128, 512 and 2,048 fibers x
              31 points clamped to a sphere inside a sphere six radii out,
              force on the sphere, GMRES 1e-5): steps/s and GMRES iterations
              per step, FP64 (up to 512 fibers) and mixed, advanced --steps
              steps after --warmup steps;
    precond   the preconditioner build (fs_build_precond: self blocks and
              their LU) of curved free-space clouds at N = 16, 32, 64 (4,096,
              2,048, 1,024 fibers): FP64 build and LU, tensor-core build with
              the FP64 LU, tensor-core build and LU; ms per build, CUDA events
              over --steps builds after --warmup."""
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    out = {"workload": args.workload, "data": "synthetic"}
    if args.workload == "precond":
        res = {}
        for N, M in ((16, 4096), (32, 2048), (64, 1024)):
            s = wl.free_space(M, N, 40.0 * (M / 1024) ** (1 / 3), seed=rank, curved_amp=0.05)
            X = torch.tensor(s.X, dtype=torch.float64, device=dev)
            L = torch.tensor(s.L, dtype=torch.float64, device=dev)
            F = torch.tensor(s.f_ext, dtype=torch.float64, device=dev)
            for name, tcb, tcl in (("fp64", 0, 0), ("tc_build", 1, 0), ("tc_build_lu", 1, 1)):
                opt = fs.fs_options_default()
                opt.tc_blocks, opt.tc_lu = tcb, tcl
                h = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, options=opt, stream=stream)
                fs.fs_set_state(h, X, L, F)
                for _ in range(args.warmup):
                    fs.fs_build_precond(h)
                stream.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    fs.fs_build_precond(h)
                e1.record(stream)
                e1.synchronize()
                res["N%d_%s" % (N, name)] = round(e0.elapsed_time(e1) / max(args.steps, 1), 3)
                fs.fs_destroy(h)
        out.update({"ms_per_build": res, "fibers": {"16": 4096, "32": 2048, "64": 1024}})
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.workload in ("confined", "batched"):
        if args.workload == "confined":
            s = wl.cfg_confined(seed=rank)
            systems = [s]
        else:
            systems = wl.batched(256, seed=rank)
        res = {}
        legs = (("mixed", fs.FS_MIXED, 0, 0), ("fp64", fs.FS_FP64, 0, 0))
        if args.workload == "batched":
            # the host-driven cycles (kernel timings), the graph cycles (one
            # graph launch per restart cycle; event records off) and the
            # autotuned launch shapes (tuned in the warm-up steps)
            legs = (("mixed", fs.FS_MIXED, 0, 0), ("mixed_graph", fs.FS_MIXED, 1, 0),
                    ("mixed_autotune", fs.FS_MIXED, 0, 1))
        for name, prec, graph, tune in legs:
            opt = fs.fs_options_default()
            opt.prec = prec
            opt.tol = 1e-8
            opt.profile = 0 if graph else 1
            opt.use_graph = graph
            opt.autotune = tune
            if args.workload == "confined":
                h = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, boundary=s.boundary, options=opt,
                                 stream=stream)
            else:
                h = fs.fs_create_batch([x.n_fibers for x in systems],
                                       np.concatenate([x.n_per_fiber for x in systems]),
                                       1.0, 1e-3, 1.0, 1e-3, options=opt, stream=stream)
            X = torch.tensor(np.concatenate([x.X for x in systems]), device=dev)
            L = torch.tensor(np.concatenate([x.L for x in systems]), device=dev)
            F = torch.tensor(np.concatenate([x.f_ext for x in systems]), device=dev)
            steps = 1 if name == "fp64" else args.steps
            ms, infos = _timed_steps(fs, torch, h, stream, X, L, F, steps, 1 if name == "fp64" else args.warmup)
            ks = fs.fs_kernel_stats(h)
            tuned = fs.fs_get_tuned_shapes(h)
            fs.fs_destroy(h)
            res[name] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "iters": [i.iters for i in infos],
                         "resid": [i.resid for i in infos],
                         "t_ms_rhs_build_solve": [round(x, 2) for x in infos[0].t_ms[:3]],
                         "kernels": {KS_NAMES[k]: [ks[k][0], round(ks[k][1], 2)] for k in range(7) if ks[k][0]}}
            if tune:
                res[name]["tuned_shapes"] = {"prec%d_hilo%d" % k: v for k, v in tuned.items()}
        pts = sum(x.n_points for x in systems)
        out.update({"points": int(pts), "systems": len(systems), "tol": 1e-8, "result": res})
        if args.workload == "confined":
            out["surface_nodes"] = int(s.boundary.nodes.shape[0])
        else:
            out["systems_per_s"] = len(systems) * res["mixed"]["steps_per_s"]
            out["systems_per_s_graph"] = len(systems) * res["mixed_graph"]["steps_per_s"]
            out["systems_per_s_autotune"] = len(systems) * res["mixed_autotune"]["steps_per_s"]
            out["fibers"] = [int(min(x.n_fibers for x in systems)), int(max(x.n_fibers for x in systems))]
    elif args.workload == "sediment":
        # Sec. 4.3: the four clouds (1,024 fibers x 16 points, L/R0 = 0.15,
        # 0.25, 0.32, 0.40, fibers at least 0.1 L apart) as one batch,
        # advanced --steps steps after one untimed step
        lens = (0.15, 0.25, 0.32, 0.40)
        clouds = [wl.sedimenting_cloud(Lr, M=1024, N=16, seed=100 * rank + k) for k, Lr in enumerate(lens)]
        opt = fs.fs_options_default()
        opt.prec = fs.FS_MIXED
        opt.tol = 1e-8
        opt.profile = 1
        h = fs.fs_create_batch([c.n_fibers for c in clouds], np.concatenate([c.n_per_fiber for c in clouds]),
                               1.0, 0.01, 3.2e-3, clouds[0].dt, options=opt, stream=stream)
        X = torch.tensor(np.concatenate([c.X for c in clouds]), device=dev)
        fs.fs_set_state(h, X, torch.tensor(np.concatenate([c.L for c in clouds]), device=dev),
                        torch.tensor(np.concatenate([c.f_ext for c in clouds]), device=dev))
        sizes = np.cumsum([0] + [c.n_points for c in clouds])
        V = torch.empty_like(X)
        Xe = torch.empty_like(X)

        def speeds():
            fs.fs_get_state(h, V=V)
            return [round(-V[sizes[k]:sizes[k + 1], 2].mean().item() / wl.cloud_velocity_scale(clouds[k]), 4)
                    for k in range(4)]

        fs.fs_step(h)
        first = speeds()
        fs.fs_get_state(h, X=Xe)
        z0 = [Xe[sizes[k]:sizes[k + 1], 2].mean().item() for k in range(4)]
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        iters = []
        for _ in range(args.steps):
            iters.append(fs.fs_step(h, info=True).iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        last = speeds()
        fs.fs_get_state(h, X=Xe)
        fs.fs_destroy(h)
        drop = [round(z0[k] - Xe[sizes[k]:sizes[k + 1], 2].mean().item(), 5) for k in range(4)]
        out.update({"L_over_R0": list(lens), "fibers_per_cloud": 1024, "points_per_fiber": 16,
                    "points": int(sizes[-1]), "dt": clouds[0].dt, "steps": args.steps,
                    "ms_per_step": ms, "steps_per_s": 1e3 / ms, "iters": iters,
                    "settling_speed_over_Vc_first_step": first, "settling_speed_over_Vc_last_step": last,
                    "centre_of_mass_drop_over_R0": drop})
    elif args.workload == "kinetics":
        # 1,024 straight microtubules (L in [5, 10] um, 32 points, eps 1e-3,
        # E = 10 pN um^2, mu = 1 pN s / um^2) in a 60 um box, at least 0.1 L
        # apart (closer pairs go unstable under plain quadrature), weak body force,
        # dynamic instability with the rates of the paper's parameter table
        # (V_g 0.12, V_s 0.288 um/s, f_cat = f_res = 0.014 / s), rescue at
        # 2 um, dt = 0.1 s; the growth term at the new time (the paper's
        # explicit term is unstable for shrinking fibers at this dt)
        mt = wl.MICROTUBULE
        s = wl.free_space(1024, 32, 60.0, seed=rank, L_range=(5.0, 10.0), mu=mt["mu"], E=mt["E"], dt=0.1,
                          min_gap=0.1)
        s.f_ext = np.tile([0.0, 0.0, -0.05], (s.n_points, 1))
        kin_args = (s.dt, mt["v_grow"], mt["v_shrink"], mt["f_cat"], mt["f_res"], 2.0)
        opt = fs.fs_options_default()
        opt.prec = fs.FS_MIXED
        opt.tol = 1e-8
        opt.profile = 1
        opt.growth_implicit = 1
        h = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, options=opt, stream=stream)
        X = torch.tensor(s.X, device=dev)
        fs.fs_set_state(h, X, torch.tensor(s.L, device=dev), torch.tensor(s.f_ext, device=dev))
        rng = np.random.default_rng(rank)
        state = np.ones(s.n_fibers, dtype=np.int32)

        def one_step(info):
            nonlocal state
            L = fs.fs_get_lengths(h, s.n_fibers)
            state, Ld = fs.fs_dynamic_instability(state, L, rng.random(s.n_fibers), *kin_args)
            fs.fs_set_growth(h, Ld)
            return fs.fs_step(h, info=info)

        for _ in range(args.warmup):
            one_step(False)
        L0 = fs.fs_get_lengths(h, s.n_fibers)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        iters = [one_step(True).iters for _ in range(args.steps)]
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / args.steps
        L1 = fs.fs_get_lengths(h, s.n_fibers)
        fs.fs_destroy(h)
        out.update({"points": int(s.n_points), "fibers": s.n_fibers, "dt_s": s.dt,
                    "steps": args.steps, "ms_per_step": 1e3 * sec, "steps_per_s": 1.0 / sec,
                    "timing": "host wall clock per step (state machine, rates upload and step)",
                    "growth": "implicit (growth_implicit = 1)",
                    "iters": iters, "mean_length_um": [float(L0.mean()), float(L1.mean())],
                    "growing_fraction": float(state.mean())})
    elif args.workload == "tree-step":
        # 1,048,576 points (32,768 straight fibers x 32 points in [0,100]^3,
        # the cloud's density; N(0,1) force per node), one mixed step at tol
        # 1e-5 with the treecode far field (order 8, theta 0.5) and one with
        # the direct far field, from the same state; velocity difference
        s = wl.free_space(32768, 32, 100.0, seed=rank)
        X = torch.tensor(s.X, device=dev)
        L = torch.tensor(s.L, device=dev)
        F = torch.tensor(s.f_ext, device=dev)
        res, V = {}, {}
        for name, order in (("tree_p8_theta0.5", 8), ("direct", 0)):
            opt = fs.fs_options_default()
            opt.prec = fs.FS_MIXED
            opt.tol = 1e-5
            opt.tree_order = order
            opt.tree_theta = 0.5
            h = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, options=opt, stream=stream)
            steps = 1 if order == 0 else max(1, min(args.steps, 3))
            ms, infos = _timed_steps(fs, torch, h, stream, X, L, F, steps, 1 if order else 0)
            V[name] = torch.empty_like(X)
            fs.fs_get_state(h, V=V[name])
            fs.fs_destroy(h)
            res[name] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "iters": [i.iters for i in infos],
                         "outer": [i.refine_sweeps for i in infos], "resid": [i.resid for i in infos],
                         "t_ms_rhs_build_solve": [round(x, 1) for x in infos[0].t_ms[:3]]}
        dv = (torch.linalg.norm(V["tree_p8_theta0.5"] - V["direct"]) / torch.linalg.norm(V["direct"])).item()
        out.update({"points": int(s.n_points), "fibers": s.n_fibers, "points_per_fiber": 32, "tol": 1e-5,
                    "result": res, "velocity_rel_difference_tree_vs_direct": dv,
                    "speedup_tree_vs_direct": res["direct"]["ms_per_step"] / res["tree_p8_theta0.5"]["ms_per_step"]})
    elif args.workload == "tree-case":
        s = wl.free_space(4096, 64, 50.0, seed=rank)
        h = fs.fs_create([], s.mu, s.eps, s.E, s.dt, stream=stream)
        X = torch.tensor(s.X, device=dev)
        Wf = torch.tensor(s.f_ext * 0.01, device=dev)
        fid = torch.tensor(s.fiber_id(), dtype=torch.int32, device=dev)
        ut = torch.empty_like(X)
        order, theta = args.tree_order, args.tree_theta
        fs.fs_stokeslet_apply_tree(h, X, Wf, X, ut, fid, fid, order=order, theta=theta)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fs.fs_stokeslet_apply_tree(h, X, Wf, X, ut, fid, fid, order=order, theta=theta)
        e1.record(stream)
        torch.cuda.synchronize()
        fs.fs_destroy(h)
        out.update({"points": int(s.n_points), "order": order, "theta": theta,
                    "ms_per_call": e0.elapsed_time(e1)})
    elif args.workload == "aster":
        res = {}
        for nf in (32, 128, 512, 2048):
            s = wl.table2_aster(nf, seed=rank)
            row = {}
            variants = [("mixed", fs.FS_MIXED)]
            if nf <= 512:   # the FP64 far field of 63,488 points costs ~0.1 s a matvec
                variants = [("fp64", fs.FS_FP64)] + variants
            for name, prec in variants:
                opt = fs.fs_options_default()
                opt.prec = prec
                opt.tol = 1e-5
                opt.max_iter = 600
                opt.profile = 1
                h = fs.fs_create_with_body(s.n_per_fiber, s.attach, s.mu, s.eps, s.E, s.dt, s.body,
                                           boundary=s.boundary, options=opt, stream=stream)
                fs.fs_set_state(h, torch.tensor(s.X, device=dev), torch.tensor(s.L, device=dev),
                                torch.tensor(s.f_ext, device=dev))
                for _ in range(args.warmup):
                    fs.fs_step(h, info=False)
                fs.fs_kernel_stats(h, reset=True)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                infos = [fs.fs_step(h, info=True) for _ in range(args.steps)]
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                ks = fs.fs_kernel_stats(h)
                _, U, _ = fs.fs_get_body(h)
                fs.fs_destroy(h)
                row[name] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms,
                             "avg_gmres_iters": float(np.mean([i.iters for i in infos])),
                             "iters": [i.iters for i in infos],
                             "outer": [i.refine_sweeps for i in infos], "U_z": float(U[2]),
                             "kernels": {KS_NAMES[k]: [ks[k][0], round(ks[k][1], 2)] for k in range(7) if ks[k][0]}}
            res[str(nf)] = row
        s = wl.table2_aster(32)
        out.update({"points_per_fiber": 31, "body_nodes": int(s.body.nodes.shape[0]),
                    "periphery_nodes": int(s.boundary.nodes.shape[0]), "dt": s.dt, "tol": 1e-5,
                    "steps": args.steps, "warmup": args.warmup, "result": res,
                    "paper_avg_gmres_iters": {"32": 3, "128": 5, "512": 9, "2048": 16}})
    else:
        s = wl.cfg_large_matvec(seed=rank)
        opt = fs.fs_options_default()
        opt.profile = 1
        h = fs.fs_create([], s.mu, s.eps, s.E, s.dt, options=opt, stream=stream)
        X = torch.tensor(s.X, device=dev)
        Wf = torch.tensor(s.f_ext * 0.01, device=dev)
        fid = torch.tensor(s.fiber_id(), dtype=torch.int32, device=dev)
        res = {}
        for name, prec, cls, nt in (("fp32_hilo", fs.FS_SUM_FP32, 0, s.n_points),
                                    ("fp32_plain", fs.FS_SUM_FP32_PLAIN, 5, s.n_points),
                                    ("float_float", fs.FS_SUM_FF, 4, s.n_points),
                                    ("fp64_sampled", fs.FS_SUM_FP64, 1, 16384)):
            idx = torch.linspace(0, s.n_points - 1, nt, device=dev).long()
            T, tf = X[idx].contiguous(), fid[idx].contiguous()
            out_u = torch.empty_like(T)
            fs.fs_stokeslet_apply(h, X, Wf, T, out_u, fid, tf, prec)
            torch.cuda.synchronize()
            fs.fs_kernel_stats(h, reset=True)
            reps = 2 if name != "fp64_sampled" else 1
            for _ in range(reps):
                fs.fs_stokeslet_apply(h, X, Wf, T, out_u, fid, tf, prec)
            st = fs.fs_kernel_stats(h, reset=True)[cls]
            pairs_s = st[2] / (st[1] * 1e-3)
            fpp = FLOPS_PER_PAIR["stokeslet_ff" if cls == 4 else "stokeslet"]
            res[name] = {"targets": int(nt), "ms_per_launch": st[1] / st[0], "pairs_per_s": pairs_s,
                         "tflops": fpp * pairs_s / 1e12,
                         "full_matvec_s": s.n_points * s.n_points / pairs_s}
        # treecode (fs_stokeslet_apply_tree) on all targets; its error on the
        # FP64 sum's sampled targets
        idx = torch.linspace(0, s.n_points - 1, 16384, device=dev).long()
        u64 = torch.empty((16384, 3), dtype=torch.float64, device=dev)
        fs.fs_stokeslet_apply(h, X, Wf, X[idx].contiguous(), u64, fid, fid[idx].contiguous(), fs.FS_SUM_FP64)
        ut = torch.empty_like(X)
        for order, theta in ((6, 0.5), (8, 0.5), (8, 0.4)):
            fs.fs_stokeslet_apply_tree(h, X, Wf, X, ut, fid, fid, order=order, theta=theta)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fs.fs_stokeslet_apply_tree(h, X, Wf, X, ut, fid, fid, order=order, theta=theta)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            err = (torch.linalg.norm(ut[idx] - u64) / torch.linalg.norm(u64)).item()
            res["tree_p%d_theta%.1f" % (order, theta)] = {
                "ms_per_call": ms, "rel_error_sampled": err,
                "speedup_vs_fp32_hilo": res["fp32_hilo"]["ms_per_launch"] / ms,
                "speedup_vs_fp32_plain": res["fp32_plain"]["ms_per_launch"] / ms}
        fs.fs_destroy(h)
        out.update({"points": int(s.n_points), "pairs_full": float(s.n_points) ** 2, "result": res,
                    "fp32_vs_fp64_pairs_per_s": res["fp32_hilo"]["pairs_per_s"] / res["fp64_sampled"]["pairs_per_s"]})
    if rank == 0:
        print(json.dumps(out), flush=True)


def serve_once(fs, systems, rate: float, slots: int, budget_gb: float, device: int, seed: int):
    """Submit `systems` (mixed precision, tol 1e-8) to a fresh fs_server with
    Poisson arrivals at `rate` per second (0: all at once); returns the wall
    time, per-request latency and queue times (ms), and the server's batch
    count.  Three warm-up requests first (kernels loaded, tables built)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=len(systems)) if rate > 0 else np.zeros(len(systems))
    sv = fs.fs_server_create(int(budget_gb * (1 << 30)), max_slots=slots, device=device)

    def submit(s):
        return fs.fs_submit(sv, s.n_per_fiber, s.X, s.L, s.mu, s.eps, s.E, s.dt, f_ext=s.f_ext,
                            prec=fs.FS_MIXED, tol=1e-8)

    for s in systems[:3]:
        fs.fs_server_wait(sv, submit(s))
    b0 = fs.fs_server_batches(sv)
    t0 = time.perf_counter()
    tickets, due = [], t0
    for s, g in zip(systems, gaps):
        due += g
        while time.perf_counter() < due:
            time.sleep(min(1e-3, max(0.0, due - time.perf_counter())))
        tickets.append(submit(s))
    res = [fs.fs_server_wait(sv, t) for t in tickets]
    wall = time.perf_counter() - t0
    batches = fs.fs_server_batches(sv) - b0
    fs.fs_server_destroy(sv)
    lat = np.array([r["info"].t_ms[6] for r in res])
    que = np.array([r["info"].t_ms[5] for r in res])
    per_batch = np.array([r["info"].t_ms[7] for r in res])
    return {"wall_s": wall, "req_per_s": len(systems) / wall, "batches": int(batches),
            "requests_per_batch_mean": float(per_batch.mean()),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                           "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
            "queue_ms": {"p50": float(np.percentile(que, 50)), "p99": float(np.percentile(que, 99))}}


def serving_leg(fs, local, rank, n_req: int = 48, slots: int = 64, budget_gb: float = 64.0):
    """The headline line's serving figures: n_req independent requests drawn
    from the batched distribution (8..512 fibers, 16/32/64 points); a burst
    gives the saturated rate, then Poisson arrivals at 0.7 x that rate give
    p50 / p99 latency."""
    systems = wl.batched(n_req, seed=200 + rank)
    burst = serve_once(fs, systems, 0.0, slots, budget_gb, local, seed=rank)
    rate = 0.7 * burst["req_per_s"]
    pois = serve_once(fs, systems, rate, slots, budget_gb, local, seed=rank + 1)
    return {"requests": n_req, "points_total": int(sum(x.n_points for x in systems)),
            "distribution": "fibers log-uniform in [8, 512], N in {16, 32, 64}, mixed, tol 1e-8",
            "saturated_req_per_s": burst["req_per_s"], "arrival_rate_per_s": rate,
            "req_per_s": pois["req_per_s"], "p50_ms": pois["latency_ms"]["p50"],
            "p99_ms": pois["latency_ms"]["p99"], "batches": pois["batches"],
            "requests_per_batch_mean": pois["requests_per_batch_mean"], "burst": burst}


def run_serve(args, ws, rank, local, fs, torch):
    """Serving: independent systems (8..512 fibers, 16/32/64 points, mixed
    precision, tol 1e-8) submitted with Poisson arrivals to an fs_server;
    reports throughput and latency percentiles, and the same systems stepped
    together in one batched context for comparison."""
    systems = wl.batched(args.serve, seed=100 + rank)
    out = serve_once(fs, systems, args.rate, args.slots, args.budget_gb, local, seed=rank)

    # the same systems in one batched context (fs_create_batch): one step for all
    opt = fs.fs_options_default()
    opt.prec = fs.FS_MIXED
    opt.tol = 1e-8
    dev = torch.device("cuda", local)
    h = fs.fs_create_batch([x.n_fibers for x in systems], np.concatenate([x.n_per_fiber for x in systems]),
                           1.0, 1e-3, 1.0, 1e-3, options=opt)
    X = torch.tensor(np.concatenate([x.X for x in systems]), device=dev)
    L = torch.tensor(np.concatenate([x.L for x in systems]), device=dev)
    F = torch.tensor(np.concatenate([x.f_ext for x in systems]), device=dev)
    bt = []
    for k in range(3):
        fs.fs_set_state(h, X, L, F)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fs.fs_step(h)
        torch.cuda.synchronize()
        bt.append(time.perf_counter() - t1)
    fs.fs_destroy(h)
    if rank == 0:
        pts = sum(x.n_points for x in systems)
        out.update({
            "mode": "serve", "requests": len(systems), "points_total": int(pts),
            "fibers": [int(min(x.n_fibers for x in systems)), int(max(x.n_fibers for x in systems))],
            "slots": args.slots, "budget_gb": args.budget_gb, "arrival_rate_per_s": args.rate,
            "throughput_req_per_s": out["req_per_s"],
            "batched_one_context": {"step_s": min(bt), "req_per_s": len(systems) / min(bt)}})
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-iters", type=int, default=12,
                    help="GMRES iterations assumed for the reference arm's extrapolation")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg of the headline line")
    ap.add_argument("--kernel", choices=["stokeslet_fp32", "stokeslet_fp64", "stokeslet_ff", "stokeslet_fp32_plain"],
                    default=None,
                    help="time only the direct-sum kernel on the cloud (fs_stokeslet_apply)")
    ap.add_argument("--points", type=int, default=0,
                    help="--kernel: use the first P points of the cloud (0 = all)")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="relative tolerance of the inner FP32-far-field solves (0 = library default)")
    ap.add_argument("--no-relax", action="store_true",
                    help="every outer direction on the float-float far field (no inexact-Krylov relaxation)")
    ap.add_argument("--tile", type=int, default=0,
                    help="far-field launch shape id (0 = default; 1..3 = targets per thread FP32 2/4/8, "
                         "float-float 1/2/4)")
    ap.add_argument("--workload", choices=["confined", "batched", "large", "sediment", "kinetics", "aster",
                                           "tree-step", "tree-case", "precond"],
                    default=None,
                    help="a secondary workload instead of the headline step benchmark")
    ap.add_argument("--tree-order", type=int, default=8, help="--workload tree-case: expansion order")
    ap.add_argument("--tree-theta", type=float, default=0.4, help="--workload tree-case: opening angle")
    ap.add_argument("--serve", type=int, default=0,
                    help="serving mode: number of independent requests (0 = the step benchmark)")
    ap.add_argument("--rate", type=float, default=0.0, help="--serve: Poisson arrival rate per s (0 = burst)")
    ap.add_argument("--slots", type=int, default=4, help="--serve: concurrent requests")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="--serve: HBM budget for the requests")
    args = ap.parse_args()
    ws, rank, local = dist_env()

    import torch
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "native" else "gloo")
    if args.impl == "reference":
        run_reference(args, ws, rank)
        if dist:
            dist.destroy_process_group()
        return

    torch.cuda.set_device(local)
    from paper_1602_05650_gb300 import build as fsbuild
    fsbuild.build()
    import paper_1602_05650_gb300 as fs
    if args.kernel:
        return run_kernel(args, ws, rank, local, fs, torch, dist)
    if args.serve:
        return run_serve(args, ws, rank, local, fs, torch)
    if args.workload:
        return run_workload(args, ws, rank, local, fs, torch)

    dev = torch.device("cuda", local)
    s = wl.cfg_cloud_mixed(seed=rank)
    stream = torch.cuda.Stream(device=dev)
    opt = fs.fs_options_default()
    opt.prec = fs.FS_MIXED
    opt.tol = 1e-8
    opt.profile = 1
    if args.inner_tol > 0:
        opt.inner_tol = args.inner_tol
    if args.no_relax:
        opt.relax = 0
    opt.tile_override = args.tile
    h = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, options=opt, stream=stream)
    X = torch.tensor(s.X, dtype=torch.float64, device=dev)
    L = torch.tensor(s.L, dtype=torch.float64, device=dev)
    F = torch.tensor(s.f_ext, dtype=torch.float64, device=dev)
    # every step starts from the initial cloud (the per-node random forcing
    # roughens the fibers within a few steps, so a free run would time a
    # degenerating state); the device-to-device reset is inside the timed region
    infos = []
    for _ in range(args.warmup):
        fs.fs_set_state(h, X, L, F)
        fs.fs_step(h, info=False)
    torch.cuda.synchronize()
    fs.fs_kernel_stats(h, reset=True)

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    n0 = fs.fs_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        fs.fs_set_state(h, X, L, F)
        infos.append(fs.fs_step(h, info=True))
    e1.record(stream)
    torch.cuda.synchronize()
    launches = fs.fs_kernel_launches() - n0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    stats = fs.fs_kernel_stats(h, reset=True)
    ms = job_time(ms, dist, dev)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    pinned = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    Xh, Lh, Fh = pinned(s.X), pinned(s.L), pinned(s.f_ext)
    Vh = torch.empty(Xh.shape, dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(2, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        fs.fs_set_state(h, Xh, Lh, Fh)
        fs.fs_step(h, info=False)
        fs.fs_get_state(h, V=Vh)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = job_time(e2e_s, dist, dev)
    h2d = Xh.nbytes + Lh.nbytes + Fh.nbytes
    d2h = Vh.nbytes
    fs.fs_destroy(h)

    # plain FP64 GPU path on the same workload (one step after one warm-up)
    fp64 = None
    if not args.no_fp64:
        o64 = fs.fs_options_default()
        o64.prec = fs.FS_FP64
        o64.tol = 1e-8
        h64 = fs.fs_create(s.n_per_fiber, s.mu, s.eps, s.E, s.dt, options=o64, stream=stream)
        fs.fs_set_state(h64, X, L, F)
        fs.fs_step(h64, info=False)
        fs.fs_set_state(h64, X, L, F)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        inf64 = fs.fs_step(h64, info=True)
        a1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"ms_per_step": a0.elapsed_time(a1), "iters": inf64.iters, "resid": inf64.resid}
        fs.fs_destroy(h64)

    # serving: continuous batching under Poisson arrivals (p50 / p99 latency)
    serve = None if args.no_serve else serving_leg(fs, local, rank)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant direct-sum kernel (CUDA events on the context's stream)
    fp32_peak = fs.fs_probe_fma(1)
    fp64_peak = fs.fs_probe_fma(0)
    per_class = {KS_NAMES[k]: {"launches": stats[k][0], "ms": stats[k][1], "pairs": stats[k][2]}
                 for k in range(7)}
    dom = max(range(7), key=lambda k: stats[k][1])
    launches_d, total_ms, pairs = stats[dom]
    kind = {2: "stresslet", 3: "stresslet", 4: "stokeslet_ff", 6: "stresslet_ff"}.get(dom, "stokeslet")
    is64 = dom in (1, 3)
    ach = FLOPS_PER_PAIR[kind] * pairs / (total_ms * 1e-3) / 1e12 if total_ms > 0 else 0.0
    sm_max = clk.get("sm_max_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    derived_fp32 = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    peak = (fp64_peak / 1e12) if is64 else derived_fp32
    roofline = {"bound": "alu", "kernel": "k_pairsum " + KS_NAMES[dom],
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak if peak else None,
                "traffic": traffic_for(KS_NAMES[dom]),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, from "
                                  "profiles/traffic.txt, used only when it was captured on the current "
                                  "source of csrc/pairsum.cu (sha1 match), else null",
                "flops_per_pair": FLOPS_PER_PAIR[kind],
                "peak_source": ("measured FP64 FMA loop (fs_probe_fma)" if is64 else
                                "%d SMs (queried) x 128 FP32 lanes x 2 x max SM clock" % n_sm),
                "launch_ms_avg": total_ms / launches_d if launches_d else None,
                "measured_fp32_fma_tflops": fp32_peak / 1e12,
                "measured_fp64_fma_tflops": fp64_peak / 1e12,
                "frac_of_measured_fma_loop": (ach * 1e12 / (fp64_peak if is64 else fp32_peak)
                                              if (fp64_peak if is64 else fp32_peak) else None),
                "fma_pipe_active_ncu": traffic_for(KS_NAMES[dom], "pipe_util.txt"),
                "fma_pipe_active_source": "ncu sm__pipe_fma_cycles_active of the dominant kernel, from "
                                          "profiles/pipe_util.txt, used only when it was captured on the "
                                          "current source of csrc/pairsum.cu (sha1 match), else null"}
    # the Stokeslet pair rate of the step's FP32 sum (the dominant kernel)
    st32 = per_class["stokeslet_fp32_plain"]
    pairs_per_s = st32["pairs"] / (st32["ms"] * 1e-3) if st32["ms"] > 0 else None
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = oracle_baseline(s, fp64["iters"] if fp64 else args.ref_iters)
    value = job_rate(1.0, ws, ms * 1e-3)
    line = {
        "metric": "implicit steps/s (%s; mixed FP32/FP64, GMRES 1e-8)" % WORKLOAD,
        "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 far field + f64", "data": "synthetic",
        "config": workload_config(s, ws, opt.inner_tol, opt.relax),
        "roofline": roofline,
        "cpu_baseline": ({"value": cpu["value"], "unit": "steps/s", "cores": cpu["cores"], "cpu": cpu["cpu"],
                          "kind": "oracle", "sample": cpu["sample"]} if cpu else None),
        "e2e": {"value": job_rate(1.0, ws, e2e_s), "unit": "steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "clocks": clk,
        "stokeslet_pairs_per_s_fp32": pairs_per_s,
        "kernels": per_class,
        "step": {"inner_gmres_iters": [i.iters for i in infos],
                 "outer_steps": [i.refine_sweeps for i in infos],
                 "resid": [i.resid for i in infos],
                 "t_ms_rhs_build_solve": [[round(i.t_ms[0], 2), round(i.t_ms[1], 2), round(i.t_ms[2], 2)]
                                          for i in infos]},
        "fp64_path": fp64,
        "mixed_speedup_vs_fp64": (fp64["ms_per_step"] / ms) if fp64 else None,
        "serving": serve,
    }
    if serve:
        line.update({"p50_ms": serve["p50_ms"], "p99_ms": serve["p99_ms"], "req_per_s": serve["req_per_s"]})
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
