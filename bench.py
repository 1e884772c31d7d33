#!/usr/bin/env python3
"""Benchmark of the RKL-multigrid Poisson solver on GB300.

Workload (one "step" = one complete solve through the library's public API):
  uniform-density sphere (R = 0.25, rho = 1) centred in [-1, 1]^3 on a 256^3
  cell-centred grid, Dirichlet faces from the analytic sphere potential,
  4 pi G = 1; RKL2-smoothed V-cycle (s = 3, tau = 0.9 tau_max, N_pre = 5,
  N_post = 3 on the finest level, 3 and 2 on the levels below it), five
  levels down to 16^3, accelerated-RKL coarsest solve;
  FP32 V-cycle inside an FP64 residual / defect-correction loop; solved to
  relative residual 1e-8.  Each step resets the density (device copy) and
  solves from phi = 0.

Metric: solves/s (whole job; N ranks solve independent instances: weak
scaling, no collective).  The K timed steps are independent solves of the
workload, four in flight at a time: one grid per CUDA stream, each driven by
its own host thread, so that the solves fill each other's idle SMs; value =
K / the device time from the first launch to the last completion.  Inputs
(256^3 x 8 B = 134 MB per array, working set about 1 GB per solve) are larger
than the 129 MB L2.  The line also reports one solve at a time (`sequential`:
L2 flushed by a 512 MB write before each solve, CUDA events per solve).

End to end (`e2e`): the density comes from pinned host memory and the
potential goes back to it through the C ABI every step, the same four grids
in flight (one grid's copies, by the copy engines, overlap the others'
solves); the strictly sequential figure (copy in, solve, copy out) beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 256
LEVELS = 5
TOL = 1e-8
# RKL2 smoother, s = 3 (odd: the checkerboard mode keeps a factor of 0.55 per
# super-step), tau = 0.9 tau_max, N_pre = 5, N_post = 3 on the finest level and
# 3, 2 on the levels between it and the two coarsest: the fastest measured RKL2
# setting on this workload whose s is odd (6 V-cycles).
# independent solves in flight: one grid per CUDA stream, one host thread each
INFLIGHT = 4
SOLVER = dict(rkl_order=2, s_smooth=3, tau_frac=0.9, n_pre=5, n_post=3, inner_n_pre=3, inner_n_post=2,
              coarse_tol=1e-2, coarse_max_ss=64)
METRIC = "Poisson solves/s to rel. residual 1e-8 at 256^3"
FALLBACK_HBM_GBS = 6800.0
# FP64 instructions per cell and stage of the FP64 stage kernel, averaged over
# an s = 3 RKL2 super-step (one first stage, 13.5; two later ones, 16.5), as
# counted by ncu (smsp__inst_executed_pipe_fp64) on 256^3 launches
FP64_INSTR_PER_STAGE_CELL = 15.5


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="only run this many solves of the sphere workload (for ncu captures; no JSON line)")
    ap.add_argument("--n", type=int, default=N, help="grid size of --profile-solves")
    ap.add_argument("--smoother", choices=["rkl", "gsrb"], default="rkl",
                    help="smoother of --profile-solves (rkl: the bench's RKL2 settings; gsrb: red-black GS)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed",
                    help="precision of --profile-solves")
    ap.add_argument("--gravity", action="store_true",
                    help="with --profile-solves: after each solve, one acceleration pass (sg_gravity)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Ranks:
    """Cross-rank reductions of the timing figures (identities with one rank).
    `dist` is torch.distributed with an initialised process group, or None."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)


def smoothing_count(solver, level):
    """Super-steps per cycle on a level: N_pre + N_post on the finest, the inner
    counts (when set, else the same) on the levels below it."""
    pre, post = solver["n_pre"], solver["n_post"]
    if level > 0:
        pre = solver.get("inner_n_pre", -1) if solver.get("inner_n_pre", -1) >= 0 else pre
        post = solver.get("inner_n_post", -1) if solver.get("inner_n_post", -1) >= 0 else post
    return pre + post


def unblocked_bytes_per_solve(level_cells, solver, cycles, coarse_stage_cells):
    """HBM bytes one solve would move if every kernel ran unfused, each array
    read or written once per sweep (the per-cell figures of the kernels'
    algorithmic-byte table): per cycle, on every level but the coarsest,
    N_pre + N_post RKL2 super-steps (levels below the finest: the inner
    counts) of s FP32 stages (16 B/cell for the
    first stage, 24 for the others), the residual + restriction and the
    prolongation + correction (8.5 B/cell each), the FP64 update of the
    finest level (40 B/cell); the coarsest level's stages (16 B/cell each);
    and once per solve the start and confirmation residuals (20 + 28 B/cell).
    The fused kernels move less, so the effective rate below may pass the
    copy bandwidth; that is the point of the temporal blocking."""
    s = solver["s_smooth"]
    per_cycle = 0.0
    for l, n in enumerate(level_cells[:-1]):
        n_relax = smoothing_count(solver, l)
        per_cycle += n * (n_relax * (16.0 + 24.0 * (s - 1)) + 8.5 + 8.5)
    per_cycle += 40.0 * level_cells[0]
    return cycles * per_cycle + 16.0 * coarse_stage_cells + 48.0 * level_cells[0]


def throughput(world, steps, max_total_ms):
    """Whole-job solves/s: every rank solves `steps` instances, and the job
    takes as long as its slowest rank."""
    return world * steps / (max_total_ms * 1e-3)


def config(world):
    return {"workload": f"sphere{N}", "grid": [N, N, N], "levels": LEVELS, "tol": TOL,
            "precision": "mixed (FP32 V-cycle; FP64 residual carried by exact recurrence, confirmed at the end by an FP64 residual whose stencil sum is exact in 64-bit fixed point; FP64 defect correction)",
            "smoother": "RKL2 s=3 tau=0.9 tau_max, N_pre=5, N_post=3 (levels 1-2: 3, 2)",
            "coarse": "accelerated RKL1 on 16^3, coarse_tol=1e-2",
            "boundary": "Dirichlet from analytic sphere potential",
            "per_gpu_instances": INFLIGHT, "instances_total": world * INFLIGHT,
            "l2": "inputs > L2 (134 MB per array, working set > 1 GB per solve, solves in flight); "
                  "the sequential figure and the kernel profile flush L2 (512 MB write) before each solve",
            "parallelism": f"replicas x{world}"}


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            sel = ["-i", self.uuid] if self.uuid else []
            self.proc = subprocess.Popen(["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken between wall-clock times t0 and t1."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons, power, allsm = [], [], set(), [], []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                vals = (float(parts[1]), float(parts[2]), float(parts[3]))
            except (ValueError, IndexError):
                continue
            allsm.append(vals[0])
            if t0 is not None and not (t0 - 0.15 <= ts <= t1 + 0.15):
                continue
            sm.append(vals[0])
            smax.append(vals[1])
            power.append(vals[2])
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:          # timed region shorter than the sampling period: all samples
            sm = allsm
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# Source files of the kernel whose DRAM bytes `roofline.traffic` reports (the
# fused level-0 super-step) and the header it includes.
TRAFFIC_SOURCES = ("kernels_superstep.cu", "sg_internal.cuh")


def kernel_source_hash():
    """Hash of the dominant kernel's sources: DRAM counters taken on other
    code of that kernel are not reported."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_05332_gb300", "csrc")
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(cls, cells):
    """DRAM bytes per launch of kernel class `cls` from the committed ncu
    summary, scaled by cells; None if absent or taken on other kernel sources.
    The level-0 super-steps of a cycle are one launch from Y0 = 0 and
    N_pre + N_post - 1 general ones: their figures are mixed in that ratio."""
    path = os.path.join(ROOT, "profiles", "ncu_dram_per_cell.txt")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    if not m or m.group(1) != kernel_source_hash():
        return None

    def fig(name):
        mm = re.search(rf"^{name}\s+([0-9.eE+-]+)\s*$", text, re.M)
        return float(mm.group(1)) if mm else None

    if cls == "rkl_stage_l0":
        z, gen = fig("rkl_stage_l0_zero"), fig("rkl_stage_l0_general")
        if z is None or gen is None:
            return None
        n = SOLVER["n_pre"] + SOLVER["n_post"]
        return (z + (n - 1) * gen) / n * cells
    v = fig(cls)
    return v * cells if v is not None else None


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------
def oracle_vcycle_seconds(p, reps=1, levels=LEVELS):
    import numpy as np
    import oracle as O
    opts = O.Options(**SOLVER)
    h = O.spacing(p.shape, p.lo, p.hi)
    f = O.source(p.rho, 1.0, p.bc)
    phi = np.zeros(p.shape)
    t = []
    for _ in range(reps):
        t0 = time.perf_counter()
        phi = O.vcycle(phi, f, h, p.bc, p.faces, levels, opts)
        O.l2norm(O.residual(phi, f, h, p.bc, p.faces))
        t.append(time.perf_counter() - t0)
    return statistics.median(t)


def _vcycle_worker(n):
    """One 256^3 oracle V-cycle in a fresh (spawned) process; returns seconds."""
    import workloads as W
    return oracle_vcycle_seconds(W.sphere(n), 1)


def _parallel_replicas():
    """Oracle replicas that fit this host: one per core, at most as many as
    the available memory holds at about 4 GB per 256^3 V-cycle."""
    cores = os.cpu_count() or 1
    try:
        with open("/proc/meminfo") as f:
            avail_kb = next(int(l.split()[1]) for l in f if l.startswith("MemAvailable:"))
        by_mem = max(1, int(avail_kb / (4 * 2 ** 20)))
    except Exception:
        by_mem = 1
    return max(1, min(cores, by_mem, 16))


def cpu_baseline_obj(p, cycles, all_cores=True):
    """The oracle timed on the host cores: one direct 256^3 V-cycle on one core,
    and (all_cores) one V-cycle in each of k concurrent spawned processes (the
    numpy oracle is single-threaded, so the cores serve independent instances).
    A solve is `cycles` V-cycles (the oracle's own count on this workload)."""
    t = oracle_vcycle_seconds(p, 1)
    per_solve = cycles * t
    out = {"value": 1.0 / per_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
           "sample": f"1 V-cycle + residual norm of the numpy FP64 oracle at {N}^3, timed directly "
                     f"({t:.2f} s), x {cycles} V-cycles per solve (the oracle's own count on this workload)",
           "vcycle_s": t, "cycles_per_solve": cycles, "nproc": os.cpu_count()}
    if all_cores:
        import multiprocessing as mp
        k = _parallel_replicas()
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(k) as pool:
            ts = pool.map(_vcycle_worker, [N] * k)
        wall = time.perf_counter() - t0
        slowest = max(ts)
        out["all_cores"] = {"value": k / (cycles * slowest), "unit": "solves/s", "cores": k,
                            "sample": f"{k} concurrent oracle processes, one 256^3 V-cycle each "
                                      f"(slowest {slowest:.2f} s, wall {wall:.1f} s with start-up), "
                                      f"x {cycles} V-cycles per solve"}
    return out


# ---------------------------------------------------------------------------
# Reference arm: the oracle, timed on the host cores
# ---------------------------------------------------------------------------
def oracle_cycles_per_solve():
    """V-cycles the FP64 oracle needs on this workload, written by
    tests/golden/make_oracle_cycles.py (a run of the oracle itself)."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_cycles_sphere256.json")
    with open(path) as f:
        return int(json.load(f)["cycles"])


def run_reference(a, world, rank):
    """The oracle as the reference arm: each step times one V-cycle of the
    256^3 workload directly (about 8 s on the GPU host's cores); a solve is the
    oracle's own cycle count of V-cycles, so value = 1 / (cycles x mean step)."""
    if rank != 0:
        return
    import workloads as W
    p = W.sphere(N)
    for _ in range(a.warmup):
        oracle_vcycle_seconds(p, 1)
    ts = [oracle_vcycle_seconds(p, 1) for _ in range(a.steps)]
    cycles = oracle_cycles_per_solve()
    step_s = statistics.mean(ts)
    value = 1.0 / (cycles * step_s)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(world),
            "step_definition": f"one V-cycle + residual norm of the FP64 oracle at {N}^3 (a solve is "
                               f"{cycles} of them: value = 1 / ({cycles} x ms_per_step))",
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: 1 V-cycle + residual norm of the numpy FP64 oracle on the "
                                       f"{N}^3 workload, timed directly; x {cycles} cycles per solve (the "
                                       f"oracle's own count on this workload)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def single_level_race(sg, W, torch, stream, n=128, bound=1e-10):
    """App. B's comparison without multigrid: Gauss-Seidel, SOR (App. B's
    omega) and the accelerated RKL1 schedule, each a single-level FP64 solve of
    the smooth-sphere problem of Sec. 4.1 at n^3 until max |L phi - f| <= bound.
    Wall time of each solve (host loop included: one residual read back per
    sweep or super-step, as each method needs for its stopping test)."""
    p = W.smooth_sphere(n)
    gr = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="fp64", stream=stream.cuda_stream)
    gr.set_boundary(p.faces)
    rho = torch.tensor(p.rho, device="cuda")
    out = {"n": n, "max_residual_bound": bound}
    for name, opts in (("gs", dict(smoother="gsrb", omega=1.0)), ("sor", dict(smoother="gsrb", omega=0.0)),
                       ("rkl", dict(smoother="rkl"))):
        gr.set_options(max_residual_tol=bound, max_cycles=200000, **opts)
        gr.set_density(rho, p.four_pi_G)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = gr.solve(tol=0.0, levels=1, check=False)
        torch.cuda.synchronize()
        out[name] = {"ms": (time.perf_counter() - t0) * 1e3, "iterations": info["cycles"],
                     "max_residual": info["max_residual"], "status": info["status"]}
    for name in ("gs", "sor"):
        out[f"{name}_over_rkl"] = out[name]["ms"] / out["rkl"]["ms"]
    del gr
    return out


def run_ours(a, world, rank, local):
    import numpy as np
    import torch

    import paper_2306_05332_gb300 as sg
    import workloads as W

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    ranks = Ranks(dist, dev)
    barrier, max_ranks, sum_ranks = ranks.barrier, ranks.max, ranks.sum

    p = W.sphere(N)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="mixed", stream=stream.cuda_stream)
    g.set_boundary(p.faces)
    g.set_options(**SOLVER)
    rho_dev = torch.tensor(p.rho, device=dev)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)

    def step():
        g.set_density(rho_dev, 1.0)
        return g.solve(tol=TOL, levels=LEVELS)

    # INFLIGHT independent solves of the workload at a time: one grid per
    # stream, each driven by its own host thread (the library's calls release
    # the interpreter lock); the solves fill each other's idle SMs (small
    # coarse-level kernels, the one-cluster launch, the one-thread loop kernels)
    streams = [stream] + [torch.cuda.Stream(dev) for _ in range(INFLIGHT - 1)]
    grids = [g]
    for st in streams[1:]:
        gi = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="mixed", stream=st.cuda_stream)
        gi.set_boundary(p.faces)
        gi.set_options(**SOLVER)
        grids.append(gi)

    def run_inflight(k_total, one_step):
        """k_total steps spread over the grids, one host thread per grid;
        returns (device ms from the first launch to the last completion, infos)."""
        out = [[] for _ in grids]

        def worker(i):
            for _ in range(i, k_total, len(grids)):
                out[i].append(one_step(grids[i], i))

        torch.cuda.synchronize()
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(streams[0])
        for st in streams[1:]:
            st.wait_event(ev0)
        threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(grids))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for st in streams[1:]:
            done = torch.cuda.Event()
            done.record(st)
            streams[0].wait_event(done)
        ev1.record(streams[0])
        torch.cuda.synchronize()
        barrier()
        return ev0.elapsed_time(ev1), [x for o in out for x in o]

    def dev_step(gi, i):
        gi.set_density(rho_dev, 1.0)
        return gi.solve(tol=TOL, levels=LEVELS)

    for _ in range(max(3, a.warmup)):
        for gi in grids:
            dev_step(gi, 0)
    torch.cuda.synchronize()
    barrier()
    # one solve at a time (L2 flushed before each, CUDA events per solve): the
    # per-solve device time, reported beside the in-flight throughput
    seq_ms = []
    for k in range(max(3, min(a.steps, 10))):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        step()
        s1.record(stream)
        torch.cuda.synchronize()
        seq_ms.append(s0.elapsed_time(s1))
    seq_step = max_ranks(statistics.mean(seq_ms))
    torch.cuda.synchronize()
    barrier()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    clocks = Clocks(uuid)
    clocks.start()
    time.sleep(0.5)                   # let nvidia-smi start sampling
    wall0 = time.perf_counter()
    epoch0 = time.time()
    dev_ms, infos = run_inflight(a.steps, dev_step)
    wall = time.perf_counter() - wall0
    epoch1 = time.time()
    clk = clocks.stop(epoch0, epoch1)
    total_ms = max_ranks(dev_ms)
    ms_per_step = total_ms / a.steps
    value = throughput(world, a.steps, total_ms)
    cycles = infos[-1]["cycles"]
    su = statistics.mean(i["stage_cell_updates"] for i in infos)
    launches = int(sum(i["kernel_launches"] for i in infos) + a.steps)   # + one source kernel per step
    launches = int(sum_ranks(launches))

    # ---- end to end: host (pinned) density in, host potential out ----
    # Every step copies its density from pinned host memory, solves and reads
    # the potential back into pinned host memory through the C ABI, the copies
    # by the copy engines (the library's default), so that one grid's copies
    # overlap the other grids' solves.  The same INFLIGHT grids and threads as
    # the device-resident value; the strictly sequential figure (one grid:
    # copy in, solve, copy out) beside it.  No L2 flush between these steps:
    # each moves 268 MB over the CPU-GPU link and the solve's working set is
    # over 1 GB.
    rho_host = torch.tensor(p.rho).pin_memory()
    phi_hosts = [torch.empty(p.shape, dtype=torch.float64).pin_memory() for _ in grids]

    def host_step(gi, i):
        gi.set_density(rho_host, 1.0)
        inf = gi.solve(tol=TOL, levels=LEVELS)
        gi.potential(phi_hosts[i])
        return inf

    e2e_ms = []
    for k in range(2 + max(1, min(a.steps, 10))):      # two untimed warm-up passes of the host path
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = host_step(g, 0)
        if k >= 2:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    seq_e2e = max_ranks(statistics.mean(e2e_ms))
    for i, gi in enumerate(grids[1:], 1):              # warm the other grids' host path
        host_step(gi, i)
    k2 = max(a.steps, 2 * len(grids))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    _, infos2 = run_inflight(k2, host_step)
    e2e_step = max_ranks((time.perf_counter() - t0) * 1e3 / k2)
    for inf in infos2:
        assert inf["cycles"] == info["cycles"] and inf["rel_residual"] <= TOL, inf
    n0 = N ** 3
    e2e = {"value": world * 1000.0 / e2e_step, "unit": "solves/s",
           "h2d_bytes_per_step": 8 * n0, "d2h_bytes_per_step": 8 * n0 + 36 * (info["cycles"] + 1),
           "ms_per_step": e2e_step, "steps": k2,
           "pattern": f"{INFLIGHT} grids in flight on {INFLIGHT} streams, one host thread each; "
                      "host copies by the copy engines, overlapping the other grids' solves",
           "sequential": {"value": world * 1000.0 / seq_e2e, "ms_per_step": seq_e2e,
                          "pattern": "one grid: copy in, solve, copy out, step after step"},
           "l2": "not flushed: each step moves 268 MB over the CPU-GPU link, working set > 1 GB"}
    del grids[1:]

    # ---- roofline of the dominant kernel: per-kernel CUDA events in a profiled pass ----
    roof = None
    kernels = None
    if not a.no_profile:
        g.set_profiling(True)
        for _ in range(max(1, min(a.steps, 5))):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        kernels = g.kernel_stats()
        g.set_profiling(False)
        tot = sum(v["ms"] for v in kernels.values())
        dom = max(kernels, key=lambda k: kernels[k]["ms"])
        d = kernels[dom]
        peak, src = hbm_peak()
        ach = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
        per_launch = d["bytes"] / max(1, d["launches"])
        traffic = ncu_traffic(dom, 1.0) if dom in ("rkl_stage_l0", "residual_l0", "update_residual") else None
        if traffic is not None:
            cells_per_launch = n0
            traffic = traffic * cells_per_launch
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": f"of {src}", "traffic": traffic,
                "algorithmic_bytes_per_launch": per_launch, "launches": d["launches"],
                "avg_launch_us": d["ms"] * 1e3 / max(1, d["launches"]),
                "share_of_kernel_time": d["ms"] / tot if tot > 0 else None}
        kernels = {k: {"launches": v["launches"], "ms_per_solve": v["ms"] / max(1, min(a.steps, 5)),
                       "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else 0.0,
                       "share": v["ms"] / tot if tot > 0 else 0.0} for k, v in kernels.items()}

    extra = {}
    if not a.no_extra:
        # the plain FP64 GPU solve of the same problem, and an RKL1-smoothed variant
        g64 = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="fp64", stream=stream.cuda_stream)
        g64.set_boundary(p.faces)
        g64.set_options(**SOLVER)
        g64.set_density(rho_dev, 1.0)
        g64.solve(tol=TOL, levels=LEVELS)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        i64 = g64.solve(tol=TOL, levels=LEVELS)
        t64 = (time.perf_counter() - t0) * 1e3
        # its roofline: the level-0 stage kernels are bound by the FP64 pipe, not
        # HBM; FP64 instructions per cell counted by ncu on these kernels
        # (13.5 in a first stage, 16.5 in a later one: 15.5 on average over an
        # s = 3 super-step), against this GPU's measured FP64 FMA rate
        fp64_tflops, _ = sg.measure_fp64_rate()
        g64.set_density(rho_dev, 1.0)
        g64.set_profiling(True)
        g64.solve(tol=TOL, levels=LEVELS)
        torch.cuda.synchronize()
        st64 = g64.kernel_stats()["rkl_stage_l0"]
        g64.set_profiling(False)
        n0c = N ** 3
        instr = FP64_INSTR_PER_STAGE_CELL * n0c * st64["launches"]
        achieved = instr / (st64["ms"] * 1e-3)
        peak_instr = fp64_tflops * 1e12 / 2.0
        peak_hbm, _src = hbm_peak()
        extra["fp64_gpu_solve"] = {"solves_per_s": 1000.0 / t64, "ms": t64, "cycles": i64["cycles"],
                                   "roofline_level0_stages": {
                                       "bound": "fp64", "achieved_fp64_instr_per_s": achieved,
                                       "peak_fp64_instr_per_s": peak_instr, "frac": achieved / peak_instr,
                                       "fp64_tflops_measured": fp64_tflops,
                                       "hbm_frac": st64["bytes"] / (st64["ms"] * 1e-3) / 1e9 / peak_hbm,
                                       "fp64_instr_per_stage_cell": FP64_INSTR_PER_STAGE_CELL,
                                       "launches": st64["launches"], "ms": st64["ms"]}}
        del g64
        g.set_options(**dict(SOLVER, rkl_order=1, s_smooth=2, tau_frac=0.75, n_pre=2, n_post=1, inner_n_pre=-1,
                             inner_n_post=-1))
        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        i1 = step()
        t1 = (time.perf_counter() - t0) * 1e3
        extra["rkl1_s2_smoother"] = {"solves_per_s": 1000.0 / t1, "ms": t1, "cycles": i1["cycles"]}
        # the paper's own smoother (GS-RB sweeps, N_pre = 2, N_post = 1) in the same V-cycle
        g.set_options(**dict(SOLVER, smoother="gsrb", n_pre=2, n_post=1, inner_n_pre=-1, inner_n_post=-1))
        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ig = step()
        tg = (time.perf_counter() - t0) * 1e3
        extra["gsrb_smoother"] = {"solves_per_s": 1000.0 / tg, "ms": tg, "cycles": ig["cycles"]}
        g.set_options(**SOLVER)
        extra["single_level_race_128"] = single_level_race(sg, W, torch, stream)

    if not a.no_extra:
        # autotuned smoother for this grid, keeping the configured RKL2 order
        g.set_density(rho_dev, 1.0)
        tuned, table = g.autotune(levels=LEVELS, keep_order=True)
        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        itn = step()
        tt = (time.perf_counter() - t0) * 1e3
        extra["autotuned_rkl2"] = {"solves_per_s": 1000.0 / tt, "ms": tt, "cycles": itn["cycles"],
                                   "s_smooth": tuned["s_smooth"], "tau_frac": tuned["tau_frac"],
                                   "n_pre": tuned["n_pre"], "n_post": tuned["n_post"],
                                   "inner_n_pre": tuned["inner_n_pre"], "inner_n_post": tuned["inner_n_post"],
                                   "tile_rows": tuned["tile_rows"],
                                   "fused": tuned["fused"], "candidates": len(table)}
        # the acceleration of the solution (Sec. 3, fourth order), device buffers:
        # reads phi (8 B/cell), writes three components (24 B/cell), 12 FP64
        # instructions per cell (two subtractions, one FMA, one multiply per axis)
        gout = torch.empty((3,) + tuple(p.shape), dtype=torch.float64, device=dev)
        g.gravity(out=gout)
        g.set_profiling(True)
        for _ in range(5):
            torch.cuda.synchronize()
            flush.fill_(1.0)
            g.gravity(out=gout)
        torch.cuda.synchronize()
        sgv = g.kernel_stats()["gravity"]
        g.set_profiling(False)
        per_ms = sgv["ms"] / max(1, sgv["launches"])
        # the combinations are exact in 64-bit fixed point: one FP64 product per
        # component, three FP64 instructions per cell (a scale pre-pass included in the time)
        extra["gravity_256"] = {"us_per_call": per_ms * 1e3,
                                "GBps_algorithmic": 32.0 * n0 / (per_ms * 1e-3) / 1e9,
                                "hbm_frac": 32.0 * n0 / (per_ms * 1e-3) / 1e9 / hbm_peak()[0],
                                "fp64_instr_per_cell": 3,
                                "arithmetic": "exact 64-bit fixed point, rounded to FP64 once per component"}
        del gout
        g.set_options(**SOLVER, fused=1)
        del g
        torch.cuda.empty_cache()
        # batched workload: 64 independent blob problems, N in {32, 64, 96, 128}
        probs = W.blob_batch(64, seed=0)
        grids, rhos = [], []
        for pb in probs:
            gb = sg.Grid(pb.shape, pb.lo, pb.hi, pb.bc, precision="mixed", stream=stream.cuda_stream)
            gb.set_boundary(pb.faces)
            rb = torch.tensor(pb.rho, device=dev)
            gb.set_density(rb, 1.0)
            grids.append(gb)
            rhos.append(rb)
        cells = sum(int(np.prod(pb.shape)) for pb in probs)
        sg.solve_batch(grids, tol=TOL)
        torch.cuda.synchronize()
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            for gb, rb in zip(grids, rhos):
                gb.set_density(rb, 1.0)
            binfo = sg.solve_batch(grids, tol=TOL)
        torch.cuda.synchronize()
        tb = (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        for gb, rb in zip(grids, rhos):
            gb.set_density(rb, 1.0)
            gb.solve(tol=TOL)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        # autotuned per size class: the smoother (order kept), s, tau, smoothing
        # counts, fused on / off and the fused kernel's tile rows picked on the
        # first instance of each size, then given to every instance of that size
        tuned = {}
        for gb, pb, rb in zip(grids, probs, rhos):
            n = pb.shape[0]
            if n not in tuned:
                gb.set_density(rb, 1.0)
                opts, _table = gb.autotune(keep_order=True)
                tuned[n] = {k: opts[k] for k in ("rkl_order", "s_smooth", "tau_frac", "n_pre", "n_post",
                                                 "inner_n_pre", "inner_n_post", "fused", "tile_rows")}
        for gb, pb in zip(grids, probs):
            gb.set_options(**tuned[pb.shape[0]])
        for gb, rb in zip(grids, rhos):
            gb.set_density(rb, 1.0)
        sg.solve_batch(grids, tol=TOL)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for gb, rb in zip(grids, rhos):
                gb.set_density(rb, 1.0)
            tinfo = sg.solve_batch(grids, tol=TOL)
        torch.cuda.synchronize()
        tt = (time.perf_counter() - t0) / reps
        extra["batch64_blobs"] = {"instances": len(grids), "cells": cells, "batched_s": tb,
                                  "batched_solves_per_s": len(grids) / tb, "sequential_s": ts,
                                  "sequential_solves_per_s": len(grids) / ts,
                                  "max_cycles": max(i["cycles"] for i in binfo),
                                  "max_rel_residual": max(i["rel_residual"] for i in binfo),
                                  "autotuned_per_size": {str(k): v for k, v in tuned.items()},
                                  "autotuned_batched_s": tt, "autotuned_batched_solves_per_s": len(grids) / tt,
                                  "autotuned_max_cycles": max(i["cycles"] for i in tinfo),
                                  "autotuned_max_rel_residual": max(i["rel_residual"] for i in tinfo),
                                  "structure": "one CUDA graph launch per batch: a branch per instance, each "
                                               "a WHILE loop of V-cycles whose condition a one-thread kernel "
                                               "sets from the residual on the device"}
        del grids, rhos

    effective = None
    try:
        cells = [(N >> l) ** 3 for l in range(LEVELS)]
        smoothing = cycles * SOLVER["s_smooth"] * sum(smoothing_count(SOLVER, l) * c for l, c in enumerate(cells[:-1]))
        coarse_stage_cells = max(0.0, su - smoothing)     # the solve's count minus the smoothing stages
        ub = unblocked_bytes_per_solve(cells, SOLVER, cycles, coarse_stage_cells)
        gbps = ub / (ms_per_step * 1e-3) / 1e9
        peak, src = hbm_peak()
        effective = {"GBps": gbps, "frac": gbps / peak, "peak_source": f"of {src}", "bytes_per_solve": ub,
                     "definition": "bytes the solve would move unfused (each sweep reading and writing its "
                                   "arrays once) / device time per solve; above 1 means the fused "
                                   "kernels save that traffic"}
    except Exception as exc:          # the line must still print
        effective = {"error": str(exc)}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline_obj(p, oracle_cycles_per_solve())

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": config(world),
                "cell_updates_per_s": world * su / (ms_per_step * 1e-3),
                "roofline_effective": effective,
                "cycles_per_solve": cycles, "final_rel_residual": infos[-1]["rel_residual"],
                "wall_s_timed_region": wall,
                "inflight": {"solves": INFLIGHT, "pattern": f"{INFLIGHT} independent solves in flight, one grid per "
                             "stream, one host thread each; value = all steps / device time from the first "
                             "launch to the last completion"},
                "sequential": {"value": world * 1000.0 / seq_step, "ms_per_step": seq_step,
                               "pattern": "one solve at a time, L2 flushed before each, CUDA events per solve"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "kernels": kernels, "extra": extra}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_profile_solves(a):
    """A bare sequence of solves of the n^3 sphere workload with the bench's
    solver settings, for profiler captures: no timing contract, no extras."""
    import torch
    import paper_2306_05332_gb300 as sg
    import workloads as W
    p = W.sphere(a.n)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision=a.precision, stream=stream.cuda_stream)
    g.set_boundary(p.faces)
    # use_graph = 2: each V-cycle a captured graph and the loop on the host, so
    # that a profiler sees every kernel (it cannot see into the kernel nodes of
    # the default solve graph, whose loop runs in conditional nodes)
    g.set_options(**SOLVER, smoother=a.smoother, use_graph=2)
    rho = torch.tensor(p.rho, device="cuda")
    gout = torch.empty((3,) + tuple(p.shape), dtype=torch.float64, device="cuda") if a.gravity else None
    for k in range(a.profile_solves):
        g.set_density(rho, 1.0)
        info = g.solve(tol=TOL, levels=LEVELS)
        if gout is not None:
            g.gravity(out=gout)
        print(k, info["cycles"], round(info["elapsed_ms"], 3), info["coarse_ss"][:5], flush=True)


def main():
    a = args_()
    world, rank, local = dist_env()
    if a.profile_solves > 0:
        run_profile_solves(a)
        return
    if a.impl == "reference":
        run_reference(a, world, rank)
        return
    run_ours(a, world, rank, local)


if __name__ == "__main__":
    main()
