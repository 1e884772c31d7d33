"""The multi-rank path of bench.py on CPU: two gloo ranks reduce their timing
figures (max of the per-rank totals, sum of launch counts) and the whole-job
throughput divides all ranks' solves by the slowest rank's time.  The CPU
reference arm prints on rank 0 only."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
rank = dist.get_rank()
r = bench.Ranks(dist, "cpu")
r.barrier()
total_ms = [400.0, 500.0][rank]          # per-rank sum of step times
launches = [100, 120][rank]
out = {{"rank": rank, "max": r.max(total_ms), "sum": r.sum(launches),
        "value": bench.throughput(dist.get_world_size(), 10, r.max(total_ms))}}
print(json.dumps(out), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_timings():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["max"] == 500.0                 # the slowest rank's total
        assert o["sum"] == 220.0                 # launches of both ranks
        assert o["value"] == pytest.approx(2 * 10 / 0.5)   # 20 solves in 0.5 s


def test_single_rank_reductions_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(None)
    r.barrier()
    assert r.max(3.5) == 3.5 and r.sum(7) == 7.0
    assert bench.throughput(1, 30, 600.0) == pytest.approx(50.0)


def test_reference_arm_prints_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    # rank 1 of 2 returns at once without work or output
    assert bench.run_reference(A(), 2, 1) is None


def test_unblocked_bytes_model():
    # two levels of 8 and 1 cells, RKL2 s = 3, (2, 1) smoothing, 2 cycles,
    # 10 coarse stage-cells: per cycle 8 (3 (16 + 2 24) + 8.5 + 8.5) + 40 8,
    # twice, + 16 10 + (20 + 28) 8
    sys.path.insert(0, ROOT)
    import bench
    solver = dict(bench.SOLVER, s_smooth=3, n_pre=2, n_post=1, inner_n_pre=-1, inner_n_post=-1)
    assert bench.unblocked_bytes_per_solve([8, 1], solver, 2, 10) == 4528.0
    # inner levels with their own counts: level 1 of [64, 8, 1] smooths 2 + 1 = 3
    # times where the finest smooths 5 + 3 = 8: per cycle 64 (8 64 + 17) + 8 (3 64 + 17) + 40 64
    solver = dict(bench.SOLVER, s_smooth=3, n_pre=5, n_post=3, inner_n_pre=2, inner_n_post=1)
    assert bench.unblocked_bytes_per_solve([64, 8, 1], solver, 1, 0) == (64 * (8 * 64 + 17) + 8 * (3 * 64 + 17)
                                                                          + 40 * 64 + 48 * 64)


def test_oracle_cycle_count_matches_bench_settings():
    # the stored oracle cycle count must have been taken with the settings the
    # bench times (tests/golden/make_oracle_cycles.py writes them out)
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "tests", "golden", "oracle_cycles_sphere256.json")) as f:
        g = json.load(f)
    fields = dict(kv.split("=") for kv in g["solver"].split()[1:])
    S = bench.SOLVER
    assert g["solver"].split()[0] == f"RKL{S['rkl_order']}"
    assert int(fields["s"]) == S["s_smooth"] and float(fields["tau_frac"]) == S["tau_frac"]
    assert int(fields["n_pre"]) == S["n_pre"] and int(fields["n_post"]) == S["n_post"]
    assert int(fields.get("inner_n_pre", -1)) == S.get("inner_n_pre", -1)
    assert int(fields.get("inner_n_post", -1)) == S.get("inner_n_post", -1)
    assert float(fields["coarse_tol"]) == S["coarse_tol"] and int(fields["coarse_max_ss"]) == S["coarse_max_ss"]
    assert g["levels"] == bench.LEVELS and g["tol"] == bench.TOL
