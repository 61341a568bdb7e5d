#!/usr/bin/env python
"""Benchmark of the flow-shop B&B hot path: subproblems bounded per second
on the 20 jobs x 20 machines workload.

Step = one branch-and-bound iteration on the device (selection of the deepest
parents, branching, bounding, elimination against the UB and compaction onto
the stack) whose pool holds 2^18 children, started from a frontier of 20 x 20
nodes: the bounding workload of seed 1 (p uniform [1,99]; prefixes of random
permutations, depth uniform [1,19]; depth-19 nodes are complete-but-one and
never wait on a stack, so the frontier keeps depths <= 18), UB = makespan of
a random permutation.  Every step restarts from the same frontier, so every
step does identical work.  Extra lines of the same JSON object report the
bounding kernel alone on the 2^12..2^20 pools, the roofline, the CPU oracle
on a bounded sample, and the end-to-end call with host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

N_JOBS, N_MACH, SEED = 20, 20, 1
POOL = 2**18
FRONTIER = 2**18
BOUND_POOLS = (2**12, 2**15, 2**18, 2**20)
METRIC = "subproblems bounded/s at 20x20 (plain vs learned pair order, bit-exact); solve time"
UNIT = "subproblems/s"
L2_FLUSH_BYTES = 512 << 20
SMS, INT_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
# The ALU pipe (logic, min/max, the add-max instructions) retires 64 lanes per clock per SM: ncu
# reports sm__inst_executed_pipe_alu.avg.peak_sustained = 2 warp instructions per cycle per SM
# against sm__inst_executed.avg.peak_sustained = 4 (the issue ceiling above, 4 x 32 lanes), in a
# capture of `bench.py --profile-case`.
ALU_LANES_PER_SM = 64
# DRAM bytes (read + write) of one launch of the dominant kernel (k_branch_family on the step), from
# one ncu capture of `bench.py --profile-case` (dram__bytes_read.sum + dram__bytes_write.sum); set to
# None when that kernel changes, until it is captured again.  The kernel has changed since the last
# capture (its staged p values are now loaded four at a time), so the value is None and the last
# capture's figure is reported beside it as such.
BB_TRAFFIC_BYTES = None
BB_TRAFFIC_LAST_CAPTURE = 1080320


def work_ops(depth, n=N_JOBS, m=N_MACH):
    """Algorithmic integer ops to bound one node of depth d (r = n - d):
    prefix release times 2md, remaining sums/min tails 3mr, one-machine bounds
    3m, two-machine Johnson recurrences 4Pr, max over pairs 2P."""
    P = m * (m - 1) // 2
    d = np.asarray(depth, np.int64)
    r = n - d
    return 2 * m * d + 3 * m * r + 3 * m + 4 * P * r + 2 * P


def workload(count=FRONTIER):
    from paper_1206_4973_gb300 import inputs
    p, ub_perm, rec = inputs.pool_workload(N_JOBS, N_MACH, SEED, count)
    frontier = rec[rec[:, N_JOBS] <= N_JOBS - 2]
    return p, ub_perm, rec, frontier


def children_depths(frontier, pool):
    """Depths of the children one iteration bounds (the selection rule: top
    parents while their children fit in the pool, at least one)."""
    n = N_JOBS
    depths, total = [], 0
    for rec in frontier[::-1]:
        r = n - int(rec[n])
        if depths and total + r > pool:
            break
        depths.append((int(rec[n]) + 1, r))
        total += r
    return np.repeat([d for d, _ in depths], [r for _, r in depths]), total


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({nm for r in self.rows if len(r) >= 8 for nm, v in zip(names, r[4:8])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(self.rows[0][1]),
                "reasons": reasons, "samples": len(sm),
                "power_w_max": max(float(r[2]) for r in self.rows if len(r) >= 8 and r[2][:1].isdigit())}


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def whole_job_rate(units_local, seconds_local, world, device=None):
    """Whole-job throughput of a timed region: the units all ranks processed
    over the slowest rank's time (an all-reduce sum of the units and max of
    the seconds; one rank needs no collective).  Returns (rate, seconds)."""
    if world == 1:
        return units_local / seconds_local, seconds_local
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds_local)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()) / float(t.item()), float(t.item())


def step_config(frontier, ub, n_children, world):
    """The workload both arms report: one B&B iteration with a pool of 2^18
    children from the 20x20 seed-1 frontier."""
    return {"workload": "20x20 B&B iteration, pool 2^18 children, from the seed-1 frontier",
            "n": N_JOBS, "m": N_MACH, "seed": SEED, "pool": POOL,
            "frontier_nodes": int(len(frontier)), "ub": int(ub), "children_per_step": int(n_children),
            "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MiB write, outside the step events)",
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    """The CPU oracle timed as the reference arm (host cores, one thread)."""
    if rank != 0:
        return
    import oracle
    p, ub_perm, _, frontier = workload()
    ub = oracle.makespan(p, ub_perm)
    sample_pool = 2**15
    for _ in range(args.warmup):
        oracle.solve(p, ub0=ub, pool=sample_pool, init_nodes=frontier, max_iterations=1)
    bounded, t0 = 0, time.perf_counter()
    for _ in range(args.steps):
        r = oracle.solve(p, ub0=ub, pool=sample_pool, init_nodes=frontier, max_iterations=1)
        bounded += r["bounded"]
    dt = time.perf_counter() - t0
    value = bounded / dt
    sample = (f"each step one B&B iteration of the same workload with a pool of {sample_pool} children "
              f"(of the 2^18) from the 20x20 seed-1 frontier, x{args.steps} steps, serial C oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": step_config(frontier, ub, children_depths(frontier, POOL)[1], world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(p, ub, frontier, pool_nodes, gpu_bound_pool, budget_s=12.0):
    """The serial oracle on one host core (the paper's baseline is one CPU
    core), and the oracle's pool bound on all host cores (OpenMP over the
    nodes) on the 20x20 bounding pool, beside the GPU's fsp_bound_pool."""
    import oracle
    bounded, steps, t0 = 0, 0, time.perf_counter()
    pool = 2**16
    while steps < 8 and (time.perf_counter() - t0) < budget_s:
        r = oracle.solve(p, ub0=ub, pool=pool, init_nodes=frontier, max_iterations=1)
        bounded += r["bounded"]
        steps += 1
    dt = time.perf_counter() - t0
    sample = pool_nodes[:2**18]
    oracle.bound_pool_threads(p, sample[:4096], 0)  # threads up
    t1 = time.perf_counter()
    _, cores = oracle.bound_pool_threads(p, sample, 0)
    dt_all = time.perf_counter() - t1
    rate_all = len(sample) / dt_all
    return {"value": bounded / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} B&B iterations of {pool} children from the same 20x20 frontier "
                      f"({dt:.1f} s, serial C oracle, one host core)",
            "nproc": os.cpu_count(),
            "bound_pool_all_cores": {
                "value": rate_all, "unit": "nodes bounded/s", "cores": cores, "kind": "oracle (OpenMP over nodes)",
                "sample": f"the {len(sample)}-node 20x20 seed-1 bounding pool ({dt_all:.2f} s on {cores} threads)",
                "gpu_fsp_bound_pool_nodes_per_s": gpu_bound_pool,
                "gpu_over_all_cores": gpu_bound_pool / rate_all}}


SOLVES = (  # (n, m, seed, pool): 0 = tuned while searching
    (12, 5, 0, 1024), (20, 5, 2, 0), (50, 5, 3, 0), (100, 5, 4, 0), (20, 10, 5, 0))
SOLVE_BUDGET = 1_000_000_000
SOLVE_BUDGETS = {}  # per-instance node budgets that differ from SOLVE_BUDGET


def solve_times(fsp, budget=SOLVE_BUDGET):
    """Time to optimality of the exact solves (12x5 from UB = +inf with pool 1024;
    20x5, 50x5, 100x5, 20x10 from the device NEH makespan with the tuned pool),
    each stopped by a node budget; the NEH time is reported apart from the
    search time (time_s is their sum)."""
    from paper_1206_4973_gb300 import inputs
    out = []
    for n, m, seed, pool in SOLVES:
        p = inputs.instance(n, m, seed)
        inst = fsp.fsp_create_instance(p)
        t0 = time.perf_counter()
        if pool == 0:
            ub0, perm0 = fsp.fsp_neh(inst)
        else:
            ub0, perm0 = fsp.UB_INF, None
        t1 = time.perf_counter()
        cap = SOLVE_BUDGETS.get((n, m, seed), budget)
        r = fsp.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=pool, node_budget=cap)
        t2 = time.perf_counter()
        row = {"instance": f"{n}x{m} seed {seed}", "ub0": None if pool else ub0, "cmax": r["cmax"],
               "optimal": r["status"] == fsp.OK, "time_s": t2 - t0, "neh_s": t1 - t0, "search_s": t2 - t1,
               "node_budget": cap, "nodes_bounded": r["nodes_bounded"],
               "iterations": r["iterations"], "pool": r["tuned_pool"] if pool == 0 else pool,
               "warps_per_cta": r["tuned_warps"], "nodes_per_s": r["nodes_bounded"] / (t2 - t1)}
        if pool == 0:  # the same solve with bidirectional branching (the ends alternate)
            t3 = time.perf_counter()
            b = fsp.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=0, node_budget=cap,
                              branching=fsp.BRANCH_BIDIR)
            t4 = time.perf_counter()
            row["bidirectional"] = {"cmax": b["cmax"], "optimal": b["status"] == fsp.OK, "search_s": t4 - t3,
                                    "time_s": t4 - t3 + (t1 - t0), "nodes_bounded": b["nodes_bounded"],
                                    "pool": b["tuned_pool"], "nodes_per_s": b["nodes_bounded"] / (t4 - t3)}
        out.append(row)
        inst.close()
    return out


LEARNED = ((20, 20, 6), (50, 20, 7))
LEARNED_POOL, LEARNED_BUDGET, LOG_NODES = 2**17, 1_000_000_000, 1_000_000


def learned_vs_plain(fsp, budget=LEARNED_BUDGET):
    """Learned pair order vs the plain order on the 20x20 (seed 6) and 50x20
    (seed 7) instances: a network trained on 1e6 children a plain search logs,
    then both orders run the same depth-first search (device NEH UB, pool
    2^17, same node budget); the search must be identical, only the time may
    differ."""
    import torch
    from paper_1206_4973_gb300 import inputs
    out = []
    for n, m, seed in LEARNED:
        P = m * (m - 1) // 2
        p = inputs.instance(n, m, seed)
        inst = fsp.fsp_create_instance(p)
        ub0, perm0 = fsp.fsp_neh(inst)
        kw = dict(ub0=ub0, ub0_perm=perm0, pool_size=LEARNED_POOL)
        t0 = time.perf_counter()
        log = torch.zeros((LOG_NODES, inst.stride), dtype=torch.uint8, device="cuda")
        fsp.fsp_solve(inst, node_budget=LOG_NODES, log_nodes=log, **kw)
        x, y = fsp.fsp_node_features(inst, log)
        mlp = fsp.Mlp(2 * m + 1, 128, P, seed=seed)
        perm = torch.randperm(LOG_NODES, generator=torch.Generator().manual_seed(seed)).cuda()
        x, y = x[perm].contiguous(), y[perm].contiguous()
        B = 4096
        steps = 3 * LOG_NODES // B
        for it in range(steps):
            s = (it * B) % (LOG_NODES - B)
            loss = mlp.train_step(x[s:s + B], y[s:s + B], lr=1e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        res, phases = {}, {}
        # plain: the family kernel (certified pair skipping); plain_per_child: every
        # pair of every child evaluated (FSP_FAMILY=0); learned: the family kernel
        # with each parent's predicted pairs first
        for name, extra, env in (("plain", {}, None), ("plain_per_child", {}, "0"),
                                 ("learned", {"model": mlp, "topk": 4}, None)):
            if env is not None:
                os.environ["FSP_FAMILY"] = env
            try:
                fsp.fsp_solve(inst, node_budget=budget // 100, **kw, **extra)  # warm-up
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                r = fsp.fsp_solve(inst, node_budget=budget, trace_cap=1, **kw, **extra)
                res[name] = (r, time.perf_counter() - t1)
                q = fsp.fsp_solve(inst, node_budget=budget // 20, profile=True, **kw, **extra)  # phase times
            finally:
                os.environ.pop("FSP_FAMILY", None)
            phases[name] = {k: round(q[k] / max(1, q["iterations"]) * 1e3, 1)
                            for k in ("select_ms", "infer_ms", "bound_ms", "compact_ms")}
        (a, ta), (b, tb), (c, tc) = res["plain"], res["learned"], res["plain_per_child"]
        same = all(a[k] == b[k] == c[k] for k in ("cmax", "nodes_bounded", "nodes_branched", "nodes_pruned",
                                                  "leaves", "iterations", "incumbent_updates", "stack_left"))
        out.append({"instance": f"{n}x{m} seed {seed}", "nodes_bounded": a["nodes_bounded"],
                    "plain_nodes_per_s": a["nodes_bounded"] / ta, "learned_nodes_per_s": b["nodes_bounded"] / tb,
                    "plain_per_child_nodes_per_s": c["nodes_bounded"] / tc,
                    "speedup": ta / tb, "speedup_vs_per_child": tc / tb, "family_vs_per_child": tc / ta,
                    "identical_search": same, "cmax": a["cmax"],
                    "optimal": a["status"] == fsp.OK, "early_cut_fraction": b["early_pruned"] / max(1, b["nodes_bounded"]),
                    "train_s": t_train, "train_final_loss": loss,
                    "us_per_iteration": phases,
                    # where the family kernel's work goes: families (parents) whose children
                    # all fall to their one-machine bounds, those the predicted pairs close,
                    # and the pair evaluations left exact
                    "families": {nm: {"parents": x["nodes_branched"], "closed_by_lb1": x["families_closed_lb1"],
                                      "closed_by_predicted_pairs": x["families_closed_predicted"],
                                      "exact_pair_evals": x["exact_pair_evals"]}
                                 for nm, (x, _) in (("plain", res["plain"]), ("learned", res["learned"]))}})
        inst.close()
    return out


VARIANT_RUNS = ((20, 10, 5, 0, 0), (20, 5, 2, 0, 0), (20, 20, 6, 2**17, 200_000_000), (50, 20, 7, 2**17, 50_000_000))


def bound_variants(fsp):
    """The base bound against the heads variant (release times raised by the
    smallest heads) on the same searches: device NEH UB, the tuned pool (0) or
    a fixed one, a node budget (0 = to optimality)."""
    from paper_1206_4973_gb300 import inputs
    out = []
    for n, m, seed, pool, budget in VARIANT_RUNS:
        p = inputs.instance(n, m, seed)
        inst = fsp.fsp_create_instance(p)
        ub0, perm0 = fsp.fsp_neh(inst)
        row = {"instance": f"{n}x{m} seed {seed}", "pool": pool or "tuned", "node_budget": budget}
        for name, var in (("base", fsp.BOUND_BASE), ("heads", fsp.BOUND_HEADS)):
            inst.set_bound(var)
            fsp.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=pool or 1024, node_budget=200_000)  # warm-up
            t0 = time.perf_counter()
            r = fsp.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=pool, node_budget=budget)
            dt = time.perf_counter() - t0
            row[name] = {"time_s": dt, "nodes_bounded": r["nodes_bounded"], "cmax": r["cmax"],
                         "optimal": r["status"] == fsp.OK, "nodes_per_s": r["nodes_bounded"] / dt}
        inst.close()
        out.append(row)
    return out


BIDIR_RUNS = ((12, 5, 0), (20, 5, 2), (20, 10, 5), (15, 10, 101))


def bidir_vs_forward(fsp):
    """Forward against bidirectional branching on the same instances: device
    NEH UB, tuned pool, to optimality; the optimum must agree."""
    from paper_1206_4973_gb300 import inputs
    out = []
    for n, m, seed in BIDIR_RUNS:
        p = inputs.instance(n, m, seed)
        inst = fsp.fsp_create_instance(p)
        ub0, perm0 = fsp.fsp_neh(inst)
        row = {"instance": f"{n}x{m} seed {seed}", "ub0": ub0}
        for name, br in (("forward", fsp.BRANCH_FORWARD), ("bidirectional", fsp.BRANCH_BIDIR)):
            fsp.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=4096, node_budget=100_000, branching=br)
            t0 = time.perf_counter()
            r = fsp.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=0, node_budget=SOLVE_BUDGET, branching=br)
            dt = time.perf_counter() - t0
            row[name] = {"time_s": dt, "nodes_bounded": r["nodes_bounded"], "cmax": r["cmax"],
                         "optimal": r["status"] == fsp.OK, "nodes_per_s": r["nodes_bounded"] / dt}
        row["same_optimum"] = row["forward"]["cmax"] == row["bidirectional"]["cmax"]
        row["node_ratio"] = row["bidirectional"]["nodes_bounded"] / max(1, row["forward"]["nodes_bounded"])
        inst.close()
        out.append(row)
    return out


BATCH_COUNT, BATCH_BUDGET, LEFTOVER_BUDGET = 256, 5_000_000, 200_000_000


def batch_solve(fsp):
    """256 instances of mixed shape (n in {12,15,20,50}, m in {5,10}, seeds
    100-355): pools tuned per shape, one persistent launch (CUDA graph) with a
    per-instance node budget, then the instances the budget stopped are
    finished by the full-GPU search from the batch's incumbent."""
    import torch
    from paper_1206_4973_gb300 import inputs
    shapes = inputs.batch_shapes(BATCH_COUNT, first_seed=100)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    instances = [inputs.instance(n, m, sd) for n, m, sd in shapes]
    t0 = time.perf_counter()
    pools = fsp.fsp_batch_tune_pools(instances, probe_budget=100_000)
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    warps = fsp.fsp_batch_tune_warps(instances, pools, probe_budget=100_000)
    t_tune_w = time.perf_counter() - t0
    B = fsp.Batch(instances, pools, np.full(BATCH_COUNT, BATCH_BUDGET, np.int64))

    def timed():
        B.run()
        B.results()  # warm-up launch
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        B.run()
        out = B.results()
        return out, time.perf_counter() - t1

    res, t_batch = timed()  # whole instances, 8 warps per CTA for every shape
    solved = sum(r["status"] == fsp.OK for r in res)
    nodes = sum(r["nodes_bounded"] for r in res)
    # split mode: the roots' subtrees as work items, a shared UB per instance
    B.set_split(True)
    res_s, t_split = timed()
    # the block shape tuned per shape, whole instances and split
    B.set_warps(warps)
    B.set_split(False)
    res_w, t_w = timed()
    B.set_split(True)
    res_ws, t_ws = timed()
    B.set_split(False)
    tuned = {"whole": {"batch_s": t_w, "solved_in_batch": sum(r["status"] == fsp.OK for r in res_w),
                       "batch_nodes_per_s": sum(r["nodes_bounded"] for r in res_w) / t_w,
                       "same_results_as_8_warps": all(
                           {k: v for k, v in a.items() if k != "perm"} == {k: v for k, v in b.items() if k != "perm"}
                           for a, b in zip(res, res_w))},
             "split": {"batch_s": t_ws, "solved_in_batch": sum(r["status"] == fsp.OK for r in res_ws),
                       "batch_nodes_per_s": sum(r["nodes_bounded"] for r in res_ws) / t_ws,
                       "same_optima": all(a["cmax"] == b["cmax"] for a, b in zip(res, res_ws)
                                          if a["status"] == fsp.OK and b["status"] == fsp.OK)},
             "tune_s": t_tune_w}
    # bidirectional branching in the batch (tuned block shapes), whole instances and split
    bidir = {}
    for mode in ("whole", "split"):
        B.set_bidir(True)
        B.set_split(mode == "split")
        B.run()
        B.results()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        B.run()
        rb = B.results()
        tb = time.perf_counter() - t1
        cs = B.class_stats()  # the CTAs of this launch, per class, from the global timer
        bidir[mode] = {"batch_s": tb, "solved_in_batch": sum(r["status"] == fsp.OK for r in rb),
                       "batch_nodes_bounded": sum(r["nodes_bounded"] for r in rb),
                       "batch_nodes_per_s": sum(r["nodes_bounded"] for r in rb) / tb,
                       "same_optima_as_forward": all(a["cmax"] == b["cmax"] for a, b in zip(res, rb)
                                                     if a["status"] == fsp.OK and b["status"] == fsp.OK),
                       # CTA lifetimes summed over the SMs' time: the mean number of live batch CTAs
                       # per SM over the launch (each class's grid is one CTA per SM at these block
                       # shapes, and a 20-warp CTA's registers fill an SM, so about 1 is the ceiling)
                       "live_ctas_per_sm": (sum(c["ctas"] * c["busy_mean_ms"] for c in cs)
                                            / max(1e-9, sms * cs[0]["launch_span_ms"])),
                       "ctas_per_sm_per_class": max(c["ctas"] for c in cs) / sms,
                       "classes": [{"shape": f"{c['n']}x{c['m']}", "warps": c["warps"], "ctas": c["ctas"],
                                    "items": c["items"], "busy_mean_ms": round(c["busy_mean_ms"], 2),
                                    "busy_max_ms": round(c["busy_max_ms"], 2),
                                    "last_end_ms": round(c["last_end_ms"], 2)} for c in cs],
                       "launch_span_ms": round(cs[0]["launch_span_ms"], 2)}
    B.set_bidir(False)
    B.set_split(False)
    split = {"batch_s": t_split, "solved_in_batch": sum(r["status"] == fsp.OK for r in res_s),
             "batch_nodes_bounded": sum(r["nodes_bounded"] for r in res_s),
             "batch_nodes_per_s": sum(r["nodes_bounded"] for r in res_s) / t_split,
             "same_optima": all(a["cmax"] == b["cmax"] for a, b in zip(res, res_s)
                                if a["status"] == fsp.OK and b["status"] == fsp.OK)}
    t2 = time.perf_counter()
    finished, left_nodes = 0, 0
    for i, r in enumerate(res):  # the instances the forward batch left, by the bidirectional search
        if r["status"] == fsp.OK:
            continue
        inst = fsp.fsp_create_instance(instances[i])
        q = fsp.fsp_solve(inst, ub0=r["cmax"], ub0_perm=r["perm"], pool_size=0, node_budget=LEFTOVER_BUDGET,
                          branching=fsp.BRANCH_BIDIR)
        finished += q["status"] == fsp.OK
        left_nodes += q["nodes_bounded"]
        inst.close()
    t_left = time.perf_counter() - t2
    per_shape = {}
    for (n, m, _), r, w in zip(shapes, res, warps):
        d = per_shape.setdefault(f"{n}x{m}", {"pool": r["pool"], "warps": int(w), "solved": 0, "count": 0})
        d["count"] += 1
        d["solved"] += r["status"] == fsp.OK
    B.close()
    # the headline: the recommended configuration (block shape tuned per shape, the roots'
    # subtrees shared between CTAs, bidirectional branching); every other mode is listed beside it
    head = bidir["split"]
    return {"instances": BATCH_COUNT, "mode": "tuned block shapes, split, bidirectional",
            "solved_in_batch": head["solved_in_batch"], "batch_s": head["batch_s"],
            "batch_nodes_bounded": head["batch_nodes_bounded"], "batch_nodes_per_s": head["batch_nodes_per_s"],
            "same_optima_as_forward": head["same_optima_as_forward"],
            "live_ctas_per_sm": head["live_ctas_per_sm"], "ctas_per_sm_per_class": head["ctas_per_sm_per_class"],
            "launch_span_ms": head["launch_span_ms"],
            "classes": head["classes"],
            "tune_s": t_tune, "tune_block_shapes_s": t_tune_w,
            "forward": {"whole_8_warps": {"batch_s": t_batch, "solved_in_batch": solved,
                                          "batch_nodes_bounded": nodes, "batch_nodes_per_s": nodes / t_batch},
                        "split_8_warps": split,
                        "whole_tuned": tuned["whole"], "split_tuned": tuned["split"]},
            "bidirectional_whole_tuned": bidir["whole"],
            "node_budget_per_instance": BATCH_BUDGET, "leftovers": BATCH_COUNT - solved,
            "leftovers_from": "forward whole, 8 warps",
            "leftovers_finished": finished, "leftover_branching": "bidirectional", "leftover_s": t_left,
            "leftover_nodes": left_nodes,
            "leftover_budget_each": LEFTOVER_BUDGET, "per_shape": per_shape}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="the timed step, e2e, fsp_bound_pool and the roofline only (no solves, learned order, "
                         "batch, bound variants or bidirectional runs)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one B&B step and one 2^18-node bounding launch, nothing else (for ncu)")
    ap.add_argument("--profile-learned", action="store_true",
                    help="three plain then three learned iterations (untrained network) from the 20x20 frontier, for ncu")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_1206_4973_gb300 import build as fsp_build
    from paper_1206_4973_gb300 import fsp

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    fsp_build.build()
    fsp.load()
    dev = torch.device("cuda", local)
    if args.profile_learned:
        p1, _, _, fr = workload()
        inst1 = fsp.fsp_create_instance(p1)
        ub1, _ = fsp.fsp_neh(inst1)
        mlp = fsp.Mlp(41, 128, 190, seed=6)
        fr_dev = torch.from_numpy(fr).to(dev)
        for order in ({}, {"model": mlp, "topk": 4}):
            r = fsp.fsp_solve(inst1, ub0=ub1, pool_size=LEARNED_POOL, max_iterations=3, init_nodes=fr_dev, **order)
        torch.cuda.synchronize()
        print(json.dumps({"profile_learned": True, "bounded": r["nodes_bounded"], "early": r["early_pruned"]}))
        return

    # Rank r runs the same workload on its own GPU (independent replicas).
    p, ub_perm, pool_nodes, frontier = workload()
    inst = fsp.fsp_create_instance(p)
    st = torch.cuda.current_stream()
    full = np.zeros((1, inst.stride), np.uint8)
    full[0, :N_JOBS] = ub_perm
    full[0, N_JOBS] = N_JOBS
    ub = int(fsp.fsp_bound_pool(inst, torch.from_numpy(full).to(dev)).item())  # depth n: its makespan
    front_dev = torch.from_numpy(frontier).to(dev)
    front_host = torch.from_numpy(frontier).pin_memory()
    ws = torch.empty(fsp.fsp_solve_workspace_bytes(inst, pool_size=POOL, init_nodes=front_dev),
                     dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    depths, n_children = children_depths(frontier, POOL)
    ops_per_step = int(work_ops(depths).sum())

    # the step through the public API: a prepared fsp_solve (options, workspace and result
    # buffers built once; every run() is one call into the library)
    calls = {id(x): fsp.SolveCall(inst, ub0=ub, pool_size=POOL, init_nodes=x, max_iterations=1, workspace=ws)
             for x in (front_dev, front_host)}
    # the same call with the library's phase events (select, branch + bound, compaction), which
    # time the dominant kernel for the roofline in a second timed region of identical steps
    prof_call = fsp.SolveCall(inst, ub0=ub, pool_size=POOL, init_nodes=front_dev, max_iterations=1, workspace=ws,
                              profile=True)

    def step(init):
        return calls[id(init)].run()

    if args.profile_case:
        r = step(front_dev)
        nodes = torch.from_numpy(pool_nodes[:POOL]).to(dev)
        fsp.fsp_bound_pool(inst, nodes, ub)
        fsp.fsp_check_status(inst)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": True, "bounded": r["nodes_bounded"]}))
        return

    for _ in range(args.warmup):
        r = step(front_dev)
    assert r["nodes_bounded"] == n_children, (r["nodes_bounded"], n_children)

    # ---- timed region: K steps, L2 flushed before each, CUDA events per step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    bound_ms, launches, bounded = [], 0, 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_soak = time.perf_counter()  # identical steps, so the sampler sees the load for ~2 s
        while time.perf_counter() - t_soak < 2.0:
            step(front_dev)
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(st)
            r = step(front_dev)
            ev[i][1].record(st)
            bounded += r["nodes_bounded"]
            launches += 2 + 4 * r["iterations"]  # k_solve_init_nodes, k_init_cum; per iteration select, branch-bound, count, push
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        # the same steps with the phase events: the dominant kernel's duration (roofline)
        phases = {"select": [], "branch_bound": [], "compact": []}
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            rp = prof_call.run()
            bound_ms.append(rp["bound_ms"])
            phases["select"].append(rp["select_ms"])
            phases["branch_bound"].append(rp["bound_ms"])
            phases["compact"].append(rp["compact_ms"])
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, t_total = whole_job_rate(bounded, sum(step_ms) / 1e3, world, dev)

    # ---- end to end through the C ABI with host buffers (frontier H2D inside the call)
    e2e_ms = []
    for _ in range(3):  # warm-up: the host-buffer path's first calls
        step(front_host)
    for i in range(max(3, args.steps // 2)):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = step(front_host)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = {"value": r["nodes_bounded"] * len(e2e_ms) / (sum(e2e_ms) / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(frontier.nbytes),
           "d2h_bytes_per_step": int(4 + 4 * N_JOBS + fsp.ctypes.sizeof(fsp.fsp_stats))}

    # ---- the bounding kernel alone on the 2^12..2^20 pools (dominant kernel)
    peak_ops = SMS * INT_LANES_PER_SM * SM_MAX_MHZ * 1e6
    bp = {}
    big = pool_nodes if len(pool_nodes) >= max(BOUND_POOLS) else workload(max(BOUND_POOLS))[2]
    for cnt in BOUND_POOLS:
        nodes = torch.from_numpy(big[:cnt]).to(dev)
        out = torch.empty(cnt, dtype=torch.int32, device=dev)
        for _ in range(3):
            fsp.fsp_bound_pool(inst, nodes, ub, out)
        ts = []
        for i in range(max(5, args.steps // 2)):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fsp.fsp_bound_pool(inst, nodes, ub, out)
            b.record(st)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        ops = int(work_ops(big[:cnt, N_JOBS]).sum())
        bp[str(cnt)] = {"nodes_per_s": cnt / (ms / 1e3), "ms": ms, "int_ops_per_s": ops / (ms / 1e3),
                        "frac_of_int_peak": ops / (ms / 1e3) / peak_ops}
        fsp.fsp_check_status(inst)

    achieved = ops_per_step / (statistics.mean(bound_ms) / 1e3)
    alu_peak = SMS * ALU_LANES_PER_SM * SM_MAX_MHZ * 1e6
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                "frac": achieved / peak_ops, "traffic": BB_TRAFFIC_BYTES,
                "traffic_last_capture": {"bytes": BB_TRAFFIC_LAST_CAPTURE,
                                         "of": "the previous revision of k_branch_family (the same global "
                                               "accesses; its shared-memory staging differed)"},
                "kernel": "k_branch_family (branching + bounding of the pool's children, one warp per parent)",
                "ops_per_launch": ops_per_step, "children_per_launch": n_children,
                "peak_basis": f"{SMS} SMs x {INT_LANES_PER_SM} int32 lanes x {SM_MAX_MHZ:.0f} MHz (issue ceiling)",
                "alu_pipe": {"peak": alu_peak / 1e12, "frac": achieved / alu_peak,
                             "basis": f"{SMS} SMs x {ALU_LANES_PER_SM} ALU-pipe lanes x {SM_MAX_MHZ:.0f} MHz"},
                "work_equivalent": "achieved counts the full per-child bound (W ops); the kernels reach the same "
                                   "integers with fewer instructions",
                # fsp_bound_pool alone on the 20x20 bounding pools (arbitrary nodes, Sec. III Type 1)
                "bound_pool": {k: {"ms": round(v["ms"], 4), "nodes_per_s": v["nodes_per_s"],
                                   "frac": round(v["frac_of_int_peak"], 3),
                                   "frac_alu_pipe": round(v["frac_of_int_peak"] * peak_ops / alu_peak, 3)}
                               for k, v in bp.items()}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": step_config(frontier, ub, n_children, world),
            "roofline": roofline,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": e2e,
            "bound_pool": bp,
            "phase_ms": {k: statistics.mean(v) for k, v in phases.items()},
            "wall_s": t_wall,  # host clock over the K steps, the L2 flush before each and host waits
            "wall_s_covers": "the K timed steps plus the 512 MiB L2 flush before each (about 0.14 ms) and "
                             "host-side waits; ms_per_step is the device time of the steps alone",
        }
        if not args.no_extras:
            line["bound_variants"] = bound_variants(fsp)
            line["bidirectional"] = bidir_vs_forward(fsp)
            line["solves"] = solve_times(fsp)
            line["learned_order"] = learned_vs_plain(fsp)
            line["batch"] = batch_solve(fsp)
        if world == 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(p, ub, frontier, big, bp[str(2**18)]["nodes_per_s"])
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
