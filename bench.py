#!/usr/bin/env python
"""Benchmark of the Sinkhorn iterations of Algorithm 2 on one GB300 per rank.

A step is one Sinkhorn pass of Algorithm 2 (source update, forward sweep with the capacity
updates, sink update, backward sweep, FP64 convergence reductions) over the traffic-scale
workload: perturbed 100x100 grid road graph, L = 1024 origin-destination commodities,
T = 100, eps = 0.005.  The timed passes continue a solve that started from the initial duals
(W warm-up passes); a solve of this instance needs thousands of passes to reach marginal
error 1e-6, so full solves-to-tolerance are timed on the multi-commodity random-geometric
workload (n = 400, L = 64, T = 50, eps = 0.01) and reported as "solves_per_s".

  value   edge*commodity*timestep updates per second, whole job: 2 (T-1) nnz(K) L updates per
          Sinkhorn pass (nnz(K) = transitions of the line graph with wait loops), summed over
          ranks, divided by the slowest rank's device time (CUDA events on the solver stream)
  e2e     the same metric through the C ABI from host buffers: create (host -> device copy
          of the problem), K passes, read the flows back (device -> host), destroy
  roofline  the forward-step kernel (the dominant kernel): algorithmic bytes per launch over
          its mean duration inside the timed passes, against the measured HBM copy bandwidth
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample of the same instance

--impl reference times the oracle itself (the CPU reference of this build) on the same
workload and metric.  With torchrun (N > 1) every rank solves its own replica (seed = rank):
independent problems, no collective on the data path ("scaling": "weak").
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

METRIC = "edge*commodity*timestep updates/s and solves/s at marginal err<=1e-6; p50/p99"
UNIT = "updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200, help="timed Sinkhorn passes")
    ap.add_argument("--warmup", type=int, default=20, help="untimed passes before the timed ones")
    ap.add_argument("--solves", type=int, default=20, help="timed full solves of the RGG workload")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle sample")
    ap.add_argument("--batch", type=int, default=256,
                    help="instances of the batched workload (uneven random geometric graphs); 0 = skip")
    ap.add_argument("--batch-max-passes", type=int, default=3000)
    ap.add_argument("--single-batch", type=int, default=64,
                    help="members of the single-commodity workload (linear-domain path); 0 = skip the single-commodity legs")
    ap.add_argument("--single-reps", type=int, default=5, help="timed repetitions of the 5x5 grid solves")
    ap.add_argument("--batch-eps-factor", type=float, default=0.0,
                    help="epsilon continuation of the batched and serving workloads: start at this multiple of "
                         "each instance's epsilon (halved per stage); 0 = off (default: on these instances it "
                         "costs passes).  The one-at-a-time arm uses the same")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="profiling case only: the first N batched-workload instances, 3 graph launches of the "
                         "tick kernel, then exit (for ncu captures of k_batch_tick)")
    ap.add_argument("--profile-linear", type=int, default=0,
                    help="profiling mode: this many linear-domain passes on the 5x5 grid, 20 on a 400-node and 10 on a 2000-node "
                         "single-commodity graph (three kernel launches), then exit")
    ap.add_argument("--profile-rgg", type=int, default=0,
                    help="profiling case only: 3 untimed full solves of the n=400 random-geometric workload, then N "
                         "solves between cudaProfilerStart/Stop (for ncu --profile-from-start off), then exit")
    ap.add_argument("--serve-rates", type=str, default="2,20",
                    help="Poisson arrival rates (requests/s) of the serving workload; empty = skip.  With 5%% "
                         "traffic-scale requests (about 8 s of GPU each) the knee is near 2.5 requests/s")
    ap.add_argument("--serve-seconds", type=float, default=15.0, help="arrival window per rate")
    ap.add_argument("--serve-drain", type=float, default=15.0, help="extra time for open requests per rate")
    ap.add_argument("--serve-large-passes", type=int, default=1500,
                    help="pass limit of the traffic-scale requests in the serving mix (they run with epsilon "
                         "continuation, 8 eps -> eps in 3 stages, and need about 700 passes)")
    ap.add_argument("--no-traffic-solve", action="store_true",
                    help="skip the full solve of the traffic-scale workload (epsilon continuation)")
    ap.add_argument("--oracle-timing", action="store_true",
                    help="with --impl reference: the oracle's update rate per pass on one core and on all cores "
                         "for the four workloads, and its time to convergence on the grid and random-geometric "
                         "workloads and on 8 sampled batch instances (host only, a few minutes)")
    ap.add_argument("--horizon", type=int, default=100,
                    help="T of the traffic-scale grid (100 = the benchmark workload; smaller values only "
                         "for profiling captures that must stay within a few GB)")
    return ap.parse_args()


def combine_ranks(pg, seconds, units, device):
    """Whole-job figures of independent replicas: the slowest rank's time and the units all
    ranks processed (max and sum all-reduces; pg = torch.distributed or None for one rank)."""
    if pg is None:
        return float(seconds), float(units)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    pg.all_reduce(u, op=pg.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(seed: int, T: int = 100):
    from paper_2106_14485_gb300 import instances
    if T == 100:
        return instances.traffic_grid(seed)
    return instances.grid_traffic_instance(seed=seed, T=T)


def workload_config(inst, tol):
    return {"workload": f"traffic-scale grid 100x100 road graph, L={inst.L} OD commodities, T={inst.T}, "
                        f"eps={inst.eps}, capacities U[0.5,3]; one step = one Sinkhorn pass",
            "nodes": inst.n_nodes, "states": inst.n_states, "nnz_K": inst.nnz_line_graph(),
            "L": inst.L, "T": inst.T, "eps": inst.eps, "tol": tol,
            "cache": "inputs larger than L2: message panels of several GB per problem",
            "parallelism": "independent replicas per GPU"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("ots_kernels.cu", "ots_device.cuh", "ots_step.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2106_14485_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(horizon: int):
    """DRAM bytes per forward launch from the committed ncu summary, or None when the kernel
    sources changed since the counters were taken (or the workload differs)."""
    path = os.path.join(ROOT, "profiles", "k_forward_tma-grid100x100-L1024.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and not line.startswith(("|", " ")):
            k, _, v = line.partition(":")
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_sources_hash():
        return None
    try:
        return int(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def forward_bytes_per_launch(info, inst):
    """Algorithmic bytes of one forward-step launch: read A_{t-1} and B_{t+1}, write A_t
    (6 bytes per entry: fp32 hi + 16-bit remainder) for V x L node rows, plus the per-state vectors
    (cost, capacity, old/new duals, weights, CSR: 56 bytes per state) and the node CSR."""
    V, S, L = info["n_nodes"], info["n_states"], inst.L
    return 18 * V * L + 56 * S + 4 * (V + 1)


def backward_bytes_per_launch(info, inst):
    V, S, L = info["n_nodes"], info["n_states"], inst.L
    return 12 * V * L + 16 * S + 4 * (V + 1)


def cpu_baseline(inst, budget_s: float):
    """The oracle as it stands, on a bounded sample of the same instance: backward message
    products (Algorithm 2, Psi_{t-1} = (Psi_t .* K_L) diag(u_t) K^T) over the first l1
    commodities, repeated until the time budget is used."""
    from oracle.oracle import Oracle, get_threads
    o = Oracle(inst)
    nnz = o.nnz
    l1 = 16
    t0 = time.perf_counter()
    o.sample_backward_products(1, l1)
    one = max(time.perf_counter() - t0, 1e-3)
    k = max(1, int(budget_s / one))
    t0 = time.perf_counter()
    o.sample_backward_products(k, l1)
    dt = time.perf_counter() - t0
    updates = (k + 1) * nnz * l1            # k products after one boundary product, each nnz * l1 terms
    return {"value": updates / dt, "unit": UNIT, "cores": get_threads(), "kind": "oracle",
            "sample": f"{k} backward message products of the traffic-scale instance on commodities "
                      f"0..{l1 - 1} ({updates:.3e} updates, {dt:.1f} s, FP64 log domain)"}


def oracle_timing(args):
    """The FP64 oracle timed on the host: updates/s (2 (T-1) nnz(K) L per pass) on one core and
    on every core, per workload, and time to marginal error <= tol from the initialisation on
    the 5x5 grid, the n = 400 random geometric graph and 8 seeded samples of the batch (each
    bounded to about a minute; a bound that ends the run first is reported as such).  The
    traffic workload's pass is sampled (backward products on 16 commodities): a full pass takes
    minutes on the host and convergence hours."""
    from oracle.oracle import Oracle, get_threads, set_threads
    from paper_2106_14485_gb300 import instances as I
    cores = get_threads()
    out = {"cores": cores, "per_pass": [], "to_convergence": []}

    def pass_rate(inst, threads, passes=1):
        set_threads(threads)
        o = Oracle(inst)
        o.backward_sweep()
        t0 = time.perf_counter()
        for _ in range(passes):
            o.iteration()
        dt = time.perf_counter() - t0
        return passes * inst.n_updates_per_iteration() / dt, dt / passes

    batch = I.uneven_rgg_batch(0, count=256, workers=min(16, os.cpu_count() or 1))
    rng = np.random.default_rng(5)
    sample = [batch[int(k)] for k in rng.choice(len(batch), 8, replace=False)]
    for name, inst, passes in (("grid5x5 L=1 T=10", I.grid_single_commodity(0), 50), ("rgg400 L=64 T=50", I.rgg400(0), 2),
                               ("batch sample (mean of 8)", None, 1)):
        row = {"workload": name}
        for threads, key in ((1, "one_core"), (cores, "all_cores")):
            if inst is None:
                rates = [pass_rate(x, threads)[0] for x in sample]
                row[key + "_updates_per_s"] = float(np.mean(rates))
            else:
                row[key + "_updates_per_s"], row[key + "_s_per_pass"] = pass_rate(inst, threads, passes)
        out["per_pass"].append(row)
    traffic = workload(0, 100)
    row = {"workload": "traffic grid100x100 L=1024 T=100 (sampled: backward products, 16 commodities)"}
    for threads, key in ((1, "one_core"), (cores, "all_cores")):
        set_threads(threads)
        o = Oracle(traffic)
        t0 = time.perf_counter()
        o.sample_backward_products(3, 16)
        dt = time.perf_counter() - t0
        row[key + "_updates_per_s"] = 4 * o.nnz * 16 / dt
        del o
    out["per_pass"].append(row)
    for name, inst in [("grid5x5 L=1 T=10", I.grid_single_commodity(0)), ("rgg400 L=64 T=50", I.rgg400(0))] + \
                      [(x.name, x) for x in sample]:
        # chunks of 20 passes, each continuing from the current duals, until tol or 60 s
        threads = 1 if inst.n_updates_per_iteration() < 1e6 else cores   # tiny: threads only add overhead
        set_threads(threads)
        o = Oracle(inst)
        passes, seconds, done, status = 0, 0.0, False, 0
        while not done and seconds < 60.0:
            r = o.solve(max_iters=20, tol=args.tol)
            passes += r["iters"]
            seconds += r["seconds"]
            status = r["status"]
            done = status == 0 and r["src_resid"] <= args.tol and r["cap_viol"] <= args.tol
            if status != 0:
                break
        out["to_convergence"].append({"workload": name, "converged": bool(done), "passes": passes,
                                      "seconds": seconds, "threads": threads, "status": status,
                                      "bound": None if done else "60 s"})
    set_threads(cores)
    print(json.dumps({"impl": "reference", "oracle_timing": out}), flush=True)
    return 0


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.oracle_timing:
        return oracle_timing(args)
    inst = workload(0, args.horizon)
    from oracle.oracle import Oracle, get_threads
    o = Oracle(inst)
    nnz = o.nnz
    l1 = 16
    per_step = max(0.2, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    t0 = time.perf_counter()
    o.sample_backward_products(1, l1)
    one = max(time.perf_counter() - t0, 1e-3)
    k = max(1, int(per_step / one))
    for _ in range(args.warmup):
        o.sample_backward_products(k, l1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.sample_backward_products(k, l1)
    dt = time.perf_counter() - t0
    updates = args.steps * (k + 1) * nnz * l1
    value = updates / dt
    sample = (f"each step: {k} backward message products of the traffic-scale instance on commodities "
              f"0..{l1 - 1} (FP64 log domain, {get_threads()} threads)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(inst, args.tol), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": get_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


ORACLE_BATCH_SAMPLE = 8
TRAFFIC_SAMPLE = ((0, 4), (1020, 1024))      # commodity ranges the oracle evaluates on the traffic workload


def oracle_sample_index(st):
    """A seeded sample of converged instances of the batch for the oracle leg."""
    ok = [k for k, s in enumerate(st) if s["status"] == 0]
    if not ok:
        return []
    rng = np.random.default_rng(8)
    return sorted(int(k) for k in rng.choice(ok, min(ORACLE_BATCH_SAMPLE, len(ok)), replace=False))


def traffic_commodity_sample(ots, h, inst):
    """GPU per-commodity flows of the sampled commodities, and the duals, kept for the oracle leg."""
    ranges = [(a, b) for a, b in TRAFFIC_SAMPLE if b <= inst.L]
    return {"inst": inst, "duals": ots.ots_get_duals(h), "ranges": ranges,
            "cflows": [ots.ots_get_commodity_flows(h, 1, inst.T + 1, a, b) for a, b in ranges]}


def oracle_check(item, optimum_tol=None):
    """Oracle leg: the FP64 oracle loads the GPU's duals and evaluates Theorem 6 there.  Returns
    the flow error of the GPU against it (relative L1 and the worst entry relative to
    1e-5 F* + 1e-9 max F*) and the marginal violation the oracle measures at those duals (source
    mismatch ||P_{0,1} - R01||_1 / ||R01||_1 and, with every commodity, capacity excess
    sum_t (P_t - d)_+ / ||R01||_1).  With optimum_tol, the oracle also solves the instance from
    its own initialisation to that tolerance and the GPU's flows are compared with that optimum."""
    from oracle.oracle import Oracle
    inst = item["inst"]
    L, S, T = inst.L, inst.n_states, inst.T
    lu, U01, U0T = item["duals"]
    a = np.full((L, S), -np.inf)
    b = np.full((L, S), -np.inf)
    a[inst.src_comm, inst.src_state] = U01
    b[inst.snk_comm, inst.snk_state] = U0T
    R01 = np.zeros((L, S))
    np.add.at(R01, (inst.src_comm, inst.src_state), inst.src_mass)
    o = Oracle(inst)
    o.set_duals(lu, a, b)
    t0 = time.perf_counter()

    def elem(F, Fref):
        return float((np.abs(F - Fref) / (1e-5 * np.abs(Fref) + 1e-9 * np.abs(Fref).max())).max())

    out = {}
    if "ranges" in item:                       # sampled commodities of a large instance
        num = den = mis = mass = worst = 0.0
        for (l0, l1), P in zip(item["ranges"], item["cflows"]):
            Pref = o.projections(l0, l1)
            num += float(np.abs(P - Pref).sum())
            den += float(np.abs(Pref).sum())
            worst = max(worst, elem(P, Pref))
            mis += float(np.abs(Pref[0] - R01[l0:l1]).sum())
            mass += float(R01[l0:l1].sum())
        out.update(commodities=[list(r) for r in item["ranges"]], commodity_flow_rel_l1=num / den,
                   commodity_flow_elem_worst=worst, oracle_src_mismatch=mis / mass)
    else:                                      # every commodity
        Fref = np.zeros((T, S))
        mis = 0.0
        for l0 in range(0, L, 32):
            l1 = min(L, l0 + 32)
            Pref = o.projections(l0, l1)
            Fref += Pref.sum(axis=1)
            mis += float(np.abs(Pref[0] - R01[l0:l1]).sum())
        d = np.concatenate([inst.edge_cap, inst.wait_cap]).astype(np.float64)
        F = item["flows"]
        out.update(flow_rel_l1=float(np.abs(F - Fref).sum() / np.abs(Fref).sum()), flow_elem_worst=elem(F, Fref),
                   oracle_src_mismatch=mis / R01.sum(),
                   oracle_cap_excess=float(sum(np.maximum(Fref[t - 1] - d, 0).sum() for t in range(2, T))) / R01.sum())
        if optimum_tol is not None:
            o2 = Oracle(inst)
            r = o2.solve(max_iters=200000, tol=optimum_tol)
            Fo = o2.flows()
            out.update(optimum_tol=optimum_tol, optimum_passes=r["iters"],
                       flow_rel_l1_vs_optimum=float(np.abs(F - Fo).sum() / np.abs(Fo).sum()),
                       flow_elem_worst_vs_optimum=elem(F, Fo))
    out["oracle_seconds"] = time.perf_counter() - t0
    return out


def pct(a, q):
    return float(np.percentile(np.asarray(a), q)) if len(a) else None


def ms(x):
    return None if x is None else 1e3 * x


def plain_continuation(args, x):
    """The same epsilon stages for the one-at-a-time arm as the batch runs (eps halved per stage)."""
    if args.batch_eps_factor <= 1.0:
        return {}
    k = max(1, int(round(np.log2(args.batch_eps_factor))))
    return {"eps_start": float(2 ** k) * x.eps, "eps_stages": k}


def bench_batch(args, ots, torch, local, insts, gen_s):
    """Batched workload: args.batch uneven instances (n ~ U{50..2000} random geometric graphs of
    mean degree 6, T ~ U{10..80}, L ~ U{1..128}, capacities U[0.2,1] * mass / 8, eps = 0.01)
    solved to marginal error <= tol (a) in one batch (persistent tick kernel, captured graphs,
    autotuned thread mapping) and (b) one instance at a time with ots_sinkhorn_solve (the
    plain single-instance GPU solver, convergence tested after every pass).  Both arms start
    from host arrays and end with the flows on the host."""
    need = 0
    for x in insts:
        g = 1
        while 4 * g < x.L:
            g <<= 1
        Lp = 4 * g
        need += (x.T - 1) * x.n_nodes * Lp * 6 + 3 * x.n_nodes * Lp * 6 + (x.T + 1) * x.n_states * 24 + x.n_states * 64
    free, _ = torch.cuda.mem_get_info(local)
    pool = int(min(max(2 * need, 1 << 30), 0.6 * free))
    b = ots.ots_batch_create(device=local, pool_bytes=pool, max_instances=max(args.batch, 1), ticks_per_launch=32)
    tune_path = os.path.join(tempfile.gettempdir(), f"ots_batch_tune_dev{local}.json")
    t0 = time.perf_counter()
    ots.ots_batch_autotune(b, tune_path)
    tune_s = time.perf_counter() - t0
    mapping = {f"L<={4 << c}": ots.ots_batch_mapping(b, 4 << c) for c in range(7)}
    # warm-up: a few instances through the whole batch path
    for x in insts[:8]:
        ots.ots_batch_add(b, x, tol=args.tol, max_iters=args.batch_max_passes, eps_start=args.batch_eps_factor * x.eps if args.batch_eps_factor > 1 else 0.0)
    ots.ots_batch_run(b)
    for i in list(b.shapes):
        ots.ots_batch_remove(b, i)
    info0 = ots.ots_batch_info(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ids = [ots.ots_batch_add(b, x, tol=args.tol, max_iters=args.batch_max_passes, eps_start=args.batch_eps_factor * x.eps if args.batch_eps_factor > 1 else 0.0)
           for x in insts]
    t_add = time.perf_counter()
    ots.ots_batch_run(b)
    t_run = time.perf_counter()
    flows_b, st_b = [], []
    for i in ids:
        st_b.append(ots.ots_batch_status(b, i))
        flows_b.append(ots.ots_batch_get_flows(b, i) if st_b[-1]["status"] in (0, ots.OTS_ERR_NOT_CONVERGED) else None)
    t_end = time.perf_counter()
    sample = oracle_sample_index(st_b)
    samples = [{"inst": insts[k], "index": k, "flows": flows_b[k], "duals": ots.ots_batch_get_duals(b, ids[k])}
               for k in sample]
    info1 = ots.ots_batch_info(b)
    lat_b = [s["seconds"] for s in st_b]
    ots.ots_batch_destroy(b)

    # plain single-instance solver, one instance at a time
    lat_p, solve_p, flows_p, st_p = [], [], [], []
    launches_p = 0
    for x in insts[:4]:                      # warm-up
        h = ots.ots_create_problem(x, device=local)
        ots.ots_sinkhorn_solve(h, tol=args.tol, max_iters=args.batch_max_passes, check_every=1, raise_on_error=False,
                               **plain_continuation(args, x))
        ots.ots_destroy_problem(h)
    torch.cuda.synchronize()
    tp0 = time.perf_counter()
    for x in insts:
        ta = time.perf_counter()
        h = ots.ots_create_problem(x, device=local)
        tb = time.perf_counter()
        r = ots.ots_sinkhorn_solve(h, tol=args.tol, max_iters=args.batch_max_passes, check_every=1, **plain_continuation(args, x),
                                   raise_on_error=False)
        tc = time.perf_counter()
        F = ots.ots_get_flows(h) if r["status"] in (0, ots.OTS_ERR_NOT_CONVERGED) else None
        launches_p += ots.ots_problem_info(h)["kernels_launched"]
        ots.ots_destroy_problem(h)
        lat_p.append(time.perf_counter() - ta)
        solve_p.append(tc - tb)
        flows_p.append(F)
        st_p.append(r)
    tp1 = time.perf_counter()
    # one at a time, every instance submitted at tp0: latency from submission includes the wait
    lat_p_sub = list(np.cumsum(lat_p))
    # relative flow difference between the arms, on the instances both solved to tol (the autotuned
    # mapping of the batch sums in another order; instances that stop at the pass limit have no
    # fixed point to agree on and are reported apart)
    diffs, diffs_nc = [], []
    for fb, fp, sb, sp in zip(flows_b, flows_p, st_b, st_p):
        if fb is None or fp is None:
            continue
        d = float(np.abs(fb - fp).sum() / np.abs(fp).sum())
        (diffs if sb["status"] == 0 and sp["status"] == 0 else diffs_nc).append(d)
    n = len(insts)
    ok_b = [s["status"] == 0 for s in st_b]
    ok_p = [s["status"] == 0 for s in st_p]
    conv_b, conv_p = sum(ok_b), sum(ok_p)
    # latencies of converged solves only (the metric is solves at marginal error <= tol)
    lat_b_ok = [v for v, ok in zip(lat_b, ok_b) if ok]
    lat_p_sub_ok = [v for v, ok in zip(lat_p_sub, ok_p) if ok]
    lat_p_ok = [v for v, ok in zip(lat_p, ok_p) if ok]
    upd = sum(s["iterations"] * x.n_updates_per_iteration() for s, x in zip(st_b, insts))
    return {
        "workload": f"{n} uneven instances: random geometric graphs n~U{{50..2000}} (mean degree 6), "
                    f"T~U{{10..80}}, L~U{{1..128}}, capacities U[0.2,1]*mass/8, eps=0.01, tol={args.tol}",
        "batched": {"solves_per_s": conv_b / (t_end - t0), "solve_only_per_s": conv_b / (t_run - t_add),
                    "attempts_per_s": n / (t_end - t0), "updates_per_s": upd / (t_run - t_add),
                    "add_s": t_add - t0, "run_s": t_run - t_add, "flows_readback_s": t_end - t_run,
                    "p50_ms": ms(pct(lat_b_ok, 50)), "p99_ms": ms(pct(lat_b_ok, 99)),
                    "all_attempts_p99_ms": ms(pct(lat_b, 99)), "converged": conv_b, "not_converged": n - conv_b,
                    "passes_mean": float(np.mean([s["iterations"] for s in st_b])),
                    "max_src_residual": max(s["src_residual"] for s in st_b),
                    "max_cap_violation": max(s["cap_violation"] for s in st_b),
                    "tick_launches": int(info1["ticks"] - info0["ticks"]),
                    "graph_launches": int(info1["launches"] - info0["launches"]),
                    "mapping": mapping, "autotune_s": tune_s},
        "plain": {"solves_per_s": conv_p / (tp1 - tp0), "solve_only_per_s": conv_p / float(np.sum(solve_p)),
                  "attempts_per_s": n / (tp1 - tp0),
                  "p50_ms": ms(pct(lat_p_sub_ok, 50)), "p99_ms": ms(pct(lat_p_sub_ok, 99)),
                  "per_solve_p50_ms": ms(pct(lat_p_ok, 50)), "per_solve_p99_ms": ms(pct(lat_p_ok, 99)),
                  "converged": conv_p, "not_converged": n - conv_p, "kernel_launches": int(launches_p)},
        "latency_note": "solves_per_s and p50/p99 count converged solves only (marginal error <= tol); "
                        "not_converged instances stopped at the pass limit (their capacities admit no feasible "
                        "flow, or nearly none) and are reported apart; attempts_per_s counts every instance. "
                        "p50/p99 from submission of all instances at once (both arms); per_solve_* = one "
                        "solve timed alone, without the wait for the instances before it",
        "max_rel_flow_diff_batched_vs_plain": max(diffs) if diffs else None,
        "max_rel_flow_diff_not_converged": max(diffs_nc) if diffs_nc else None,
        "generate_s": gen_s,
        "_oracle_samples": samples,
    }


def bench_single(args, ots, torch, local):
    """Single-commodity workloads (L = 1) through the linear-domain path against the log-domain
    path.  (a) The 5x5 grid (25 nodes, T = 10, eps = 0.05): full solves to tol, one problem;
    pass throughput of both paths.  (b) Members with the uneven batch's sizes (n~U{50..2000}
    random geometric graphs, T~U{10..80}, L = 1, eps = 0.01, capacities U[0.2,1]*mass/2), from host
    arrays to flows on the host: every member in one linear-domain launch (one thread block each),
    the batched log-domain solver, and the plain one-at-a-time log-domain solver."""
    from paper_2106_14485_gb300 import instances as I
    out = {}
    g = I.grid_single_commodity(0)
    h = ots.ots_create_problem(g, device=local)
    upd = g.n_updates_per_iteration()
    ots.ots_sinkhorn_solve(h, tol=args.tol, max_iters=100000)
    ots.ots_linear_solve(h, tol=args.tol, max_iters=100000)
    reps = args.single_reps

    def timed(f):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rs = [f() for _ in range(reps)]
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps, rs[-1]

    t_log, r_log = timed(lambda: ots.ots_sinkhorn_solve(h, tol=args.tol, max_iters=100000))
    t_lin, r_lin = timed(lambda: ots.ots_linear_solve(h, tol=args.tol, max_iters=100000))
    n_it = 2000
    t_plog, _ = timed(lambda: ots.ots_iterate(h, n_it, reset=True))
    t_plin, r_plin = timed(lambda: ots.ots_linear_iterate(h, n_it, reset=True))
    lin_duals = ots.ots_get_duals(h)
    lin_flows = ots.ots_get_flows(h)
    ots.ots_linear_solve(h, tol=args.tol, max_iters=100000)
    item = {"inst": g, "duals": ots.ots_get_duals(h), "flows": ots.ots_get_flows(h)}
    ots.ots_destroy_problem(h)
    out["grid5x5"] = {
        "workload": "5x5 grid, L=1, T=10, eps=0.05, move cost 1, wait cost 0.1, Dirichlet(1) marginals over 3 nodes",
        "linear": {"solves_per_s": 1.0 / t_lin, "ms_per_solve": 1e3 * t_lin, "passes": r_lin["iterations"],
                   "linear_stats": r_lin["linear"], "pass_updates_per_s": n_it * upd / t_plin,
                   "us_per_pass": 1e6 * t_plin / n_it},
        "log_domain": {"solves_per_s": 1.0 / t_log, "ms_per_solve": 1e3 * t_log, "passes": r_log["iterations"],
                       "pass_updates_per_s": n_it * upd / t_plog, "us_per_pass": 1e6 * t_plog / n_it},
        "speedup_solves": t_log / t_lin, "speedup_passes": t_plog / t_plin}
    out["_oracle_items"] = [dict(item, name="grid5x5")]
    del lin_duals, lin_flows

    # (b) many single-commodity members
    tg = time.perf_counter()
    members = I.uneven_single_batch(0, count=args.single_batch, workers=min(16, os.cpu_count() or 1))
    gen_s = time.perf_counter() - tg
    n = len(members)
    mp = args.batch_max_passes
    for x in members[:2]:                           # warm-up of every arm
        hx = ots.ots_create_problem(x, device=local)
        ots.ots_linear_solve(hx, tol=args.tol, max_iters=mp, raise_on_error=False)
        ots.ots_sinkhorn_solve(hx, tol=args.tol, max_iters=mp, check_every=1, raise_on_error=False)
        ots.ots_destroy_problem(hx)
    # linear-domain, one launch for all members
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs = [ots.ots_create_problem(x, device=local) for x in members]
    t1 = time.perf_counter()
    reps_l, st_l = ots.ots_linear_solve_many(hs, tol=args.tol, max_iters=mp, raise_on_error=False)
    t2 = time.perf_counter()
    flows_l = [ots.ots_get_flows(hx) for hx in hs]
    t3 = time.perf_counter()
    ok_l = [r["status"] == 0 for r in reps_l]
    samp = [k for k in oracle_sample_index(reps_l)][:4]
    out["_oracle_items"] += [{"inst": members[k], "duals": ots.ots_get_duals(hs[k]), "flows": flows_l[k],
                              "name": members[k].name} for k in samp]
    upd_l = sum(r["iterations"] * x.n_updates_per_iteration() for r, x in zip(reps_l, members))
    for hx in hs:
        ots.ots_destroy_problem(hx)
    # batched log-domain solver
    need = sum((x.T + 2) * x.n_nodes * 4 * 6 + (x.T + 1) * x.n_states * 24 + x.n_states * 64 for x in members)
    free, _ = torch.cuda.mem_get_info(local)
    b = ots.ots_batch_create(device=local, pool_bytes=int(min(max(2 * need, 1 << 30), 0.6 * free)),
                             max_instances=n, ticks_per_launch=32)
    torch.cuda.synchronize()
    tb0 = time.perf_counter()
    ids = [ots.ots_batch_add(b, x, tol=args.tol, max_iters=mp) for x in members]
    ots.ots_batch_run(b)
    st_b = [ots.ots_batch_status(b, i) for i in ids]
    flows_b = [ots.ots_batch_get_flows(b, i) for i in ids]
    tb1 = time.perf_counter()
    ots.ots_batch_destroy(b)
    ok_b = [r["status"] == 0 for r in st_b]
    # plain one at a time
    torch.cuda.synchronize()
    tp0 = time.perf_counter()
    st_p, flows_p = [], []
    for x in members:
        hx = ots.ots_create_problem(x, device=local)
        st_p.append(ots.ots_sinkhorn_solve(hx, tol=args.tol, max_iters=mp, check_every=1, raise_on_error=False))
        flows_p.append(ots.ots_get_flows(hx))
        ots.ots_destroy_problem(hx)
    tp1 = time.perf_counter()
    ok_p = [r["status"] == 0 for r in st_p]
    diffs = [float(np.abs(a - c).sum() / np.abs(c).sum()) for a, c, u, v in zip(flows_l, flows_p, ok_l, ok_p) if u and v]
    upd_b = sum(r["iterations"] * x.n_updates_per_iteration() for r, x in zip(st_b, members))
    upd_p = sum(r["iterations"] * x.n_updates_per_iteration() for r, x in zip(st_p, members))
    # the largest member that every arm solved, alone: linear-domain (a cluster of blocks) against the
    # log-domain solver, from host arrays to flows on the host
    both = [k for k in range(n) if ok_l[k] and ok_p[k]]
    alone = None
    if both:
        k = max(both, key=lambda q: members[q].n_states * members[q].T)
        x = members[k]
        times = {}
        for arm in ("linear", "log_domain"):
            for rep in range(2):                       # the first is a warm-up
                torch.cuda.synchronize()
                ta = time.perf_counter()
                hx = ots.ots_create_problem(x, device=local)
                if arm == "linear":
                    rr = ots.ots_linear_solve(hx, tol=args.tol, max_iters=mp, raise_on_error=False)
                else:
                    rr = ots.ots_sinkhorn_solve(hx, tol=args.tol, max_iters=mp, check_every=1, raise_on_error=False)
                ots.ots_get_flows(hx)
                ots.ots_destroy_problem(hx)
                times[arm] = (time.perf_counter() - ta, rr["iterations"], rr["status"])
        alone = {"member": x.name, "states": x.n_states, "T": x.T,
                 **{arm: {"seconds": t, "passes": it, "status": stt,
                          "updates_per_s": it * x.n_updates_per_iteration() / t} for arm, (t, it, stt) in times.items()}}
    out["uneven_single"] = {
        "workload": f"{n} members: random geometric graphs n~U{{50..2000}} (mean degree 6, bridged), T~U{{10..80}}, "
                    f"L=1, capacities U[0.2,1]*mass/2, eps=0.01, tol={args.tol}, pass limit {mp}",
        "linear_many": {"solves_per_s": sum(ok_l) / (t3 - t0), "converged": sum(ok_l), "create_s": t1 - t0,
                        "solve_s": t2 - t1, "flows_s": t3 - t2, "updates_per_s": upd_l / (t3 - t0),
                        "solve_only_updates_per_s": upd_l / (t2 - t1),
                        "linear_stats": st_l, "passes_mean": float(np.mean([r["iterations"] for r in reps_l]))},
        "batched_log": {"solves_per_s": sum(ok_b) / (tb1 - tb0), "converged": sum(ok_b), "seconds": tb1 - tb0,
                        "updates_per_s": upd_b / (tb1 - tb0)},
        "plain_log": {"solves_per_s": sum(ok_p) / (tp1 - tp0), "converged": sum(ok_p), "seconds": tp1 - tp0,
                      "updates_per_s": upd_p / (tp1 - tp0)},
        "largest_member_alone": alone,
        "max_rel_flow_diff_linear_vs_plain": max(diffs) if diffs else None,
        "generate_s": gen_s,
        "note": "solves_per_s and updates_per_s (passes run x 2(T-1) nnz(K) L) over the whole call sequence "
                "(create from host arrays, solve, flows to host; solves count converged members, marginal error "
                "<= tol); the linear arm confirms each member with log-domain passes at tol"}
    return out


def bench_serve(args, ots, torch, local, small, large):
    """Serving workload: Poisson arrivals at each rate of a request mix drawn from the batched
    workload's instances (95%) and traffic-scale instances (5%, pass limit
    --serve-large-passes), each request solved to marginal error <= tol from host arrays to
    flows on the host.  Served (a) by the continuous-batching server and (b) by the same server
    in plain mode (one request at a time, single-instance solver).  Latency = submit -> result,
    queueing included.  solves_per_s, p50_ms and p99_ms count the requests solved to tol; requests
    that finished without reaching it (pass limit; capacities with no feasible flow) are counted
    as failed, and requests still open after the window plus the drain time as open ("censored":
    their latencies are unknown).  all_* percentiles take every request, the open ones at their
    age at the deadline (a lower bound)."""
    rates = [float(r) for r in args.serve_rates.split(",") if r.strip()]
    out = {"workload": f"Poisson arrivals; 95% drawn from the {len(small)} batched-workload instances, 5% "
                       f"traffic-scale grid (n={large.n_nodes}, L={large.L}, T={large.T}, eps={large.eps}, "
                       f"epsilon continuation from {8 * large.eps:g} in 3 stages, <= {args.serve_large_passes} "
                       f"passes); tol={args.tol}",
           "window_s": args.serve_seconds, "drain_s": args.serve_drain, "rates": []}
    for rate in rates:
        rng = np.random.default_rng(int(rate))
        n_req = max(1, int(rng.poisson(rate * args.serve_seconds)))
        arrivals = np.sort(rng.uniform(0.0, args.serve_seconds, n_req))
        kinds = rng.random(n_req) < 0.05
        picks = rng.integers(0, len(small), n_req)
        row = {"rate": rate, "requests": n_req, "large_requests": int(kinds.sum())}
        for mode, name in ((0, "batched"), (1, "plain")):
            srv = ots.ots_server_create(device=local, pool_bytes=int(0.5 * torch.cuda.mem_get_info(local)[0]),
                                        max_instances=256, ticks_per_launch=8, builder_threads=4, mode=mode)
            tickets = []
            t0 = time.perf_counter()
            for k in range(n_req):
                now = time.perf_counter() - t0
                if arrivals[k] > now:
                    time.sleep(arrivals[k] - now)
                if kinds[k]:
                    tk = ots.ots_server_submit(srv, large, tol=args.tol, max_iters=args.serve_large_passes,
                                               check_every=10, eps_start=8 * large.eps, eps_stages=3)
                else:
                    tk = ots.ots_server_submit(srv, small[picks[k]], tol=args.tol, max_iters=args.batch_max_passes,
                                               eps_start=args.batch_eps_factor * small[picks[k]].eps if args.batch_eps_factor > 1 else 0.0)
                tickets.append((tk, bool(kinds[k])))
            deadline = t0 + args.serve_seconds + args.serve_drain
            for tk, _ in tickets:
                left = (deadline - time.perf_counter()) * 1e3
                if left <= 0:
                    break
                ots.ots_server_wait(srv, tk, left)
            t_end = time.perf_counter()
            lat = {False: [], True: []}        # solved requests (marginal error <= tol)
            lat_all = {False: [], True: []}    # every request; open ones at their age at the deadline (lower bound)
            solved = {False: 0, True: 0}
            failed = {False: 0, True: 0}       # finished without reaching tol (pass limit, infeasible)
            open_ = {False: 0, True: 0}
            for k, (tk, big) in enumerate(tickets):
                r = ots.ots_server_poll(srv, tk)
                if r["status"] == ots.OTS_PENDING:
                    open_[big] += 1
                    lat_all[big].append((t_end - t0 - arrivals[k]) * 1e3)
                    continue
                ms = ots.ots_server_timing(srv, tk)["total_ms"]
                lat_all[big].append(ms)
                if r["status"] == 0:
                    lat[big].append(ms)
                    solved[big] += 1
                else:
                    failed[big] += 1
            info = ots.ots_server_info(srv)
            ots.ots_server_destroy(srv)
            span = t_end - t0
            row[name] = {"solves_per_s": (solved[False] + solved[True]) / span,
                         "small": {"p50_ms": pct(lat[False], 50), "p99_ms": pct(lat[False], 99),
                                   "all_p50_ms": pct(lat_all[False], 50), "all_p99_ms": pct(lat_all[False], 99),
                                   "solved": solved[False], "failed": failed[False], "open": open_[False]},
                         "large": {"p50_ms": pct(lat[True], 50), "p99_ms": pct(lat[True], 99),
                                   "all_p50_ms": pct(lat_all[True], 50), "all_p99_ms": pct(lat_all[True], 99),
                                   "solved": solved[True], "failed": failed[True], "open": open_[True]},
                         "p50_ms": pct(lat[False] + lat[True], 50), "p99_ms": pct(lat[False] + lat[True], 99),
                         "all_p99_ms": pct(lat_all[False] + lat_all[True], 99),
                         "censored": bool(open_[False] + open_[True]),
                         "span_s": span, "batch_launches": int(info["batch_launches"])}
        out["rates"].append(row)
    return out


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2106_14485_gb300 import build, ots
    build.build()
    ots.load_library()

    inst = workload(rank, args.horizon)
    upd_per_pass = inst.n_updates_per_iteration()
    h = ots.ots_create_problem(inst, device=local)
    info = ots.ots_problem_info(h)
    stream = torch.cuda.ExternalStream(ots.ots_problem_stream(h), device=local)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    ots.ots_iterate(h, args.warmup, reset=True)
    barrier()
    launches0 = ots.ots_problem_info(h)["kernels_launched"]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        r = ots.ots_iterate(h, args.steps, reset=False)
        ev1.record(stream)
        ev1.synchronize()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = ots.ots_problem_info(h)["kernels_launched"] - launches0
    tm = ots.ots_last_pass_timing(h)
    fwd_ms = [tm["forward_ms"] / (inst.T - 2)]
    bwd_ms = [tm["backward_ms"] / (inst.T - 2)]
    final = r
    barrier()
    checks = {"timed_passes": traffic_commodity_sample(ots, h, inst)} if rank == 0 else {}

    updates = args.steps * upd_per_pass
    elapsed_ms, updates_all = combine_ranks(pg, elapsed_ms, float(updates), "cuda")
    value = updates_all / (elapsed_ms / 1e3)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        ots.ots_destroy_problem(h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h_e = ots.ots_create_problem(inst, device=local)
        ots.ots_iterate(h_e, args.steps, reset=True)
        F = ots.ots_get_flows(h_e)
        st = ots.ots_problem_info(h_e)
        ots.ots_destroy_problem(h_e)
        t_e = time.perf_counter() - t0
        assert F.shape[0] == inst.T
        t_all, u_all = combine_ranks(pg, t_e, float(args.steps * upd_per_pass), "cuda")
        e2e_val = u_all / t_all
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(st["h2d_bytes"]) // args.steps,
               "d2h_bytes_per_step": int(st["d2h_bytes"]) // args.steps,
               "note": f"one call sequence of {args.steps} passes: create from host arrays, passes, flows to host, destroy"}

    # ---- one full solve of the traffic-scale workload to tol, with epsilon continuation ----
    traffic = None
    if not args.no_traffic_solve:
        h_t = ots.ots_create_problem(inst, device=local)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rt = ots.ots_sinkhorn_solve(h_t, tol=args.tol, max_iters=20000, eps_start=8 * inst.eps, eps_stages=3,
                                    raise_on_error=False)
        torch.cuda.synchronize()
        t_t = time.perf_counter() - t0
        if rank == 0:
            checks["traffic_solve"] = traffic_commodity_sample(ots, h_t, inst)
        ots.ots_destroy_problem(h_t)
        traffic = {"workload": workload_config(inst, args.tol)["workload"],
                   "continuation": f"eps {8 * inst.eps:g} -> {inst.eps:g} in 3 warm-start stages (stage tol 1e-4)",
                   "status": rt["status"], "passes": rt["iterations"], "seconds": t_t,
                   "solves_per_s": 1.0 / t_t if rt["status"] == 0 else 0.0,
                   "final_src_residual": rt["src_residual"], "final_cap_violation": rt["cap_violation"]}

    # ---- full solves to marginal error <= tol on the random-geometric workload ----
    solves = None
    if args.solves > 0:
        from paper_2106_14485_gb300 import instances
        rg = instances.rgg400(rank)
        hs = ots.ots_create_problem(rg, device=local)
        for _ in range(3):
            ots.ots_sinkhorn_solve(hs, tol=args.tol)
        lat = []
        passes_s = 0
        for _ in range(args.solves):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rs = ots.ots_sinkhorn_solve(hs, tol=args.tol, check_every=2)
            lat.append(time.perf_counter() - t0)
            passes_s += rs["iterations"]
        checks["rgg400"] = {"inst": rg, "duals": ots.ots_get_duals(hs), "flows": ots.ots_get_flows(hs)}
        ots.ots_destroy_problem(hs)
        lat = np.array(lat)
        solves = {"workload": f"random geometric graph n={rg.n_nodes}, L={rg.L}, T={rg.T}, eps={rg.eps}, "
                              f"capacities U[0.2,1]*mass/8",
                  "value": float(len(lat) / lat.sum()), "unit": "solves/s",
                  "updates_per_s": float(passes_s * rg.n_updates_per_iteration() / lat.sum()),
                  "passes_per_solve": passes_s / len(lat), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                  "p99_ms": float(np.percentile(lat, 99) * 1e3), "final_src_residual": rs["src_residual"],
                  "final_cap_violation": rs["cap_violation"]}

    batch = serve = None
    if args.batch > 0 or args.serve_rates.strip():
        from paper_2106_14485_gb300 import instances as _inst
        tg = time.perf_counter()
        c4 = _inst.uneven_rgg_batch(0, count=max(args.batch, 64), workers=min(16, os.cpu_count() or 1))
        gen_s = time.perf_counter() - tg
        if args.batch > 0:
            batch = bench_batch(args, ots, torch, local, c4[:args.batch], gen_s)
        if args.serve_rates.strip():
            serve = bench_serve(args, ots, torch, local, c4, inst)

    single = None
    if args.single_batch > 0:
        single = bench_single(args, ots, torch, local)

    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return 0

    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    fwd_launch_ms = float(np.mean(fwd_ms))
    fb = forward_bytes_per_launch(info, inst)
    achieved = fb / (fwd_launch_ms * 1e-3) / 1e9
    bb = backward_bytes_per_launch(info, inst)
    bwd_launch_ms = float(np.mean(bwd_ms))
    # the state-level bytes of one forward step (read hatPsi_t and Psi_t, write hatPsi_{t+1}, FP32 per
    # state and commodity: 12 S L): what the step moves without the node-level factorisation
    sl_bytes = 12 * info["n_states"] * inst.L
    roof = {"kernel": "k_forward (fused capacity update + node-level LSE message step)",
            "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "peak_source": peak_src, "traffic": measured_traffic(args.horizon), "bytes_per_launch": fb,
            "launch_ms": fwd_launch_ms,
            "state_level_equivalent": {
                "bytes_per_launch": sl_bytes, "achieved": sl_bytes / (fwd_launch_ms * 1e-3) / 1e9,
                "frac": sl_bytes / (fwd_launch_ms * 1e-3) / 1e9 / hbm,
                "note": "12 bytes per state and commodity per forward step, as the state-level step counts them; the "
                        "node-level factorisation moves bytes_per_launch instead, so frac above (own bytes) is the "
                        "kernel's roofline and this one the step's rate in the state-level method's bytes"},
            "backward": {"kernel": "k_backward", "achieved": bb / (bwd_launch_ms * 1e-3) / 1e9,
                         "frac": bb / (bwd_launch_ms * 1e-3) / 1e9 / hbm, "bytes_per_launch": bb,
                         "launch_ms": bwd_launch_ms}}
    cpu = None
    oracle_error = None
    samples = batch.pop("_oracle_samples", []) if batch else []
    single_items = single.pop("_oracle_items", []) if single else []
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(inst, args.cpu_seconds)
        # oracle leg: the FP64 oracle evaluated at the GPU's results (duals and flows)
        oracle_error = {"timed_passes": oracle_check(checks["timed_passes"])}
        if traffic is not None:
            traffic["oracle_error"] = oracle_error["traffic_solve"] = oracle_check(checks["traffic_solve"])
        if solves is not None:
            solves["oracle_error"] = oracle_error["rgg400_solves"] = oracle_check(checks["rgg400"], optimum_tol=1e-11)
        if samples:
            errs = [dict(oracle_check(x), index=x["index"], name=x["inst"].name) for x in samples]
            batch["oracle_error"] = oracle_error["batch_sample"] = {
                "instances": len(errs), "max_flow_rel_l1": max(e["flow_rel_l1"] for e in errs),
                "max_flow_elem_worst": max(e["flow_elem_worst"] for e in errs),
                "max_oracle_src_mismatch": max(e["oracle_src_mismatch"] for e in errs),
                "max_oracle_cap_excess": max(e["oracle_cap_excess"] for e in errs), "per_instance": errs}
        if single is not None:
            errs = [dict(oracle_check(x), name=x["name"]) for x in single_items]
            single["oracle_error"] = oracle_error["single_commodity"] = errs
        oracle_error["note"] = ("FP64 oracle at the GPU's duals: flow error of the GPU (relative L1; worst entry as "
                                "|F-F*| / (1e-5 F* + 1e-9 max F*), <= 1 passes) and the marginal violation the oracle "
                                "measures there; traffic workload on sampled commodities")
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32",
            "number_format": "log2 messages as an fp32 part on a power-of-two grid plus a 16-bit integer "
                             "remainder (float-float arithmetic in f32); f64 convergence sums, boundary updates "
                             "and flows",
            "data": "synthetic", "config": workload_config(inst, args.tol),
            "solves_per_s": solves, "traffic_solve": traffic, "batch": batch, "serving": serve,
            "single_commodity": single,
            "passes_timed": args.steps, "src_residual_after": final["src_residual"],
            "cap_violation_after": final["cap_violation"],
            "roofline": roof, "cpu_baseline": cpu, "oracle_error": oracle_error, "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def profile_batch(args):
    import torch
    from paper_2106_14485_gb300 import build, instances, ots
    build.build()
    ots.load_library()
    insts = instances.uneven_rgg_batch(0, count=args.profile_batch, workers=min(16, os.cpu_count() or 1))
    b = ots.ots_batch_create(pool_bytes=6 << 30, max_instances=args.profile_batch, ticks_per_launch=32)
    for x in insts:
        ots.ots_batch_add(b, x, tol=args.tol, max_iters=args.batch_max_passes, eps_start=args.batch_eps_factor * x.eps if args.batch_eps_factor > 1 else 0.0)
    ots.ots_batch_run(b, 3)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "batch", "instances": len(insts), "info": ots.ots_batch_info(b)}), flush=True)
    ots.ots_batch_destroy(b)
    return 0


def profile_rgg(args):
    import torch
    from paper_2106_14485_gb300 import build, instances, ots
    build.build()
    ots.load_library()
    rg = instances.rgg400(0)
    h = ots.ots_create_problem(rg)
    for _ in range(3):
        ots.ots_sinkhorn_solve(h, tol=args.tol)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    lat, passes = [], 0
    for _ in range(args.profile_rgg):
        t0 = time.perf_counter()
        r = ots.ots_sinkhorn_solve(h, tol=args.tol, check_every=2)
        lat.append(time.perf_counter() - t0)
        passes += r["iterations"]
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile": "rgg400", "solves": len(lat), "passes": passes, "solve_ms": [x * 1e3 for x in lat],
                      "pass_timing_ms": ots.ots_last_pass_timing(h)}), flush=True)
    ots.ots_destroy_problem(h)
    return 0


def profile_linear(args):
    """Three launches of the linear-domain kernel for an ncu capture: the 5x5 grid (every array in
    shared memory) for args.profile_linear passes, a 400-node single-commodity random geometric
    graph (T = 50, arrays in L2, one block) for 20 passes, and a 2000-node one (T = 80, an 8-block
    cluster) for 10 passes."""
    import torch
    from paper_2106_14485_gb300 import build, instances, ots
    build.build()
    ots.load_library()
    out = {"profile": "linear"}
    g = instances.grid_single_commodity(0)
    h = ots.ots_create_problem(g)
    out["grid5x5"] = ots.ots_linear_iterate(h, args.profile_linear, reset=True)
    ots.ots_destroy_problem(h)
    r = instances.rgg_instance(seed=3, n=400, L=1, T=50, eps=0.01, cap_div=2.0, connect="bridge")
    h = ots.ots_create_problem(r)
    out["rgg400_L1"] = ots.ots_linear_iterate(h, 20, reset=True)
    ots.ots_destroy_problem(h)
    r = instances.rgg_instance(seed=3, n=2000, L=1, T=80, eps=0.01, cap_div=2.0, connect="bridge")
    h = ots.ots_create_problem(r)
    out["rgg2000_L1"] = ots.ots_linear_iterate(h, 10, reset=True)
    ots.ots_destroy_problem(h)
    torch.cuda.synchronize()
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.profile_batch > 0:
        return profile_batch(args)
    if args.profile_linear > 0:
        return profile_linear(args)
    if args.profile_rgg > 0:
        return profile_rgg(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
