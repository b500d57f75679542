#!/usr/bin/env python
"""Benchmark of the GPU EMT network solve (bus-steps per second).

Default workload: the 11,456-bus network (64 seeded 179-bus tiles, 4-level
hierarchy, 16 leaves of 716 buses), dt = 50 us, 512 scenarios (source and load
amplitudes scaled by 1 + N(0, 5%) per column), 1,000 time steps. One bench
"step" is the whole run: every time step updates all branch histories, injects
the sources, applies the hierarchical inverse to the 512 right-hand sides
(split-BF16 tensor-core products with FP32 accumulation) and refines once
against the float-float residual r = i - G v. Accuracy is measured against the
CPU oracle (FP64, exact hierarchical store) on 8 columns over all 1,000 steps.
The same JSON line carries, as secondary keys, the single 1,432-bus simulation
(20,000 steps with a line trip; FF64, FP32 + refinement and FP64 variants) and
the single-vector apply on the 11,456-bus store (the HBM-bound form).

--config picks one workload alone (1: 179 buses; 2: 1,432 buses; 3: N-1
screening; 4: scenarios; 5: serving; 6: d_th sweep; 7: three phases; 41: the
single apply). --gpus N splits the columns (3, 4) or the request stream (5)
over N ranks, one per GPU; without an outside launcher it starts the ranks
itself under torch.distributed.run.

  python bench.py [--gpus N --steps K --warmup W] [--config C] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DT = 50e-6
N_MON = 16
ERR_TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--time-steps", type=int, default=0,
                    help="time steps per bench step (default: the workload's own; smaller values are for "
                         "profiling captures, not bench lines)")
    ap.add_argument("--variants", default="ff64,fp32,fp64")
    ap.add_argument("--config", type=int, default=0, choices=[0, 1, 2, 3, 4, 5, 6, 7, 41],
                    help="0 (default): config 4 with configs 2 and 41 as secondary keys of the same line; "
                         "1: single 179-bus simulation; 2: single 1,432-bus simulation; 3: N-1 screening, 256 "
                         "contingencies; 4: 11,456-bus network, 512 scenarios; 5: serving, Poisson stream of "
                         "2,000 requests; 6: PAPER-mode d_th sweep (approximation error, build and modification "
                         "cost); 7: three-phase 1,432-bus network (4,296 nodes): apply, line trip vs rebuild; "
                         "41: single apply on the 11,456-bus store")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--profile", type=int, default=0,
                    help="for profiler captures: run only the stepping of configs 3/4 (this many time steps) or this "
                         "many applies of config 41, with no oracle, no e2e and no JSON line")
    ap.add_argument("--apply-kernels", type=int, default=0, help="config 41 with --profile: emt_apply_tune kernels")
    ap.add_argument("--columns", type=int, default=0, help="configs 3/4 with --profile: columns (default: all)")
    ap.add_argument("--tune", default="", help="rows_per_cta,kernels: fixed launch shape instead of the autotuner "
                                               "(with kernels 4, rows_per_cta is the cluster size)")
    ap.add_argument("--cpu-worker", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-col", type=int, default=-1, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-steps", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(rank: int = 0, cfg: int = 2):
    import numpy as np
    import netgen
    net = netgen.tile(1_000_000) if cfg == 1 else netgen.tiled(2, 4)
    trip = netgen.pick_branch(net, seed=7 + rank)
    mon = np.sort(np.random.default_rng(17).choice(net["n_bus"], N_MON, replace=False))
    return net, trip, mon


# ---------------------------------------------------------------- CPU oracle (test infrastructure)
def multi_workload(cfg: int, world: int = 1, rank: int = 0) -> dict:
    """Configs 3 and 4: network, monitored buses, steps, levels, and this rank's block [c0, c1) of
    the R columns with its trips (keyed by local column) and source/load scales (rows of the block)."""
    import numpy as np
    import netgen
    if cfg == 3:
        net = netgen.tiled(2, 4)
        R, steps, levels = 256, 5000, 3
        br = netgen.pick_branches(net, R, seed=11)
        trips = {c: (1000, int(br[c])) for c in range(R)}
        ss = ls = None
    else:
        net = netgen.config_network(4)
        R, steps, levels = 512, 1000, 4
        trips = {}
        ss, ls = netgen.scenario_scales(net, R, seed=13)
    mon = np.sort(np.random.default_rng(17).choice(net["n_bus"], N_MON, replace=False))
    c0, c1 = rank_columns(R, world, rank)
    return dict(net=net, mon=mon, R=R, steps=steps, levels=levels, c0=c0, c1=c1,
                trips={c - c0: trips[c] for c in range(c0, c1) if c in trips},
                ss=None if ss is None else np.ascontiguousarray(ss[c0:c1]),
                ls=None if ls is None else np.ascontiguousarray(ls[c0:c1]),
                global_trips=trips, global_ss=ss, global_ls=ls)


def rank_columns(R: int, world: int, rank: int):
    """Contiguous block [c0, c1) of the R columns that rank `rank` of `world` steps; the blocks of
    all ranks cover every column exactly once."""
    return R * rank // world, R * (rank + 1) // world


def rank_share(items, world: int, rank: int):
    """Round-robin share of a request stream: the (global index, item) pairs rank `rank` serves."""
    return [(i, x) for i, x in enumerate(items) if i % world == rank]


def accuracy_columns(n_cols: int):
    """Local columns the oracle checks: first, last, both sides of the 192-column tensor-core tile
    edge, the middle and the ragged last tile (8 distinct columns when there are that many)."""
    want = [0, 1, 191, 192, n_cols // 2, n_cols - 65, n_cols - 2, n_cols - 1]
    return sorted({c for c in want if 0 <= c < n_cols})


def cpu_worker(out_prefix: str, n_steps: int, cfg: int = 2, col: int = -1):
    """Run the oracle on the workload single-threaded; write the monitored
    trajectory and the wall time."""
    import numpy as np
    from oracle import emt as oemt
    t0 = time.perf_counter()
    if cfg in (1, 2):
        net, trip, mon = workload(0, cfg)
        nw = oemt.Network(net, DT, levels=2 if cfg == 1 else 3)
        half = n_steps // 2
        traj, _ = oemt.simulate(nw, n_steps, [(half, oemt.TRIP, trip, 0.0)], solver="exact", monitor=mon)
    else:
        w = multi_workload(cfg)
        trips, ss, ls = w["global_trips"], w["global_ss"], w["global_ls"]
        nw = oemt.Network(w["net"], DT, levels=w["levels"])
        ev = [(trips[col][0], oemt.TRIP, trips[col][1], 0.0)] if col in trips else []
        traj, _ = oemt.simulate(nw, n_steps, ev, solver="exact", monitor=w["mon"],
                                src_scale=None if ss is None else ss[col], load_scale=None if ls is None else ls[col])
    t1 = time.perf_counter()
    np.save(out_prefix + ".npy", traj)
    json.dump({"seconds": t1 - t0, "steps": n_steps}, open(out_prefix + ".json", "w"))


def run_cpu_oracle(n_steps: int, cfg: int = 2, col: int = -1):
    trajs, secs = run_cpu_oracle_columns(n_steps, cfg, [col])
    return trajs[0], secs[0]


def run_cpu_oracle_columns(n_steps: int, cfg: int, cols):
    """The oracle on several columns, each in its own single-threaded process, at most one process
    per host core at a time; returns the trajectories and each process's own wall seconds."""
    import numpy as np
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cols = list(cols)
    par = max(1, min(len(cols), os.cpu_count() or 1))
    trajs, secs = [None] * len(cols), [0.0] * len(cols)
    with tempfile.TemporaryDirectory() as td:
        for k0 in range(0, len(cols), par):
            procs = []
            for k in range(k0, min(len(cols), k0 + par)):
                pre = os.path.join(td, f"oracle{k}")
                procs.append((k, pre, subprocess.Popen(
                    [sys.executable, os.path.abspath(__file__), "--cpu-worker", pre, "--cpu-steps", str(n_steps),
                     "--config", str(cfg), "--cpu-col", str(cols[k])], env=env)))
            for k, pre, p in procs:
                if p.wait() != 0:
                    raise RuntimeError(f"oracle worker for column {cols[k]} failed")
                trajs[k] = np.load(pre + ".npy")
                secs[k] = json.load(open(pre + ".json"))["seconds"]
    return trajs, secs


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is None:
            os.unlink(self.f.name)
            return summarize_clocks([])
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        with open(self.f.name) as fh:
            lines = fh.readlines()
        os.unlink(self.f.name)
        return summarize_clocks(lines)


def summarize_clocks(lines) -> dict:
    """Median SM clock, maximum SM clock and the throttle reasons seen, from the CSV rows (no header,
    no units) of `nvidia-smi --query-gpu=<Clocks.Q>`; rows that do not parse are skipped."""
    import numpy as np
    out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return out
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = set()
    for r in rows:
        for k, name in enumerate(names):
            if r[5 + k].lower().startswith("active"):
                reasons.add(name)
    out["sm_mhz"] = float(np.median(sm)) if sm else None
    out["sm_max_mhz"] = max(mx) if mx else None
    out["reasons"] = sorted(reasons)
    out["samples"] = len(rows)
    return out


def job_ms(ms: float, world: int, device=None) -> float:
    """Whole-job time of one timed step: the maximum over ranks of each rank's own time."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units processed by all ranks per second (independent replicas, weak scaling)."""
    return world * units_per_rank / (ms / 1e3)


def job_units(local_units: float, world: int, device=None) -> float:
    """Units processed by all ranks together, each rank counting only the distinct units it ran."""
    import torch
    t = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def launch_ranks(args):
    """`--gpus N` with no launcher around this process: start N ranks, one per GPU, under
    torch.distributed.run and return their exit status. None when this process is a rank already
    (WORLD_SIZE set) or N is 1."""
    if args.gpus <= 1 or "WORLD_SIZE" in os.environ:
        return None
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def rel_err(got, ref):
    import numpy as np
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


# ---------------------------------------------------------------- reference arm (the oracle)
def workload_name(cfg: int) -> str:
    return (("1432-bus network (8 seeded 179-bus tiles), 3-level hierarchy, 20,000 time steps of 50 us, one line "
             "trip at step 10,000, 16 monitored buses") if cfg == 2 else
            ("179-bus tile, 2-level hierarchy (4 leaves), 2,000 time steps of 50 us, one line trip at step 1,000, "
             "16 monitored buses"))


def multi_name(cfg: int) -> str:
    return ("N-1 screening: 256 contingencies on the 1432-bus network, each trips a different branch at step "
            "1000, 5000 steps" if cfg == 3 else
            "11456-bus network (64 tiles), 4-level hierarchy, 512 scenarios (+-5% source/load), 1000 steps")


def reference_arm(args):
    """The oracle as it stands, single-threaded on the host cores, on a bounded sample of the
    workload the native arm runs (same config, metric and unit). Rank 0 only."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import numpy as np
    cfg = 4 if args.config in (0, 4) else args.config
    if cfg in (3, 4):
        from oracle import emt as oemt
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        w = multi_workload(cfg)
        net, R, T = w["net"], w["R"], w["steps"]
        n = net["n_bus"]
        nw = oemt.Network(net, DT, levels=w["levels"])    # partition and network set-up, once
        trips, ss, ls = w["global_trips"], w["global_ss"], w["global_ls"]
        sample = 20 if cfg == 4 else 200                   # time steps of one column per bench step
        times = []
        for i in range(args.warmup + args.steps):
            col = (i * 97) % R
            ev = [(trips[col][0], oemt.TRIP, trips[col][1], 0.0)] if col in trips else []
            t0 = time.perf_counter()
            oemt.simulate(nw, sample, ev, solver="exact", monitor=w["mon"],
                          src_scale=None if ss is None else ss[col], load_scale=None if ls is None else ls[col])
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
        t = float(np.mean(times))
        v = n * sample / t
        desc = (f"{sample} time steps of one column per step (columns 97 i mod {R}), FP64 exact hierarchical store "
                "built once, single thread")
        config = {"workload": multi_name(cfg), "buses": n, "columns": R, "time_steps_per_step": T,
                  "sample_time_steps": sample}
        ms = t * 1e3
    else:
        net, _, _ = workload(0, 2 if cfg not in (1, 2) else cfg)
        sample = 2000
        times = []
        for i in range(args.warmup + args.steps):
            _, sec = run_cpu_oracle(sample, 2 if cfg not in (1, 2) else cfg)
            if i >= args.warmup:
                times.append(sec)
        t = float(np.mean(times))
        v = net["n_bus"] * sample / t
        desc = (f"{sample} time steps of the {net['n_bus']}-bus workload (trip at step {sample // 2}), FP64 exact "
                "hierarchical store, single thread")
        config = {"workload": workload_name(2 if cfg not in (1, 2) else cfg), "time_steps_per_step": 20000,
                  "buses": net["n_bus"], "mode": "exact", "sample_time_steps": sample}
        ms = t * 1e3
    print(json.dumps({
        "impl": "reference", "metric": "bus-steps/sec at rel err <=1e-8 vs FP64 oracle", "value": v,
        "unit": "bus-steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": v, "unit": "bus-steps/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "bus-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- native arm
def ranks():
    """(rank, world size, local rank) of this process; the CUDA device is the local rank's."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    return rank, world, local


def step4_ceilings(n_cta: int, sm_mhz: float, store_bytes_per_step: float, ff_fma_per_step: float) -> dict:
    """On-chip time bounds of one time step of the persistent cluster kernel, whose store lives in
    the shared memory of its n_cta CTAs (one per SM): reading the store once from shared memory at
    128 B per clock per SM, and its float-float FMAs at about 14 per clock per SM (measured at
    full occupancy); in microseconds."""
    hz = sm_mhz * 1e6
    return {"smem_read_us": store_bytes_per_step / (n_cta * 128.0 * hz) * 1e6,
            "ff_fma_us": ff_fma_per_step / (n_cta * 14.0 * hz) * 1e6,
            "smem_peak_gbs": n_cta * 128.0 * hz / 1e9}


def native_arm(args, cfg: int):
    """Configs 1 and 2: one simulation per rank (replicas). Returns the JSON line on rank 0."""
    import numpy as np
    import torch
    import paper_2105_10661_gb300._lib as L

    rank, world, local = ranks()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    T = (args.time_steps or 20000) if cfg == 2 else (args.time_steps or 2000)
    LV = 3 if cfg == 2 else 2
    net, trip, mon = workload(rank, cfg)
    n = net["n_bus"]
    prec = {"ff64": L.EMT_PREC_FF64, "fp32": L.EMT_PREC_FP32, "fp64": L.EMT_PREC_FP64}
    names = [v for v in args.variants.split(",") if v]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # end to end through the C ABI from host buffers, with the launch shape emt_sim_create picks on
    # its own (before this process autotunes anything, so no tuned shape is cached yet)
    e2e = {}
    rec_host = torch.empty(T, N_MON, dtype=torch.float64, pin_memory=True)
    h2d = sum(int(np.asarray(net[k]).nbytes) for k in ("br_a", "br_b", "kind", "R", "L", "C", "shunt_C", "src_bus",
                                                          "src_Vm", "src_phi", "src_Rs"))
    for name in names:
        e2e_times = []
        for i in range(max(1, min(args.steps, 3)) + 1):
            barrier()
            t0 = time.perf_counter()
            s2 = L.emt_sim_create(net, DT, levels=LV, mode=L.EMT_MODE_EXACT, precision=prec[name])
            L.emt_sim_schedule(s2, T // 2, L.EMT_EVENT_TRIP, trip)
            L.emt_sim_monitor(s2, mon)
            rec2 = torch.empty(T, N_MON, dtype=torch.float64, device=dev)
            L.emt_step(s2, T, rec2, stream)
            rec_host.copy_(rec2, non_blocking=True)
            torch.cuda.synchronize()
            del s2
            t1 = time.perf_counter()
            if i > 0:
                e2e_times.append(t1 - t0)
        e2e[name] = job_ms(float(np.mean(e2e_times)) * 1e3, world, dev)

    # oracle trajectory (accuracy reference and CPU baseline), rank 0 only, in a subprocess
    ref = None
    cpu_sec = None
    if rank == 0:
        ref, cpu_sec = run_cpu_oracle(T, cfg)

    results = {}
    clocks = Clocks(local)
    for name in names:
        sim = L.emt_sim_create(net, DT, levels=LV, mode=L.EMT_MODE_EXACT, precision=prec[name])
        L.emt_sim_schedule(sim, T // 2, L.EMT_EVENT_TRIP, trip)
        L.emt_sim_monitor(sim, mon)
        if args.tune:
            rpc, kern = (int(v) for v in args.tune.split(","))
            L.emt_sim_tune(sim, rpc, kern)
            tuned = (rpc, kern)
        else:
            tuned = L.emt_sim_autotune(sim, 512, stream)
        rec = torch.zeros(T, N_MON, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            L.emt_sim_reset(sim, stream)
            L.emt_step(sim, T, rec, stream)
        barrier()
        l0 = L.emt_sim_stats(sim)["launches"]
        times = []
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.emt_sim_reset(sim, stream)
            L.emt_step(sim, T, rec, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        launches = L.emt_sim_stats(sim)["launches"] - l0
        ms = job_ms(float(np.mean(times)), world, dev)
        traj = rec.cpu().numpy()
        err = rel_err(traj, ref) if ref is not None else None
        results[name] = dict(sim=sim, ms=ms, err=err, launches=launches // args.steps,
                             tuned={"rows_per_cta": tuned[0], "kernels": tuned[1]})
    clk = clocks.stop()

    ok = [k for k in names if results[k]["err"] is not None and results[k]["err"] <= ERR_TOL]
    head = min(ok or names, key=lambda k: results[k]["ms"])
    H = results[head]
    sim = H["sim"]
    st = L.emt_sim_stats(sim)
    value = job_rate(n * T, world, H["ms"])

    # roofline of the dominant kernel (timed alone: a graph of back-to-back launches, or one
    # persistent launch running `reps` steps)
    reps = 2000
    kt = {}
    for which in (0, 1):
        L.emt_sim_bench_kernel(sim, which, reps, stream)   # instantiate + warm
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.emt_sim_bench_kernel(sim, which, reps, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        kt[which] = e0.elapsed_time(e1) / reps * 1e3   # us per launch (per time step for generation 4)
    L.emt_sim_reset(sim, stream)
    gen4 = H["tuned"]["kernels"] == 4
    s_bytes = 4 if head == "fp32" else 8
    pld = (-(-n // st["n_leaf"]) + 3) // 4 * 4
    b_partial = st["leaf_elems"] * s_bytes + st["n_incidence"] * 48 + st["n_cta"] * pld * 8
    b_sweep = st["factor_elems"] * s_bytes + st["core_elems"] * s_bytes + n * 8 * 2
    dom = 0 if kt[0] >= kt[1] else 1
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    # per bus-step bytes of the method's own data (store rows and the state a step touches), the
    # HBM-roofline accounting of the measurement plan: s (b + sum over the path of k) + 60 B
    leaf_b = st["leaf_elems"] / max(n, 1)
    path_k = st["factor_elems"] / max(n, 1)
    plan_bytes = (s_bytes * (leaf_b + path_k) + 60.0) * n
    if gen4:
        # the store lives in the shared memory of one cluster: the step is bound on chip (shared-
        # memory reads of the store and float-float FMAs on n_cta SMs) and by the latency of its
        # phase chain, not by HBM
        cs = H["tuned"]["rows_per_cta"]
        byts = b_partial + b_sweep
        ff = st["leaf_elems"] + st["factor_elems"] + st["s_total"] * st["n_cut_rows"]   # leaf, expansion, s = K y_cut
        ceil = step4_ceilings(cs, clk.get("sm_mhz") or 2070.0, byts, ff)
        ach = byts / (kt[0] * 1e-6) / 1e9
        roofline = {"bound": "smem", "kernel": "k_step4", "achieved": ach, "peak": ceil["smem_peak_gbs"],
                    "unit": "GB/s", "frac": ach / ceil["smem_peak_gbs"], "traffic": None,
                    "us_per_step": kt[0], "algorithmic_bytes_per_step": byts, "cluster_ctas": cs,
                    "ceilings_us_per_step": {"smem_read": ceil["smem_read_us"], "ff_fma": ceil["ff_fma_us"]},
                    "hbm_view": {"bytes_per_step": plan_bytes, "achieved_gbs": plan_bytes / (kt[0] * 1e-6) / 1e9,
                                 "frac_of_hbm": plan_bytes / (kt[0] * 1e-6) / 1e9 / peaks["hbm_gbs"]},
                    "peak_source": f"shared-memory read bandwidth of {cs} SMs (128 B/clock each) at the median "
                                   "SM clock sampled in the timed region",
                    "note": "store resident in the shared memory of one thread-block cluster; the per-step chain "
                            "of dependent phases (latency) bounds it, far above both on-chip ceilings"}
    else:
        ach = (b_partial if dom == 0 else b_sweep) / (kt[dom] * 1e-6) / 1e9
        roofline = {"bound": "hbm", "kernel": "k_step_partial" if dom == 0 else "k_step_sweep", "achieved": ach,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None,
                    "us_per_launch": {"k_step_partial": kt[0], "k_step_sweep": kt[1]},
                    "algorithmic_bytes_per_launch": {"k_step_partial": b_partial, "k_step_sweep": b_sweep},
                    "peak_source": "measured" if "when" in peaks else "fallback"}

    if rank != 0:
        return None
    return {
        "metric": "bus-steps/sec at rel err <=1e-8 vs FP64 oracle", "value": value, "unit": "bus-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": H["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": head, "data": "synthetic",
        "config": {"workload": workload_name(cfg),
                   "time_steps_per_step": T, "buses": n, "mode": "exact", "l2": "flushed between timed steps",
                   "parallelism": f"replicas x{world}"},
        "accuracy": {k: results[k]["err"] for k in names},
        "variants_ms_per_step": {k: results[k]["ms"] for k in names},
        "autotuned": {k: results[k]["tuned"] for k in names},
        "variants_bus_steps_per_s": {k: world * n * T / (results[k]["ms"] / 1e3) for k in names},
        "roofline": roofline,
        "cpu_baseline": {"value": n * T / cpu_sec, "unit": "bus-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"full workload ({T} time steps incl. the trip), FP64 exact hierarchical "
                                   "store with explicit recomputation at the trip, single thread"},
        "e2e": {"value": job_rate(n * T, world, e2e[head]), "unit": "bus-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": T * N_MON * 8,
                "variants": {k: job_rate(n * T, world, v) for k, v in e2e.items()},
                "includes": "emt_sim_create from host arrays (partition, GPU build, the launch shape it picks "
                            "itself), emt_step, D2H of the record; measured before any autotuning in this process"},
        "gpu_launches": int(H["launches"]),
        "clocks": clk,
    }


# ---------------------------------------------------------------- configs 3 and 4 (many columns)
def multi_arm(args, cfg: int):
    """Configs 3 and 4: R columns stepped together, split into one contiguous block per rank (no
    collective on the data path). Returns the JSON line on rank 0, None elsewhere."""
    import numpy as np
    import torch
    import paper_2105_10661_gb300._lib as L

    rank, world, local = ranks()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = multi_workload(cfg, world, rank)
    net, mon, R, levels = w["net"], w["mon"], w["R"], w["levels"]
    T = args.time_steps or w["steps"]
    Rl = w["c1"] - w["c0"]
    trips, ss, ls = w["trips"], w["ss"], w["ls"]
    n = net["n_bus"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    tune = [int(x) for x in args.tune.split(",")] if args.tune else None

    def create():
        sm = L.emt_sim_create(net, DT, levels=levels, mode=L.EMT_MODE_EXACT, nrhs=Rl, src_scale=ss, load_scale=ls)
        if tune:
            L.emt_sim_tune(sm, *tune)
        for c, (st_, e) in trips.items():
            L.emt_sim_schedule(sm, st_, L.EMT_EVENT_TRIP, e, 0.0, c)
        L.emt_sim_monitor(sm, mon)
        return sm

    # end to end through the C ABI from host arrays, first, in a process that has timed nothing yet:
    # build, schedule, step, record read back to pinned host memory
    rec = torch.zeros(T, Rl, N_MON, dtype=torch.float64, device=dev)
    rec_host = torch.empty(T, Rl, N_MON, dtype=torch.float64, pin_memory=True)
    h2d = sum(int(np.asarray(net[k]).nbytes) for k in ("br_a", "br_b", "kind", "R", "L", "C", "shunt_C", "src_bus",
                                                          "src_Vm", "src_phi", "src_Rs"))
    h2d += (0 if ss is None else np.asarray(ss).nbytes) + (0 if ls is None else np.asarray(ls).nbytes)
    e2e_times = []
    for i in range(max(1, min(args.steps, 2)) + 1):
        barrier()
        t0 = time.perf_counter()
        s2 = create()
        L.emt_step(s2, T, rec, stream)
        rec_host.copy_(rec, non_blocking=True)
        torch.cuda.synchronize()
        del s2
        t1 = time.perf_counter()
        if i > 0:
            e2e_times.append(t1 - t0)

    sim = create()
    tuned = None
    if not tune:
        # block tiles, product kinds and the injection kernel timed on this simulation
        t0 = time.perf_counter()
        tn, kind = L.emt_sim_autotune(sim, 64, stream)
        tuned = {"leaf_tile_columns": tn, "kernels": kind,
                 "inject_columns_per_thread": L.emt_sim_stats(sim)["inject_columns_per_thread"],
                 "seconds": time.perf_counter() - t0, "probe_steps": 64}
    for _ in range(args.warmup):
        L.emt_sim_reset(sim, stream)
        L.emt_step(sim, T, rec, stream)
    barrier()
    clocks = Clocks(local)
    l0 = L.emt_sim_stats(sim)["launches"]
    times = []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.emt_sim_reset(sim, stream)
        L.emt_step(sim, T, rec, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    launches = (L.emt_sim_stats(sim)["launches"] - l0) // args.steps
    ms = job_ms(float(np.mean(times)), world, dev)
    units = job_units(n * Rl * T, world, dev)     # each column counted once, on the rank that ran it
    value = units / (ms / 1e3)
    e2e_ms = job_ms(float(np.mean(e2e_times)) * 1e3, world, dev)
    e2e_val = units / (e2e_ms / 1e3)
    traj = rec.cpu().numpy()
    st = L.emt_sim_stats(sim)

    # the kernels of a time step, timed alone on the operands of the last pass: 0 leaf GEMM, 1 BF16
    # split of its right-hand sides, 2 sweep GEMM, 3 expansion (each twice per time step), 4 history
    # update and injection, 5 residual (once)
    reps = 200
    kus = {}
    for which in (0, 1, 2, 3, 4, 5):
        L.emt_sim_bench_kernel(sim, which, reps, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.emt_sim_bench_kernel(sim, which, reps, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        kus[which] = e0.elapsed_time(e1) / reps * 1e3
    L.emt_sim_reset(sim, stream)

    # accuracy: the oracle on 8 of this rank's columns over every time step (rank 0; one
    # single-threaded process per column)
    errs, cpu_rate, acc_cols = {}, None, []
    if rank == 0:
        acc_cols = accuracy_columns(Rl)
        refs, secs = run_cpu_oracle_columns(T, cfg, [w["c0"] + c for c in acc_cols])
        for c, ref in zip(acc_cols, refs):
            errs[w["c0"] + c] = rel_err(traj[:, c, :], ref)
        cpu_rate = n * T * len(acc_cols) / sum(secs)
    # leaf GEMM: 2 sum(b_j^2) R algorithmic flops per launch (FP32-grade products, each formed as
    # three BF16 tensor-core products hi*hi + hi*lo + lo*hi)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
    flops_gemm = 2 * st["leaf_elems"] * Rl
    peak_tf = peaks["bf16_tflops"] / 3.0
    hbm = peaks.get("hbm_gbs", 6800.0)
    fp32_peak = 69.4   # TFLOP/s FP32 FMA (2 flops per FMA), measured by the probe on this GB300
    # algorithmic work per launch: flops of the products; bytes of the streaming parts (split:
    # read FP32, write BF16 hi + lo; expansion epilogue: read Y, read and write float-float V)
    # injection: element histories read + written (two parity buffers, one word per element), own
    # and neighbour voltages, source terms, X (float-float) and Xf written; residual: X and the
    # CSR neighbours' V read, Xf written (neighbour re-reads hit L2: counted once)
    n_el = st["n_elements"]
    n_terms_b = len(net["src_bus"]) + len(net.get("load_bus", []))
    inj_bytes = (2 * n_el * 8 + n * 8 + n_terms_b * 16 + n * 12) * Rl
    res_bytes = n * (8 + 8 + 4) * Rl
    per = {
        "k_mc_umma<leaf> (tcgen05 BF16x3)": (kus[0], 2, "tensor", flops_gemm / 1e12, peak_tf, "TFLOP/s"),
        "k_split_b (BF16 hi/lo split)": (kus[1], 2, "hbm", n * Rl * 8 / 1e9, hbm, "GB/s"),
        "k_mc_sweep_gemm (FP32 SIMT, split-K over nonzero column pieces)":
            (kus[2], 2, "alu", 2 * st["s_total"] * st["n_cut_rows"] * Rl / 1e12, fp32_peak, "TFLOP/s"),
        "expansion (tcgen05 k_mc_umma<expand> when it has a tile per SM, else SIMT k_mc_expand_tiled)":
            (kus[3], 2, "hbm", n * Rl * 20 / 1e9, hbm, "GB/s"),
        inject_name(st): (kus[4], 1, "hbm", inj_bytes / 1e9, hbm, "GB/s"),
        residual_name(st): (kus[5], 1, "hbm", res_bytes / 1e9, hbm, "GB/s"),
    }
    kernels = {}
    my_ms = float(np.mean(times))
    for name, (us, per_step, bound, work, peak, unit) in per.items():
        ach = work / (us * 1e-6)
        kernels[name] = {"us_per_launch": us, "launches_per_time_step": per_step, "bound": bound, "achieved": ach,
                         "peak": peak, "unit": unit, "frac": ach / peak,
                         "share_of_step": per_step * us * T / 1e3 / my_ms}
    dom = max(kernels, key=lambda k: kernels[k]["share_of_step"])
    if rank != 0:
        return None
    name = multi_name(cfg)
    return {
        "metric": "bus-steps/sec at rel err <=1e-8 vs FP64 oracle", "value": value, "unit": "bus-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "bf16x3-f32acc+ff64-refine", "data": "synthetic",
        "config": {"workload": name, "buses": n, "columns": R, "columns_per_rank": Rl, "time_steps_per_step": T,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"columns split over {world} rank(s), no collective on the data path"},
        "accuracy": {"sampled_columns": {str(k): v for k, v in errs.items()}, "sampled_steps": T,
                     "max": max(errs.values()) if errs else None, "tolerance": ERR_TOL},
        "autotuned": tuned,
        "roofline": dict(kernels[dom], kernel=dom, traffic=ncu_traffic(dom, n, Rl),
                         peak_source=("measured" if "when" in peaks else "fallback")
                         + " (tensor: bf16 burst / 3, three BF16 products per FP32-grade product; hbm: copy; "
                           "alu: FP32 FMA rate of the probe)",
                         kernels=kernels),
        "e2e": {"value": e2e_val, "unit": "bus-steps/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": T * Rl * N_MON * 8,
                "includes": "emt_sim_create from host arrays (partition, GPU build), trip scheduling, emt_step, "
                            "D2H of the record; measured first, in a process that had run nothing else"},
        "cpu_baseline": {"value": cpu_rate, "unit": "bus-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"columns {[w['c0'] + c for c in acc_cols]}, {T} steps each, FP64 exact "
                                   "hierarchical store, each column single-threaded in its own process"},
        "gpu_launches": int(launches), "clocks": clk,
    }


def inject_name(st):
    v = st["inject_variant"]
    if v >= 2:
        kb, mb = {2: (6, 2), 3: (3, 3), 4: (2, 4)}[v]
        return (f"k_mc_inject2<{kb},{mb}> (histories + injection, float-float, two columns per thread, "
                f"{kb} element ends per round trip, {mb} CTAs per SM)")
    return "k_mc_inject (histories + injection, float-float)"


def residual_name(st):
    if st["residual_columns_per_thread"] == 2:
        return "k_mc_residual2 (float-float r = x - G'v, two columns per thread)"
    return "k_mc_residual (float-float r = x - G'v)"


# DRAM bytes (read + write) per launch, keyed by (kernel, buses, columns), from one ncu capture of
# dram__bytes_read.sum and dram__bytes_write.sum of the kernel as it stands (python bench.py
# --config 4 --profile 6, third launch of each; profiles/multi_column_11456bus_512col_*_ncu_*.md)
NCU_TRAFFIC = {("k_mc_inject2<2,4>", 11456, 512): 211.768832e6 + 148.137472e6,
               ("k_mc_residual2", 11456, 512): 94.539264e6 + 9.608960e6}


def ncu_traffic(kernel, n, cols):
    return NCU_TRAFFIC.get((kernel.split(" ")[0], n, cols))


# ---------------------------------------------------------------- config 5 (serving)
PRIV_BASE = 100   # request network index >= PRIV_BASE: private network PRIV_BASE + j of the pool


def serve_requests(nets, n_req, seed, rate, steps_lo=1000, steps_hi=10000, priv=None, priv_frac=0.0):
    import numpy as np
    import netgen
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_req):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        if priv and rng.random() < priv_frac:
            j = int(rng.integers(len(priv)))
            k, net = PRIV_BASE + j, priv[j]
        else:
            k = int(rng.integers(len(nets)))
            net = nets[k][0]
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        if rng.random() < 0.5:
            out.append((k, t, steps, 0, int(rng.integers(len(net["br_a"]))), 0.0, int(rng.integers(1, steps)), 0))
        else:
            st = int(rng.integers(1, max(2, steps - 400)))
            out.append((k, t, steps, 1, int(rng.integers(net["n_bus"])), 10.0, st, 400))
    return out


def serve_arm(args):
    """Config 5. With N ranks the stream carries N times the requests at N times the rate, dealt
    round-robin, so every rank (one server per GPU) sees the one-GPU load (weak scaling);
    latencies of all ranks' requests are gathered for p50/p99. Returns the JSON line on rank 0."""
    import numpy as np
    import torch
    import netgen
    import paper_2105_10661_gb300._lib as L
    from oracle import emt as oemt

    rank, world, local = ranks()
    dev = torch.device("cuda", local)
    nets = [(netgen.tile(1_000_000), 2, 256), (netgen.tiled(2, 4), 3, 256), (netgen.config_network(4), 4, 128)]
    mons = [np.sort(np.random.default_rng(17 + i).choice(n[0]["n_bus"], N_MON, replace=False)) for i, n in enumerate(nets)]
    # private networks: a pool of seeded 179-bus tiles that requests bring with them (10 % of the
    # requests); each is built on its first arrival and then served from the resident copy
    priv = [netgen.tile(3_000_000 + j) for j in range(16)]
    priv_mon = np.arange(0, 179, 12)[:N_MON]
    priv_frac = 0.1

    def make_server():
        srv = L.emt_server_create(100, 96 << 30)
        ids = [L.emt_server_add_network(srv, n[0], DT, levels=n[1], max_slots=n[2], monitor=mons[i])
               for i, n in enumerate(nets)]
        return srv, ids

    def submit(srv, ids, r):
        if r[0] >= PRIV_BASE:
            return L.emt_server_submit_network(srv, priv[r[0] - PRIV_BASE], DT, *r[1:], levels=2, monitor=priv_mon)
        return L.emt_server_submit(srv, ids[r[0]], *r[1:])

    # calibration: a burst at t = 0 measures the saturated request rate
    srv, ids = make_server()
    cal = serve_requests(nets, 300, 99, 0.0, priv=priv, priv_frac=priv_frac)
    for r in cal:
        submit(srv, ids, r)
    L.emt_server_run(srv)
    cst = L.emt_server_stats(srv)
    # one GPU's saturated rate, averaged over the ranks' calibrations
    sat_rate = job_units(cst["finished"] / cst["wall_s"], world, dev) / world
    del srv
    # the measured run: Poisson arrivals at 80% of the saturated rate per GPU
    rate = 0.8 * sat_rate * world
    reqs_all = serve_requests(nets, args.requests * world, 17, rate, priv=priv, priv_frac=priv_frac)
    mine = rank_share(reqs_all, world, rank)
    reqs = [r for _, r in mine]
    srv, ids = make_server()
    rids = [submit(srv, ids, r) for r in reqs]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = Clocks(local)
    L.emt_server_run(srv)
    clk = clocks.stop()
    st = L.emt_server_stats(srv)
    lat = []
    for rid in rids:
        _, tm = L.emt_server_result(srv, rid)
        lat.append(float(tm[2] - tm[0]))
    wall = job_ms(st["wall_s"] * 1e3, world, dev) / 1e3
    bus_steps = job_units(st["bus_steps"], world, dev)
    if world > 1:
        import torch.distributed as dist
        gathered = [None] * world
        dist.all_gather_object(gathered, lat)
        lat = [x for part in gathered for x in part]
    if rank != 0:
        return None
    lat_np = np.asarray(lat)
    # accuracy: oracle on sampled short requests of the two smaller networks
    errs = {}
    cpu_sec = 0.0
    cpu_bus_steps = 0.0
    picks = [i for i, r in enumerate(reqs) if r[0] in (0, 1) and r[2] <= 2500][:4]
    picks += [i for i, r in enumerate(reqs) if r[0] >= PRIV_BASE and r[2] <= 2500][:2]
    for i in picks:
        k, _, steps, kind, target, value, ev, ln = reqs[i]
        net, levels = (priv[k - PRIV_BASE], 2) if k >= PRIV_BASE else nets[k][:2]
        mon = priv_mon if k >= PRIV_BASE else mons[k]
        t0 = time.perf_counter()
        nw = oemt.Network(net, DT, levels=levels)
        evs = ([(ev, oemt.TRIP, target, 0.0)] if kind == 0 else
               [(ev, oemt.FAULT_ON, target, value), (ev + ln, oemt.FAULT_OFF, target, 0.0)])
        ref, _ = oemt.simulate(nw, steps, evs, solver="exact", monitor=mon)
        cpu_sec += time.perf_counter() - t0
        cpu_bus_steps += steps * net["n_bus"]
        got, _ = L.emt_server_result(srv, rids[i])
        errs[str(i)] = rel_err(got, ref)
    return {
        "metric": "bus-steps/sec at rel err <=1e-8 vs FP64 oracle; p50/p99 served latency", "value": bus_steps / wall,
        "unit": "bus-steps/s", "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": wall * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3-f32acc+ff64-refine",
        "data": "synthetic",
        "config": {"workload": f"serving: Poisson stream of {args.requests} requests per GPU over resident "
                               "179/1432/11456-bus networks (10% bring one of 16 private 179-bus networks, built on "
                               "first arrival), 1000-10000 steps each, a line trip or a 10-ohm 400-step bus fault per "
                               "request",
                   "arrival_rate_req_per_s": rate, "saturated_rate_req_per_s_per_gpu": sat_rate, "tick_steps": 100,
                   "slots": [n[2] for n in nets],
                   "parallelism": f"requests dealt round-robin over {world} rank(s), one server per GPU"},
        "latency_s": {"p50": float(np.percentile(lat_np, 50)), "p99": float(np.percentile(lat_np, 99)),
                      "max": float(lat_np.max()), "requests": len(lat)},
        "served": {k: st[k] for k in ("wall_s", "bus_steps", "max_queue", "ticks", "finished")},
        "private_networks": {"requests": sum(1 for r in reqs if r[0] >= PRIV_BASE), "pool": len(priv),
                             "builds": st["builds"], "cache_hits": st["cache_hits"], "build_s": st["build_s"],
                             "evictions": st["evictions"]},
        "accuracy": {"sampled_requests": errs, "max": max(errs.values()) if errs else None},
        "cpu_baseline": {"value": cpu_bus_steps / cpu_sec if cpu_sec else None, "unit": "bus-steps/s", "cores": 1,
                         "kind": "oracle", "sample": f"{len(picks)} sampled requests, exact hierarchical store"},
        "clocks": clk,
    }


# ---------------------------------------------------------------- config 4': single-vector apply, HBM bound
def apply_arm(args):
    import numpy as np
    import torch
    import netgen
    import paper_2105_10661_gb300._lib as L
    from oracle import emt as oemt
    from oracle import hinv as ohinv

    if int(os.environ.get("RANK", "0")) != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    net = netgen.config_network(4)
    n = net["n_bus"]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    x = torch.tensor(np.random.default_rng(5).standard_normal(n), dtype=torch.float64, device=dev)
    res = {}
    clocks = Clocks(dev.index)
    paths = {}
    for pname, p in (("fp64", L.EMT_PREC_FP64), ("ff64", L.EMT_PREC_FF64)):
        h = L.emt_build_hinv_from_network(net, DT, levels=4, precision=p)
        # mode 2: one cooperative launch (k_apply_persist); 1: three chained kernels (the default)
        for mode, mname in ((2, "single_launch"), (1, "three_kernels")):
            L.emt_apply_tune(h, mode)
            v = torch.zeros(n, dtype=torch.float64, device=dev)
            for _ in range(args.warmup):
                L.emt_apply(h, x, v, stream=stream)
            used = L.emt_apply_tune(h, mode)
            ts = []
            for _ in range(max(args.steps, 10)):
                # the flush (a 512 MB write, longer than the apply) is queued ahead of the timed
                # apply, so the apply's launch is submitted while the GPU is still busy and the
                # event interval is device time, not host launch latency
                torch.cuda.synchronize()
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                L.emt_apply(h, x, v, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            name = f"{pname}_{mname}"
            res[name] = (float(np.median(ts)), v.cpu().numpy())
            paths[name] = {2: "single launch", 1: "three kernels", 0: "small-store kernels"}[used]
        L.emt_apply_tune(h, 0)
    clk = clocks.stop()
    # oracle: exact hierarchical apply of the same vector (CPU, single thread)
    t0 = time.perf_counter()
    nw = oemt.Network(net, DT, levels=4)
    H = ohinv.HInv(nw.G, nw.tree, nw.g_series, ohinv.EXACT)
    t1 = time.perf_counter()
    ref = H.apply(x.cpu().numpy())
    t2 = time.perf_counter()
    tree = nw.tree
    leaf = sum(int(tree["hi"][j] - tree["lo"][j]) ** 2 for j in tree["leaves"])
    fac = sum(int(tree["hi"][p] - tree["lo"][p]) * int(tree["cut_ptr"][p + 1] - tree["cut_ptr"][p])
              for p in range(len(tree["lo"])) if tree["left"][p] >= 0)
    byts = (leaf + fac) * 8 + n * 8 * 3
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    head = min(res, key=lambda k: res[k][0])
    ms = res[head][0]
    ach = byts / (ms * 1e-3) / 1e9
    return {
        "metric": "bus-steps/sec at rel err <=1e-8 vs FP64 oracle", "value": n / (ms * 1e-3), "unit": "bus-steps/s",
        "n_gpus": 1, "steps": max(args.steps, 10), "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": head.split("_")[0], "data": "synthetic",
        "config": {"workload": "single-vector apply v = Ginv i on the 11456-bus store (16 leaves of 716), "
                               "L2 flushed before every apply", "store_bytes_fp64": (leaf + fac) * 8},
        "variants_ms": {k: v[0] for k, v in res.items()},
        "accuracy": {k: rel_err(v[1], ref) for k, v in res.items()},
        "paths": paths,
        "roofline": {"bound": "hbm", "kernel": ("k_apply_persist (the whole apply in one launch)" if
                                               paths[head] == "single launch" else
                                               "whole apply (k_leaf_stream + k_sweep_matrix + k_expand_stream)"),
                     "achieved": ach,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None,
                     "algorithmic_bytes": byts},
        "cpu_baseline": {"value": n / (t2 - t1), "unit": "bus-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "one exact hierarchical apply of the same vector (store build excluded)"},
        "clocks": clk,
    }


# ---------------------------------------------------------------- config 6 (d_th sweep)
def hier_solve_flops(tree: dict, p: int = 0, paper: bool = False) -> int:
    """Additions and multiplications of one solve with the store of node p's subtree, in the
    recursive order of Eq. 9: every leaf y_j = L_j x_j (b^2 products, b(b-1) additions); at every
    internal node with k cut columns, t_p (k products by -g, the other half is a gather),
    s_p = C_p t_p (EXACT: 4k^2 products and 2k(2k-1) additions; PAPER: C_p = [[0, I], [I, 0]] is a
    swap) and the correction of its n_p rows by P s_1 or Q s_2 (k products, k additions a row)."""
    lo, hi, left, right, cut_ptr = (tree[k] for k in ("lo", "hi", "left", "right", "cut_ptr"))
    total = 0
    stack = [p]
    while stack:
        q = stack.pop()
        n_q = int(hi[q] - lo[q])
        if left[q] < 0:
            total += 2 * n_q * n_q - n_q
        else:
            k = int(cut_ptr[q + 1] - cut_ptr[q])
            total += k + (0 if paper else 8 * k * k - 2 * k) + 2 * n_q * k
            stack += [int(left[q]), int(right[q])]
    return total


def leaf_inverse_flops(b: int) -> int:
    """Direct inversion of an SPD leaf block (Cholesky L L^T, W = L^-1, then W^T W for one triangle;
    divisions and square roots count one each)."""
    chol = sum((b - j) * (2 * j + 1) for j in range(b))
    trinv = b + sum((b - d) * 2 * d for d in range(1, b))
    wtw = sum((j + 1) * (2 * (b - j) - 1) for j in range(b))
    return chol + trinv + wtw


def _alg1_node_flops(tree: dict, p: int) -> int:
    """Algorithm 1's work at node p: a leaf's direct inverse, or the k cut columns of P and Q."""
    lo, hi, left, right, cut_ptr = (tree[k] for k in ("lo", "hi", "left", "right", "cut_ptr"))
    if left[p] < 0:
        return leaf_inverse_flops(int(hi[p] - lo[p]))
    k = int(cut_ptr[p + 1] - cut_ptr[p])
    return k * (hier_solve_flops(tree, int(left[p]), True) + hier_solve_flops(tree, int(right[p]), True))


def alg1_build_flops(tree: dict) -> int:
    """Algorithm 1 (PAPER store): every leaf inverted directly, and at every internal node the k
    cut columns of P and of Q, each one solve of -g e_a (resp. e_b) through the child's store."""
    return sum(_alg1_node_flops(tree, p) for p in range(len(tree["lo"])))


def alg2_flops(tree: dict, a_pos: int, b_pos: int = -1) -> int:
    """Algorithm 2 (Sec. IV) for a change at positions a_pos, b_pos (-1: to ground): the leaves
    holding them re-inverted directly and Algorithm 1's cut columns recomputed at every internal
    node on their paths up to the lowest common ancestor (Theorem 1), nothing above it."""
    lo, hi, left, parent = (tree[k] for k in ("lo", "hi", "left", "parent"))

    def leaf_of(x):
        q = 0
        while left[q] >= 0:
            q = int(left[q]) if x < hi[int(left[q])] else int(tree["right"][q])
        return q

    la = leaf_of(a_pos)
    lb = leaf_of(b_pos) if b_pos >= 0 else la
    up, q = set(), la
    while q >= 0:
        up.add(q)
        q = int(parent[q])
    top = lb
    while top not in up:
        top = int(parent[top])
    nodes = set()
    for leaf in {la, lb}:
        q = leaf
        while True:
            nodes.add(q)
            if q == top:
                break
            q = int(parent[q])
    return sum(_alg1_node_flops(tree, q) for q in nodes)


def lu_flops(n_bus: int, br_a, br_b) -> dict:
    """Additions, multiplications and divisions of the sparse-LU alternative (SuperLU through SciPy,
    minimum-degree ordering of A + A^T, no pivoting) on the pattern of G: a weighted Laplacian of the
    branches plus a positive diagonal (fill depends on the pattern only). Factorisation: l_k divisions
    and l_k u_k multiply-adds at pivot k (l_k, u_k: nonzeros below and right of it). Solve: one
    multiply-add per off-diagonal nonzero of L and U, one division per row."""
    import numpy as np
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    a, b = np.asarray(br_a), np.asarray(br_b)
    ones = np.ones(len(a))
    A = sp.coo_matrix((np.concatenate([-ones, -ones]), (np.concatenate([a, b]), np.concatenate([b, a]))),
                      shape=(n_bus, n_bus)).tocsr()
    deg = -np.asarray(A.sum(axis=1)).ravel()
    A = (A + sp.diags(deg + 1.0)).tocsc()
    lu = spla.splu(A, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0, options={"SymmetricMode": True})
    Lm, Um = lu.L.tocsc(), lu.U.tocsr()
    Lm.eliminate_zeros()
    Um.eliminate_zeros()
    l_k = np.diff(Lm.indptr) - 1            # below the unit diagonal, per column
    u_k = np.diff(Um.indptr) - 1            # right of the diagonal, per row
    factor = int(np.sum(l_k) + 2 * np.sum(l_k * u_k))
    solve = int(2 * np.sum(l_k) + 2 * np.sum(u_k) + n_bus)
    return {"factor": factor, "solve": solve, "nnz_L": int(Lm.nnz), "nnz_U": int(Um.nnz)}


def flop_table(shapes=((1, 1), (1, 2), (2, 2), (2, 4), (3, 4)), dths=(45, 179)) -> list:
    """FLOPs on the tiled arrays (Sec. V-B): Algorithm 1's build (E2), Algorithm 2 for a fault and
    for a trip of a root cut branch (Theorem 1), and one solve per time step with the PAPER and the
    EXACT store (E3), partitions from the library's host-side tree build, against the sparse-LU
    solve and factorisation and the dense mat-vec."""
    import netgen
    import paper_2105_10661_gb300._lib as L
    rows = []
    for (r, c) in shapes:
        net = netgen.tile(1_000_000) if r * c == 1 else netgen.tiled(r, c)
        n = int(net["n_bus"])
        lu = lu_flops(n, net["br_a"], net["br_b"])
        row = {"n_bus": n, "lu_solve": lu["solve"], "lu_factor": lu["factor"], "dense_matvec": 2 * n * n - n}
        for d in dths:
            tree = L.emt_tree_build(n, net["br_a"], net["br_b"], d_th=d)
            row[f"solve_paper_dth{d}"] = hier_solve_flops(tree, paper=True)
            row[f"solve_exact_dth{d}"] = hier_solve_flops(tree)
            row[f"alg1_build_dth{d}"] = alg1_build_flops(tree)
            # Algorithm 2: a fault at bus N/3 (one leaf), and a trip of the root's first cut branch
            # (paths up to the root: Theorem 1's worst case)
            pos = {int(bus): i for i, bus in enumerate(tree["perm"])}
            row[f"alg2_fault_dth{d}"] = alg2_flops(tree, pos[n // 3])
            if tree["left"][0] >= 0 and tree["cut_ptr"][1] > 0:
                row[f"alg2_root_trip_dth{d}"] = alg2_flops(tree, int(tree["cut_a"][0]), int(tree["cut_b"][0]))
        rows.append(row)
    return rows


def dth_arm(args):
    """PAPER-mode store (Algorithm 1) on tiled arrays of 1..12 tiles, leaves of at most d_th buses.

    Per (network, d_th): the approximation error of the PAPER inverse against the exact one (Fig. 5,
    from identity applies of a PAPER and an EXACT store), the GPU build time (Algorithm 1), and the
    time of Algorithm 2 for a 10-ohm bus fault against rebuilding the store of the faulted network
    (Theorem 1, Sec. V-C.2); with the element saving 1 - (b / N)^2 of inverting one b-bus leaf
    instead of the whole matrix."""
    import numpy as np
    import torch
    import netgen
    import paper_2105_10661_gb300._lib as L

    if int(os.environ.get("RANK", "0")) != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    shapes = [(1, 1), (1, 2), (2, 2), (2, 4), (3, 4)]
    dths = [22, 45, 90, 179]
    fault_ohm = 10.0
    rows = []

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) * 1e3

    def inverse(h, n):
        eye = torch.eye(n, dtype=torch.float64, device=dev)
        out = torch.empty_like(eye)
        L.emt_apply(h, eye, out, nrhs=n, stream=stream)
        torch.cuda.synchronize()
        return out

    clocks = Clocks(dev.index)
    for (r, c) in shapes:
        net = netgen.tile(1_000_000) if r * c == 1 else netgen.tiled(r, c)
        n = net["n_bus"]
        # the fault as a zero-volt source behind 10 ohm: G' = G + (1/10) e_a e_a^T
        bus = n // 3
        netf = dict(net)
        for k, v in (("src_bus", bus), ("src_Vm", 0.0), ("src_phi", 0.0), ("src_Rs", fault_ohm)):
            netf[k] = np.concatenate([np.asarray(net[k]), np.asarray([v], dtype=np.asarray(net[k]).dtype)])
        he = L.emt_build_hinv_from_network(net, DT, d_th=max(dths))   # exact store (single leaf up to 179)
        Gi = inverse(he, n)
        for d in dths:
            if d > n and d != dths[0]:
                continue
            L.emt_build_hinv_from_network(net, DT, d_th=d, mode=L.EMT_MODE_PAPER)   # warm (allocator, kernels)
            h, build_ms = timed(lambda: L.emt_build_hinv_from_network(net, DT, d_th=d, mode=L.EMT_MODE_PAPER))
            Gp = inverse(h, n)
            err = float(torch.linalg.norm(Gp - Gi) / torch.linalg.norm(Gi))
            tr = h.tree()
            leaves = [j for j in range(len(tr["lo"])) if tr["left"][j] < 0]
            bmax = max(int(tr["hi"][j] - tr["lo"][j]) for j in leaves)
            _, mod_ms = timed(lambda: L.emt_modify_branch(h, bus, -1, 1.0 / fault_ohm, stream=stream))
            hf, rebuild_ms = timed(lambda: L.emt_build_hinv_from_network(netf, DT, d_th=d, mode=L.EMT_MODE_PAPER))
            # literal Algorithm 2 stops at the lowest common ancestor; a rebuild also changes the
            # ancestors' factors: their gap
            Gm, Gf = inverse(h, n), inverse(hf, n)
            gap = float(torch.linalg.norm(Gm - Gf) / torch.linalg.norm(Gf))
            # the EXACT store: the local update continued to the root, against its rebuild
            hx = L.emt_build_hinv_from_network(net, DT, d_th=d)
            _, xmod_ms = timed(lambda: L.emt_modify_branch(hx, bus, -1, 1.0 / fault_ohm, stream=stream))
            hxf, xrebuild_ms = timed(lambda: L.emt_build_hinv_from_network(netf, DT, d_th=d))
            xgap = float(torch.linalg.norm(inverse(hx, n) - inverse(hxf, n)) / torch.linalg.norm(Gi))
            rows.append({"n_bus": n, "d_th": d, "n_leaf": len(leaves), "max_leaf": bmax,
                         "paper_rel_err_vs_exact": err, "build_ms": build_ms, "modify_ms": mod_ms,
                         "rebuild_ms": rebuild_ms, "time_saved": 1.0 - mod_ms / rebuild_ms,
                         "algorithm2_vs_rebuild_rel_diff": gap,
                         "exact_modify_ms": xmod_ms, "exact_rebuild_ms": xrebuild_ms,
                         "exact_modify_vs_rebuild_rel_diff": xgap,
                         "element_saving": 1.0 - (bmax / n) ** 2})
    # scaling of the build time with N at each d_th (least-squares slope of log t vs log N)
    clk = clocks.stop()
    slopes = {}
    for d in dths:
        pts = [(x["n_bus"], x["build_ms"]) for x in rows if x["d_th"] == d]
        if len(pts) >= 3:
            lx, ly = np.log([p[0] for p in pts]), np.log([p[1] for p in pts])
            slopes[str(d)] = float(np.polyfit(lx, ly, 1)[0])
    head = [x for x in rows if x["n_bus"] == max(y["n_bus"] for y in rows) and x["d_th"] == 45][0]
    # the oracle's Algorithm 2 on the same fault, 179-bus tile, d_th 45 (one core)
    from oracle import emt as oemt, hinv as ohinv, modify as omod, partition as opart
    t_net = netgen.tile(1_000_000)
    nw = oemt.Network(t_net, DT, want_tree=False)
    tree = opart.build_tree(t_net["n_bus"], nw.series_frm, nw.series_to, 0, 45)
    H = ohinv.HInv(nw.G, tree, nw.g_series, ohinv.PAPER)
    t0 = time.perf_counter()
    omod.algorithm2(H, nw.series_frm, nw.series_to, t_net["n_bus"] // 3, -1, 1.0 / fault_ohm)
    cpu_ms = (time.perf_counter() - t0) * 1e3
    return {
        "metric": "share of rebuild time saved by Algorithm 2 (10-ohm bus fault, PAPER store)",
        "value": head["time_saved"], "unit": "fraction", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": head["modify_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "PAPER-mode d_th sweep on seeded tiled arrays (179..2148 buses), d_th in "
                               f"{dths}, 10-ohm fault at bus N/3", "headline": "2148 buses, d_th 45"},
        "table": rows, "build_time_exponent_vs_N": slopes, "flops_e2_e3": flop_table(),
        "cpu_baseline": {"value": cpu_ms, "unit": "ms per Algorithm 2", "cores": 1, "kind": "oracle",
                         "sample": "179-bus tile, d_th 45, the same fault"},
        "gpu_launches": None, "clocks": clk,
    }


# ---------------------------------------------------------------- config 7 (three-phase buses)
def three_phase_arm(args):
    """Three nodes per bus with mutually coupled RL branches: single-vector apply, and a
    three-phase line trip as exact rank-1 node updates against rebuilding the store; the bus-level
    partition with block cuts (the default) beside the node-level one."""
    import numpy as np
    import torch
    import netgen
    import paper_2105_10661_gb300._lib as L
    from oracle import companion as ocm, dense as odense, modify as omod

    if int(os.environ.get("RANK", "0")) != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    net = netgen.three_phase(netgen.tiled(2, 4))
    nn = 3 * net["n_bus"]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    x = torch.tensor(np.random.default_rng(5).standard_normal(nn), dtype=torch.float64, device=dev)

    def sync_time(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) * 1e3

    # reference solution of the oracle's G (CPU), also the timed CPU baseline
    gr = ocm.three_phase_graph(net, DT)
    G0 = ocm.assemble_dense(gr)
    t0 = time.perf_counter()
    ref = odense.DenseSolver(G0).solve(x.cpu().numpy())
    cpu_ms = (time.perf_counter() - t0) * 1e3
    # three-phase trip of the first RL branch: 15 exact rank-1 node updates, negative (cross-phase)
    # branches first so every intermediate G stays positive definite
    e = next(k for k in range(len(net["br_a"])) if net["kind"][k] == 0)
    a, b = int(net["br_a"][e]), int(net["br_b"][e])
    Y = ocm.coupled_rl_admittance(float(net["R"][e]), float(net["L"][e]), float(net["L_mut"][e]), DT)
    ups = ([(3 * a + p, 3 * b + q, Y[p, q]) for p in range(3) for q in range(3) if p != q]
           + [(3 * z + p, 3 * z + q, -Y[p, q]) for z in (a, b) for p in range(3) for q in range(p + 1, 3)]
           + [(3 * a + p, 3 * b + p, Y[p, p]) for p in range(3)])
    Gt = G0
    for xx, yy, g in ups:
        Gt = omod.modified_G(Gt, xx, yy, -g)
    ref_trip = odense.DenseSolver(Gt).solve(x.cpu().numpy())
    keep = [k for k in range(len(net["br_a"])) if k != e]
    net_t = dict(net)
    for k in ("br_a", "br_b", "kind", "R", "L", "C", "L_mut"):
        net_t[k] = np.asarray(net[k])[keep]

    def measure(npb, clocks=None):
        L.emt_build_hinv_from_network3(net, DT, levels=3, nodes_per_bus=npb)   # warm
        h, build_ms = sync_time(lambda: L.emt_build_hinv_from_network3(net, DT, levels=3, nodes_per_bus=npb))
        v = torch.zeros(nn, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            L.emt_apply(h, x, v, stream=stream)
        clk = Clocks(dev.index) if clocks else None
        ts = []
        t_end = time.perf_counter() + (0.8 if clocks else 0.0)   # long enough for clock samples
        while len(ts) < max(args.steps, 10) or time.perf_counter() < t_end:
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.emt_apply(h, x, v, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        clk = clk.stop() if clk else None
        v_before = v.cpu().numpy()
        err = rel_err(v_before, ref)
        cuts = int(len(h.tree()["cut_b"]))

        def trip():
            for xx, yy, g in ups:
                L.emt_modify_branch(h, xx, yy, -g, stream=stream)
        _, trip_ms = sync_time(trip)
        _, rebuild_ms = sync_time(lambda: L.emt_build_hinv_from_network3(net_t, DT, levels=3, nodes_per_bus=npb))
        L.emt_apply(h, x, v, stream=stream)
        torch.cuda.synchronize()
        return {"apply_ms": float(np.median(ts)), "applies_timed": len(ts), "build_ms": build_ms, "cut_columns": cuts,
                "accuracy": {"apply": err, "after_three_phase_trip": rel_err(v.cpu().numpy(), ref_trip),
                             "solution_change_by_trip": rel_err(v.cpu().numpy(), v_before)},
                "three_phase_trip": {"node_updates": len(ups), "ms": trip_ms, "rebuild_ms": rebuild_ms,
                                     "time_saved": 1.0 - trip_ms / rebuild_ms}}, clk

    blk, clk = measure(3, clocks=True)
    node, _ = measure(1)
    apply_ms = blk["apply_ms"]
    return {
        "metric": "three-phase node solves per second (v = G^-1 i, one vector)", "value": nn / (apply_ms * 1e-3),
        "unit": "node-solves/s", "n_gpus": 1, "steps": blk["applies_timed"], "warmup": args.warmup,
        "ms_per_step": apply_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "1432-bus 8-tile network in three phases (4,296 nodes, mutual inductance U[0.2, 0.4] "
                               "of self on every RL branch), 3-level hierarchy, EXACT FP64 store, L2 flushed before "
                               "every apply", "nodes": nn,
                   "partition": "by bus (three nodes kept together), one rank-3 block cut per joined bus pair"},
        "accuracy": blk["accuracy"], "build_ms": blk["build_ms"], "three_phase_trip": blk["three_phase_trip"],
        "partitions": {"block_cuts": blk, "node_level": node},
        "cpu_baseline": {"value": nn / (cpu_ms * 1e-3), "unit": "node-solves/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": "dense Cholesky solve of the same G and vector (factorisation "
                                                     "included)"},
        "clocks": clk,
    }


def profile_run(args):
    """The kernels of one workload and nothing else, for profiler captures (no timing, no line)."""
    import numpy as np
    import torch
    import netgen
    import paper_2105_10661_gb300._lib as L
    if args.config in (3, 4):
        w = multi_workload(args.config)
        R = args.columns or w["R"]
        ss = None if w["ss"] is None else np.ascontiguousarray(w["ss"][:R])
        ls = None if w["ls"] is None else np.ascontiguousarray(w["ls"][:R])
        sim = L.emt_sim_create(w["net"], DT, levels=w["levels"], nrhs=R, src_scale=ss, load_scale=ls)
        for c, (st_, e) in w["trips"].items():
            if c < R:
                L.emt_sim_schedule(sim, st_, L.EMT_EVENT_TRIP, e, 0.0, c)
        L.emt_sim_monitor(sim, w["mon"])
        rec = torch.zeros(args.profile, R, N_MON, dtype=torch.float64, device="cuda")
        L.emt_step(sim, args.profile, rec)
    elif args.config == 41:
        net = netgen.config_network(4)
        h = L.emt_build_hinv_from_network(net, DT, levels=4, precision=L.EMT_PREC_FF64)
        L.emt_apply_tune(h, args.apply_kernels)
        x = torch.tensor(np.random.default_rng(5).standard_normal(net["n_bus"]), dtype=torch.float64, device="cuda")
        v = torch.zeros_like(x)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        for _ in range(args.profile):
            flush.zero_()
            L.emt_apply(h, x, v)
    else:
        raise SystemExit("--profile serves configs 3, 4 and 41")
    torch.cuda.synchronize()


def main():
    args = parse()
    if args.cpu_worker:
        cpu_worker(args.cpu_worker, args.cpu_steps, args.config, args.cpu_col)
        return
    if args.profile:
        profile_run(args)
        return
    rc = launch_ranks(args)
    if rc is not None:
        sys.exit(rc)
    if args.impl != "reference" and args.config in (5, 6, 41):
        # these arms time the oracle in this process and report one core: pin the BLAS pools to one
        # thread before numpy is first imported
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
    if args.impl == "reference":
        reference_arm(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.config in (0, 4):
        line = multi_arm(args, 4)
        if args.config == 0:
            # secondary keys of the same line: the single 1,432-bus simulation and the single apply on
            # the 11,456-bus store (rank 0 times the apply alone)
            sec = {"single_1432bus_20000_steps": native_arm(args, 2)}
            if int(os.environ.get("RANK", "0")) == 0:
                sec["single_apply_11456bus"] = apply_arm(args)
            if line is not None:
                line["secondary"] = sec
    elif args.config == 3:
        line = multi_arm(args, 3)
    elif args.config == 5:
        line = serve_arm(args)
    elif args.config == 41:
        line = apply_arm(args)
    elif args.config == 6:
        line = dth_arm(args)
    elif args.config == 7:
        line = three_phase_arm(args)
    else:
        line = native_arm(args, args.config)
    if line is not None:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
