#!/usr/bin/env python
"""Throughput benchmark of the GB300 DPSO hot path.

Workload (default): the bridge-shaped instance (1992 viewpoints over seven
planar faces of a deck and two piers at 1 m spacing and 2 m stand-off, 20
boxes), swarm 4096, the paper's w = 1, phi1 = phi2 = 0.4, mutation every
third generation, back-and-forth seeding and edge exchange on.  `--workload
facade` takes the office-facade-shaped instance (400 viewpoints, swarm 1024).
A step is one DPSO generation (Fig. "pseudocode"): particle update + fitness +
pbest, mutation when due, gbest, and the edge exchange whenever the gbest did
not improve.

value   particle-iterations/s = particles x generations / device time of the
        generations dpso_step replays from its CUDA graphs, with the cost
        matrix and swarm resident in HBM; the L2 is flushed between timed
        generations.  For N > 1 each rank runs an independent replica (the
        solver has no exchange step to shard).
2-opt moves/s  candidate 2-opt pairs the exchange kernel evaluated per second
        of its own device time (`two_opt_pairs_evaluated_per_s`); the pairs a
        plain best-improvement scan of the same passes would take are
        reported beside it.
e2e     the same metric through dpso_plan from pinned host buffers: copies in,
        cost matrix, initialisation, `steps` generations, best tour out.
roofline  the 2-opt kernel: 8 bytes of C per candidate pair evaluated (two
        int32 entries) over its CUDA-event time inside the timed generations,
        against the L2 read bandwidth measured in this run (the cost matrix is
        L2-resident; rows are staged from L2).
fitness_roofline  the tour-fitness kernel (Eq. min) over the swarm's tours:
        4 n bytes of C gathered per tour over its CUDA-event time, against the
        random 4-byte gather rate from an L2-resident buffer measured in this
        run.

`--impl reference` times the CPU oracle on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DPSO particle-iterations/s and 2-opt moves/s per GB300; batched p99 latency"
UNIT = "particle-iterations/s"
BYTES_PER_PAIR = 8          # 2-opt: C[x_i][x_j] + C[x_i+1][x_j+1], int32 each
BYTES_PER_SWAP_PAIR = 16    # node swap: the four new edges' costs, int32 each
DEFAULT_STEPS = {"bridge": 20, "facade": 100, "tiny": 100, "batched": 3, "astar": 20,
                 "two-opt": 3, "serving": 1}


def cpu_sample_shape(n: int, threads: int, node_swap: bool = False) -> tuple[int, int]:
    """(particles, generations) of the oracle sample for the bench's
    cpu_baseline, sized to a few tens of seconds on `threads` host threads
    (each particle's edge exchange runs on one thread): an early generation
    costs the oracle about n^3 per particle (2-opt from the initial tours),
    about 0.1 s at n = 400 and 10-30 s at n = 1992; the node swap about twice
    the 2-opt."""
    if n > 1000:
        return threads, 1
    if n > 600:
        return 2 * threads, 1
    return 8 * threads, (2 if node_swap else 4)


def reference_swarm(n: int, threads: int) -> int:
    """Particles of the reference arm's oracle swarm: one per host thread for
    the long tours (a generation then costs about one particle's exchange,
    5-30 s at n = 1992), more for short ones."""
    return threads if n > 1000 else (4 * threads if n > 300 else 8 * threads)


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def workload(name: str):
    from paper_1706_04399_gb300 import inputs
    if name == "batched":      # the oracle arm times one member of the batch
        return inputs.batched()[0]
    if name == "serving":      # ... or the first request of the stream
        return inputs.serving(count=1)[0][1]
    if name in ("astar", "two-opt"):  # ... or the facade's swarm
        return inputs.facade()
    return inputs.CONFIGS[name]()


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ----------------------------------------------------------------- CPU oracle

def oracle_sample(inst, swarm: int, warmup: int, generations: int, threads: int, flags=None):
    """Times the oracle on `generations` generations of a `swarm`-particle
    swarm over the same instance, the edge exchange of each particle on one
    of `threads` host threads (the oracle's arithmetic is its plain
    single-threaded C; particles' exchanges are independent); returns
    (value, seconds)."""
    import oracle
    C, _ = oracle.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle.Swarm(C, inst.tags, swarm=swarm, seed=inst.seed,
                      flags=oracle.ALL if flags is None else flags)
    for _ in range(warmup):
        sw.iterate_threaded(threads)
    t0 = time.perf_counter()
    for _ in range(generations):
        sw.iterate_threaded(threads)
    dt = time.perf_counter() - t0
    return swarm * generations / dt, dt


def _oracle_instance_worker(job):
    """One spawned process: the oracle on one instance with `swarm`
    particles for `generations` generations; returns (units, seconds)."""
    inst, swarm, generations = job
    import oracle
    C, _ = oracle.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle.Swarm(C, inst.tags, swarm=swarm, seed=inst.seed)
    t0 = time.perf_counter()
    sw.run(generations)
    return swarm * generations, time.perf_counter() - t0


def oracle_pool_sample(insts, swarm: int, generations: int, procs: int):
    """Times the oracle with one spawned process per host core over the
    instances (each a `swarm`-particle swarm for `generations` generations);
    returns (particle-iterations/s over the wall time, wall seconds).  The
    pool is spawned, not forked, so it may start after CUDA is in use."""
    import multiprocessing as mp
    jobs = [(inst, min(swarm, inst.swarm), generations) for inst in insts]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        got = pool.map(_oracle_instance_worker, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    return sum(u for u, _ in got) / wall, wall


def swarm_config(inst, exchange: str, world: int, steps: int) -> dict:
    """The `config` of a swarm workload's bench line (both arms)."""
    node_swap = exchange == "node-swap"
    return {"workload": f"{inst.name}-{inst.n}vp-{inst.swarm}p" + ("-nodeswap" if node_swap else ""),
            "n": inst.n, "swarm": inst.swarm, "exchange": exchange,
            "generations_timed": steps, "boxes": inst.m,
            "l2": "flushed between timed generations (256 MiB write)",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    inst = workload(args.workload)
    import oracle
    node_swap = args.exchange == "node-swap"
    flags = oracle.ALL | (oracle.NODE_SWAP if node_swap else 0)
    C, _ = oracle.cost_matrix(inst.xyz, inst.boxes)
    threads = cpu_cores()
    swarm = reference_swarm(inst.n, threads)
    sw = oracle.Swarm(C, inst.tags, swarm=swarm, seed=inst.seed, flags=flags)
    for _ in range(args.warmup):
        sw.iterate_threaded(threads)
    per_step = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sw.iterate_threaded(threads)
        per_step.append(time.perf_counter() - t0)
    total = sum(per_step)
    value = swarm * args.steps / total
    sample = (f"{inst.name} instance (n={inst.n}): an oracle swarm of {swarm} particles "
              f"(the workload's is {inst.swarm}) from its own initial swarm, "
              f"{args.warmup} untimed + {args.steps} timed generations, each particle's edge "
              f"exchange on one of {threads} host threads")
    config = swarm_config(inst, args.exchange, args.gpus, args.steps)
    config["sample_swarm"] = swarm
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU helpers

class ClockSampler:
    """nvidia-smi clock / throttle samples every 50 ms while running.  When
    start() / stop() mark a window, summary() keeps the samples whose
    timestamps fall inside it (the process is started earlier, so its start-up
    does not eat a short timed region)."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index: str | None):
        self.index = index
        self.proc = None
        self.window = None
        self.out = os.path.join("/tmp", f"dpso_clocks_{os.getpid()}.csv")

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if self.index is not None:
            cmd += ["-i", self.index]
        try:
            self.fh = open(self.out, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def start(self):
        self.window = [time.time(), None]

    def stop(self):
        if self.window:
            self.window[1] = time.time()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    @staticmethod
    def _stamp(text):
        import datetime
        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        if self.proc is None or not os.path.exists(self.out):
            return None
        rows = []
        with open(self.out) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out)
        total = len(rows)
        if self.window and self.window[1] is not None:
            lo, hi = self.window[0] - 0.05, self.window[1] + 0.05
            stamped = [(self._stamp(r[0]), r) for r in rows]
            if all(t is not None for t, _ in stamped):
                rows = [r for t, r in stamped if lo <= t <= hi]
        rows = [r[1:] for r in rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "samples_under_load": 0, "samples_all": total}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        util = [num(r[7]) for r in rows]
        loaded = [num(r[0]) for r in rows if num(r[7]) is not None and num(r[7]) > 50
                  and num(r[0]) is not None] or sm
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(num(r[1]) or 0 for r in rows),
                "reasons": reasons, "samples": len(rows),
                "samples_under_load": sum(1 for u in util if u is not None and u > 50),
                "samples_all": total,
                "window": "timed region" if self.window else "whole run"}


def gpu_index_for_smi(local_rank: int) -> str | None:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank].strip()
    return str(local_rank)


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def fitness_roofline(dpso, C, n: int, X, stream, workload_name: str, reps: int = 20) -> dict:
    """Times dpso_fitness over the tours X (count x n uint16, host) on `stream`:
    mean CUDA-event duration of `reps` back-to-back launches after three warm-up
    launches (the cost matrix stays L2-resident, as in a generation), against
    the L2 random-gather rate measured by dpso_probe_l2_gather_gbs on a buffer
    of the cost matrix's size (at least 8 MiB)."""
    import numpy as np
    import torch
    count = X.shape[0]
    T = torch.from_numpy(np.ascontiguousarray(X).view(np.int16)).cuda()
    out = torch.empty(count, dtype=torch.int64, device="cuda")
    for _ in range(3):
        dpso.dpso_fitness(C, n, T, count, out, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        dpso.dpso_fitness(C, n, T, count, out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    probe_bytes = max(8 << 20, 4 * n * n)
    peak = dpso.dpso_probe_l2_gather_gbs(probe_bytes, 64, stream)
    algo = 4 * n * count
    achieved = algo / (ms / 1e3) / 1e9
    return {"kernel": "fitness_kernel", "bound": "l2_gather", "bytes_per_launch": algo,
            "tours": count, "ms_per_launch": ms, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak if peak else None,
            "traffic": dram_traffic("fitness_kernel", workload_name),
            "peak_source": f"random 4-byte gathers from an L2-resident {probe_bytes >> 20} MiB "
                           "buffer measured in this run by dpso_probe_l2_gather_gbs "
                           "(best of 5)"}


def dram_traffic(kernel: str, workload_name: str):
    """DRAM bytes per launch of `kernel` on `workload_name` from the committed
    ncu summary, if it was taken from the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        recs = json.load(open(path))["records"]
    except (OSError, ValueError, KeyError):
        return None
    for rec in recs:
        if rec.get("kernel") != kernel or rec.get("workload") != workload_name:
            continue
        try:
            digest = hashlib.sha256(open(os.path.join(ROOT, rec["source"]), "rb").read()).hexdigest()
        except (OSError, KeyError):
            return None
        return rec.get("dram_bytes_per_launch") if rec.get("source_sha256") == digest else None
    return None


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def gpu_line(args):
    import numpy as np
    import torch

    from paper_1706_04399_gb300 import dpso

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    inst = workload(args.workload)
    if args.swarm:                 # a smaller swarm of the same instance (profiling)
        inst = dataclasses.replace(inst, swarm=args.swarm)
    seed = inst.seed + rank        # independent replica per rank
    S, n = inst.swarm, inst.n
    stream = torch.cuda.current_stream()

    xyz = torch.from_numpy(inst.xyz).cuda()
    boxes = torch.from_numpy(inst.boxes).cuda()
    C = torch.empty((n, n), dtype=torch.int32, device="cuda")
    dpso.dpso_cost_matrix(xyz, n, boxes, inst.m, dpso.default_cost_params(), C, stream)
    node_swap = args.exchange == "node-swap"
    flags = dpso.FLAGS_ALL | (dpso.FLAG_NODE_SWAP if node_swap else 0)
    params = dpso.default_params(swarm=S, flags=flags)
    sw = dpso.Swarm(C, n, inst.tags, params, seed, stream)
    sampler = ClockSampler(gpu_index_for_smi(local))
    sampler.__enter__()            # sampling from here; the timed window is marked below
    sw.step(args.warmup, stream)
    torch.cuda.synchronize()
    # timing mode: the same generation graphs, their phase-boundary event
    # nodes pointed at fresh events before every replay (turning it on clears
    # the accumulators, so only the timed generations count)
    sw.set_timing(True)
    st0 = sw.stats()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    sampler.start()
    for k in range(args.steps):
        flush.zero_()                      # evict the L2 between generations
        evs[k][0].record(stream)
        sw.step(1, stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    sampler.stop()
    sampler.__exit__(None, None, None)
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    timing = sw.timing()
    st1 = sw.stats()
    dev_ms_max = max_over_ranks(dev_ms, dist, "cuda")
    value = job_throughput(S * args.steps, world, dev_ms_max)

    pairs = st1["two_opt_pairs"] - st0["two_opt_pairs"]
    evaluated = st1["two_opt_evaluated"] - st0["two_opt_evaluated"]
    moves = st1["two_opt_moves"] - st0["two_opt_moves"]
    two_ms = timing["ms"]["two_opt"]
    launches = sum(timing["launches"].values())
    out = None
    if rank == 0:
        peaks = measured_peaks()
        probes = {f"{mb}MiB": dpso.dpso_probe_l2_read_gbs(mb << 20, max(1, 960 // mb))
                  for mb in (8, 16, 24)}
        l2 = max(probes.values())
        bpp = BYTES_PER_SWAP_PAIR if node_swap else BYTES_PER_PAIR
        # bytes of the pairs the kernel evaluated (a pass skips the rows the
        # last move left unchanged), not of the pairs a plain scan would take
        achieved = bpp * evaluated / (two_ms / 1e3) / 1e9 if two_ms > 0 else 0.0
        traffic = None if node_swap else dram_traffic("two_opt_tiled_kernel", inst.name)
        roofline = {
            "kernel": "node_swap_tiled_kernel" if node_swap else "two_opt_tiled_kernel",
            "bound": "l2", "bytes_per_pair": bpp, "pairs_evaluated": evaluated,
            "achieved": achieved, "peak": l2,
            "unit": "GB/s", "frac": achieved / l2 if l2 else None,
            "traffic": traffic,
            "peak_source": "L2 read bandwidth measured in this run by dpso_probe_l2_read_gbs "
                           "(16-byte loads of an L2-resident buffer, best of 5 runs, best of "
                           "8/16/24 MiB buffers)",
            "l2_probes_gbs": probes,
            "hbm_peak_gbs": peaks.get("hbm_gbs"),
            "frac_of_hbm_peak": achieved / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
        }
        fit_roof = fitness_roofline(dpso, C, n, sw.state()["X"], stream, inst.name)
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            threads = cpu_cores()
            cs, cg = cpu_sample_shape(n, threads, node_swap)
            cval, csec = oracle_sample(inst, cs, 0, cg, threads, flags)
            cpu = {"value": cval, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": f"{inst.name} instance (n={n}), an oracle swarm of {cs} "
                             f"particles from its own initial swarm, generations 1..{cg} "
                             f"({csec:.1f} s; early generations exchange from random "
                             f"tours and cost the oracle more per particle than the timed "
                             f"steady state), each particle's edge exchange on one of "
                             f"{threads} host threads",
                   "host_cores": cpu_cores(), "cpu": cpu_model()}
        e2e = None
        if not args.no_e2e:
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
            hx, hb, ht = pin(inst.xyz), pin(inst.boxes), pin(inst.tags)
            tour = torch.empty(n, dtype=torch.int32).pin_memory()
            import ctypes
            cost = ctypes.c_int64(0)
            cp = dpso.default_cost_params()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc = dpso.lib().dpso_plan(hx.data_ptr(), n, hb.data_ptr(), inst.m, ht.data_ptr(),
                                      ctypes.byref(cp), ctypes.byref(params), seed, args.steps,
                                      ctypes.cast(tour.data_ptr(), ctypes.POINTER(ctypes.c_int32)),
                                      ctypes.byref(cost))
            e2e_s = time.perf_counter() - t0  # dpso_plan runs the same parameters
            if rc != 0:
                raise dpso.DpsoError(rc, "dpso_plan")
            e2e = {"value": S * args.steps / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": int(hx.numel() * 8 + hb.numel() * 8 + ht.numel() * 4),
                   "d2h_bytes_per_step": int(n * 4 + 8),
                   "what": f"dpso_plan: {args.steps} generations from host buffers, including "
                           "cost matrix and initialisation"}
        phases = {k: round(v, 3) for k, v in timing["ms"].items()}
        config = swarm_config(inst, args.exchange, world, args.steps)
        config["timed_path"] = ("dpso_step replaying its generation graphs (timing mode: the "
                                "graphs' phase-boundary event nodes bound to fresh events)")
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": config,
            # the metric's "2-opt moves/s": candidate pairs the kernel evaluated
            "two_opt_pairs_evaluated_per_s": evaluated / (two_ms / 1e3) if two_ms > 0 else 0.0,
            "two_opt_pairs_evaluated": evaluated,
            # what a plain best-improvement scan of the same passes would take
            "two_opt_plain_scan_pairs": pairs,
            "two_opt_plain_scan_pairs_per_s": pairs / (two_ms / 1e3) if two_ms > 0 else 0.0,
            "two_opt_moves_applied": moves,
            "phase_ms": phases, "wall_s": wall,
            "roofline": roofline, "fitness_roofline": fit_roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": sampler.summary(),
            "gbest_cost_mm": st1["gbest_cost"],
        }
    sw.close()
    if dist:
        dist.destroy_process_group()
    return out


# ------------------------------------------------ batched and served workloads

def _same_state(a: dict, b: dict) -> bool:
    import numpy as np
    keys = ("X", "V", "P", "G", "F", "PF", "history")
    return all(np.array_equal(a[k], b[k]) for k in keys) and (a["t"], a["gf"]) == (b["t"], b["gf"])


def shard(items, rank: int, world: int):
    """The items rank `rank` of `world` takes: every world-th, from its rank
    (instances are independent, so no collective is needed)."""
    return items[rank::world]


def batched_line(args):
    """Independent instances of uneven size advanced together by dpso_batch_*
    (one set of launches per generation for all of them) against the same
    instances stepped one launch sequence per instance; both from the same
    initial swarms, so their trajectories must be identical."""
    import torch

    from paper_1706_04399_gb300 import dpso, inputs

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    all_insts = inputs.batched()[: args.instances]
    insts = shard(all_insts, rank, world)
    stream = torch.cuda.current_stream()
    Cs = []
    for inst in insts:
        C = torch.empty((inst.n, inst.n), dtype=torch.int32, device="cuda")
        boxes = torch.from_numpy(inst.boxes.reshape(-1, 6)).cuda() if inst.m else None
        dpso.dpso_cost_matrix(torch.from_numpy(inst.xyz).cuda(), inst.n, boxes, inst.m,
                              dpso.default_cost_params(), C, stream)
        Cs.append(C)

    def swarms():
        return [dpso.Swarm(C, i.n, i.tags, dpso.default_params(swarm=i.swarm), i.seed, stream)
                for C, i in zip(Cs, insts)]

    together, alone = swarms(), swarms()
    batch = dpso.Batch(together, stream)
    # the launch classes take their default shapes (from steady-state sweeps)
    # unless --autotune asks dpso_batch_autotune to time the shapes that fit
    rows, tpc, tg = batch.autotune(stream) if args.autotune else (0, 0, 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def run(step_fn, steps, per_step=None):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            step_fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in evs]
        if per_step is not None:
            per_step.extend(ms)
        return sum(ms)

    def solo_step():
        for sw in alone:
            sw.step(1, stream)

    batch.step(args.warmup, stream)
    for sw in alone:
        sw.step(args.warmup, stream)
    torch.cuda.synchronize()
    st0 = [sw.stats() for sw in together]
    sampler = ClockSampler(gpu_index_for_smi(local))
    if dist:
        dist.barrier()
    gen_ms = []
    with sampler:
        sampler.start()
        ms_batch = max_over_ranks(run(lambda: batch.step(1, stream), args.steps, gen_ms), dist,
                                  "cuda")
        sampler.stop()
        if dist:
            dist.barrier()
        ms_solo = max_over_ranks(run(solo_step, args.steps), dist, "cuda")
    st1 = [sw.stats() for sw in together]
    identical = all(_same_state(a.state(), b.state()) for a, b in zip(together, alone))
    pairs = sum(b["two_opt_pairs"] - a["two_opt_pairs"] for a, b in zip(st0, st1))
    S_job = sum(i.swarm for i in all_insts)  # every rank's particles
    value = S_job * args.steps / (ms_batch / 1e3)
    solo_value = S_job * args.steps / (ms_solo / 1e3)
    if dist:
        t = torch.tensor([1.0 if identical else 0.0], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        identical = bool(t.item() == 1.0)
    batch.close()
    for sw in together + alone:
        sw.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return None
    ns = [i.n for i in all_insts]
    import numpy as np
    gm = np.array(gen_ms)
    T = all_insts[0].iterations
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        procs = cpu_cores()
        sample = all_insts[::8]
        cval, csec = oracle_pool_sample(sample, 2, 1, procs)
        cpu = {"value": cval, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{len(sample)} of the {len(all_insts)} instances (every 8th), each an "
                         f"oracle swarm of 2 particles for its first generation, one spawned "
                         f"process per host core ({csec:.1f} s wall)",
               "cpu": cpu_model()}
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batch / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": {"workload": f"batched-{len(all_insts)}", "instances": len(all_insts),
                   "parallelism": f"instances sharded over {world} GPU(s), no collective",
                   "n_min": min(ns), "n_max": max(ns), "swarm_total": S_job,
                   "l2": "flushed between timed generations (256 MiB write)"},
        "batched": {"one_per_launch_value": solo_value, "speedup": value / solo_value,
                    "one_per_launch_ms_per_step": ms_solo / args.steps,
                    "identical_states": identical,
                    "two_opt_shapes": (f"autotuned; last class ({rows}, {tpc}, {tg})" if args.autotune
                                       else "each class's default shape"),
                    "two_opt_pairs_per_s_over_step": pairs / (ms_batch / 1e3),
                    # every member advances one generation per replay of the
                    # batch graph: a generation's latency is the latency of
                    # each member's step, and a member's solve of T
                    # generations finishes with the batch
                    "generation_latency_ms": {"p50": float(np.percentile(gm, 50)),
                                              "p99": float(np.percentile(gm, 99)),
                                              "max": float(gm.max())},
                    "instance_solve_latency_s": {
                        "generations": T,
                        "p50": float(np.percentile(gm, 50)) * T / 1e3,
                        "p99": float(np.percentile(gm, 99)) * T / 1e3,
                        "what": "T generations at the measured per-generation p50 / p99"}},
        "gpu_launches": None, "roofline": None, "cpu_baseline": cpu, "e2e": None,
        "clocks": sampler.summary(),
    }


def serving_line(args):
    """A Poisson stream of re-planning requests served by dpso_server_* with
    continuous batching, against the same requests solved one at a time
    (dpso_plan); tours must be identical."""
    import numpy as np
    import torch

    from paper_1706_04399_gb300 import dpso, inputs

    torch.cuda.set_device(0)
    # the stream's requests with at most --max-n viewpoints, arrival times kept
    full = inputs.serving()
    stream_reqs = [r for r in full if r[1].n <= args.max_n][: args.requests]
    cp = dpso.default_cost_params()
    params = [dpso.default_params(swarm=inst.swarm) for _, inst in stream_reqs]
    # one request alone first: loads the kernels so neither arm pays for it
    _, w = stream_reqs[0]
    dpso.dpso_plan(w.xyz, w.boxes, w.tags, cp, params[0], w.seed, 1)

    policy = dpso.SERVE_SHORTEST_FIRST if args.policy == "shortest" else dpso.SERVE_ARRIVAL_ORDER
    server = dpso.Server(dpso.default_server_params(max_active=args.max_active, policy=policy,
                                                    lanes=args.lanes))
    sampler = ClockSampler(gpu_index_for_smi(0))
    ids = []
    with sampler:
        t0 = time.perf_counter()
        for (arrival, inst), p in zip(stream_reqs, params):
            delay = arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(server.submit(inst.xyz, inst.boxes, inst.tags, cp, p, inst.seed,
                                     inst.iterations))
        results = []
        for rid in ids:
            if server.wait(rid, 3600.0) != 1:
                raise RuntimeError(f"request {rid} failed: {server.poll(rid)[0]}")
            results.append(server.poll(rid))
        served_s = time.perf_counter() - t0
    sstats = server.stats()
    server.close()
    lat = np.array([r[3] for r in results])

    t1 = time.perf_counter()
    solo = [dpso.dpso_plan(inst.xyz, inst.boxes, inst.tags, cp, p, inst.seed, inst.iterations)
            for (_, inst), p in zip(stream_reqs, params)]
    solo_s = time.perf_counter() - t1
    identical = all(r[2] == c and np.array_equal(r[1], t) for r, (t, c) in zip(results, solo))
    units = sum(inst.swarm * inst.iterations for _, inst in stream_reqs)
    ns = [inst.n for _, inst in stream_reqs]
    rate = len(stream_reqs) / stream_reqs[-1][0]
    return {
        "metric": METRIC, "value": units / served_s, "unit": UNIT, "n_gpus": 1,
        "steps": len(stream_reqs), "warmup": 1, "ms_per_step": 1000 * served_s / len(stream_reqs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
        "data": "synthetic",
        "config": {"workload": f"serving-{len(stream_reqs)}req-n{args.max_n}",
                   "requests": len(stream_reqs), "offered_rate_hz": rate,
                   "stream": f"first {len(stream_reqs)} requests with n <= {args.max_n} of the "
                             f"{len(full)}-request Poisson stream (200 req/s, n log-uniform "
                             "50..3000), arrival times kept",
                   "n_min": min(ns), "n_max": max(ns),
                   "swarm": stream_reqs[0][1].swarm, "iterations": stream_reqs[0][1].iterations,
                   "l2": "inputs per request exceed L2 in aggregate; no flush"},
        "serving": {"requests_per_s": len(stream_reqs) / served_s,
                    "p50_latency_s": float(np.percentile(lat, 50)),
                    "p99_latency_s": float(np.percentile(lat, 99)),
                    "max_latency_s": float(lat.max()),
                    "one_per_launch_requests_per_s": len(stream_reqs) / solo_s,
                    "speedup": solo_s / served_s, "identical_tours": identical,
                    "peak_active": sstats["peak_active"], "ticks": sstats["ticks"],
                    "policy": args.policy, "max_active": args.max_active,
                    "lanes": args.lanes},
        "gpu_launches": None, "roofline": None, "cpu_baseline": None,
        "e2e": {"value": units / served_s, "unit": UNIT,
                "h2d_bytes_per_step": int(np.mean([i.xyz.nbytes + i.boxes.nbytes + i.tags.nbytes
                                                   for _, i in stream_reqs])),
                "d2h_bytes_per_step": int(np.mean([4 * i.n + 8 for _, i in stream_reqs])),
                "what": "requests submitted from host buffers, tours read back; a step is one "
                        "request"},
        "clocks": sampler.summary(),
    }


def astar_line(args):
    """A* edge costs (Sec. 2.2) for every viewpoint pair of the facade or
    bridge workload on a 0.5 m voxel grid with its boxes inflated by a 0.5 m
    UAV: occupancy plus the full matrix per step."""
    import numpy as np
    import torch

    from paper_1706_04399_gb300 import dpso, inputs

    torch.cuda.set_device(0)
    inst = inputs.CONFIGS[args.astar_instance]()
    voxel = 0.5
    origin, dims = inputs.voxel_grid(inst, voxel)
    ap = dpso.astar_params(origin, voxel, dims, inflate_r2=inputs.inflate_r2(0.5, voxel),
                           unit_mm=int(round(1000 * voxel)))
    n = inst.n
    npairs = n * (n - 1) // 2
    stream = torch.cuda.current_stream()
    xyz = torch.from_numpy(inst.xyz).cuda()
    boxes = torch.from_numpy(inst.boxes).cuda()
    occ = torch.empty(int(np.prod(dims)), dtype=torch.uint8, device="cuda")
    C = torch.empty((n, n), dtype=torch.int32, device="cuda")

    def step():
        dpso.dpso_voxel_occupancy(boxes, inst.m, ap, occ, stream)
        dpso.dpso_cost_matrix_astar(xyz, n, occ, ap, C, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = ClockSampler(gpu_index_for_smi(0))
    with sampler:
        for k in range(args.steps):
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    Cn = C.cpu().numpy()
    blocked = int((Cn == ap.blocked_cost).sum() // 2)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        k = min(n, 400)  # the whole facade matrix; the first 400 viewpoints of the bridge
        occ_ref = oracle.voxel_occupancy(origin, voxel, dims, inst.boxes, ap.inflate_r2)
        t0 = time.perf_counter()
        Cref, _ = oracle.cost_matrix_astar(inst.xyz[:k], occ_ref, origin, voxel, dims,
                                           unit_mm=ap.unit_mm, blocked_cost=ap.blocked_cost,
                                           max_expansions=ap.max_expansions)
        csec = time.perf_counter() - t0
        cpu = {"value": k * (k - 1) / 2 / csec, "unit": "viewpoint-pairs/s", "cores": 1,
               "kind": "oracle", "sample": f"A* matrix of the first {k} viewpoints ({csec:.2f} s)",
               "matches_gpu": bool(np.array_equal(Cref, Cn[:k, :k])), "cpu": cpu_model()}
    return {
        "metric": METRIC, "value": npairs / (ms / 1e3), "unit": "viewpoint-pairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32/f64", "data": "synthetic",
        "config": {"workload": f"astar-{inst.name}-{n}vp", "n": n, "voxel_m": voxel,
                   "grid": [int(v) for v in dims], "inflate_r2": ap.inflate_r2,
                   "weights": list(ap.weights), "max_expansions": ap.max_expansions,
                   "blocked_pairs": blocked,
                   "l2": "inputs rebuilt every step (occupancy and matrix)"},
        "gpu_launches": None, "roofline": None, "cpu_baseline": cpu, "e2e": None,
        "clocks": sampler.summary(),
    }


def two_opt_line(args):
    """Standalone edge exchange: dpso_two_opt over `--tours` random tours of the
    facade or bridge instance, each taken through at most `--max-moves` moves
    (0: to 2-optimality), timed with CUDA events per call.  A small, bounded
    case of the swarm's 2-opt kernel shapes (the launch shape follows the tour
    count), e.g. for ncu captures."""
    import numpy as np
    import torch

    from paper_1706_04399_gb300 import dpso, inputs

    inst = inputs.CONFIGS[args.two_opt_instance]()
    n = inst.n
    stream = torch.cuda.current_stream()
    C = torch.empty((n, n), dtype=torch.int32, device="cuda")
    dpso.dpso_cost_matrix(torch.from_numpy(inst.xyz).cuda(), n, torch.from_numpy(inst.boxes).cuda(),
                          inst.m, dpso.default_cost_params(), C, stream)
    tours = inputs.random_tours(n, args.tours, 5)
    cost = torch.empty(args.tours, dtype=torch.int64, device="cuda")
    ms, pairs, moves = [], 0, 0
    for k in range(args.warmup + args.steps):
        T = torch.from_numpy(tours.view(np.int16).copy()).cuda()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pairs, moves = dpso.dpso_two_opt(C, n, T, args.tours, cost, args.max_moves, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms.append(e0.elapsed_time(e1))
    mean = sum(ms) / len(ms)
    return {
        "metric": METRIC, "value": pairs / (mean / 1e3), "unit": "2-opt candidate pairs/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
        "data": "synthetic",
        "config": {"workload": f"two-opt-{inst.name}-{n}vp-{args.tours}tours",
                   "n": n, "tours": args.tours, "max_moves": args.max_moves,
                   "what": "dpso_two_opt on the same random tours each step (plain-scan pairs)",
                   "l2": "cost matrix L2-resident after the first call"},
        "two_opt_pairs": pairs, "two_opt_moves_applied": moves,
        "gpu_launches": None, "roofline": None, "cpu_baseline": None, "e2e": None,
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default by workload: bridge 20, facade 100, ...)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="bridge",
                    choices=["tiny", "facade", "bridge", "batched", "serving", "astar",
                             "two-opt"])
    ap.add_argument("--astar-instance", default="facade", choices=["facade", "bridge"],
                    help="astar: whose viewpoints and boxes")
    ap.add_argument("--two-opt-instance", default="bridge", choices=["facade", "bridge"],
                    help="two-opt: whose cost matrix")
    ap.add_argument("--tours", type=int, default=152, help="two-opt: random tours per call")
    ap.add_argument("--max-moves", type=int, default=30, help="two-opt: move cap per tour")
    ap.add_argument("--instances", type=int, default=256, help="batched: instances")
    ap.add_argument("--autotune", action="store_true",
                    help="batched: dpso_batch_autotune the launch classes' shapes")
    ap.add_argument("--requests", type=int, default=48, help="serving: requests")
    ap.add_argument("--max-n", type=int, default=400, help="serving: largest request taken")
    ap.add_argument("--policy", default="arrival", choices=["arrival", "shortest"],
                    help="serving: admission order")
    ap.add_argument("--max-active", type=int, default=16, help="serving: running requests at most")
    ap.add_argument("--lanes", type=int, default=4,
                    help="serving: size-class lanes (1: one lock-step batch)")
    ap.add_argument("--exchange", default="2-opt", choices=["2-opt", "node-swap"],
                    help="edge exchange of the swarm workloads")
    ap.add_argument("--swarm", type=int, default=0,
                    help="bridge/facade/tiny: particles instead of the workload's (small "
                         "profiling cases; the bench line then names that swarm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args(argv)
    if args.steps is None:
        args.steps = DEFAULT_STEPS.get(args.workload, 20)
    if args.warmup < 3 and args.impl == "gb300":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        out = batched_line(args)
    elif args.workload == "serving":
        out = serving_line(args)
    elif args.workload == "astar":
        out = astar_line(args)
    elif args.workload == "two-opt":
        out = two_opt_line(args)
    else:
        out = gpu_line(args)
    if out is not None:
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
