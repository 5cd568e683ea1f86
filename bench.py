#!/usr/bin/env python
"""Benchmark of the RIS hot path (GreediRIS, arXiv 2408.10982) on GB300.

One step = the whole hot path over one batch of synthetic input:
  RRR sampling of theta sets (im_sample_rrr: walk kernel, scan, per-set sort)
  -> covering-subset index (histogram, scan, scatter)
  -> plain greedy max-k-cover                        (im_max_k_cover, greedy)
  -> RandGreedi: 148 vertex parts, lazy local greedy, then the streaming
     threshold buckets over the first ceil(k/4) local seeds of every part,
     counted for all buckets at once over per-set bucket masks
                                                     (im_max_k_cover, RandGreedi)
Workload: R-MAT scale 20 (1,048,576 vertices, 16,777,216 edges, a/b/c/d =
0.57/0.19/0.19/0.05, seed 42), LT weights 1/in-degree quantised to uint32,
theta = 4,194,304, k = 100, delta = 0.077.

`value` is RRR edges examined per second over whole steps (the in-edges a
cumulative-weight scan would decide over, identical to the oracle's count;
the GPU walk does not read them -- a division by the vertex's common in-weight
(or one 16-byte cut point) decides each step --
so `walk_steps_per_s` and `roofline` give its real rate), with the graph
resident in HBM.  `e2e` is the same metric through the C ABI
from pinned host arrays: graph upload, LT index build, sampling, both covers
and the read-back of seeds every step.

Beside the step, the line carries three sections measured after it:
`batched` (256 queries of the batched mix in one im_solve_batch call against
the one-query path), `served` (Poisson arrivals at 200/s through im_server
against the one-query path as a FIFO server: q/s, p50/p99 latency) and `ic`
(IC sampling on the LiveJournal-shaped graph).

--impl reference runs the CPU oracle (oracle/, the plain definition) on a
bounded sample of the same workload on rank 0.

Multi-GPU: one process per GPU; every rank runs its own replica with its own
disjoint sample ids (weak scaling, no data-path collective; the path's only
exchange step is not needed when ranks solve independent problems).
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

from paper_2408_10982_gb300 import inputs  # noqa: E402

THETA = 4_194_304
K = 100
PARTS = 148
ALPHA = (1, 4)
DELTA = 0.077
SEED = 42
SERVE_WORKERS = 3            # im_server workers in the served section
SERVE_HEAVY = 1 << 24        # its heavy lane: requests of >= 2^24 estimated RRR members
METRIC = "RRR edges/s + max-k-cover ms (HBM %); served q/s, p50/p99 vs plain; bit-exact"
WORKLOAD = ("rmat20-lt: R-MAT scale 20 (1,048,576 vertices, 16,777,216 edges, a/b/c=0.57/0.19/0.19, "
            "seed 42), LT 1/in-degree as uint32, theta=4,194,304 RRR sets, k=100; plain greedy "
            "+ RandGreedi (148 partitions, streamed top ceil(k/4), delta=0.077)")
# DRAM bytes per launch from an ncu capture, valid while the kernel source is
# unchanged (sha256 of the kernel's source text, see kernel_sha).  k_sample_lt1 was captured on
# the same graph at theta = 1,048,576 (42.82 M walk steps, 2.5637 GB read +
# written, profiles/ncu_sample_lt1_rmat20_theta1M.txt); traffic grows with the
# walk steps, so a full launch (171.49 M steps) moves 2.5637 * 171.49 / 42.82 GB.
TRAFFIC: dict = {"sample_lt": {"src_sha": "5dfa6a69246f81f9",
                               "bytes_per_launch": int(2.5637e9 * 171.49 / 42.82)}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--theta", type=int, default=THETA, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--rg-fused", type=int, default=0,
                    help="RandGreedi as one cooperative launch (1) or two launches (0)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the IC, batched and served sections")
    ap.add_argument("--served-no-orkut", action="store_true",
                    help="serve the batched mix alone, without the 5%% Orkut-shaped queries")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def replica_first_id(rank: int, theta: int) -> int:
    """Weak scaling: rank r solves its own replica over sample ids
    [r theta, (r + 1) theta), disjoint from every other rank's."""
    return rank * theta


def max_over_ranks(x: float, dist, device=None) -> float:
    """The slowest rank's time (the job's time); x itself on one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region:
    the sampler is running (its first line read) before the region starts,
    every line is stamped when it arrives, and only the lines stamped inside
    the region are summarised."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[tuple[float, str]] = []

    def start(self, wait_s: float = 10.0):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t_end = time.perf_counter() + wait_s
        while not self.lines and self.proc.poll() is None and time.perf_counter() < t_end:
            time.sleep(0.005)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t0: float, t1: float) -> dict:
        """Summary of the samples stamped in [t0, t1] (host perf_counter times
        of the timed region's start and end)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(self.INTERVAL_MS / 1000.0)  # the sample that closes the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        inside = [ln for t, ln in self.lines if t0 <= t <= t1 + self.INTERVAL_MS / 1000.0]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "interval_ms": self.INTERVAL_MS}


def kernel_sha(file: str, kernel: str) -> str:
    """sha256 of one kernel's source text (from its __global__ line to the
    brace that closes its body), so an ncu capture stays tied to that kernel
    and not to unrelated edits of the same file."""
    import hashlib
    text = open(os.path.join(ROOT, "paper_2408_10982_gb300", "csrc", file)).read()
    start = text.index(kernel + "(")
    start = text.rindex("__global__", 0, start)
    depth, i = 0, text.index("{", start)
    while True:
        if text[i] == "{":
            depth += 1
        elif text[i] == "}":
            depth -= 1
            if depth == 0:
                break
        i += 1
    return hashlib.sha256(text[start:i + 1].encode()).hexdigest()[:16]


# ---------------------------------------------------------------------------
# CPU oracle (the reference arm, and the cpu_baseline of our arm)
# ---------------------------------------------------------------------------

def oracle_step(g, first: int, count: int, sampler=None):
    """Oracle over a bounded sample: sample, covering subsets, both covers.
    With a sampler (oracle/parallel.py) the sampling is split by sample id
    over its worker processes (the same sets); the covering subsets and both
    covers stay single-threaded (the plain definitions).  Returns the total
    time, the pool and the sampling time."""
    import oracle as O
    t0 = time.perf_counter()
    if sampler is not None:
        pool = sampler.sample(O.LT, SEED, first, count)
    else:
        pool = O.sample(O.LT, g, SEED, first, count)
    t_samp = time.perf_counter() - t0
    inv = O.invert(g.n, pool)
    O.greedy(g.n, pool, inv, K)
    O.randgreedi(g.n, pool, inv, K, PARTS, SEED, O.trunc_count(K, *ALPHA), DELTA)
    return time.perf_counter() - t0, pool, t_samp


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    g = inputs.graph_lt_scale20(SEED)
    from oracle import parallel as OP
    cores = host_cores()
    count = 65536
    total_t, total_e = 0.0, 0
    with OP.Sampler(g, cores) as sampler:
        for w in range(args.warmup):
            oracle_step(g, w * count, count, sampler)
        for s in range(args.steps):
            dt, pool, _ = oracle_step(g, (args.warmup + s) * count, count, sampler)
            total_t += dt
            total_e += pool.examined
    value = total_e / total_t
    sample = (f"{count} LT RRR sets per step (of {THETA}), sampled over {cores} worker "
              f"processes, plus their index, plain greedy k={K} and RandGreedi P={PARTS} "
              f"single-threaded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2408_10982_gb300 import build, im
    build.build_library()
    theta = args.theta
    first = replica_first_id(rank, theta)        # disjoint sample ids per replica
    g = inputs.graph_lt_scale20(SEED)
    G = im.Graph(g)
    cap = theta * 64
    pool = im.Pool(G, theta, cap)
    opts_rg = im.cover_opts(im.IM_RANDGREEDI, PARTS, ALPHA, DELTA, SEED, fused=bool(args.rg_fused))
    dev = torch.device("cuda", local)
    # launch-shape knobs (results never depend on them) picked by timing a probe
    tuned = im.im_autotune(G.handle, im.IM_LT, SEED, theta, K, opts_rg)   # probe: the full workload
    out = dict(seeds=torch.zeros(K, dtype=torch.int32, device=dev),
               gains=torch.zeros(K, dtype=torch.int64, device=dev),
               ns=torch.zeros(1, dtype=torch.int32, device=dev),
               cov=torch.zeros(1, dtype=torch.int64, device=dev))
    stream = torch.cuda.current_stream()

    def step():
        pool.reset()
        pool.sample(im.IM_LT, SEED, first, theta)
        im.im_max_k_cover(pool.handle, K, None, out["seeds"], out["gains"], out["ns"],
                          out["cov"], stream)
        im.im_max_k_cover(pool.handle, K, opts_rg, out["seeds"], out["gains"], out["ns"],
                          out["cov"], stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    _, total, examined = pool.info()
    sbytes = pool.sample_bytes()

    im.im_profile_reset()
    im.im_profile_enable(True)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    nvtx = getattr(torch.cuda, "nvtx", None)
    if nvtx:
        nvtx.range_push("timed")             # lets ncu select the timed launches (--nvtx)
    t_region = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    if nvtx:
        nvtx.range_pop()
    torch.cuda.synchronize()
    t_region_end = time.perf_counter()
    if dist:
        dist.barrier()
    clk = clocks.stop(t_region, t_region_end)
    im.im_profile_enable(False)
    prof = im.im_profile_read()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    ms_step = elapsed_ms / args.steps
    value = world * examined / (ms_step / 1000.0)

    # per-kernel times (CUDA events on the launching stream, timed region)
    per = {k: (n / args.steps, ms / args.steps) for k, (n, ms) in prof.items()}
    launches = sum(n for n, _ in prof.values())
    plain_ms = per.get("greedy", (0, 0))[1]
    rg_ms = sum(v[1] for k, v in per.items() if k.startswith("randgreedi") or
                k.startswith("partition") or k == "max_subset_size")
    hbm, peak_kind = measured_peaks()
    samp_name = "sample_lt"
    samp_launch_ms = per[samp_name][1] / max(per[samp_name][0], 1)
    achieved = sbytes / (samp_launch_ms / 1000.0) / 1e9
    dominant = max(per.items(), key=lambda kv: kv[1][1])[0]
    traffic = None
    tr = TRAFFIC.get(samp_name)
    if tr and tr["src_sha"] == kernel_sha("sample.cu", "k_sample_lt1"):
        traffic = tr["bytes_per_launch"]
    roofline = {"kernel": samp_name, "bound": "hbm", "achieved": round(achieved, 1),
                "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "peak_kind": f"{peak_kind} hbm_gbs (copy, burst)", "traffic": traffic,
                "traffic_over_alg": round(traffic / sbytes, 3) if traffic else None,
                "alg_bytes_per_launch": sbytes,
                "alg_bytes": "the walk kernel's own loads and stores, counted by the kernel: "
                             "per step a 16 B vertex record, then the 4 B source of the "
                             "picked in-edge when the vertex's in-edges weigh the same, else "
                             "a 16 B cut point (+ 8 B per search probe when the draw lies "
                             "past it); 4 B per member, 12 B per set",
                "launch_ms": round(samp_launch_ms, 4),
                "walk_steps_per_launch": total,
                "dominant_kernel": dominant,
                "share": round(per[samp_name][1] / ms_step, 4)}

    line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "theta_per_gpu": theta,
                       "l2": "inputs larger than L2 (graph + LT index 277 MB, pool 1.4 GB)",
                       "parallelism": f"replicas x{world}",
                       "tuned": {k2: v for k2, v in tuned.items() if k2 != "ms"}},
            "value_note": "examined edges = the in-edges a cumulative-weight scan would "
                          "decide over (the oracle's count, identical); the GPU walk does "
                          "not read them: one division by the common in-weight (or one "
                          "16-byte cut point) decides each step; walk_steps_per_s is the "
                          "walk's own rate",
            "sets_per_s": world * theta / (ms_step / 1000.0),
            "entries_per_s": world * total / (ms_step / 1000.0),
            "walk_steps_per_s": world * total / (ms_step / 1000.0),
            "max_k_cover_ms": {"plain_greedy": round(plain_ms, 3),
                               "randgreedi": round(rg_ms, 3)},
            "phase_ms": {k: round(v[1], 3) for k, v in sorted(per.items())},
            "gpu_launches": launches, "roofline": roofline, "clocks": clk}

    pool_stats = cover_stats(im, pool, g.n, theta, K, opts_rg)
    cover_paths = bench_cover_paths(im, pool, opts_rg) if not args.no_extras else None
    spread = bench_spread(im, torch, G, pool, g.n, theta) if not args.no_extras else None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["bit_exact"], line["cpu_baseline"] = cpu_baseline_and_check(g, pool, first)
    if not args.no_e2e:
        line["e2e"] = e2e(args, g, im, torch, dev, stream, first, dist)
    pool.close()
    G.close()
    line["kernels"] = kernel_rooflines(im, pool_stats, per, hbm)
    if spread:
        line["spread"] = spread
    if cover_paths:
        line["cover_paths"] = cover_paths
    if not args.no_extras:
        line["batched"] = bench_batched(im, torch)
        line["served"] = bench_served(im, torch, not args.served_no_orkut)
        lj = inputs.graph_livejournal_like_both(SEED)
        line["ic"] = bench_ic(im, torch, lj["trivalency"])
        line["imm"] = bench_imm(im, torch, lj["wc"])
        del lj
        line["paper_weights"] = bench_paper_weights(im, torch)
        line["opim"] = bench_opim(im, torch)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def cpu_baseline_and_check(g, pool, first):
    """Time the oracle on a bounded sample (same graph, first ids of this
    step) at one thread and with its sampling spread over every host core,
    and check the GPU's sets for those ids bit for bit."""
    import oracle as O
    from oracle import parallel as OP
    O.build()
    count = 262144
    cores = host_cores()
    dt1, ref, ts1 = oracle_step(g, first, count)
    if cores > 1:
        with OP.Sampler(g, cores) as sampler:
            oracle_step(g, first, 4 * cores, sampler)          # workers up and loaded
            dtn, refn, tsn = oracle_step(g, first, count, sampler)
    else:
        dtn, refn, tsn = dt1, ref, ts1
    set_off, members = pool.export()
    exact = (np.array_equal(set_off[: count + 1], ref.set_off) and
             np.array_equal(members[: ref.set_off[-1]], ref.members) and
             np.array_equal(refn.set_off, ref.set_off) and
             np.array_equal(refn.members, ref.members))
    sample = (f"{count} LT RRR sets (ids {first}..{first + count - 1} of {THETA}) with their "
              f"index, plain greedy k={K} and RandGreedi P={PARTS}; sampling over {cores} "
              f"worker processes, index and covers single-threaded")
    return bool(exact), {"value": ref.examined / dtn, "unit": "edges/s", "cores": cores,
                         "kind": "oracle", "sample": sample, "seconds": round(dtn, 2),
                         "sampling_seconds": round(tsn, 2),
                         "single_thread": {"value": ref.examined / dt1, "unit": "edges/s",
                                           "cores": 1, "seconds": round(dt1, 2),
                                           "sampling_seconds": round(ts1, 2)}}


def e2e(args, g, im, torch, dev, stream, first, dist):
    """Same metric through the C ABI from pinned host buffers, copies included."""
    pin = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
           for k, a in (("in_off", g.in_off), ("in_src", g.in_src), ("w", g.w))}
    res = {k: torch.zeros(sz, dtype=dt).pin_memory() for k, sz, dt in
           (("seeds", K, torch.int32), ("gains", K, torch.int64), ("ns", 1, torch.int32),
            ("cov", 1, torch.int64))}
    opts_rg = im.cover_opts(im.IM_RANDGREEDI, PARTS, ALPHA, DELTA, SEED, fused=bool(args.rg_fused))
    steps = max(1, min(args.steps, 10))
    examined = 0

    def one():
        nonlocal examined
        gh = im.im_graph_create(pin["in_off"], pin["in_src"], pin["w"], g.n, g.m, stream)
        ph = im.im_pool_create(gh, args.theta, args.theta * 64)
        im.im_sample_rrr(gh, im.IM_LT, SEED, first, args.theta, ph, stream)
        for o in (None, opts_rg):
            im.im_max_k_cover(ph, K, o, res["seeds"], res["gains"], res["ns"], res["cov"], stream)
        examined = im.im_pool_info(ph)[2]
        im.im_pool_destroy(ph)
        im.im_graph_destroy(gh)

    one()                                   # warm-up
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    dt = max_over_ranks((time.perf_counter() - t0) / steps, dist, dev)
    world = dist.get_world_size() if dist else 1
    h2d = 8 * (g.n + 1) + 4 * g.m + 4 * g.m
    d2h = 2 * (4 * K + 8 * K + 4 + 8)
    return {"value": world * examined / dt, "unit": "edges/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": round(1000 * dt, 3), "steps": steps}


# ---------------------------------------------------------------------------
# per-kernel rooflines
# ---------------------------------------------------------------------------

def cover_stats(im, pool, n, theta, k, opts_rg):
    """Counts the algorithmic-byte formulas of the index and cover kernels need:
    T, sum over the greedy's seeds of |S(v)|, sum over the sets it covers of
    |R(i)| and their number, and the RandGreedi producers' scanned entries."""
    set_off, _ = pool.export()
    vtx_off, set_ids = pool.index()
    c = pool.cover(k)
    sizes = np.diff(set_off)
    seeds = c.seeds.astype(np.int64)
    s_seed = int(np.sum(vtx_off[seeds + 1] - vtx_off[seeds]))
    covered = np.unique(np.concatenate([set_ids[vtx_off[v]:vtx_off[v + 1]] for v in seeds])) \
        if len(seeds) else np.zeros(0, np.int64)
    pool.cover(k, opts_rg)
    st = im.im_randgreedi_stats(pool.handle, PARTS, 63)
    return {"T": int(set_off[-1]), "n": n, "theta": theta, "k": k, "s_seed": s_seed,
            "covered": int(covered.size), "r_covered": int(np.sum(sizes[covered])),
            "rg_eval": int(st[:PARTS, 4].sum()), "rg_cover": int(st[:PARTS, 5].sum())}


def bench_cover_paths(im, pool, opts_rg):
    """The other max-k-cover paths on the step's pool (after the timed region):
    the standard greedy by its counts-decrement kernel and by the lazy kernel
    (Alg. 2) at two widths -- the same seeds -- and RandGreedi with Alg. 4's
    non-streaming global step next to the streaming one.  Kernel time per
    cover (CUDA events, mean of 3), coverage, and the lazy kernel's counters."""
    paths = [("greedy_counts", 0, None),
             ("greedy_lazy_w8", 8, im.cover_opts(im.IM_GREEDY_LAZY)),
             ("greedy_lazy_w32", 32, im.cover_opts(im.IM_GREEDY_LAZY)),
             ("randgreedi_stream", 0, opts_rg),
             ("randgreedi_naive", 16, im.cover_opts(im.IM_RANDGREEDI, PARTS, ALPHA, DELTA, SEED,
                                                    fused=False, aggregator=im.IM_AGG_GREEDY))]
    out, ref = {}, None
    for name, width, opts in paths:
        im.im_tune_set(im.IM_TUNE_GREEDY_EVALS, width)
        pool.cover(K, opts)                              # warm-up
        im.im_profile_reset()
        im.im_profile_enable(True)
        for _ in range(3):
            c = pool.cover(K, opts)
        im.im_profile_enable(False)
        prof = im.im_profile_read()
        ms = sum(v[1] for v in prof.values()) / 3
        e = {"kernel_ms": round(ms, 3), "coverage": int(c.coverage), "seeds": int(len(c.seeds)),
             "kernels": {k2: round(v[1] / 3, 3) for k2, v in sorted(prof.items())}}
        if name == "greedy_counts":
            ref = c
        elif name.startswith("greedy_lazy"):
            e["same_as_counts"] = bool(c.seeds.tolist() == ref.seeds.tolist() and
                                       c.coverage == ref.coverage)
        if "lazy" in name or "naive" in name:
            e["lazy_stats"] = im.im_greedy_stats(pool.handle)
        out[name] = e
    im.im_tune_set(im.IM_TUNE_GREEDY_EVALS, 0)
    return out


def kernel_rooflines(im, cs, per, hbm):
    """Achieved GB/s and fraction of measured HBM of the step's kernels, from
    the algorithmic-byte formulas of each (see the design notes) and the
    kernels' CUDA-event times inside the timed region."""
    T, n, th, k = cs["T"], cs["n"], cs["theta"], cs["k"]
    passes = max(1, -(-max(n - 1, 0).bit_length() // 8))    # radix passes of <= 8 bits
    alg = {
        "sort_sets_warp": 8 * T + 16 * th,
        "index_hist": 12 * T,
        "index_scatter": 16 * T + 16 * th,
        # per pass: keys read by the count, keys + values read and written by
        # the scatter (the first pass reads members only, with set ids from set_off)
        "index_radix": 16 * T + (passes - 1) * 20 * T + 8 * th,
        "index_bounds": 4 * T + 8 * n,
        "greedy": 4 * n * k + 4 * cs["s_seed"] + 16 * cs["covered"] + 12 * cs["r_covered"] + th // 8,
        "randgreedi_local": 4 * (cs["rg_eval"] + cs["rg_cover"]) + PARTS * th // 8,
    }
    out = {}
    for name, (launches, ms) in sorted(per.items()):
        if ms <= 0.05:
            continue
        e = {"ms": round(ms, 3)}
        if name in alg and launches > 0:
            gbs = alg[name] / (ms / 1000.0) / 1e9
            e.update({"alg_bytes": int(alg[name]), "gbs": round(gbs, 1), "frac": round(gbs / hbm, 4)})
        out[name] = e
    return out


# ---------------------------------------------------------------------------
# IC sampling, IMM, batched queries, served queries
# ---------------------------------------------------------------------------

class OneQuery:
    """The plain one-query-at-a-time GPU path: im_sample_rrr into a reused pool
    of the query's graph, then im_max_k_cover (plain greedy), seeds read back."""

    def __init__(self, im, G):
        self.im, self.G = im, G
        self.pools = {}
        self.caps = {}
        self.per_set = {}

    def solve(self, name, model, k, theta, seed, opts=None):
        im = self.im
        p = self.pools.get(name)
        per = self.per_set.get((name, model), 32.0)     # members per set seen so far
        want = int(theta * per * 1.25) + 1024
        if p is None:
            self.caps[name] = (max(theta, 1), want)
            p = self.pools[name] = im.Pool(self.G[name], *self.caps[name])
        while True:
            sets, ents = self.caps[name]
            if theta > sets or want > ents:
                self.caps[name] = (max(sets, theta), max(ents, want))
                im.im_pool_reserve(p.handle, *self.caps[name])
            p.reset()
            try:
                p.sample(model, seed, 0, theta)
                break
            except im.ImError as e:
                if e.status != im.IM_ERR_CAPACITY:
                    raise
                sets, ents = self.caps[name]
                self.caps[name] = (sets, ents * 4)
                im.im_pool_reserve(p.handle, *self.caps[name])
        total = p.info()[1]
        self.per_set[(name, model)] = max(self.per_set.get((name, model), 0.0),
                                          total / max(theta, 1))
        c = p.cover(k, opts)
        return c.seeds, c.coverage

    def close(self):
        for p in self.pools.values():
            p.close()


def _batched_graphs(im):
    graphs = {f"rmat{s}": inputs.batched_graph(s, SEED) for s in inputs.BATCH_SCALES}
    return graphs, {name: im.Graph(g) for name, g in graphs.items()}


def _mix_opts(im, i, partitions):
    """Every other query of the mix selects its seeds with RandGreedi (alpha
    1/4, delta 0.077); partitions 0 leaves the count to the batch."""
    if i % 2:
        return None
    return im.cover_opts(im.IM_RANDGREEDI, partitions, ALPHA, DELTA, SEED, fused=False)


def bench_batched(im, torch):
    """256 queries of the batched mix (every other one with RandGreedi, its
    partition count picked by the batch) in one im_solve_batch call versus the
    one-query path run back to back with the same counts; results compared
    query by query."""
    specs = inputs.batched_queries(256, SEED)
    graphs, G = _batched_graphs(im)
    qlist = [(G[q.graph].handle, q.model, q.k, q.theta, q.seed, _mix_opts(im, i, 0))
             for i, q in enumerate(specs)]
    batch = im.im_batch_create()
    im.im_solve_batch(batch, qlist, 100)          # warm-up: arenas, partition counts
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = im.im_solve_batch(batch, qlist, 100, with_partitions=True)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    # the same call again with per-kernel events, for the phase breakdown
    im.im_profile_reset()
    im.im_profile_enable(True)
    im.im_solve_batch(batch, qlist, 100)
    torch.cuda.synchronize()
    im.im_profile_enable(False)
    phases = {k: round(v[1], 2) for k, v in sorted(im.im_profile_read().items()) if v[1] >= 1.0}
    im.im_batch_destroy(batch)
    parts = [o[4] for o in out]
    one = OneQuery(im, G)
    for i, q in enumerate(specs[:8]):                     # warm-up
        one.solve(q.graph, q.model, q.k, q.theta, q.seed, _mix_opts(im, i, parts[i]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [one.solve(q.graph, q.model, q.k, q.theta, q.seed, _mix_opts(im, i, parts[i]))
             for i, q in enumerate(specs)]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    one.close()
    same = all(a[0].tolist() == b[0].tolist() and a[2] == b[1] for a, b in zip(out, plain))
    entries = sum(o[3] for o in out)
    for g in G.values():
        g.close()
    chosen = sorted({p for p in parts if p})
    return {"workload": "256 queries: R-MAT scales 12..18 (edge factor 16), IC (weighted cascade "
                        "1/in-degree) or LT (1/in-degree), k in [5,100], theta in [2^14,2^20]; "
                        "every other query RandGreedi (alpha 1/4, partition count picked by "
                        "the batch)",
            "queries": len(specs), "sets": sum(q.theta for q in specs), "entries": entries,
            "randgreedi_queries": sum(1 for p in parts if p), "partition_counts_chosen": chosen,
            "q_per_s": round(len(specs) / t_batch, 2), "ms": round(1000 * t_batch, 2),
            "plain_q_per_s": round(len(specs) / t_plain, 2), "plain_ms": round(1000 * t_plain, 2),
            "speedup_vs_plain": round(t_plain / t_batch, 3), "bit_exact_vs_plain": bool(same),
            "phase_ms": phases}


def bench_served(im, torch, orkut: bool):
    """Poisson arrivals (mean 200/s) replayed in real time into im_server
    (continuous batching), versus the one-query path as a FIFO server: each
    query's service time is measured back to back and the trace is replayed
    through a single queue (done_i = max(arrival_i, done_{i-1}) + service_i).
    The trace draws from the batched mix (every other mix query RandGreedi with
    64 parts) plus 5% Orkut-shaped queries (IC p = 0.01, plain greedy)."""
    nq = 512
    specs = inputs.served_trace(nq, SEED, orkut_frac=0.05 if orkut else 0.0)
    graphs, G = _batched_graphs(im)
    if any(q.graph == "orkut" for q in specs):
        G["orkut"] = im.Graph(inputs.graph_orkut_like(SEED))
    opts = [None if q.graph == "orkut" else _mix_opts(im, i, 64) for i, q in enumerate(specs)]
    srv = im.im_server_create(workers=SERVE_WORKERS, max_batch=8, mem_budget=96 << 30,
                              heavy_members=SERVE_HEAVY)
    try:
        warm = [im.im_server_submit(srv, G[q.graph].handle, q.model, q.k, q.theta, q.seed, o)
                for q, o in zip(specs[:16], opts[:16])]
        for t in warm:
            im.im_server_wait(srv, t, 100, 600)
        b0, q0, _ = im.im_server_stats(srv)
        tickets = []
        t0 = time.perf_counter()
        for q, o in zip(specs, opts):
            delay = q.arrival_s - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(im.im_server_submit(srv, G[q.graph].handle, q.model, q.k, q.theta,
                                               q.seed, o))
        res = [im.im_server_wait(srv, t, 100, 600) for t in tickets]
        t_all = time.perf_counter() - t0
        b1, q1, _ = im.im_server_stats(srv)
    finally:
        im.im_server_destroy(srv)        # joins the workers: no batch left in flight
    lat = np.array([r[2] for r in res])
    one = OneQuery(im, G)
    for q, o in zip(specs[:8], opts[:8]):
        one.solve(q.graph, q.model, q.k, q.theta, q.seed, o)
    torch.cuda.synchronize()
    service, plain = [], []
    for q, o in zip(specs, opts):
        t1 = time.perf_counter()
        plain.append(one.solve(q.graph, q.model, q.k, q.theta, q.seed, o))
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t1)
    one.close()
    done, plat = 0.0, []
    for q, sv in zip(specs, service):
        done = max(q.arrival_s, done) + sv
        plat.append(1000 * (done - q.arrival_s))
    plat = np.array(plat)
    same = all(a[0].tolist() == b[0].tolist() and a[1] == b[1] for a, b in zip(res, plain))
    n_ork = sum(1 for q in specs if q.graph == "orkut")
    for g in G.values():
        g.close()
    return {"workload": f"{nq} Poisson arrivals at 200/s from the batched mix (every other mix "
                        "query RandGreedi, 64 parts)"
                        + (f", {n_ork} Orkut-shaped (3,072,441 vertices, 234,369,798 edges, IC "
                           "p=0.01, theta in [2^6,2^10])" if orkut else "")
                        + f"; im_server: {SERVE_WORKERS} workers, batches of up to 8, requests "
                          f"of >= {SERVE_HEAVY:,} estimated members on worker 0 only",
            "queries": nq, "orkut_queries": n_ork, "span_s": round(specs[-1].arrival_s, 3),
            "q_per_s": round(nq / t_all, 2), "p50_ms": round(float(np.percentile(lat, 50)), 2),
            "p99_ms": round(float(np.percentile(lat, 99)), 2),
            "batches": int(b1 - b0), "mean_batch": round((q1 - q0) / max(b1 - b0, 1), 2),
            "plain_q_per_s": round(nq / max(done, specs[-1].arrival_s), 2),
            "plain_p50_ms": round(float(np.percentile(plat, 50)), 2),
            "plain_p99_ms": round(float(np.percentile(plat, 99)), 2),
            "plain_busy_s": round(float(sum(service)), 3),
            "bit_exact_vs_plain": bool(same)}


def bench_spread(im, torch, G, pool, n, theta):
    """Quality of the plain greedy's seeds: forward simulation of 1,024 runs
    in fresh live-edge worlds (sample ids from 2^30) against the RIS estimate
    n * coverage / theta of the pool they were selected on."""
    c = pool.cover(K)
    runs = 1024
    act = np.zeros(runs, np.int64)
    im.im_spread(G.handle, im.IM_LT, c.seeds, SEED, 1 << 30, 64, None, None)   # warm-up
    torch.cuda.synchronize()
    im.im_profile_reset()
    im.im_profile_enable(True)
    t0 = time.perf_counter()
    tot = im.im_spread(G.handle, im.IM_LT, c.seeds, SEED, 1 << 30, runs, act, None)
    dt = time.perf_counter() - t0
    im.im_profile_enable(False)
    k_ms = im.im_profile_read().get("spread_lt", (1, 0.0))[1]
    mean = tot / runs
    return {"workload": f"LT forward simulation of the plain greedy's {K} seeds on rmat20-lt, "
                        f"{runs} runs (sample ids from 2^30)",
            "sigma_mc": round(mean, 1), "sigma_mc_stderr": round(float(act.std() / np.sqrt(runs)), 1),
            "sigma_ris": round(n * c.coverage / theta, 1), "ms": round(1000 * dt, 2),
            "kernel_ms": round(k_ms, 2), "activations_per_s": tot / dt}


def bench_imm(im, torch, g):
    """IMM (Alg. 1) through im_solve on the LiveJournal-shaped graph, IC with
    weighted-cascade probabilities, eps = 0.13, l = 1, k = 200."""
    G = im.Graph(g)
    im.im_solve(G.handle, im.IM_IC, 200, 0.5, 1.0, SEED + 1)   # warm-up (LT-free, small)
    torch.cuda.synchronize()
    im.im_profile_reset()
    im.im_profile_enable(True)
    t0 = time.perf_counter()
    seeds, cov, theta, info = im.im_solve(G.handle, im.IM_IC, 200, 0.13, 1.0, SEED)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    im.im_profile_enable(False)
    prof = im.im_profile_read()
    G.close()
    return {"workload": "LiveJournal-shaped R-MAT (4,847,571 vertices, 69,000,000 edges), IC "
                        "weighted cascade (1/in-degree), eps=0.13, l=1, k=200",
            "ms": round(1000 * dt, 2), "rounds": int(info.rounds),
            "theta_rounds": [int(x) for x in info.theta_rounds[:info.rounds]],
            "lb": info.lb, "theta": int(theta), "round_entries": int(info.round_entries),
            "final_entries": int(info.final_entries), "coverage": int(cov),
            "num_seeds": int(len(seeds)), "final_examined_edges": int(info.examined),
            "phase_ms": {k: round(v[1], 3) for k, v in sorted(prof.items())}}


def bench_opim(im, torch):
    """OPIM with GreediRIS-trunc seed selection, the setting of the paper's
    Table 6 (k = 1000, eps = 0.01, halves capped at 2^20 sets, bucket spacing
    0.0562 for 63 buckets, delta = 1/n) on the rmat20-lt graph: per truncation
    alpha, the seed-selection time over all rounds, the rounds' sampling and
    scoring time, and the instance-wise guarantee; the plain greedy beside it."""
    g = inputs.graph_lt_scale20(SEED)
    G = im.Graph(g)
    k, eps, cap = 1000, 0.01, 1 << 20
    out = {"workload": "rmat20-lt, OPIM: k=1000, eps=0.01, delta=1/n, R1/R2 capped at 2^20 "
                       "sets each; GreediRIS-trunc 148 parts, bucket delta 0.0562 (B=63)"}
    im.im_opim(G.handle, im.IM_LT, 10, 0.5, 0.01, SEED, 1 << 14)     # warm-up
    runs = [("plain_greedy", None)] + [
        (f"alpha_{a[0]}/{a[1]}", im.cover_opts(im.IM_RANDGREEDI, PARTS, a, 0.0562, SEED,
                                               fused=False))
        for a in ((1, 1), (1, 2), (1, 4), (1, 8))]
    for name, opts in runs:
        im.im_profile_reset()
        im.im_profile_enable(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seeds, info = im.im_opim(G.handle, im.IM_LT, k, eps, 1.0 / g.n, SEED, cap, opts)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        im.im_profile_enable(False)
        prof = im.im_profile_read()
        sel = sum(v[1] for kk, v in prof.items() if kk.startswith(("randgreedi", "greedy",
                                                                     "partition", "max_subset")))
        samp = sum(v[1] for kk, v in prof.items() if kk.startswith(("sample", "sort_sets", "scan")))
        idx = sum(v[1] for kk, v in prof.items() if kk.startswith("index"))
        score = sum(v[1] for kk, v in prof.items() if kk.startswith("opim"))
        r = info.rounds
        out[name] = {"ms": round(1000 * dt, 1), "seed_select_ms": round(sel, 2),
                     "index_ms": round(idx, 2), "sampling_ms": round(samp, 2),
                     "scoring_ms": round(score, 2), "rounds": r,
                     "theta_per_half": int(info.theta[r - 1]),
                     "guarantee": round(info.guarantee, 4),
                     "guarantee_per_round": [round(x, 4) for x in info.alpha[:r]],
                     "num_seeds": int(len(seeds))}
    G.close()
    return out


def bench_paper_weights(im, torch):
    """The paper's own weight model (Sec. 4.1, U[0, 0.1] per edge) on R-MAT
    scale 20: IC with 16,384 sets (15% of them hold a ~10^5-vertex giant
    component) and LT (the same draws scaled per vertex to sum to at most 1)
    with 1,048,576 sets; sampling, plain greedy and RandGreedi (148 parts,
    alpha 1/4) at k = 100.  The first 16 IC sets are checked against the
    oracle."""
    import oracle as O
    opts_rg = im.cover_opts(im.IM_RANDGREEDI, PARTS, ALPHA, DELTA, SEED, fused=False)
    out = {}
    for model, wts, theta in ((im.IM_IC, "u0.1", 16384), (im.IM_LT, "lt-u0.1", 1 << 20)):
        g = inputs.rmat_graph(1 << 20, 1 << 24, SEED, wts)
        G = im.Graph(g)
        cap = theta * (40000 if model == im.IM_IC else 64)
        p = im.Pool(G, theta, cap)
        p.sample(model, SEED, 0, min(theta, 1024))       # warm-up (builds the LT index)
        p.reset()
        im.im_profile_reset()
        im.im_profile_enable(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.sample(model, SEED, 0, theta)
        torch.cuda.synchronize()
        t_s = time.perf_counter() - t0
        c = p.cover(K)
        torch.cuda.synchronize()
        t_g = time.perf_counter() - t0 - t_s
        r = p.cover(K, opts_rg)
        torch.cuda.synchronize()
        t_r = time.perf_counter() - t0 - t_s - t_g
        im.im_profile_enable(False)
        prof = im.im_profile_read()
        _, total, examined = p.info()
        e = {"theta": theta, "entries": total, "examined_edges": examined,
             "sample_ms": round(1000 * t_s, 2), "edges_per_s": examined / t_s,
             "greedy_ms": round(1000 * t_g, 2), "randgreedi_ms": round(1000 * t_r, 2),
             "coverage_greedy": int(c.coverage), "coverage_randgreedi": int(r.coverage),
             "phase_ms": {k2: round(v[1], 3) for k2, v in sorted(prof.items())}}
        if model == im.IM_IC:
            set_off, members = p.export()
            ref = O.sample(O.IC, g, SEED, 0, 16)
            e["bit_exact_first_16"] = bool(np.array_equal(set_off[:17], ref.set_off) and
                                           np.array_equal(members[:ref.set_off[-1]], ref.members))
        out["ic" if model == im.IM_IC else "lt"] = e
        p.close()
        G.close()
    out["workload"] = ("R-MAT scale 20 (1,048,576 vertices, 16,777,216 edges), edge probabilities "
                       "U[0, 0.1] (IC; LT scaled per vertex to sum <= 1), k=100")
    return out


def bench_ic(im, torch, g):
    """IC sampling on the LiveJournal-shaped graph (trivalency), 8,192 sets."""
    G = im.Graph(g)
    theta = 8192
    p = im.Pool(G, theta, theta * 600_000)
    p.sample(im.IM_IC, SEED, 0, 1024)                  # warm-up
    p.reset()
    im.im_profile_reset()
    im.im_profile_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p.sample(im.IM_IC, SEED, 1 << 20, theta)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    im.im_profile_enable(False)
    prof = im.im_profile_read()
    _, total, examined = p.info()
    sbytes = p.sample_bytes()
    k_ms = prof.get("sample_ic", (1, 0.0))[1] + prof.get("sample_ic_big", (1, 0.0))[1]
    hbm, _ = measured_peaks()
    p.close()
    G.close()
    return {"workload": "LiveJournal-shaped R-MAT (4,847,571 vertices, 69,000,000 edges), IC "
                        "trivalency, 8,192 RRR sets", "edges_per_s": examined / dt,
            "entries": total, "ms": round(1000 * dt, 3),
            "kernel_ms": round(k_ms, 3),   # both sampling passes
            "kernel_gbs": round(sbytes / (k_ms / 1000) / 1e9, 1) if k_ms else None,
            "kernel_frac": round(sbytes / (k_ms / 1000) / 1e9 / hbm, 4) if k_ms else None,
            "phase_ms": {k: round(v[1], 3) for k, v in sorted(prof.items())}}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
