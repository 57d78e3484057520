"""RASTER benchmark: points/s of the whole hot path on one GB300 (or N replicas).

A step is one pass of the plain RASTER hot path over the 500M-point workload
(1,000,000 square clusters of 475 points in [0, 3000)^2 plus 25M uniform
noise points, shuffled; precision 2, tau 5, mu 4):
    reset -> contract (projection + tile counting) -> agglomerate (tau filter,
    8-connected components, mu filter, cluster ids) -> per-point labels.

value : points/s with the points already resident in HBM (CUDA events).
e2e   : the same step through the host-buffer entry points (pinned host
        points in, labels out), copies inside the timed region.
roofline : the contraction phase, algorithmic bytes (16 B per point read +
        12 B per distinct tile written) over its measured time, against the
        measured HBM copy bandwidth.
cpu_baseline : the CPU oracle on a bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
       (N > 1 under torch.distributed.run: one independent replica per GPU.)
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gen  # noqa: E402

TILE_BYTES = 12          # algorithmic bytes per distinct tile (key + count written once)
POINT_BYTES = 16         # algorithmic bytes per point (x, y read once)

# DRAM bytes (read + write) of one contraction phase (k_part, k_region_items,
# k_bucket and k_insert_fresh, the pass 2 of a round into a table void since
# its reset) in a steady-state step, from one ncu capture
# with one pass per launch on the 100M-point case of the same workload
# (`--points 100000000`: 1.6 GB of points, a 91M-slot table).  The traffic
# grows with the points (16 B read, each point's key stored, keys staged
# twice) and with the table slots (each written once, with the selected
# significant rows beside them), so it scales to a full launch as
# per_point * n + per_slot * slots.  Valid only for the contraction kernels'
# sources it was measured with (their digest); reported as null otherwise.
MEASURED_CONTRACT_TRAFFIC = {"sources": "42f19a62f49a1162", "case_points": 100_000_000, "case_slots": 91_226_112,
                             "per_point": 5.515e9 / 100_000_000, "per_slot": 1.549e9 / 91_226_112}


def kernel_sources_digest() -> str:
    """Digest of the sources of the contraction kernels (the device code of
    k_part, k_bucket, k_insert_fresh, k_insert_bucket and their helpers)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1907_03620_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("raster_block.cuh", "raster_device.cuh", "raster_project.cuh", "raster_region.cuh",
              "raster_single_contract.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="500m", choices=sorted(gen.NAMED))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=10_000_000, help="points of the oracle sample")
    ap.add_argument("--cpu-parallel-sample", type=int, default=500_000_000,
                    help="points of the multi-threaded P-RASTER sample")
    ap.add_argument("--profile", action="store_true", help="short run for ncu (no clocks/e2e/cpu legs)")
    ap.add_argument("--points", type=int, default=0, help="use only the first N points (profiling cases)")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and served legs")
    ap.add_argument("--loop-seconds", type=float, default=8.0, help="time budget of each single-call loop baseline")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="duration of each Poisson serving run")
    ap.add_argument("--serve-rates", default="0.5,0.8,0.95", help="arrival rates as fractions of saturated throughput")
    ap.add_argument("--serve-pool", type=int, default=512, help="requests staged on the device for the served leg")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device) -> float:
    """The largest value over all ranks (timings: the job is as slow as its
    slowest replica); the value itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, seconds: float) -> float:
    """Weak scaling: every rank processes its own copy of the workload, so the
    job processes world * units in the (max-over-ranks) time."""
    return world * units_per_rank / seconds


def workload_config(w: gen.Workload, name: str) -> dict:
    return {"workload": f"raster-{name}", "n_points": w.n, "clusters": w.clusters,
            "cluster_points": w.cluster_points, "canvas": [0.0, w.canvas], "precision": w.precision,
            "tau": w.tau, "mu": w.mu, "point_dtype": "float64x2", "order": "shuffled", "seed": w.seed,
            "l2": "inputs (16 B/point) far larger than L2; no flush needed"}


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        hi = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(hi), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (the reference arm and the cpu_baseline leg)

def oracle_sample(w: gen.Workload, sample: int):
    """Time the oracle (contraction, agglomeration, labels) on the first
    `sample` points of the workload; returns points/s and a description."""
    import oracle
    xy = gen.points(w, 0, min(sample, w.n))
    oracle.build()  # compiled before the clock starts
    t0 = time.perf_counter()
    o = oracle.Oracle(w.precision, w.tau, w.mu)
    o.add(xy)
    o.finish()
    o.labels(xy)
    dt = time.perf_counter() - t0
    return xy.shape[0] / dt, dt, f"first {xy.shape[0]:,} points of the workload (contract + agglomerate + labels)"


def praster_sample(w: gen.Workload, sample: int) -> dict:
    """Time P-RASTER (Sect. 3.5, Alg. 2-3; the oracle library's multi-threaded
    form) on all host cores over the first `sample` points of the workload:
    contraction (per-thread maps, join), agglomeration (slices, border joins)
    and labels."""
    import oracle
    xy = gen.points(w, 0, min(sample, w.n))
    threads = os.cpu_count() or 1
    oracle.build_praster()  # compiled before the clock starts
    t0 = time.perf_counter()
    res, _, secs = oracle.praster(xy, w.precision, w.tau, w.mu, threads, with_labels=True, sort=False)
    dt = time.perf_counter() - t0
    return {"value": xy.shape[0] / dt, "unit": "points/s", "cores": threads, "kind": "P-RASTER (oracle library)",
            "sample": f"first {xy.shape[0]:,} points of the workload (contract + agglomerate + labels)",
            "seconds": dt, "phases_s": secs}


def run_reference(args):
    world, rank, _ = dist_env()
    w = gen.NAMED[args.workload]
    if rank != 0:
        return
    times = []
    sample = max(1, args.cpu_sample // 5)
    for i in range(args.warmup + args.steps):
        rate, dt, desc = oracle_sample(w, sample)
        if i >= args.warmup:
            times.append(dt)
    v = sample / statistics.mean(times)
    line = {"impl": "reference", "metric": "points_per_s", "value": v, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(workload_config(w, args.workload), parallelism=f"replicas{world}"),
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {sample:,} points of the workload per step",
                             "host_cores": os.cpu_count()},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------

def single_call_loops(items, seconds: float) -> dict:
    """Two loops of plain single-instance calls over the same instances, each
    time-bounded, one instance at a time with a synchronisation after each:
    `reuse` keeps one handle per (precision, tau, mu) and resets it between
    instances (raster_reset); `create` creates and destroys a handle per
    instance.  items: (xy or list of chunk views, precision, tau, mu, chunks)."""
    import torch

    import paper_1907_03620_gb300 as R
    out = {}
    for mode in ("reuse", "create"):
        handles = {}
        lat, pts = [], 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for xy, p, tau, mu, _ in items:
            views = xy if isinstance(xy, list) else [xy]
            t1 = time.perf_counter()
            if mode == "reuse":
                h = handles.get((p, tau, mu))
                if h is None:
                    h = handles[(p, tau, mu)] = R.Raster(p, tau, mu)
                h.reset()
            else:
                h = R.Raster(p, tau, mu)
            for v in views:
                h.contract(v)
            h.agglomerate(copy=False, raw=True)
            if mode == "create":
                h.close()
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - t1) * 1e3)
            pts += sum(int(v.shape[0]) for v in views)
            if time.perf_counter() - t0 > seconds:
                break
        for h in handles.values():
            h.close()
        out[mode] = {"value": pts / (sum(lat) / 1e3), "unit": "points/s", "instances": len(lat), "points": pts,
                     "latency_p50_ms": float(np.percentile(lat, 50)), "latency_p99_ms": float(np.percentile(lat, 99)),
                     "calls": ("one handle per (p, tau, mu): reset, contract per chunk, agglomerate" if mode == "reuse"
                               else "create, contract per chunk, agglomerate, destroy")}
    return out


def batched_leg(args, dev):
    """Batched form: the 4096-instance workload in one graph launch, against a
    loop of plain single-instance calls (create, contract, agglomerate,
    destroy) on the same GPU."""
    import torch

    import paper_1907_03620_gb300 as R
    from paper_1907_03620_gb300 import tune
    from paper_1907_03620_gb300.batch import RasterBatch

    ws = gen.batch_instances()
    offs = np.cumsum([0] + [w.n for w in ws])
    total = int(offs[-1])
    flat = torch.empty((total, 2), dtype=torch.float64, device=dev)
    host = np.empty((int(max(w.n for w in ws)), 2), dtype=np.float64)
    for i, w in enumerate(ws):
        gen.points_into(host[: w.n], w)
        flat[offs[i]:offs[i + 1]].copy_(torch.from_numpy(host[: w.n]))
    inst = [(flat[offs[i]:offs[i + 1]], w.precision, w.tau, w.mu) for i, w in enumerate(ws)]
    t0 = time.perf_counter()
    cfg = tune.tune_batch(inst)
    tune_s = time.perf_counter() - t0
    b = RasterBatch(inst, **cfg)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 1)):
        b.run()
    b.wait()
    times = []
    for _ in range(max(args.steps, 3)):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        b.run()
        s1.record(stream)
        b.wait()
        times.append(s0.elapsed_time(s1))
    ms = statistics.mean(times)
    launches_per_run = 9
    n_clusters = sum(b.counts(i).n_clusters for i in range(len(ws)))
    dev_bytes = b.device_bytes
    b.close()
    loops = single_call_loops([(inst[i][0], ws[i].precision, ws[i].tau, ws[i].mu, 1) for i in range(len(ws))],
                              args.loop_seconds)
    best = max(loops.values(), key=lambda v: v["value"])
    del flat
    torch.cuda.empty_cache()
    q = lambda v, p: float(np.percentile(np.array(v), p))  # noqa: E731
    return {"metric": "points_per_s", "value": total / (ms / 1e3), "unit": "points/s",
            "instances": len(ws), "points": total, "ms_per_run": ms, "runs": len(times),
            "latency_p50_ms": q(times, 50), "latency_p99_ms": q(times, 99),
            "clusters": n_clusters, "device_bytes": dev_bytes, "config": cfg, "tune_seconds": tune_s,
            "gpu_launches_per_run": launches_per_run,
            "loop_baseline": loops,
            "speedup_vs_loop": (total / (ms / 1e3)) / best["value"],
            "speedup_vs_loop_against": best["calls"]}


def served_leg(args, dev):
    """Served form: Poisson arrivals of requests into the continuous-batching
    engine for --serve-seconds at each rate in --serve-rates (fractions of the
    saturated throughput).  Requests follow the serving workload: sizes
    log-uniform in [1e4, 2e7), 1..8 chunks, per-request p/tau/mu.  Their points
    come from a pool of --serve-pool requests drawn from that distribution and
    staged on the device (arrival k takes a pseudo-random pool entry), since
    60 s of arrivals would be terabytes of input."""
    import torch

    from paper_1907_03620_gb300.serve import RasterServer

    pool_n = args.serve_pool
    ws = [gen._instance(5, i, gen._log_uniform_size(5, i, 10_000, 20_000_000), 0.10) for i in range(pool_n)]
    nchunks = [int(1 + gen.rng_at(5, 15, i) % 8) for i in range(pool_n)]
    offs = np.cumsum([0] + [w.n for w in ws])
    flat = torch.empty((int(offs[-1]), 2), dtype=torch.float64, device=dev)
    stage = torch.empty((max(w.n for w in ws), 2), dtype=torch.float64, pin_memory=True)
    for i, w in enumerate(ws):
        gen.points_into(stage[: w.n].numpy(), w)
        flat[offs[i]:offs[i + 1]].copy_(stage[: w.n])
    del stage
    pool = []
    for i, w in enumerate(ws):
        xy = flat[offs[i]:offs[i + 1]]
        pool.append((w, [xy[lo:hi] for lo, hi in gen.chunk_bounds(w.n, nchunks[i])]))
    mean_pts = float(offs[-1]) / pool_n
    srv = RasterServer(max_active=4096, reserve_bytes=8 << 30)
    done_lat, done_pts = [], [0]
    lock = threading.Lock()
    stop = [False]

    def poller():
        while not stop[0]:
            r = srv.poll(wait_ms=20, rows=False)
            if r is None:
                continue
            rid, res, lat = r
            srv.release(rid)
            with lock:
                done_lat.append(lat)
                done_pts[0] += res.n_points

    def submit(rid, k):
        w, views = pool[k]
        srv.submit(rid, w.precision, w.tau, w.mu, w.n, len(views))
        for v in views:
            srv.push(rid, v)

    def wait_done(count):
        while True:
            with lock:
                if len(done_lat) >= count:
                    return
            time.sleep(0.002)

    def take():
        with lock:
            lat, pts = list(done_lat), done_pts[0]
            done_lat.clear()
            done_pts[0] = 0
        return lat, pts

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    for k in range(pool_n):  # warm-up: every request once (the engine maps its pages on first use)
        submit(10**9 + k, k)
    wait_done(pool_n)
    take()
    # saturation: the whole pool submitted at once
    t0 = time.perf_counter()
    for k in range(pool_n):
        submit(k, k)
    wait_done(pool_n)
    t_sat = time.perf_counter() - t0
    _, sat_pts = take()
    sat_rate = sat_pts / t_sat
    runs = []
    rid = 10**6
    peak_bytes = 0
    for frac in [float(f) for f in args.serve_rates.split(",") if f]:
        req_rate = frac * sat_rate / mean_pts
        arrivals = gen.serve_requests(rate_per_s=req_rate, duration_s=args.serve_seconds, seed=7)
        picks = [int(gen.rng_at(7, 16, k) % pool_n) for k in range(len(arrivals))]
        t0 = time.perf_counter()
        for k, rq in enumerate(arrivals):
            delay = rq.arrival_s - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            submit(rid, picks[k])
            rid += 1
            if k % 256 == 0:
                peak_bytes = max(peak_bytes, srv.stats()["device_bytes"])
        wait_done(len(arrivals))
        wall = time.perf_counter() - t0
        lat, pts = take()
        runs.append({"load_fraction": frac, "requests": len(arrivals), "offered_req_per_s": req_rate,
                     "offered_points_per_s": frac * sat_rate, "points_per_s": pts / wall,
                     "latency_p50_ms": float(np.percentile(lat, 50)), "latency_p99_ms": float(np.percentile(lat, 99)),
                     "seconds": wall})
    stop[0] = True
    th.join()
    st = srv.stats()
    srv.close()
    loops = single_call_loops([(views, w.precision, w.tau, w.mu, len(views)) for w, views in pool],
                              args.loop_seconds)
    best = max(loops.values(), key=lambda v: v["value"])
    del pool, flat
    torch.cuda.empty_cache()
    return {"metric": "points_per_s", "saturated_points_per_s": sat_rate, "saturated_burst_requests": pool_n,
            "mean_request_points": mean_pts, "runs": runs, "engine_steps": st["steps"],
            "engine_peak_device_bytes": peak_bytes, "admission": "free device memory less an 8 GiB reserve",
            "loop_baseline": loops, "speedup_vs_loop": sat_rate / best["value"],
            "speedup_vs_loop_per_run": {str(r["load_fraction"]): r["points_per_s"] / best["value"] for r in runs},
            "speedup_vs_loop_against": best["calls"],
            "request_data": (f"pool of {pool_n} requests drawn from the serving workload's distribution, staged on "
                             f"the device; arrival k uses a pseudo-random pool entry")}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1907_03620_gb300 as R

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = gen.NAMED[args.workload]
    if args.points:  # same density, fewer points: scale clusters and canvas area
        f = args.points / w.n
        w = gen.Workload(**dict(w.asdict(), n=args.points, clusters=max(1, round(w.clusters * f)),
                                cluster_points=round(w.cluster_points * f), canvas=w.canvas * f ** 0.5))
    L = R.lib()

    # inputs: pinned host copy (for e2e) and a device-resident copy
    host = torch.empty((w.n, 2), dtype=torch.float64, pin_memory=True)
    gen.points_into(host.numpy(), w)
    xy = host.to(dev, non_blocking=False)
    labels = torch.empty(w.n, dtype=torch.int64, device=dev)
    keys = torch.empty(w.n, dtype=torch.int64, device=dev)  # every point's tile key, written by the contraction
    stream = torch.cuda.current_stream()

    r = R.Raster(w.precision, w.tau, w.mu)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(record=None):
        e0, e1, e2, e3, e4 = ev(), ev(), ev(), ev(), ev()
        e0.record(stream)
        r.reset()
        e1.record(stream)
        r.contract_keys(xy, keys)  # contraction, storing each point's tile key
        e2.record(stream)
        res = r.agglomerate(copy=False, raw=True)
        e3.record(stream)
        r.key_labels(keys, out=labels)  # RASTER* labels read from the stored keys
        e4.record(stream)
        if record is not None:
            record.append((e0, e1, e2, e3, e4, res))
        return res

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    if not args.profile:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = L.raster_kernel_launches()
    recs = []
    t_start, t_end = ev(), ev()
    t_start.record(stream)
    for _ in range(args.steps):
        step(recs)
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = L.raster_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if not args.profile else None

    total_ms = max_over_ranks(t_start.elapsed_time(t_end), dev)
    phase = {"reset": [], "contract": [], "agglomerate": [], "labels": []}
    for (e0, e1, e2, e3, e4, res) in recs:
        phase["reset"].append(e0.elapsed_time(e1))
        phase["contract"].append(e1.elapsed_time(e2))
        phase["agglomerate"].append(e2.elapsed_time(e3))
        phase["labels"].append(e3.elapsed_time(e4))
    res = recs[-1][5]
    ms_step = total_ms / args.steps
    # for comparison, outside the timed steps and with the label index already
    # built: the labels of the same points projected again from their
    # coordinates (raster_point_labels) and read from the stored keys
    lp_ms, lk_ms = [], []
    for rep in range(3):
        l0, l1, l2 = ev(), ev(), ev()
        l0.record(stream)
        r.point_labels(xy, out=labels)
        l1.record(stream)
        r.key_labels(keys, out=labels)
        l2.record(stream)
        torch.cuda.synchronize()
        lp_ms.append(l0.elapsed_time(l1))
        lk_ms.append(l1.elapsed_time(l2))
    value = whole_job_rate(world, w.n, ms_step / 1e3)

    peaks = measured_peaks()
    contract_ms = statistics.mean(phase["contract"])
    alg_bytes = POINT_BYTES * w.n + TILE_BYTES * res.n_distinct
    achieved = alg_bytes / (contract_ms / 1e3) / 1e9
    traffic = None
    if kernel_sources_digest() == MEASURED_CONTRACT_TRAFFIC["sources"]:
        traffic = round(MEASURED_CONTRACT_TRAFFIC["per_point"] * w.n + MEASURED_CONTRACT_TRAFFIC["per_slot"] * r.capacity)
    roofline = {"bound": "hbm", "kernel": "contraction phase: k_part + k_region_items + k_bucket + k_insert_fresh",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"] + " (copy bandwidth)",
                "traffic": traffic,
                "traffic_unit": ("bytes per contraction phase (ncu dram__bytes read+write on the 100M-point case, "
                                 "scaled per point and per table slot)"),
                "algorithmic_bytes": alg_bytes, "algorithmic": "16 B/point + 12 B/distinct tile",
                "also_stored": "8 B/point of tile keys for the labels (not counted as algorithmic bytes)",
                "phase_ms": contract_ms}
    # the other phases of the step, against the same peak
    ag_bytes = 12 * res.n_distinct + 24 * res.n_significant + 20 * int(res.key.numel())
    lb_bytes = 16 * w.n
    roofline_phases = {
        "agglomerate": {"algorithmic_bytes": ag_bytes, "algorithmic": "12 B/tile + 24 B/significant + 20 B/kept row",
                        "ms": statistics.mean(phase["agglomerate"]),
                        "frac": ag_bytes / (statistics.mean(phase["agglomerate"]) / 1e3) / 1e9 / peaks["hbm_gbs"]},
        "labels": {"algorithmic_bytes": lb_bytes, "algorithmic": "8 B/point key read + 8 B/point label written",
                   "ms": statistics.mean(phase["labels"]),
                   "frac": lb_bytes / (statistics.mean(phase["labels"]) / 1e3) / 1e9 / peaks["hbm_gbs"]}}

    line = {"metric": "points_per_s", "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(w, args.workload), parallelism=f"replicas{world}"),
            "phases_ms": {k: statistics.mean(v) for k, v in phase.items()},
            "step": ("raster_reset; raster_contract_keys (contraction, storing each point's tile key); "
                     "raster_agglomerate; raster_key_labels (labels read from the stored keys)"),
            "labels_without_index_build_ms": {"from_points": statistics.mean(lp_ms[1:]),
                                              "from_keys": statistics.mean(lk_ms[1:])},
            "stats": {"n_distinct": res.n_distinct, "n_significant": res.n_significant,
                      "n_clusters": res.n_clusters, "kept_tiles": int(res.key.numel()),
                      "table_slots": r.capacity, "table": r.table_stats()},
            "roofline": roofline, "roofline_phases": roofline_phases, "gpu_launches": int(launches),
            "clocks": clocks}

    # the same workload streamed as 10 chunks of 50M through raster_contract
    # into one table (chunked processing): same step, chunked contraction
    if not args.profile and w.n % 10 == 0:
        m = w.n // 10
        chunk_ms = []
        for rep in range(3):
            c0, c1 = ev(), ev()
            c0.record(stream)
            r.reset()
            for c in range(10):
                r.contract_keys(xy[c * m:(c + 1) * m], keys[c * m:(c + 1) * m])
            r.agglomerate(copy=False, raw=True)
            r.key_labels(keys, out=labels)
            c1.record(stream)
            torch.cuda.synchronize()
            if rep:
                chunk_ms.append(c0.elapsed_time(c1))
        cms = max_over_ranks(statistics.mean(chunk_ms), dev)
        line["streamed_10_chunks"] = {"value": whole_job_rate(world, w.n, cms / 1e3), "unit": "points/s",
                                      "ms_per_step": cms, "chunks": 10, "chunk_points": m}

    # RASTER' grouped output (Sect. 3.4) on the same workload: the handle is
    # agglomerated; point_groups re-projects every point and groups the
    # indices of points in kept tiles by result row
    if not args.profile:
        res = r.agglomerate(copy=False, raw=True)
        k = int(res.key.numel())
        gbuf = (torch.empty(k + 1, dtype=torch.int64, device=dev), torch.empty(w.n, dtype=torch.int64, device=dev))
        g_ms = []
        for rep in range(4):
            g0, g1 = ev(), ev()
            g0.record(stream)
            _, gidx = r.point_groups(xy, k, out=gbuf)
            g1.record(stream)
            torch.cuda.synchronize()
            if rep:
                g_ms.append(g0.elapsed_time(g1))
        gms = max_over_ranks(statistics.mean(g_ms), dev)
        g_bytes = POINT_BYTES * w.n + 8 * int(gidx.numel()) + 8 * (k + 1)
        line["raster_prime_groups"] = {
            "value": whole_job_rate(world, w.n, gms / 1e3), "unit": "points/s", "ms": gms,
            "grouped_points": int(gidx.numel()), "rows": k, "algorithmic_bytes": g_bytes,
            "algorithmic": "16 B/point read + 8 B/grouped point + 8 B/row written",
            "frac": g_bytes / (gms / 1e3) / 1e9 / peaks["hbm_gbs"]}
        del gbuf, gidx

    # the extensions on the same workload and step: the 2 x 2 group rule
    # (Sect. 3.6) and other neighbourhoods neighbors(u, delta) (Sect. 3.2)
    if not args.profile and not args.no_forms:
        ext = {}
        for name, kw in (("groups_2x2", dict(groups=True)), ("chebyshev_delta2", dict(delta=2)),
                         ("manhattan_delta2", dict(metric=R.MANHATTAN, delta=2))):
            rx = R.Raster(w.precision, w.tau, w.mu, **kw)
            times = {"contract": [], "agglomerate": [], "labels": []}
            for rep in range(4):
                e0, e1, e2, e3 = ev(), ev(), ev(), ev()
                e0.record(stream)
                rx.reset()
                rx.contract_keys(xy, keys)
                e1.record(stream)
                resx = rx.agglomerate(copy=False, raw=True)
                e2.record(stream)
                rx.key_labels(keys, out=labels)
                e3.record(stream)
                torch.cuda.synchronize()
                if rep:
                    times["contract"].append(e0.elapsed_time(e1))
                    times["agglomerate"].append(e1.elapsed_time(e2))
                    times["labels"].append(e2.elapsed_time(e3))
            ms = {k: statistics.mean(v) for k, v in times.items()}
            step_ms = max_over_ranks(sum(ms.values()), dev)
            ext[name] = {"value": whole_job_rate(world, w.n, step_ms / 1e3), "unit": "points/s", "ms_per_step": step_ms,
                         "phases_ms": ms, "n_significant": resx.n_significant, "n_clusters": resx.n_clusters,
                         "kept_tiles": int(resx.key.numel())}
            rx.close()
        # three coordinates per point (Sect. 3.6, higher dimensions): 100M points
        # in 100,000 cubes of side 0.1 plus 10M noise points in [0, 100)^3
        c3 = gen.CUBES_100M
        xyz = torch.from_numpy(gen.cubes3(**c3)).to(dev)
        n3 = xyz.shape[0]
        lab3 = torch.empty(n3, dtype=torch.int64, device=dev)
        key3 = torch.empty(n3, dtype=torch.int64, device=dev)
        r3 = R.Raster(1.5, 5, 4, dims=3)
        times = {"contract": [], "agglomerate": [], "labels": []}
        for rep in range(4):
            e0, e1, e2, e3 = ev(), ev(), ev(), ev()
            e0.record(stream)
            r3.reset()
            r3.contract_keys(xyz, key3)
            e1.record(stream)
            res3 = r3.agglomerate(copy=False, raw=True)
            e2.record(stream)
            r3.key_labels(key3, out=lab3)
            e3.record(stream)
            torch.cuda.synchronize()
            if rep:
                times["contract"].append(e0.elapsed_time(e1))
                times["agglomerate"].append(e1.elapsed_time(e2))
                times["labels"].append(e2.elapsed_time(e3))
        ms = {k: statistics.mean(v) for k, v in times.items()}
        step_ms = max_over_ranks(sum(ms.values()), dev)
        ext["three_coordinates"] = {
            "value": whole_job_rate(world, n3, step_ms / 1e3), "unit": "points/s", "ms_per_step": step_ms,
            "phases_ms": ms, "workload": dict(c3, precision=1.5, tau=5, mu=4, dims=3),
            "n_distinct": res3.n_distinct, "n_significant": res3.n_significant, "n_clusters": res3.n_clusters,
            "contraction_frac": (24 * n3 + 12 * res3.n_distinct) / (ms["contract"] / 1e3) / 1e9 / peaks["hbm_gbs"]}
        r3.close()
        del xyz, lab3, key3
        line["extensions"] = ext

    # e2e: host buffers through the C ABI, copies inside the timed region: one
    # call (raster_cluster_host) copies the points in once, contracts,
    # agglomerates, labels and copies the labels back
    if not args.no_e2e and not args.profile:
        lab_host = torch.empty(w.n, dtype=torch.int64, pin_memory=True)

        def e2e_step():
            r.reset()
            res, _ = r.cluster_host(host, out=lab_host, copy=False, raw=True)
            return res

        e2e_step()
        torch.cuda.synchronize()
        # the machine's host link, for context: 2 GB of points in and 1 GB of labels
        # out on a copy stream, timed with CUDA events on that stream, best of 3
        q = w.n // 4
        cs = torch.cuda.Stream()
        link = {"h2d": 0.0, "d2h": 0.0}
        with torch.cuda.stream(cs):
            for _ in range(3):
                for name, dst, src, nbytes in (("h2d", xy[:q], host[:q], POINT_BYTES * q),
                                               ("d2h", lab_host[:q], labels[:q], 8 * q)):
                    a0, a1 = ev(), ev()
                    a0.record(cs)
                    dst.copy_(src, non_blocking=True)
                    a1.record(cs)
                    a1.synchronize()
                    link[name] = max(link[name], nbytes / (a0.elapsed_time(a1) / 1e3) / 1e9)
        h2d_gbs, d2h_gbs = link["h2d"], link["d2h"]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 3))
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / n_e2e, dev)
        line["e2e"] = {"value": whole_job_rate(world, w.n, dt), "unit": "points/s", "h2d_bytes_per_step": POINT_BYTES * w.n,
                       "d2h_bytes_per_step": 8 * w.n, "ms_per_step": dt * 1e3, "steps": n_e2e,
                       "call": "raster_cluster_host (points copied once; labels copied back)",
                       "link_gbs": {"h2d": h2d_gbs, "d2h": d2h_gbs}}

    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.profile:
        rate, dt, desc = oracle_sample(w, args.cpu_sample)
        line["cpu_baseline"] = {"value": rate, "unit": "points/s", "cores": 1, "kind": "oracle",
                                "sample": desc, "seconds": dt, "host_cores": os.cpu_count(),
                                "parallel": praster_sample(w, args.cpu_parallel_sample)}

    r.close()
    del xy, labels, host
    torch.cuda.empty_cache()
    if not args.no_forms and not args.profile:
        line["batched"] = batched_leg(args, dev)
        line["served"] = served_leg(args, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
