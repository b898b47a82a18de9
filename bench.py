#!/usr/bin/env python
"""Benchmark of the GB300 voxel map update (G-VOM per-scan update).

Workload (default, the headline): the plain high-speed workload -- a
128-beam lidar (262,144 points per scan) at 12 m/s over seeded procedural
terrain with vegetation clusters, 40 scans at 10 Hz into a 512 x 512 x 64
map at 0.1 m (201 MB of counts, more than the 129 MB L2) with a window
shift every scan. One step = one scan through the whole path: shift the
window, ingest the scan (transform, hits, exact traversal passes), and
extract every 2D product (height, obstacles, density, slope, roughness,
negative obstacles). Steps cycle through the 40 scans.

Also measured (key "sequence"): the plain sequence workload -- a 64-beam
lidar (131,072 points per scan), 20 scans along a 4.5 m/s sinusoidal path,
into a 256 x 256 x 64 map at 0.2 m. --workload sequence swaps the two
(both arms). The batched (64 maps), served (32 robots) and next-row legs
(pipeline, lookup-table export, scan buffer, several sensors) follow.

Metric: rays integrated per second (valid rays / GPU time), with map updates
per second beside it. The L2 is flushed (a 256 MiB write) between timed
steps; each step is timed with CUDA events on the stream that runs it.

--impl reference times the CPU oracle (the plain FP64 statement of the
method) on the same workload, one scan per step.
Multi-GPU (torchrun): every rank updates its own map from its own seeded
robot (replicas, weak scaling); no data-path collective.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rays integrated/s (plain high-speed map update: shift + ingest + extract)"
UNIT = "rays/s"
METRIC_SEQUENCE = "rays integrated/s (plain sequence map update: shift + ingest + extract)"
SEQUENCE_WORKLOAD = ("plain sequence: 64-beam 64x2048 = 131,072 pts/scan, 20 scans at 10 Hz, 4.5 m/s, "
                     "map 256x256x64 @ 0.2 m, shift every scan")
L2_FLUSH_BYTES = 256 << 20
L2_NOTE = ("flushed between timed steps: a 256 MiB write, then a 256 MiB read of another buffer (no step data "
           "cached, no dirty lines left to write back inside the step)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--cpu-sample-s", type=float, default=12.0, help="oracle time budget for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-maps leg")
    ap.add_argument("--batched-maps", type=int, default=64)
    ap.add_argument("--batched-steps", type=int, default=10, help="timed steps of the batched leg")
    ap.add_argument("--retune", action="store_true", help="ignore cached tuning and search again")
    ap.add_argument("--tuning", default=None,
                    help="walk shape seg_len/march_block/blocks_per_sm/fused_ingest for the plain legs instead of "
                         "the tuner's (e.g. 64/128/0/1 for the fused ingest)")
    ap.add_argument("--no-served", action="store_true", help="skip the served leg")
    ap.add_argument("--served-seconds", type=float, default=60.0, help="length of the replayed arrival stream")
    ap.add_argument("--no-next-rows", action="store_true", help="skip the pipeline / LUT / buffer / multi-sensor legs")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the other plain workload's leg (sequence when the main leg is high_speed)")
    ap.add_argument("--high-speed-scans", type=int, default=40, help="generated scans of the high-speed workload")
    ap.add_argument("--workload", choices=["sequence", "high_speed"], default="high_speed",
                    help="workload of the main leg; the other one is measured as a sub-object")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(times, counts, device):
    """Replica aggregation: each time is the slowest rank's, each count the
    sum over ranks (the whole job's work in the whole job's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor(list(counts), dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(v) for v in t], [float(v) for v in c]


def gen_workers() -> int:
    return max(1, min(16, (os.cpu_count() or 2) - 1))


def host_cpu() -> dict:
    """The host the CPU baselines ran on: logical CPUs and the CPU model."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key, _, val = line.partition(":")
                fields.setdefault(key.strip(), val.strip())
    except OSError:
        pass
    import platform
    model = fields.get("model name") or fields.get("Model") or ""
    if not model and "CPU part" in fields:  # Arm: implementer and part numbers
        model = f"{platform.machine()} (implementer {fields.get('CPU implementer', '?')}, part {fields['CPU part']})"
    return {"nproc": os.cpu_count() or 0, "model": model or platform.machine()}


def make_inputs(rank: int, workload: str = "high_speed", n_scans: int = 40):
    """The plain workload's scans (high_speed: the first n_scans of 40)."""
    if workload == "high_speed":
        return make_high_speed_inputs(rank, n_scans)
    import synth
    seed = synth.SEEDS["sequence"] + 1000 * rank
    cfg, scans = synth.sequence_scans("sequence", seed=seed, workers=gen_workers())
    return cfg, scans


def workload_text(workload: str, n_scans: int) -> str:
    return HIGH_SPEED_WORKLOAD.format(n=n_scans) if workload == "high_speed" else SEQUENCE_WORKLOAD


def metric_of(workload: str) -> str:
    return METRIC if workload == "high_speed" else METRIC_SEQUENCE


def config_of(workload: str, cfg, n_scans: int, world: int) -> dict:
    """The workload as both arms name it (identical dicts)."""
    ms = cfg.map
    return {"workload": workload_text(workload, n_scans), "map": [ms.nx, ms.ny, ms.nz], "res_m": ms.res,
            "points_per_scan": cfg.lidar.n, "scans": n_scans, "l2": L2_NOTE,
            "parallelism": f"replicas x{world} (one map per GPU)"}


def summary_of(line: dict) -> dict:
    """The headline figures of every leg in a few hundred characters, last
    in the line (so that a reader keeping only the line's tail still sees
    them)."""
    out = {"value_M": round(line["value"] / 1e6, 1), "e2e_M": round(line["e2e"]["value"] / 1e6, 1),
           "walk_frac_coalesced": round(line["roofline"]["frac"], 3),
           "walk_us": round(line["roofline"]["launch_us"], 1)}
    other = line.get("sequence") or line.get("high_speed")
    if other:
        out["other_M"] = round(other["value"] / 1e6, 1)
        out["other_e2e_M"] = round(other["e2e"]["value"] / 1e6, 1)
    b = line.get("batched")
    if b:
        out["batched"] = {"M": round(b["rays_per_s_batched"] / 1e6, 1), "plain_M": round(b["rays_per_s_plain"] / 1e6, 1),
                          "speedup": round(b["speedup"], 3), "ms": round(b["ms_per_step_batched"], 3),
                          "graph_fixed_us": round(b["graph_fixed_cost"]["empty_step_us_median"], 1)}
    v = line.get("served")
    if v:
        out["served"] = {"p50_ms": round(v["realtime"]["p50_ms"], 2), "p99_ms": round(v["realtime"]["p99_ms"], 2),
                         "max_load_p99_lt_100ms": v["max_load_with_p99_under_100ms"],
                         "sweep_p99_ms": {str(p["load"]): round(p["p99_ms"], 1) for p in v["load_sweep"]},
                         "saturated_M": round(v["saturated"]["rays_per_s"] / 1e6, 1)}
    n = line.get("next_rows")
    if n:
        out["pipeline_M"] = round(n["pipeline_e2e"]["value"] / 1e6, 1)
    return out


BATCHED_WORKLOAD = ("batched: {m} independent maps 256x256x64 @ 0.2 m, each its own terrain and trajectory, "
                    "scan sizes log-uniform in [8,192, 262,144] (subsets of a 128x2048 scan), 2 generated steps cycled")


SERVED_WORKLOAD = ("served: 32 robots, mixed sensors (16/64/128 beams) and maps (128x128x32 @ 0.2 m, "
                   "256x256x64 @ 0.2 m, 512x512x64 @ 0.1 m), exponential inter-arrival times (mean 100 ms), "
                   "{s:g} s stream replayed in real time; each arrival posed on its robot's own trajectory "
                   "(2-12 m/s), its points one of 8 casts per robot spread over the stream")
SERVED_LOADS = (2.0, 4.0, 8.0, 16.0, 24.0, 32.0)   # offered-load factors of the sweep
SERVED_SWEEP_WINDOW_S = 10.0           # replay window per sweep point


def make_served_inputs(rank: int, seconds: float):
    import synth
    return synth.served_stream(n_robots=32, duration_s=seconds, seed=synth.SEEDS["served"] + 1000 * rank,
                               workers=gen_workers())


HIGH_SPEED_WORKLOAD = ("plain high-speed: 128-beam 128x2048 = 262,144 pts/scan at 10 Hz, 12 m/s, map 512x512x64 @ 0.1 m "
                       "(201 MB of counts, larger than L2), shift every scan; {n} generated scans cycled")


def make_high_speed_inputs(rank: int, n_scans: int):
    import synth
    return synth.sequence_scans("high_speed", n_scans=n_scans, seed=synth.SEEDS["high_speed"] + 1000 * rank,
                                workers=gen_workers())


def make_batched_inputs(rank: int, n_maps: int):
    import synth
    return synth.batched_scans(n_maps=n_maps, n_steps=2, seed=synth.SEEDS["batched"] + 1000 * rank,
                               workers=gen_workers())


def oracle_params(ms):
    import oracle
    return oracle.OracleParams(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))


def run_oracle_steps(cfg, scans, n_steps: int, time_budget_s: float | None = None):
    """Runs the oracle step by step (shift + ingest + extract); returns per-step (rays, seconds)."""
    import oracle
    params = oracle_params(cfg.map)
    om = oracle.OracleMap(params)
    out = []
    t_all = time.perf_counter()
    for k in range(n_steps):
        s = scans[k % len(scans)]
        t0 = time.perf_counter()
        om.shift_for_pose(s.vehicle_xyz)
        st = om.ingest(s.points, s.T_ws)
        om.extract()
        out.append((st.rays_valid, time.perf_counter() - t0))
        if time_budget_s is not None and time.perf_counter() - t_all > time_budget_s and k >= 1:
            break
    return out


def roofline_step(atomics, red_peak, V, ms, n_points, hbm_gbs, step_s):
    """The whole update's roofline time: the larger of its atomics at the
    measured L2 reduction rate and its HBM bytes (points read, state read by
    the column pass, products written) at the measured copy rate; beside it
    the sum of the two, for phases that run one after the other."""
    px = ms.nx * ms.ny
    hbm_bytes = 12 * n_points + 12 * V + 17 * px
    t_atom = atomics / red_peak
    t_hbm = hbm_bytes / (hbm_gbs * 1e9) if hbm_gbs else 0.0
    t = max(t_atom, t_hbm)
    return {"roofline_us": 1e6 * t, "measured_us": 1e6 * step_s, "frac": t / step_s,
            "serial_roofline_us": 1e6 * (t_atom + t_hbm), "frac_serial": (t_atom + t_hbm) / step_s,
            "atomic_us": 1e6 * t_atom, "hbm_us": 1e6 * t_hbm,
            "rule": "max(atomics / measured L2 RED rate, (12 B/point + 12 B/voxel + 17 B/px) / measured HBM rate)"}


def _oracle_map_job(args):
    """One map's scans through the oracle (shift + ingest + extract each), in
    a worker process; returns (valid rays, seconds)."""
    ms, scans = args
    import oracle
    om = oracle.OracleMap(oracle_params(ms))
    rays = 0
    t0 = time.perf_counter()
    for s in scans:
        om.shift_for_pose(s.vehicle_xyz)
        rays += om.ingest(s.points, s.T_ws).rays_valid
        om.extract()
    return rays, time.perf_counter() - t0


def oracle_batched_baseline(inputs, n_maps: int):
    """The batched workload's first step on the oracle, maps in parallel
    processes (spawn) over the host's cores, for the first n_maps maps."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    cfg4, steps = inputs
    jobs = [(cfg4.map, [steps[0][m]]) for m in range(min(n_maps, len(steps[0])))]
    cores = max(1, min(len(jobs), os.cpu_count() or 1))
    t0 = time.perf_counter()
    with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_map_job, jobs))
    wall = time.perf_counter() - t0
    rays = sum(r for r, _ in res)
    return {"value": rays / wall, "unit": UNIT, "cores": cores, "kind": "oracle", "host": host_cpu(),
            "sample": f"first step of the first {len(jobs)} maps, one map per process (spawned), wall time "
                      "including process start"}


def oracle_served_baseline(inputs, time_budget_s: float):
    """The served workload's requests in arrival order on the oracle (one
    thread, each robot its own map) until the time budget is spent."""
    import oracle
    robots, arrivals = inputs
    maps = {}
    rays, n, t_all = 0, 0, time.perf_counter()
    per = []
    for _, rid, k, c, T, veh in arrivals:
        r = robots[rid]
        om = maps.get(rid)
        if om is None:
            om = maps[rid] = oracle.OracleMap(oracle_params(r["map"]))
        t0 = time.perf_counter()
        om.shift_for_pose(veh)
        rays += om.ingest(r["casts"][c].points, T).rays_valid
        om.extract()
        per.append(time.perf_counter() - t0)
        n += 1
        if time.perf_counter() - t_all > time_budget_s:
            break
    return {"value": rays / sum(per), "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"first {n} requests in arrival order, each robot's own map, one thread",
            "mean_ms_per_request": 1e3 * statistics.fmean(per)}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.fh.close()
        except Exception:
            pass

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        loaded = [v for v in sm if smax and v > 0.5 * max(smax)] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def measure_red_peak(gv, torch, coalesced: bool = False):
    """L2 reduction-atomic throughput (increments/s) over a map-sized buffer:
    scattered single words, or (coalesced) 32 lanes on one 128-byte line."""
    words = 16 << 20  # 64 MiB, the size of one count array of the map
    buf = torch.zeros(words, dtype=torch.int32, device="cuda")
    ops = 1 << 28
    fn = gv.gvom_microbench_red_coalesced if coalesced else gv.gvom_microbench_red
    for _ in range(2):
        fn(buf, ops, seed=7)
    torch.cuda.synchronize()
    best = 0.0
    for r in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn(buf, ops, seed=11 + r)
        e1.record()
        e1.synchronize()
        best = max(best, ops / (e0.elapsed_time(e1) * 1e-3))
    del buf
    return best


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# the CUDA source each profiled kernel is compiled from (besides the headers)
KERNEL_SOURCES = {"k_march": "ingest.cu", "k_rays": "ingest.cu", "k_ingest": "ingest.cu",
                  "k_ingest_fused": "ingest.cu", "k_columns_tma": "extract.cu", "k_slope_negative": "extract.cu"}


def source_digest(kernel: str) -> str:
    """Digest of the sources a kernel is built from: its .cu file (every .cu
    file for a kernel not listed, or whose file is missing), the library's
    headers and the public header. A change elsewhere leaves it unchanged."""
    import hashlib
    src = os.path.join(ROOT, "paper_2109_13176_gb300", "csrc")
    names = sorted(os.listdir(src))
    own = KERNEL_SOURCES.get(kernel)
    if own in names:
        files = [own] + [f for f in names if f.endswith((".cuh", ".h"))]
    else:
        files = [f for f in names if f.endswith((".cu", ".cuh", ".h"))]
    paths = [os.path.join(src, f) for f in files]
    pub = os.path.join(ROOT, "include", "gvom.h")
    if os.path.exists(pub):
        paths.append(pub)
    h = hashlib.sha256()
    for q in paths:
        with open(q, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    sources are the ones it was measured on."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    digest = source_digest(kernel)
    with open(p) as fh:
        for line in fh:
            parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
            if parts.get("kernel") == kernel and parts.get("workload") == workload and parts.get("src") == digest:
                return float(parts["dram_bytes_per_launch"])
    return None


def run_reference(args, rank, world):
    if rank != 0:
        return
    # the steps cycle the workload's scans; only the ones they reach are cast
    n = args.warmup + args.steps
    cfg, scans = make_inputs(0, args.workload, max(1, min(args.high_speed_scans, n)))
    res = run_oracle_steps(cfg, scans, n)
    timed = res[args.warmup:]
    rays = sum(r for r, _ in timed)
    secs = sum(t for _, t in timed)
    v = rays / secs
    line = {"impl": "reference", "metric": metric_of(args.workload), "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded procedural terrain and lidar model)",
            "config": config_of(args.workload, cfg, args.high_speed_scans if args.workload == "high_speed" else 20,
                                args.gpus),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": f"{len(timed)} full scans of the workload (shift + ingest + extract each)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "map_updates_per_s": len(timed) / secs}
    print(json.dumps(line), flush=True)


def run_batched(args, gv, tune, torch, inputs, flush, stream):
    """The batched workload: the same maps and scans stepped as one batch
    (graph replay) and as one plain update + extraction per map."""
    import numpy as np
    cfg4, steps = inputs
    ms = cfg4.map
    nm = len(steps[0])
    mk = lambda: [gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
                  for _ in range(nm)]
    maps_b, maps_p = mk(), mk()
    dev = [[torch.from_numpy(s.points).cuda() for s in st] for st in steps]
    poses = [[s.T_ws for s in st] for st in steps]
    vehs = [[s.vehicle_xyz for s in st] for st in steps]
    max_pts = max(sum(int(p.shape[0]) for p in d) for d in dev)
    batch = gv.MapBatch(nm, max_pts, graph=True)
    outs_b = [m.alloc_maps() for m in maps_b]
    outs_p = [m.alloc_maps() for m in maps_p]
    for m in maps_p:
        m.reserve(max(int(d[i].shape[0]) for d in dev for i in range(nm)))
    best, entry = tune.tune_batch(batch, maps_b, [(vehs[k], dev[k], poses[k]) for k in range(len(steps))],
                                  flush=flush, refresh=args.retune)
    for m in maps_p:
        m.set_tuning(*best)
    for m in maps_b:  # the search stepped these maps: start both sets empty
        m.reset((0, 0, 0))
        m.reset_stats()

    def plain_step(k):
        j = k % len(steps)
        for i, m in enumerate(maps_p):
            m.update(vehs[j][i], dev[j][i], poses[j][i])
            m.extract_maps(outs_p[i])

    def batched_step(k):
        j = k % len(steps)
        batch.step(maps_b, vehs[j], dev[j], poses[j], outs=outs_b)

    def timed(fn, maps):
        for k in range(args.warmup):
            fn(k)
        torch.cuda.synchronize()
        st0 = [m.stats()["rays_valid"] for m in maps]
        l0 = gv.gvom_kernel_launches()
        evs = []
        for k in range(args.batched_steps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(args.warmup + k)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms_ = [a.elapsed_time(b) for a, b in evs]
        launches = (gv.gvom_kernel_launches() - l0) / args.batched_steps
        rays = sum(m.stats()["rays_valid"] for m in maps) - sum(st0)
        return rays / (sum(ms_) * 1e-3), statistics.median(ms_), launches, rays / args.batched_steps

    p_rate, p_ms, p_l, p_rays = timed(plain_step, maps_p)
    b_rate, b_ms, b_l, b_rays = timed(batched_step, maps_b)
    # the two forms computed the same maps
    same = all(torch.equal(outs_b[i]["flags"], outs_p[i]["flags"]) for i in range(nm))
    # fixed cost of the step's graph: the same maps, no points and no window
    # motion, no extraction, so its kernels (shift, per-point pass, walk) find
    # no work: what is left is launch and drain
    empty = [torch.empty((0, 3), dtype=torch.float32, device="cuda") for _ in range(nm)]
    # a vehicle position whose window origin is the map's current one
    half = np.array([ms.nx // 2, ms.ny // 2, ms.nz // 2], dtype=np.float64)
    veh0 = [(np.asarray(maps_b[i].origin, dtype=np.float64) + half + 0.5) * ms.res for i in range(nm)]
    for _ in range(3):
        batch.step(maps_b, veh0, empty, poses[0])
    torch.cuda.synchronize()
    e_ms = []
    for _ in range(20):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # keep the GPU busy (~1 ms spin) while the host marshals the step, so
        # that the events bracket device time only
        torch.cuda._sleep(2_000_000)
        e0.record(stream)
        batch.step(maps_b, veh0, empty, poses[0])
        e1.record(stream)
        e1.synchronize()
        e_ms.append(e0.elapsed_time(e1))
    empty_launches = 3
    batch.close()
    for m in maps_b + maps_p:
        m.close()
    return {"workload": BATCHED_WORKLOAD.format(m=nm), "maps": nm, "rays_per_step": b_rays,
            "points_per_step": [int(sum(int(p.shape[0]) for p in d)) for d in dev],
            "rays_per_s_batched": b_rate, "rays_per_s_plain": p_rate, "speedup": b_rate / p_rate,
            "ms_per_step_batched": b_ms, "ms_per_step_plain": p_ms,
            "map_updates_per_s_batched": nm * 1e3 / b_ms, "map_updates_per_s_plain": nm * 1e3 / p_ms,
            "gpu_launches_per_step_batched": b_l, "gpu_launches_per_step_plain": p_l,
            "graph": True, "tuning": {"seg_len": best[0], "march_block": best[1], "march_blocks_per_sm": best[2]},
            "outputs_identical": bool(same), "steps": args.batched_steps,
            "graph_fixed_cost": {"empty_step_us_median": 1e3 * statistics.median(e_ms), "kernels": empty_launches,
                                 "per_kernel_us": 1e3 * statistics.median(e_ms) / empty_launches,
                                 "share_of_step_for_all_kernels": (1e3 * statistics.median(e_ms) / empty_launches)
                                 * b_l / (1e3 * b_ms),
                                 "note": "graph replay of a step with no points, no window motion and no "
                                         "extraction (shift, per-point pass and walk launch with nothing to do)"},
            "l2": L2_NOTE}


def run_next_rows(args, gv, torch, cfg, scans, tuning, flush, stream, serial_e2e, hbm_peak):
    """The widened rows on the plain-sequence workload: the asynchronous
    pipeline end to end, the lookup-table export, a 10-scan buffer, and four
    sensors per scan folded in one launch."""
    from paper_2109_13176_gb300 import tune
    ms = cfg.map
    dev_pts = [torch.from_numpy(s.points).cuda() for s in scans]
    host_pts = [torch.from_numpy(s.points).pin_memory() for s in scans]
    kw = dict(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
    n_steps = args.steps
    ns = len(scans)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {}

    # asynchronous pipeline: pinned host scan in, pinned host products out
    m = gv.VoxelMap(**kw)
    tune.apply_walk(m, tuning)
    pipe = gv.Pipeline(m, max(int(p.shape[0]) for p in host_pts))
    houts = [pipe.alloc_host_outs() for _ in range(3)]
    t = 0
    for k in range(args.warmup):
        s = scans[k % ns]
        t = pipe.submit(s.vehicle_xyz, host_pts[k % ns], s.T_ws, houts[k % 3])
    pipe.wait(t)
    # a window of many scans (host wall clock), the median of three windows
    n_pipe = max(n_steps, 200)
    walls, rays = [], 0
    for rep in range(3):
        r0 = m.stats()["rays_valid"]
        torch.cuda.synchronize()
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        for i in range(n_pipe):
            k = args.warmup + i
            s = scans[k % ns]
            t = pipe.submit(s.vehicle_xyz, host_pts[k % ns], s.T_ws, houts[k % 3])
        pipe.wait(t)
        walls.append(time.perf_counter() - t0)
        gc.enable()
        rays = m.stats()["rays_valid"] - r0
    wall = statistics.median(walls)
    out["pipeline_e2e"] = {"value": rays / wall, "unit": UNIT, "ms_per_scan": 1e3 * wall / n_pipe,
                           "vs_serial_e2e": rays / wall / serial_e2e if serial_e2e else None, "depth": 3,
                           "scans_per_window": n_pipe,
                           "timing": "host wall clock from submit of the first scan to the last scan's products "
                                     "in pinned host memory, median of three windows; steps overlap, so L2 is "
                                     "not flushed between them"}
    pipe.close()

    # lookup-table export of the map the pipeline left
    V = ms.nx * ms.ny * ms.nz
    lut = torch.empty(V, dtype=torch.int64, device="cuda")
    dh = torch.empty(V, dtype=torch.int32, device="cuda")
    dp = torch.empty(V, dtype=torch.int32, device="cuda")
    dm = torch.empty(V, dtype=torch.float32, device="cuda")
    n_occ = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(args.warmup):
        gv.gvom_export_lut(m.handle, lut, dh, dp, dm, V, n_occ, stream)
    lut_ms = []
    for _ in range(n_steps):
        flush()
        e0, e1 = ev(), ev()
        e0.record(stream)
        gv.gvom_export_lut(m.handle, lut, dh, dp, dm, V, n_occ, stream)
        e1.record(stream)
        e1.synchronize()
        lut_ms.append(e0.elapsed_time(e1))
    occ = int(n_occ.item())
    lut_bytes = 20 * V + 12 * occ
    lut_s = statistics.mean(lut_ms) * 1e-3
    out["lut_export"] = {"ms": 1e3 * lut_s, "voxels": V, "occupied": occ,
                         "algorithmic_bytes": lut_bytes, "achieved_gbs": lut_bytes / lut_s / 1e9,
                         "frac_hbm": lut_bytes / lut_s / 1e9 / hbm_peak if hbm_peak else None,
                         "bytes_rule": "12 B/voxel read + 8 B/voxel table write + 12 B per occupied voxel",
                         "kernels": 3}
    m.close()

    def timed_steps(mp, fn):
        for k in range(args.warmup):
            fn(k)
        torch.cuda.synchronize()
        r0 = mp.stats()["rays_valid"]
        l0 = gv.gvom_kernel_launches()
        # like the main leg: events around each step, one synchronisation at
        # the end (the host enqueues ahead of the device)
        evs = []
        for i in range(n_steps):
            flush()
            e0, e1 = ev(), ev()
            e0.record(stream)
            fn(args.warmup + i)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ts = [a.elapsed_time(b) for a, b in evs]
        return ((mp.stats()["rays_valid"] - r0) / (sum(ts) * 1e-3), statistics.median(ts),
                (gv.gvom_kernel_launches() - l0) / n_steps)

    # 10-scan buffer: the same step on a map that holds its last 10 scans
    mb = gv.VoxelMap(scan_buffer=10, **kw)
    tune.apply_walk(mb, tuning)
    ob = mb.alloc_maps()

    def buffered_step(k):
        s = scans[k % ns]
        mb.update(s.vehicle_xyz, dev_pts[k % ns], s.T_ws)
        mb.extract_maps(ob)
    rate, med, launches = timed_steps(mb, buffered_step)
    out["scan_buffer"] = {"K": 10, "value": rate, "unit": UNIT, "ms_per_step_median": med,
                          "gpu_launches_per_step": launches,
                          "note": "shift of all slots + eviction of the oldest slot + ingest into map and slot + extract"}
    mb.close()

    # four sensors per scan (each scan cut into four quarters, one pose each)
    quarters = [[p[j * (p.shape[0] // 4):(j + 1) * (p.shape[0] // 4)] for j in range(4)] for p in dev_pts]
    mm, mseq = gv.VoxelMap(**kw), gv.VoxelMap(**kw)
    tune.apply_walk(mm, tuning)
    tune.apply_walk(mseq, tuning)

    def multi_step(k):
        s = scans[k % ns]
        mm.shift(mm.origin_for_pose(s.vehicle_xyz))
        mm.ingest_multi(quarters[k % ns], [s.T_ws] * 4)

    def seq_step(k):
        s = scans[k % ns]
        mseq.shift(mseq.origin_for_pose(s.vehicle_xyz))
        for q in quarters[k % ns]:
            mseq.ingest(q, s.T_ws)
    r_m, med_m, l_m = timed_steps(mm, multi_step)
    r_s, med_s, l_s = timed_steps(mseq, seq_step)
    same = all(torch.equal(a, b) for a, b in zip(mm.extract_voxels(), mseq.extract_voxels()))
    out["multi_sensor"] = {"sensors": 4, "value_one_launch": r_m, "value_sequential": r_s, "unit": UNIT,
                           "ms_per_step_one_launch": med_m, "ms_per_step_sequential": med_s,
                           "gpu_launches_per_step_one_launch": l_m, "gpu_launches_per_step_sequential": l_s,
                           "state_identical": bool(same), "note": "shift + ingest only (no extraction)"}
    mm.close()
    mseq.close()
    out["l2"] = L2_NOTE + "; the pipeline is not flushed"
    return out


def measure_plain(args, gv, tune, torch, inputs, flush, stream, world=1, clocks=None, e2e_steps=200):
    """One plain workload through the public API: the timed steps (shift +
    ingest + extract, CUDA events per step on the launching stream, L2
    flushed between steps, one synchronisation at the end), then the same
    update end to end with host buffers (pinned H2D copy of the scan,
    gvom_update_extract, one D2H copy of the packed products, per step).
    Returns the raw figures; the map is closed."""
    import contextlib
    cfg, scans = inputs
    ms = cfg.map
    ns = len(scans)
    dev_pts = [torch.from_numpy(s.points).cuda() for s in scans]
    host_pts = [torch.from_numpy(s.points).pin_memory() for s in scans]
    gmap = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
    out = gmap.alloc_maps()
    # launch shape for this workload: cached, or searched on its first scans
    nt = min(4, ns)
    if getattr(args, "tuning", None):
        # a walk shape named on the command line instead of the tuner's
        tuning = tuple(int(v) for v in args.tuning.split("/"))
        tune.apply_walk(gmap, tuning)
        tune_entry = {"forced": args.tuning}
    else:
        tuning, tune_entry = tune.tune_map(gmap, dev_pts[:nt], [s.T_ws for s in scans[:nt]],
                                           [s.vehicle_xyz for s in scans[:nt]], flush=flush, refresh=args.retune)
    # extraction shapes, on the state those scans left
    ext_tuning, ext_entry = tune.tune_extract(gmap, out, flush=flush, refresh=args.retune)
    gmap.reset((0, 0, 0))
    gmap.reset_stats()

    def step(k, ev_ingest0=None, ev_ingest1=None):
        s = scans[k % ns]
        gmap.shift(gmap.origin_for_pose(s.vehicle_xyz))
        if ev_ingest0 is not None:
            ev_ingest0.record(stream)
        gmap.ingest(dev_pts[k % ns], s.T_ws)
        if ev_ingest1 is not None:
            ev_ingest1.record(stream)
        gmap.extract_maps(out)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    st0 = gmap.stats()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    launches0 = gv.gvom_kernel_launches()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    gc.collect()
    gc.disable()
    with (clocks if clocks is not None else contextlib.nullcontext()):
        for i in range(args.steps):
            flush()
            e = ev[i]
            e[0].record(stream)
            step(args.warmup + i, e[1], e[2])
            e[3].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = gv.gvom_kernel_launches() - launches0  # this library's kernels only
    st1 = gmap.stats()
    r = {"step_ms": [e[0].elapsed_time(e[3]) for e in ev], "ingest_ms": [e[1].elapsed_time(e[2]) for e in ev],
         "extract_ms": [e[2].elapsed_time(e[3]) for e in ev],
         "shift_ms": [e[0].elapsed_time(e[1]) for e in ev],
         "rays": st1["rays_valid"] - st0["rays_valid"], "visits": st1["pass_visits"] - st0["pass_visits"],
         "hits": st1["hits_in_window"] - st0["hits_in_window"], "launches": launches,
         "tuning": tuning, "tune_entry": tune_entry, "ext_tuning": ext_tuning, "ext_entry": ext_entry,
         "cfg": cfg, "n_scans": ns}
    r["total_s"] = sum(r["step_ms"]) * 1e-3

    # the walk by itself: a caller event recorded by the library between the
    # per-point pass and the segment walk (a separate loop, so the marker
    # does not touch the timed steps above)
    wk_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    for e in wk_ev:
        for x in e:
            x.record(stream)  # creates the events before their handles are passed on
    torch.cuda.synchronize()
    sw0 = gmap.stats()
    for i in range(args.steps):
        flush()
        s = scans[(args.warmup + i) % ns]
        e = wk_ev[i]
        gmap.shift(gmap.origin_for_pose(s.vehicle_xyz))
        e[0].record(stream)
        gv.gvom_set_walk_marker(gmap.handle, e[1])
        gmap.ingest(dev_pts[(args.warmup + i) % ns], s.T_ws)
        e[2].record(stream)
        gmap.extract_maps(out)
    gv.gvom_set_walk_marker(gmap.handle, None)
    torch.cuda.synchronize()
    sw1 = gmap.stats()
    r["walk_ms"] = [e[1].elapsed_time(e[2]) for e in wk_ev]
    r["rays_pass_ms"] = [e[0].elapsed_time(e[1]) for e in wk_ev]
    r["walk_visits"] = sw1["pass_visits"] - sw0["pass_visits"]
    r["walk_hits"] = sw1["hits_in_window"] - sw0["hits_in_window"]
    r["fused"] = len(tuning) > 3 and bool(tuning[3])

    # end to end through the public API with host buffers
    h2d = sum(p.numel() * 4 for p in host_pts) / ns
    packed_dev, packed_out = gmap.alloc_maps_packed()
    packed_host = torch.empty(packed_dev.numel(), dtype=torch.uint8, pin_memory=True)
    staging = torch.empty((max(int(p.shape[0]) for p in dev_pts), 3), dtype=torch.float32, device="cuda")
    e2e_ms = []
    for i in range(e2e_steps):
        flush()
        k = args.warmup + args.steps + i
        s = scans[k % ns]
        hp = host_pts[k % ns]
        view = staging[:hp.shape[0]]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        view.copy_(hp, non_blocking=True)
        gmap.update_extract(s.vehicle_xyz, view, s.T_ws, packed_out)
        packed_host.copy_(packed_dev, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    st2 = gmap.stats()
    r.update({"e2e_ms": e2e_ms, "e2e_s": sum(e2e_ms) * 1e-3, "rays_e2e": st2["rays_valid"] - st1["rays_valid"],
              "h2d": int(h2d), "d2h": int(packed_dev.numel())})

    # end to end through the asynchronous pipeline (gvom_pipeline_*): the same
    # scans from pinned host memory, every product back in pinned host
    # memory, with the copies of neighbouring scans overlapping the compute;
    # host wall clock from the first submit to the last scan's products
    pipe = gv.Pipeline(gmap, max(int(p.shape[0]) for p in host_pts))
    houts = [pipe.alloc_host_outs() for _ in range(3)]
    tk = 0
    for i in range(6):
        s = scans[i % ns]
        tk = pipe.submit(s.vehicle_xyz, host_pts[i % ns], s.T_ws, houts[i % 3])
    pipe.wait(tk)
    torch.cuda.synchronize()
    p0 = gmap.stats()["rays_valid"]
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        k = args.warmup + i
        s = scans[k % ns]
        tk = pipe.submit(s.vehicle_xyz, host_pts[k % ns], s.T_ws, houts[i % 3])
    pipe.wait(tk)
    wall = time.perf_counter() - t0
    gc.enable()
    r.update({"e2e_pipe_s": wall, "rays_e2e_pipe": gmap.stats()["rays_valid"] - p0, "e2e_pipe_steps": e2e_steps,
              "d2h_pipe": int(sum(v.numel() * v.element_size() for v in houts[0].values()))})
    pipe.close()
    gmap.close()
    return r


def walk_roofline(r, steps, red_coalesced, red_scattered, workload):
    """The dominant kernel, the segment walk (k_march), timed by itself with
    the library's walk marker: its pass increments per launch over its
    average duration, against the L2's best-case increment rate (warp-wide
    reduction atomics on one 128-byte line, measured in this run); beside it
    the rate for scattered single-word atomics, which the walk's run merging
    can exceed."""
    fused = r.get("fused", False)
    # the fused kernel also lists the scan: its hit and lowest-return atomics count too
    inc = (r["walk_visits"] + (2 * r["walk_hits"] if fused else 0)) / steps
    t = statistics.mean(r["walk_ms"]) * 1e-3
    achieved = inc / t
    kernel = "k_ingest_fused" if fused else "k_march"
    return {"kernel": kernel, "bound": "l2_atomic", "achieved": achieved / 1e9, "peak": red_coalesced / 1e9,
            "unit": "Gincrement/s", "frac": achieved / red_coalesced,
            "traffic": profile_traffic(kernel, "plain_" + workload),
            "launch_us": 1e6 * t, "increments_per_launch": inc,
            "peak_source": "measured in this run: 32-bit reduction atomics, 32 lanes on one 128-byte line per warp "
                           "instruction, over 64 MiB (gvom_microbench_red_coalesced)",
            "peak_scattered": red_scattered / 1e9, "frac_vs_scattered": achieved / red_scattered,
            "algorithmic": "pass increments (ray/voxel crossings counted) per launch",
            "timing": "CUDA events on the launching stream around the walk (library walk marker), mean of the "
                      "timed steps of a separate loop"}


def ingest_roofline(r, steps, red_peak, workload):
    """The ingest (per-point pass + segment walk, one timed region) against
    the measured L2 reduction-atomic rate."""
    atom = (r["visits"] + 2 * r["hits"]) / steps
    achieved = atom / (statistics.mean(r["ingest_ms"]) * 1e-3)
    return {"kernel": "k_rays + k_march", "bound": "l2_atomic", "achieved": achieved / 1e9, "peak": red_peak / 1e9,
            "unit": "Gatomic/s", "frac": achieved / red_peak,
            "traffic": profile_traffic("k_ingest", "plain_" + workload),
            "peak_source": "measured in this run: scattered 32-bit reduction atomics over 64 MiB (gvom_microbench_red)",
            "algorithmic": "pass visits + 2 atomics per in-window hit, per launch"}


def extract_roofline(r, ms, hbm_peak, peak_kind):
    V = ms.nx * ms.ny * ms.nz
    b = 12 * V + (4 + 4 + 1 + 4 + 4) * ms.nx * ms.ny
    t = statistics.mean(r["extract_ms"]) * 1e-3
    return {"kernels": "k_columns + k_slope_negative", "bound": "hbm", "achieved": b / t / 1e9, "peak": hbm_peak,
            "unit": "GB/s", "frac": b / t / 1e9 / hbm_peak if hbm_peak else None, "algorithmic_bytes": b,
            "bytes_rule": "12 B/voxel read + 17 B/px written", "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}


def e2e_object(r):
    """End to end through the public API: the asynchronous pipeline (the
    value), with one synchronised scan at a time beside it."""
    return {"value": r["rays_e2e_pipe"] / r["e2e_pipe_s"], "unit": UNIT, "h2d_bytes_per_step": r["h2d"],
            "d2h_bytes_per_step": r["d2h_pipe"], "ms_per_step": 1e3 * r["e2e_pipe_s"] / r["e2e_pipe_steps"],
            "steps": r["e2e_pipe_steps"],
            "call": "gvom_pipeline_submit per scan (pinned host points in; shift, ingest and every product; each "
                    "scan's products back in pinned host memory), three scans in flight, host wall clock from the "
                    "first submit to the last scan's products; no L2 flush (scans overlap)",
            "serial": {"value": r["rays_e2e"] / r["e2e_s"], "ms_per_step_p50": statistics.median(r["e2e_ms"]),
                       "ms_per_step_p99": sorted(r["e2e_ms"])[int(0.99 * (len(r["e2e_ms"]) - 1))],
                       "d2h_bytes_per_step": r["d2h"], "steps": len(r["e2e_ms"]),
                       "call": "one scan at a time: pinned H2D copy, gvom_update_extract, one D2H copy of the "
                               "packed products, synchronised, CUDA events per scan"}}


def plain_summary(args, r, workload, red_peak, red_coalesced, hbm_peak, peak_kind):
    """The sub-object of a plain workload measured beside the main leg."""
    cfg = r["cfg"]
    ms = cfg.map
    steps = args.steps
    return {"workload": workload_text(workload, r["n_scans"]), "metric": metric_of(workload),
            "value": r["rays"] / r["total_s"], "unit": UNIT, "map_updates_per_s": steps / r["total_s"],
            "ms_per_step_mean": 1e3 * r["total_s"] / steps, "ms_per_step_median": statistics.median(r["step_ms"]),
            "rays_per_step": r["rays"] / steps, "pass_visits_per_step": r["visits"] / steps,
            "hits_per_step": r["hits"] / steps, "shift_ms_mean": statistics.mean(r["shift_ms"]),
            "ingest_ms_mean": statistics.mean(r["ingest_ms"]), "extract_ms_mean": statistics.mean(r["extract_ms"]),
            "per_point_pass_ms_mean": statistics.mean(r["rays_pass_ms"]), "walk_ms_mean": statistics.mean(r["walk_ms"]),
            "roofline": walk_roofline(r, steps, red_coalesced, red_peak, workload),
            "roofline_ingest": ingest_roofline(r, steps, red_peak, workload),
            "roofline_step": roofline_step((r["visits"] + 2 * r["hits"]) / steps, red_peak, ms.nx * ms.ny * ms.nz, ms,
                                           cfg.lidar.n, hbm_peak, r["total_s"] / steps),
            "roofline_extract": extract_roofline(r, ms, hbm_peak, peak_kind),
            "e2e": e2e_object(r), "gpu_launches_per_step": r["launches"] / steps,
            "tuning": {"seg_len": r["tuning"][0], "march_block": r["tuning"][1],
                       "march_blocks_per_sm": r["tuning"][2], "fused_ingest": int(r["fused"]),
                       "px_tile": r["ext_tuning"][0], "col_shape": r["ext_tuning"][1]},
            "l2": L2_NOTE}


def oracle_plain_baseline(inputs, time_budget_s: float, workload: str):
    """The oracle on the first scans of a plain workload (one thread)."""
    cfg, scans = inputs
    res = run_oracle_steps(cfg, scans, len(scans) * 10, time_budget_s=time_budget_s)
    return {"value": sum(r for r, _ in res) / sum(t for _, t in res), "unit": UNIT, "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": f"first {len(res)} scans of the {workload} workload, shift + ingest + extract each, "
                      "single thread"}


def served_pools(torch, robots, arrivals):
    """scans[robot][k] for the server: the arrival's cast (pinned host
    memory, shared by the arrivals of one span) with the arrival's pose."""
    casts = {i: [torch.from_numpy(c.points).pin_memory() for c in r["casts"]] for i, r in enumerate(robots)}
    pools = {i: {} for i in range(len(robots))}
    for t, rid, k, c, T, veh in arrivals:
        pools[rid][k] = dict(points=casts[rid][c], T_ws=T, vehicle_xyz=veh)
    return pools


def run_served(args, gv, torch, inputs):
    """The served workload: real-time replay with continuous batching and
    per-scan admission (latency), the same stream offered 2-16 times faster
    (latency against load), then all requests at once (capacity); beside
    them one plain update per scan."""
    from paper_2109_13176_gb300.serve import Server
    robots, arrivals = inputs
    specs = {i: r["map"] for i, r in enumerate(robots)}
    pools = served_pools(torch, robots, arrivals)
    arr = [(t, rid, k) for t, rid, k, *_ in arrivals]
    max_pts = sum(max(int(c.points.shape[0]) for c in r["casts"]) for r in robots)

    def replay(stream, realtime=True, scale=1.0):
        srv = Server(specs, slots=2, max_batch_maps=len(robots), max_batch_points=max_pts, reserve_bytes=2 << 30)
        # the collector stays off during each replay, as in the main leg's timed region
        gc.collect()
        gc.disable()
        try:
            out = srv.run(stream, pools, realtime=realtime, time_scale=scale).summary()
        finally:
            gc.enable()
            srv.close()
        return out

    rt = replay(arr)
    sweep = [dict(load=1.0, offered_scans_per_s=len(arr) / args.served_seconds, window_s=args.served_seconds,
                  **{k: rt[k] for k in ("requests", "p50_ms", "p99_ms", "max_ms", "mean_batch_maps", "rays_per_s",
                                        "deferred")})]
    for f in SERVED_LOADS:
        # the first f * window seconds of the stream, offered f times faster
        part = [a for a in arr if a[0] < f * SERVED_SWEEP_WINDOW_S]
        st = replay(part, scale=f)
        sweep.append(dict(load=f, offered_scans_per_s=f * len(arr) / args.served_seconds,
                          window_s=min(SERVED_SWEEP_WINDOW_S, args.served_seconds / f),
                          **{k: st[k] for k in ("requests", "p50_ms", "p99_ms", "max_ms", "mean_batch_maps",
                                                "rays_per_s", "deferred")}))
    ok = [p["load"] for p in sweep if p["p99_ms"] is not None and p["p99_ms"] < 100.0]
    sat = replay(arr, realtime=False)
    # the plain path on the same requests: one update + extraction + readback per scan, in order
    maps = {i: gv.VoxelMap(nx=sp.nx, ny=sp.ny, nz=sp.nz, res=sp.res, neg_max_px=int(math.ceil(2.0 / sp.res)))
            for i, sp in specs.items()}
    outs = {i: m.alloc_maps() for i, m in maps.items()}
    host = {i: {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in o.items()} for i, o in outs.items()}
    staging = torch.empty((max(int(c.points.shape[0]) for r in robots for c in r["casts"]), 3), device="cuda")
    r0 = {i: m.stats()["rays_valid"] for i, m in maps.items()}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t, rid, k in arr:
        sc = pools[rid][k]
        n = int(sc["points"].shape[0])
        view = staging[:n]
        view.copy_(sc["points"], non_blocking=True)
        maps[rid].update(sc["vehicle_xyz"], view, sc["T_ws"])
        maps[rid].extract_maps(outs[rid])
        for key, v in outs[rid].items():
            host[rid][key].copy_(v, non_blocking=True)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_rays = sum(m.stats()["rays_valid"] - r0[i] for i, m in maps.items())
    for m in maps.values():
        m.close()
    return {"workload": SERVED_WORKLOAD.format(s=args.served_seconds), "robots": len(robots),
            "requests": len(arr), "realtime": rt, "load_sweep": sweep,
            "max_load_with_p99_under_100ms": max(ok) if ok else None,
            "saturated": sat,
            "plain_sequential": {"rays_per_s": plain_rays / plain_s, "wall_s": plain_s},
            "capacity_speedup_vs_plain": sat["rays_per_s"] / (plain_rays / plain_s),
            "slots": 2, "admission": "per scan, device-memory budget (free memory at start - 2 GiB - staging); "
                                     "maps created on a robot's first scan",
            "latency": "arrival to 2D products in pinned host memory (device event times)"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    # inputs first: the generator's process pools start before any CUDA call
    main_wl = args.workload
    other_wl = "sequence" if main_wl == "high_speed" else "high_speed"
    inputs = make_inputs(rank, main_wl, args.high_speed_scans)
    other_inputs = None if args.no_other else make_inputs(rank, other_wl, args.high_speed_scans)
    seq_inputs = inputs if main_wl == "sequence" else other_inputs
    if seq_inputs is None and not args.no_next_rows:
        seq_inputs = make_inputs(rank, "sequence")
    batched_inputs = None if args.no_batched else make_batched_inputs(rank, args.batched_maps)
    served_inputs = None if args.no_served else make_served_inputs(rank, args.served_seconds)

    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2109_13176_gb300 import build as gvbuild
    gvbuild.build()
    import paper_2109_13176_gb300 as gv
    from paper_2109_13176_gb300 import tune

    flush_buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    clean_buf = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    flush_k = [0]

    def flush():
        # write a buffer larger than L2 (no step data stays cached), then read
        # another one, so that the write's dirty lines are written back here
        # and not inside the next timed step
        flush_k[0] += 1
        flush_buf.fill_(flush_k[0] & 0xff)
        clean_buf.sum()

    # the main leg: timed steps with clocks sampled, then e2e
    clocks = ClockSampler(local)
    r = measure_plain(args, gv, tune, torch, inputs, flush, stream, world=world, clocks=clocks,
                      e2e_steps=max(args.steps, 200))
    total_s, e2e_s, rays, rays_e2e = r["total_s"], r["e2e_pipe_s"], r["rays"], r["rays_e2e_pipe"]
    if world > 1:
        (total_s, e2e_s), (rays, rays_e2e) = reduce_over_ranks([total_s, e2e_s], [rays, rays_e2e], "cuda")

    if rank != 0:
        dist.destroy_process_group() if world > 1 else None
        return

    peaks, peak_kind = read_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    red_peak = measure_red_peak(gv, torch)
    red_coalesced = measure_red_peak(gv, torch, coalesced=True)
    cfg = r["cfg"]
    ms = cfg.map

    other = None
    if other_inputs is not None:
        ro = measure_plain(args, gv, tune, torch, other_inputs, flush, stream)
        other = plain_summary(args, ro, other_wl, red_peak, red_coalesced, hbm_peak, peak_kind)
        if not args.no_cpu_baseline:
            other["cpu_baseline"] = oracle_plain_baseline(other_inputs, 6.0, other_wl)
    batched = None
    if batched_inputs is not None:
        batched = run_batched(args, gv, tune, torch, batched_inputs, flush, stream)
        if not args.no_cpu_baseline:
            batched["cpu_baseline"] = oracle_batched_baseline(batched_inputs, 16)
    served = None
    if served_inputs is not None:
        served = run_served(args, gv, torch, served_inputs)
        if not args.no_cpu_baseline:
            served["cpu_baseline"] = oracle_served_baseline(served_inputs, 8.0)
    next_rows = None
    if not args.no_next_rows:
        seq_cfg, seq_scans = seq_inputs
        seq_tuning = r["tuning"] if main_wl == "sequence" else (
            tuple(other["tuning"][k] for k in ("seg_len", "march_block", "march_blocks_per_sm", "fused_ingest"))
            if other else (16, 256, 0, 0))
        seq_e2e = (r["rays_e2e"] / r["e2e_s"]) if main_wl == "sequence" else (
            other["e2e"]["serial"]["value"] if other else None)
        next_rows = run_next_rows(args, gv, torch, seq_cfg, seq_scans, seq_tuning, flush, stream, seq_e2e, hbm_peak)

    cpu = None
    if not args.no_cpu_baseline:
        cpu = oracle_plain_baseline(inputs, args.cpu_sample_s, main_wl)

    steps = args.steps
    atom_per_launch = (r["visits"] + 2 * r["hits"]) / steps
    line = {
        "metric": metric_of(main_wl), "value": rays / total_s, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 transform, int32 traversal, u32 counts, f32 maps",
        "data": f"synthetic (seeded procedural terrain, boxes, ditches; {cfg.lidar.beams}-beam lidar model)",
        "config": config_of(main_wl, cfg, r["n_scans"], world),
        "map_updates_per_s": steps * world / total_s,
        "rays_per_step": rays / (steps * world),
        "pass_visits_per_step": r["visits"] / steps,
        "step_ms": {"median": statistics.median(r["step_ms"]),
                    "p99": sorted(r["step_ms"])[int(0.99 * (len(r["step_ms"]) - 1))],
                    "shift_avg": statistics.mean(r["shift_ms"]), "ingest_avg": statistics.mean(r["ingest_ms"]),
                    "extract_avg": statistics.mean(r["extract_ms"]),
                    "per_point_pass_avg": statistics.mean(r["rays_pass_ms"]), "walk_avg": statistics.mean(r["walk_ms"])},
        "roofline": walk_roofline(r, steps, red_coalesced, red_peak, main_wl),
        "roofline_ingest": ingest_roofline(r, steps, red_peak, main_wl),
        "roofline_step": roofline_step(atom_per_launch, red_peak, ms.nx * ms.ny * ms.nz, ms, cfg.lidar.n, hbm_peak,
                                      r["total_s"] / steps),
        "roofline_extract": extract_roofline(r, ms, hbm_peak, peak_kind),
        "cpu_baseline": cpu,
        "e2e": dict(e2e_object(r), value=rays_e2e / e2e_s),
        "gpu_launches": int(r["launches"]),
        "clocks": clocks.summary(),
        "tuning": {"seg_len": r["tuning"][0], "march_block": r["tuning"][1], "march_blocks_per_sm": r["tuning"][2],
                   "fused_ingest": int(r["fused"]), "px_tile": r["ext_tuning"][0], "col_shape": r["ext_tuning"][1],
                   "search_us": r["tune_entry"].get("us"), "extract_search_us": r["ext_entry"].get("us")},
        other_wl: other,
        "batched": batched,
        "served": served,
        "next_rows": next_rows,
    }
    line["summary"] = summary_of(line)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
