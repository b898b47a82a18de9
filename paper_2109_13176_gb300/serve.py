"""Serving loop: continuous batching of arriving scans over resident maps.

Many robots stream scans at their own rates; every robot's map stays
resident on the GPU. Scans are admitted and batched as they arrive: whenever
one of the server's stream slots is free, the scans that are ready (at most
one per robot, and none for a robot whose previous scan is still on the
GPU, so each map sees its scans in arrival order) form one batch step
(gvom_batch_step: shift, ingest and extract for every map of the batch),
whose work overlaps on the device with the batches of the other slots. A
scan's latency runs from its arrival to the moment its 2D products are back
in host memory; the device timestamps of completion events are mapped to
the host clock, so no polling delay enters the figures.

Admission by device memory: a robot's map is created only while free
device memory minus a reserve covers it (else the robot is refused), and a
batch takes only as many points as its slot's staging buffer holds (the
rest wait for the next slot).

Scheduler and Admission are plain host logic (tested on CPU with fakes);
Server drives the GPU through the library's batch API.
"""
from __future__ import annotations

import collections
import math
import statistics
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    robot: int
    n_points: int
    arrival: float        # seconds on the server clock
    payload: object = None
    seq: int = 0          # per-robot sequence number
    done: float = math.nan


class Scheduler:
    """Per-robot FIFO queues and continuous batch formation."""

    def __init__(self, max_batch_maps: int, max_batch_points: int):
        self.max_maps = max_batch_maps
        self.max_points = max_batch_points
        self.queues: dict[int, collections.deque] = collections.defaultdict(collections.deque)
        self.busy: set[int] = set()   # robots with a scan on the GPU
        self.order: collections.deque = collections.deque()  # robots in order of their oldest waiting scan

    def arrive(self, req: Request) -> None:
        q = self.queues[req.robot]
        if not q:
            self.order.append(req.robot)
        q.append(req)

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values())

    def next_batch(self) -> list[Request]:
        """The oldest waiting scan of each idle robot, oldest first, within
        the batch's map and point limits."""
        batch, pts = [], 0
        skipped = []
        while self.order and len(batch) < self.max_maps:
            r = self.order.popleft()
            q = self.queues[r]
            if not q:
                continue
            if r in self.busy or pts + q[0].n_points > self.max_points:
                skipped.append(r)
                continue
            req = q.popleft()
            batch.append(req)
            pts += req.n_points
            self.busy.add(r)
            if q:
                skipped.append(r)
        # robots passed over keep their place at the front
        self.order.extendleft(reversed(skipped))
        return batch

    def finish(self, batch: list[Request]) -> None:
        for req in batch:
            self.busy.discard(req.robot)


class Admission:
    """Creates a robot's map only while free device memory covers it."""

    def __init__(self, mem_free_fn, reserve_bytes: int):
        self.mem_free = mem_free_fn
        self.reserve = reserve_bytes
        self.refused: list[int] = []

    def admit(self, robot: int, map_bytes: int) -> bool:
        free = self.mem_free()
        if free - map_bytes < self.reserve:
            self.refused.append(robot)
            return False
        return True


def map_bytes(spec, scan_buffer: int = 0) -> int:
    """Device memory of one map: 12 bytes per voxel (and as much again per
    slot of a scan buffer) plus 2D scratch and outputs."""
    return 12 * (1 + scan_buffer) * spec.nx * spec.ny * spec.nz + (4 + 17) * spec.nx * spec.ny + 4096


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    batches: int = 0
    batch_sizes: list = field(default_factory=list)
    rays: int = 0
    points: int = 0
    wall_s: float = 0.0
    refused_robots: list = field(default_factory=list)
    deferred: int = 0          # scans that waited past a free slot (busy robot or full staging)

    def summary(self) -> dict:
        lat = sorted(self.latencies_ms)

        def pct(p):
            return lat[min(len(lat) - 1, int(math.ceil(p / 100.0 * len(lat))) - 1)] if lat else None
        return {"requests": len(lat), "p50_ms": pct(50), "p99_ms": pct(99), "max_ms": lat[-1] if lat else None,
                "mean_ms": statistics.fmean(lat) if lat else None, "batches": self.batches,
                "mean_batch_maps": statistics.fmean(self.batch_sizes) if self.batch_sizes else 0.0,
                "rays": self.rays, "points": self.points, "wall_s": self.wall_s,
                "rays_per_s": self.rays / self.wall_s if self.wall_s > 0 else 0.0,
                "refused_robots": list(self.refused_robots), "deferred": self.deferred}


class Server:
    """Resident maps for many robots; continuous batching over stream slots."""

    def __init__(self, robot_specs: dict, slots: int = 2, max_batch_maps: int = 64,
                 max_batch_points: int = 4 << 20, reserve_bytes: int = 1 << 30, mem_free_fn=None,
                 graph: bool = True):
        import torch

        import paper_2109_13176_gb300 as gv
        self.torch = torch
        self.gv = gv
        mem = mem_free_fn or (lambda: torch.cuda.mem_get_info()[0])
        self.admission = Admission(mem, reserve_bytes)
        self.maps, self.outs, self.host_outs = {}, {}, {}
        for rid, spec in robot_specs.items():
            if not self.admission.admit(rid, map_bytes(spec)):
                continue
            m = gv.VoxelMap(nx=spec.nx, ny=spec.ny, nz=spec.nz, res=spec.res,
                            neg_max_px=int(math.ceil(2.0 / spec.res)))
            self.maps[rid] = m
            self.outs[rid] = m.alloc_maps()
            self.host_outs[rid] = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                                   for k, v in self.outs[rid].items()}
        self.sched = Scheduler(max_batch_maps, max_batch_points)
        self.slots = []
        for _ in range(slots):
            self.slots.append({
                "stream": torch.cuda.Stream(),
                "batch": gv.MapBatch(max_batch_maps, max_batch_points, graph=graph),
                "staging": torch.empty((max_batch_points, 3), dtype=torch.float32, device="cuda"),
                "event": None, "reqs": None,
            })

    def close(self):
        for s in self.slots:
            s["batch"].close()
        for m in self.maps.values():
            m.close()

    # one batch on a free slot
    def _launch(self, slot, batch):
        torch = self.torch
        st = slot["stream"]
        with torch.cuda.stream(st):
            off, views = 0, []
            for req in batch:
                n = req.n_points
                view = slot["staging"][off:off + n]
                if n:
                    view.copy_(req.payload["points"], non_blocking=True)
                views.append(view)
                off += n
            maps = [self.maps[r.robot] for r in batch]
            outs = [self.outs[r.robot] for r in batch]
            slot["batch"].step(maps, [r.payload["vehicle_xyz"] for r in batch], views,
                               [r.payload["T_ws"] for r in batch], outs=outs, stream=st)
            for r in batch:
                for k, v in self.outs[r.robot].items():
                    self.host_outs[r.robot][k].copy_(v, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
        slot["event"], slot["reqs"] = ev, batch

    def run(self, arrivals: list, scans: dict, realtime: bool = True, on_done=None) -> ServeStats:
        """arrivals: time-ordered (t_s, robot, pool_index); scans[robot][pool_index]
        = dict(points=pinned float32 (n,3) tensor, T_ws, vehicle_xyz). realtime:
        admit each scan at its arrival time; else all at once (saturation).
        on_done(req) is called after each scan's maps are back on the host."""
        torch = self.torch
        stats = ServeStats(refused_robots=list(self.admission.refused))
        reqs = []
        seq = collections.Counter()
        for t, rid, k in arrivals:
            if rid not in self.maps:
                continue
            sc = scans[rid][k]
            reqs.append(Request(rid, int(sc["points"].shape[0]), t if realtime else 0.0, sc, seq[rid]))
            seq[rid] += 1
        stats0 = {rid: m.stats()["rays_valid"] for rid, m in self.maps.items()}
        # host clock <-> device event clock
        ref = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ref.record()
        ref.synchronize()
        t0 = time.perf_counter()
        i, done = 0, 0
        while done < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                self.sched.arrive(reqs[i])
                i += 1
            progressed = False
            for slot in self.slots:
                ev = slot["event"]
                if ev is not None and ev.query():
                    t_done = ref.elapsed_time(ev) * 1e-3
                    for r in slot["reqs"]:
                        r.done = t_done
                        stats.latencies_ms.append(1e3 * (t_done - r.arrival))
                        stats.points += r.n_points
                        if on_done is not None:
                            on_done(r)
                    self.sched.finish(slot["reqs"])
                    done += len(slot["reqs"])
                    slot["event"], slot["reqs"] = None, None
                    progressed = True
                if slot["event"] is None:
                    waiting = self.sched.pending()
                    batch = self.sched.next_batch()
                    if batch:
                        stats.deferred += waiting - len(batch)
                        self._launch(slot, batch)
                        stats.batches += 1
                        stats.batch_sizes.append(len(batch))
                        progressed = True
            if not progressed:
                if i < len(reqs) and all(s["event"] is None for s in self.slots) and not self.sched.pending():
                    time.sleep(max(0.0, min(0.001, reqs[i].arrival - (time.perf_counter() - t0))))
                else:
                    time.sleep(20e-6)
        torch.cuda.synchronize()
        stats.wall_s = time.perf_counter() - t0
        stats.rays = sum(m.stats()["rays_valid"] - stats0[rid] for rid, m in self.maps.items())
        return stats
