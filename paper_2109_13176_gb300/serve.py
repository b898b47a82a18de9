"""Serving loop: continuous batching of arriving scans over resident maps.

Many robots stream scans at their own rates; every admitted robot's map
stays resident on the GPU. Scans are admitted and batched as they arrive:
whenever one of the server's stream slots is free, the scans that are ready
(at most one per robot, and none for a robot whose previous scan is still on
the GPU, so each map sees its scans in arrival order) form one batch step
(gvom_batch_step: shift, ingest and extract for every map of the batch),
whose work overlaps on the device with the batches of the other slots. A
scan's latency runs from its arrival to the moment its 2D products are back
in host memory; the device timestamps of completion events are mapped to
the host clock, so no polling delay enters the figures.

Admission by device memory, per scan: the server holds a device-memory
budget (free memory at start-up minus a reserve, less its own staging
buffers). A scan enters the scheduler only when its robot holds a map; a
robot's first scan creates the map if the budget still covers it, else the
robot's scans wait, in order, and are offered again whenever memory is
released. A robot that has been idle (nothing queued or in flight) for
`idle_release_s` gives its map back to the budget; its next scan starts a
new, empty map. A scan with more points than a batch's staging buffer holds
is refused outright. The rest of a batch's limit (points per batch) is
applied by the scheduler: scans that do not fit wait for the next slot.

Scheduler, Admission and FrontDoor are plain host logic (tested on CPU with
fakes); Server drives the GPU through the library's batch API.
"""
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
    """A device-memory budget shared by the robots' maps."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.used = 0
        self.held: dict = {}
        self.refusals = 0        # requests for memory that the budget did not cover
        self.releases = 0        # bumps whenever memory is given back

    @classmethod
    def from_free_memory(cls, mem_free_fn, reserve_bytes: int, extra_bytes: int = 0):
        """Budget = free device memory now - reserve - what the caller is
        about to allocate outside the budget (extra_bytes)."""
        return cls(max(0, int(mem_free_fn()) - int(reserve_bytes) - int(extra_bytes)))

    def try_hold(self, key, nbytes: int) -> bool:
        if key in self.held:
            return True
        if self.used + nbytes > self.budget:
            self.refusals += 1
            return False
        self.held[key] = int(nbytes)
        self.used += int(nbytes)
        return True

    def release(self, key) -> None:
        nb = self.held.pop(key, None)
        if nb is not None:
            self.used -= nb
            self.releases += 1


class FrontDoor:
    """Per-scan admission in front of the scheduler.

    offer(req): a scan whose robot holds a map goes to the scheduler; a robot
    without one gets it now if the memory budget covers it (create_map is
    called), else the scan waits behind the robot's earlier waiting scans.
    retry(): after memory was released, offers the waiting robots again, in
    the order their first scan arrived. release_idle(): robots with nothing
    queued, waiting or in flight since `idle_s` give their map back
    (release_map is called). Scans larger than max_points are refused."""

    def __init__(self, admission: Admission, sched: "Scheduler", bytes_of, create_map, release_map,
                 max_points: int):
        self.adm = admission
        self.sched = sched
        self.bytes_of = bytes_of
        self.create_map = create_map
        self.release_map = release_map
        self.max_points = max_points
        self.waiting: collections.OrderedDict = collections.OrderedDict()  # robot -> deque of requests
        self.has_map: set = set()
        self.last_seen: dict = {}
        self.rejected: list = []
        self.ever_waited: set = set()
        self._seen_releases = admission.releases

    def _admit_robot(self, robot) -> bool:
        if robot in self.has_map:
            return True
        if not self.adm.try_hold(robot, self.bytes_of(robot)):
            return False
        self.create_map(robot)
        self.has_map.add(robot)
        return True

    def offer(self, req: "Request", now: float) -> str:
        self.last_seen[req.robot] = now
        if req.n_points > self.max_points:
            self.rejected.append(req)
            return "rejected"
        if req.robot in self.waiting:
            self.waiting[req.robot].append(req)
            return "waiting"
        if self._admit_robot(req.robot):
            self.sched.arrive(req)
            return "admitted"
        self.waiting[req.robot] = collections.deque([req])
        self.ever_waited.add(req.robot)
        return "waiting"

    def retry(self, now: float) -> int:
        """Offers waiting robots again if memory was released since the last
        try; returns the number of scans that entered the scheduler."""
        if self.adm.releases == self._seen_releases or not self.waiting:
            return 0
        self._seen_releases = self.adm.releases
        moved = 0
        for robot in list(self.waiting):
            if not self._admit_robot(robot):
                continue
            q = self.waiting.pop(robot)
            while q:
                self.sched.arrive(q.popleft())
                moved += 1
        return moved

    def release_idle(self, now: float, idle_s: float) -> list:
        out = []
        for robot in list(self.has_map):
            if robot in self.sched.busy or self.sched.queues.get(robot) or robot in self.waiting:
                continue
            if now - self.last_seen.get(robot, now) >= idle_s:
                self.has_map.discard(robot)
                self.release_map(robot)
                self.adm.release(robot)
                out.append(robot)
        return out

    def pending(self) -> int:
        return sum(len(q) for q in self.waiting.values())


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
    refused_robots: list = field(default_factory=list)   # robots that had to wait for memory
    waited_scans: int = 0      # scans that waited for their robot's map (memory)
    rejected_scans: int = 0    # scans larger than a batch's staging buffer
    unserved_scans: int = 0    # scans still waiting for memory when nothing else was left
    released_maps: int = 0     # maps given back after idling
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
                "refused_robots": list(self.refused_robots), "waited_scans": self.waited_scans,
                "rejected_scans": self.rejected_scans, "unserved_scans": self.unserved_scans,
                "released_maps": self.released_maps, "deferred": self.deferred}


class Server:
    """Resident maps for many robots; per-scan admission by device memory;
    continuous batching over stream slots."""

    def __init__(self, robot_specs: dict, slots: int = 2, max_batch_maps: int = 64,
                 max_batch_points: int = 4 << 20, reserve_bytes: int = 1 << 30, mem_free_fn=None,
                 graph: bool = True, budget_bytes: int | None = None, idle_release_s: float | None = None):
        import torch

        import paper_2109_13176_gb300 as gv
        self.torch = torch
        self.gv = gv
        self.specs = dict(robot_specs)
        self.idle_release_s = idle_release_s
        staging_bytes = slots * max_batch_points * 12
        if budget_bytes is not None:
            self.admission = Admission(budget_bytes)
        else:
            mem = mem_free_fn or (lambda: torch.cuda.mem_get_info()[0])
            self.admission = Admission.from_free_memory(mem, reserve_bytes, staging_bytes)
        self.maps, self.outs, self.host_outs = {}, {}, {}
        self.sched = Scheduler(max_batch_maps, max_batch_points)
        self.door = FrontDoor(self.admission, self.sched, lambda r: map_bytes(self.specs[r]),
                              self._create_map, self._release_map, max_batch_points)
        self.rays_released = 0
        self._rays_base = {}   # rays of a map before the current run
        self.slots = []
        for _ in range(slots):
            self.slots.append({
                "stream": torch.cuda.Stream(),
                "batch": gv.MapBatch(max_batch_maps, max_batch_points, graph=graph),
                "staging": torch.empty((max_batch_points, 3), dtype=torch.float32, device="cuda"),
                "event": None, "reqs": None,
            })

    def _create_map(self, rid):
        torch, spec = self.torch, self.specs[rid]
        m = self.gv.VoxelMap(nx=spec.nx, ny=spec.ny, nz=spec.nz, res=spec.res,
                             neg_max_px=int(math.ceil(2.0 / spec.res)))
        self.maps[rid] = m
        self.outs[rid] = m.alloc_maps()
        self.host_outs[rid] = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                               for k, v in self.outs[rid].items()}

    def _release_map(self, rid):
        m = self.maps.pop(rid)
        self.rays_released += m.stats()["rays_valid"] - self._rays_base.pop(rid, 0)
        m.close()
        self.outs.pop(rid, None)
        self.host_outs.pop(rid, None)

    def admit_all(self, robots=None):
        """Creates the maps of the given robots (all known robots by default)
        up front, as far as the memory budget allows; returns those refused."""
        refused = []
        for rid in (self.specs if robots is None else robots):
            if not self.door._admit_robot(rid):
                refused.append(rid)
        return refused

    def close(self):
        for s in self.slots:
            s["batch"].close()
        for m in self.maps.values():
            m.close()
        self.maps.clear()

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

    def run(self, arrivals: list, scans: dict, realtime: bool = True, on_done=None, time_scale: float = 1.0) -> ServeStats:
        """arrivals: time-ordered (t_s, robot, key); scans[robot][key] =
        dict(points=pinned float32 (n,3) tensor, T_ws, vehicle_xyz). realtime:
        each scan arrives at t_s / time_scale seconds after the start (so
        time_scale > 1 offers the same stream faster); else all arrive at
        once (saturation). on_done(req) is called after each scan's maps are
        back on the host."""
        torch = self.torch
        stats = ServeStats()
        reqs = []
        seq = collections.Counter()
        for t, rid, k in arrivals:
            sc = scans[rid][k]
            reqs.append(Request(rid, int(sc["points"].shape[0]), t / time_scale if realtime else 0.0, sc, seq[rid]))
            seq[rid] += 1
        stats0 = {rid: m.stats()["rays_valid"] for rid, m in self.maps.items()}
        self._rays_base = dict(stats0)
        released0 = self.rays_released
        # host clock <-> device event clock
        ref = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ref.record()
        ref.synchronize()
        t0 = time.perf_counter()
        i, done = 0, 0
        door = self.door
        while True:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                r = reqs[i]
                st = door.offer(r, now)
                if st == "rejected":
                    stats.rejected_scans += 1
                elif st == "waiting":
                    stats.waited_scans += 1
                i += 1
            door.retry(now)
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
            if self.idle_release_s is not None:
                released = door.release_idle(now, self.idle_release_s)
                if released:
                    stats.released_maps += len(released)
                    door.retry(now)  # the waiting robots may fit now
            idle = all(s["event"] is None for s in self.slots) and not self.sched.pending()
            if i >= len(reqs) and idle:
                # everything offered has been served, except scans still
                # waiting for memory that no idle map can free any more
                if door.waiting and self.idle_release_s is not None and door.has_map:
                    pass
                else:
                    stats.unserved_scans = door.pending()
                    break
            if not progressed:
                if i < len(reqs) and idle:
                    time.sleep(max(0.0, min(0.001, reqs[i].arrival - (time.perf_counter() - t0))))
                else:
                    time.sleep(20e-6)
        torch.cuda.synchronize()
        stats.wall_s = time.perf_counter() - t0
        stats.refused_robots = sorted(door.ever_waited)
        stats.rays = (sum(m.stats()["rays_valid"] - stats0.get(rid, 0) for rid, m in self.maps.items())
                      + self.rays_released - released0)
        return stats
