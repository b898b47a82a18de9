"""Scene, trajectory and lidar models (inputs only; see the package docstring).

Recipes (seed = SEEDS[workload], sub-seeds by map/robot index):

single_scan: 16-beam lidar (+-15 deg, 1024 columns), ground z = tan(5 deg) x,
   two 1 x 1 x 2 m boxes at (5, 3) and (-4, -5), a ditch 2 m wide (x in
   [7, 9]) and 0.8 m deep spanning y in [-6, 6], and 2,000 vegetation points
   uniform in [-6, -3] x [2, 5] x [g, g + 1] (g = ground height) appended to
   the 16,384-point organised scan. Sensor at (0, 0, 1.5), identity pose.
sequence: 64-beam lidar (+-16.6 deg, 2048 columns), 20 scans at 10 Hz,
   4.5 m/s along y = 0.557 sin(2 pi x / 40) (heading follows the tangent,
   +-5 deg), pitch 5 deg sin(2 pi t / 2 s); terrain = 4 seeded sinusoid
   octaves (amplitude 0.5 m halving, wavelength 40 m halving), 30 boxes
   (footprint 0.5-2 m, height 0.5-2.5 m) and 10 ditches (width 1-3 m, depth
   0.5-1.5 m, length 3-10 m).
high_speed: 128-beam lidar (+-22.5 deg, 2048 columns), 40 scans at 12 m/s,
   the same generator plus two roughness octaves (0.15 m at 2.5 m, 0.075 m
   at 1.25 m) and vegetation clusters (radius 1-2 m, 0.5-1.5 m tall) where
   20 % of the rays entering a cluster return inside it at a uniform depth
   and the rest pass through.
batched: 64 maps of the sequence kind, each with its own terrain and
   trajectory (terrain modelled 70 m around the route; beyond it the ground
   continues at the edge height); each map's scan per step is a seeded
   random subset (scan order kept) of a 128 x 2048 scan, of size
   floor(exp U(ln 8192, ln 262144)).
served: 32 robots with mixed sensors (16/64/128 beams) and maps, each with
   its own seeded speed (2-12 m/s) and route (features lining it at the
   sequence workload's density), arrivals with exponential inter-arrival
   times (mean 100 ms) over the stream. Every arrival carries the pose of
   the robot's trajectory at its arrival time (the window moves forward
   with the robot); its points come from one of 8 lidar casts per robot,
   cast at the middle of 8 equal spans of the stream and used for the
   arrivals of that span (sensor frame, re-posed).
Every scan: range noise N(0, 0.02 m) along the beam; beams with no return
within 120 m report the zero point (which the map update drops, as it drops
returns beyond its 100 m range).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 13176
SEEDS = {"single_scan": SEED_BASE + 1, "sequence": SEED_BASE + 2, "high_speed": SEED_BASE + 3,
         "batched": SEED_BASE + 4, "served": SEED_BASE + 5}


@dataclass(frozen=True)
class MapSpec:
    nx: int
    ny: int
    nz: int
    res: float


@dataclass(frozen=True)
class LidarSpec:
    beams: int
    columns: int
    vfov_deg: float          # beams spread uniformly over [-vfov, +vfov]
    noise: float = 0.02      # range noise sigma, metres
    max_cast: float = 120.0  # beams with no return within this report zero

    @property
    def n(self) -> int:
        return self.beams * self.columns

    def directions(self) -> np.ndarray:
        """Unit beam directions in the sensor frame, beam-major (n, 3) float64."""
        el = np.deg2rad(np.linspace(-self.vfov_deg, self.vfov_deg, self.beams))
        az = 2.0 * np.pi * np.arange(self.columns) / self.columns
        ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
        d = np.stack([np.broadcast_to(ce * np.cos(az)[None, :], (self.beams, self.columns)),
                      np.broadcast_to(ce * np.sin(az)[None, :], (self.beams, self.columns)),
                      np.broadcast_to(se, (self.beams, self.columns))], axis=-1)
        return d.reshape(-1, 3)


@dataclass
class Scan:
    points: np.ndarray       # (n, 3) float32, sensor frame
    T_ws: np.ndarray         # (3, 4) float64, world <- sensor
    vehicle_xyz: np.ndarray  # (3,) float64
    t: float = 0.0           # time stamp, s


@dataclass
class Box:
    cx: float
    cy: float
    hx: float
    hy: float
    yaw: float
    z0: float
    z1: float


@dataclass
class Ditch:
    cx: float
    cy: float
    hl: float     # half length (along yaw)
    hw: float     # half width
    yaw: float
    depth: float


@dataclass
class VegCluster:
    cx: float
    cy: float
    radius: float
    z0: float
    z1: float
    p_return: float = 0.2


@dataclass
class Scene:
    tilt_x: float = 0.0                       # dz/dx of a base plane
    octaves: list = field(default_factory=list)  # (amp, wavelength, theta, phase)
    boxes: list = field(default_factory=list)
    ditches: list = field(default_factory=list)
    veg: list = field(default_factory=list)
    raster: float = 0.1                       # height raster spacing, metres
    _grid: tuple | None = None

    # --- analytic ground ---------------------------------------------------
    def ground_exact(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        h = self.tilt_x * x
        for amp, lam, th, ph in self.octaves:
            k = 2.0 * np.pi / lam
            h = h + amp * np.sin(k * (x * math.cos(th) + y * math.sin(th)) + ph)
        for d in self.ditches:
            c, s = math.cos(d.yaw), math.sin(d.yaw)
            u = (x - d.cx) * c + (y - d.cy) * s
            v = -(x - d.cx) * s + (y - d.cy) * c
            inside = (np.abs(u) <= d.hl) & (np.abs(v) <= d.hw)
            h = h - np.where(inside, d.depth, 0.0)
        return h

    def slope_bound(self) -> float:
        return abs(self.tilt_x) + sum(a * 2.0 * np.pi / lam for a, lam, _, _ in self.octaves)

    def build_raster(self, x0: float, x1: float, y0: float, y1: float) -> None:
        g = self.raster
        nxr = int(math.ceil((x1 - x0) / g)) + 2
        nyr = int(math.ceil((y1 - y0) / g)) + 2
        xs = x0 + g * np.arange(nxr)
        ys = y0 + g * np.arange(nyr)
        H = np.empty((nxr, nyr), dtype=np.float32)
        # the smooth part over the whole raster, then each ditch over the
        # raster cells of its bounding square only
        all_ditches = self.ditches
        self.ditches = []
        try:
            for i in range(0, nxr, 256):
                X, Y = np.meshgrid(xs[i:i + 256], ys, indexing="ij")
                H[i:i + 256] = self.ground_exact(X, Y)
        finally:
            self.ditches = all_ditches
        # each ditch's square is recomputed whole (smooth part and every ditch
        # that reaches the square, in list order), so the raster equals
        # ground_exact everywhere
        def square(d):
            r = d.hl + d.hw
            return (max(0, math.floor((d.cx - r - x0) / g)), min(nxr, math.floor((d.cx + r - x0) / g) + 2),
                    max(0, math.floor((d.cy - r - y0) / g)), min(nyr, math.floor((d.cy + r - y0) / g) + 2))
        squares = [square(d) for d in all_ditches]
        for i0, i1, j0, j1 in squares:
            if i0 >= i1 or j0 >= j1:
                continue
            near = [d for d, (a0, a1, b0, b1) in zip(all_ditches, squares)
                    if a0 < i1 and i0 < a1 and b0 < j1 and j0 < b1]
            X, Y = np.meshgrid(xs[i0:i1], ys[j0:j1], indexing="ij")
            self.ditches = near
            try:
                H[i0:i1, j0:j1] = self.ground_exact(X, Y)
            finally:
                self.ditches = all_ditches
        self._grid = (x0, y0, g, H)

    def ground(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        """Ground height by bilinear lookup in the raster (exact where none built)."""
        if self._grid is None:
            return self.ground_exact(x, y)
        x0, y0, g, H = self._grid
        fx = np.clip((x - x0) / g, 0.0, H.shape[0] - 1.001)
        fy = np.clip((y - y0) / g, 0.0, H.shape[1] - 1.001)
        ix = fx.astype(np.int64)
        iy = fy.astype(np.int64)
        ax = fx - ix
        ay = fy - iy
        h00 = H[ix, iy]
        h10 = H[ix + 1, iy]
        h01 = H[ix, iy + 1]
        h11 = H[ix + 1, iy + 1]
        return (h00 * (1 - ax) + h10 * ax) * (1 - ay) + (h01 * (1 - ax) + h11 * ax) * ay

    # --- ray casting -------------------------------------------------------
    def _cast_ground(self, o: np.ndarray, d: np.ndarray, t_max: float) -> np.ndarray:
        n = d.shape[0]
        t_hit = np.full(n, np.nan)
        L = self.slope_bound() + 0.05
        dxy = np.hypot(d[:, 0], d[:, 1])
        denom = np.abs(d[:, 2]) + L * dxy + 1e-9
        zmax = self._grid[3].max() + 0.01 if self._grid is not None else np.inf
        idx = np.arange(n)
        t = np.zeros(n)
        f = o[2] - self.ground(np.full(n, o[0]), np.full(n, o[1]))
        for _ in range(4000):
            if idx.size == 0:
                break
            dd = d[idx]
            step = np.clip(0.9 * f / denom[idx], 0.02, 0.5)
            tn = t + step
            px = o[0] + tn * dd[:, 0]
            py = o[1] + tn * dd[:, 1]
            pz = o[2] + tn * dd[:, 2]
            fn = pz - self.ground(px, py)
            crossed = fn < 0.0
            if crossed.any():
                lo = t[crossed].copy()
                hi = tn[crossed].copy()
                dc = dd[crossed]
                for _ in range(24):
                    mid = 0.5 * (lo + hi)
                    fm = (o[2] + mid * dc[:, 2]) - self.ground(o[0] + mid * dc[:, 0], o[1] + mid * dc[:, 1])
                    below = fm < 0.0
                    hi = np.where(below, mid, hi)
                    lo = np.where(below, lo, mid)
                t_hit[idx[crossed]] = 0.5 * (lo + hi)
            keep = ~crossed & (tn < t_max) & ~((dd[:, 2] > 0) & (pz > zmax))
            idx = idx[keep]
            t = tn[keep]
            f = fn[keep]
        return t_hit

    def _cast_boxes(self, o: np.ndarray, d: np.ndarray, reach: float = np.inf) -> np.ndarray:
        n = d.shape[0]
        best = np.full(n, np.inf)
        # rays sorted by azimuth: a box can only be hit by the rays whose
        # azimuth lies within the angle its bounding circle subtends
        az = np.arctan2(d[:, 1], d[:, 0])
        order = np.argsort(az, kind="stable")
        az_sorted = az[order]
        for b in self.boxes:
            rb = math.hypot(b.hx, b.hy)
            dist = math.hypot(b.cx - o[0], b.cy - o[1])
            if dist > reach + rb:
                continue
            if dist > rb + 1e-6:
                half = math.asin(min(1.0, rb / dist)) + 1e-9
                a0 = math.atan2(b.cy - o[1], b.cx - o[0])
                lo_a, hi_a = a0 - half, a0 + half
                idx = []
                for lo, hi in ((lo_a, hi_a), (lo_a + 2 * math.pi, hi_a + 2 * math.pi),
                               (lo_a - 2 * math.pi, hi_a - 2 * math.pi)):
                    i0, i1 = np.searchsorted(az_sorted, [lo, hi])
                    if i1 > i0:
                        idx.append(order[i0:i1])
                if not idx:
                    continue
                sel = np.concatenate(idx)
            else:
                sel = np.arange(n)
            c, s = math.cos(b.yaw), math.sin(b.yaw)
            ox, oy = o[0] - b.cx, o[1] - b.cy
            lo_ = np.array([c * ox + s * oy, -s * ox + c * oy, o[2]])
            ds = d[sel]
            ld = np.stack([c * ds[:, 0] + s * ds[:, 1], -s * ds[:, 0] + c * ds[:, 1], ds[:, 2]], axis=1)
            bmin = np.array([-b.hx, -b.hy, b.z0])
            bmax = np.array([b.hx, b.hy, b.z1])
            with np.errstate(divide="ignore", invalid="ignore"):
                inv = 1.0 / ld
                t1 = (bmin - lo_) * inv
                t2 = (bmax - lo_) * inv
            tmin = np.nanmax(np.minimum(t1, t2), axis=1)
            tmax = np.nanmin(np.maximum(t1, t2), axis=1)
            ok = (tmax >= tmin) & (tmin > 1e-6)
            cur = best[sel]
            best[sel] = np.where(ok & (tmin < cur), tmin, cur)
        return best

    def _cast_veg(self, o, d, t_hit, rng, reach: float = np.inf) -> np.ndarray:
        out = t_hit.copy()
        for v in self.veg:
            ox, oy = o[0] - v.cx, o[1] - v.cy
            if math.hypot(ox, oy) > reach + v.radius:
                continue
            a = d[:, 0] ** 2 + d[:, 1] ** 2
            bq = 2.0 * (ox * d[:, 0] + oy * d[:, 1])
            cq = ox * ox + oy * oy - v.radius ** 2
            disc = bq * bq - 4 * a * cq
            ok = (disc > 0) & (a > 1e-12)
            sq = np.sqrt(np.where(ok, disc, 0.0))
            with np.errstate(divide="ignore", invalid="ignore"):
                ta = (-bq - sq) / (2 * a)
                tb = (-bq + sq) / (2 * a)
                # clip to the cluster's height band
                tz0 = (v.z0 - o[2]) / d[:, 2]
                tz1 = (v.z1 - o[2]) / d[:, 2]
            tzl = np.where(d[:, 2] != 0, np.minimum(tz0, tz1), -np.inf)
            tzh = np.where(d[:, 2] != 0, np.maximum(tz0, tz1), np.where((o[2] >= v.z0) & (o[2] <= v.z1), np.inf, -np.inf))
            enter = np.maximum(np.maximum(ta, tzl), 0.0)
            leave = np.minimum(np.minimum(tb, tzh), out)
            hit = ok & (leave > enter)
            draw = rng.random(d.shape[0])
            depth = rng.random(d.shape[0])
            ret = hit & (draw < v.p_return)
            out = np.where(ret, enter + depth * (leave - enter), out)
        return out

    def cast(self, o: np.ndarray, d: np.ndarray, t_max: float, rng) -> np.ndarray:
        """First-return range of each unit ray from o (world frame); NaN if none."""
        tg = self._cast_ground(o, d, t_max)
        tb = self._cast_boxes(o, d, t_max)
        t = np.fmin(tg, tb)
        t = np.where(np.isinf(t), np.nan, t)
        if self.veg:
            t = self._cast_veg(o, d, np.where(np.isnan(t), np.inf, t), rng, t_max)
            t = np.where(np.isinf(t), np.nan, t)
        t = np.where(t <= t_max, t, np.nan)
        return t


def pose_matrix(vehicle_xyz, yaw: float, pitch: float, mount=(0.0, 0.0, 1.5)) -> np.ndarray:
    """World <- sensor as a 3x4 matrix: R = Rz(yaw) Ry(pitch), sensor mounted at `mount`."""
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    Rz = np.array([[cy_, -sy_, 0.0], [sy_, cy_, 0.0], [0.0, 0.0, 1.0]])
    Ry = np.array([[cp, 0.0, sp], [0.0, 1.0, 0.0], [-sp, 0.0, cp]])
    R = Rz @ Ry
    t = np.asarray(vehicle_xyz, dtype=np.float64) + R @ np.asarray(mount, dtype=np.float64)
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = t
    return T


def scan_from_pose(scene: Scene, lidar: LidarSpec, T_ws: np.ndarray, vehicle_xyz, rng,
                   subset: np.ndarray | None = None, t: float = 0.0) -> Scan:
    """Cast the lidar's beams (all, or the given beam indices) from the pose."""
    ds = lidar.directions()
    if subset is not None:
        ds = ds[subset]
    R = T_ws[:, :3]
    o = T_ws[:, 3]
    dw = ds @ R.T
    r = scene.cast(o, dw, lidar.max_cast, rng)
    noise = rng.normal(0.0, lidar.noise, size=r.shape)
    rr = np.where(np.isnan(r), 0.0, r + noise)
    rr = np.where(rr > 0.0, rr, 0.0)
    pts = (ds * rr[:, None]).astype(np.float32)
    return Scan(points=pts, T_ws=T_ws, vehicle_xyz=np.asarray(vehicle_xyz, dtype=np.float64), t=t)


# --- the single-scan test scene ----------------------------------------------
def single_scan_scene() -> Scene:
    tilt = math.tan(math.radians(5.0))
    sc = Scene(tilt_x=tilt, raster=0.05)
    sc.ditches.append(Ditch(cx=8.0, cy=0.0, hl=1.0, hw=6.0, yaw=0.0, depth=0.8))
    for cx, cy in ((5.0, 3.0), (-4.0, -5.0)):
        g = tilt * cx
        sc.boxes.append(Box(cx=cx, cy=cy, hx=0.5, hy=0.5, yaw=0.0, z0=g - 0.5, z1=g + 2.0))
    sc.build_raster(-110.0, 110.0, -110.0, 110.0)
    return sc


def single_scan(seed: int | None = None) -> Scan:
    """16,384-beam organised scan plus 2,000 appended vegetation points."""
    rng = np.random.default_rng(SEEDS["single_scan"] if seed is None else seed)
    sc = single_scan_scene()
    lidar = LidarSpec(16, 1024, 15.0)
    T = pose_matrix((0.0, 0.0, 0.0), 0.0, 0.0)
    s = scan_from_pose(sc, lidar, T, (0.0, 0.0, 0.0), rng)
    vx = rng.uniform(-6.0, -3.0, 2000)
    vy = rng.uniform(2.0, 5.0, 2000)
    g = sc.ground_exact(vx, vy)
    vz = g + rng.uniform(0.0, 1.0, 2000)
    w = np.stack([vx, vy, vz], axis=1)
    ps = (w - T[:, 3]) @ T[:, :3]  # R^T (w - t)
    s.points = np.concatenate([s.points, ps.astype(np.float32)], axis=0)
    return s


# --- sequence scenes (sequence, high_speed, batched, served) ---------------
def random_scene(rng, x_range, y_range, rough: float = 0.0, veg_clusters: int = 0,
                 n_boxes: int = 30, n_ditches: int = 10, raster: float = 0.1,
                 path=None) -> Scene:
    sc = Scene(raster=raster)
    for o in range(4):
        sc.octaves.append((0.5 * 2.0 ** -o, 40.0 / 2.0 ** o, rng.uniform(0, np.pi), rng.uniform(0, 2 * np.pi)))
    if rough > 0:
        sc.octaves.append((rough, 2.5, rng.uniform(0, np.pi), rng.uniform(0, 2 * np.pi)))
        sc.octaves.append((rough / 2, 1.25, rng.uniform(0, np.pi), rng.uniform(0, 2 * np.pi)))
    (x0, x1), (y0, y1) = x_range, y_range

    def off_path(x, y, clear):
        return path is None or abs(y - path(x)) > clear

    while len(sc.ditches) < n_ditches:
        cx, cy = rng.uniform(x0, x1), rng.uniform(y0, y1)
        if not off_path(cx, cy, 6.0):
            continue
        sc.ditches.append(Ditch(cx, cy, rng.uniform(1.5, 5.0), rng.uniform(0.5, 1.5),
                                rng.uniform(0, np.pi), rng.uniform(0.5, 1.5)))
    while len(sc.boxes) < n_boxes:
        cx, cy = rng.uniform(x0, x1), rng.uniform(y0, y1)
        if not off_path(cx, cy, 2.5):
            continue
        hx, hy = rng.uniform(0.25, 1.0), rng.uniform(0.25, 1.0)
        g = float(sc.ground_exact(np.array([cx]), np.array([cy]))[0])
        sc.boxes.append(Box(cx, cy, hx, hy, rng.uniform(0, np.pi), g - 1.0, g + rng.uniform(0.5, 2.5)))
    centres = []
    tries = 0
    while len(centres) < veg_clusters and tries < 10000:
        tries += 1
        cx, cy = rng.uniform(x0, x1), rng.uniform(y0, y1)
        r = rng.uniform(1.0, 2.0)
        if not off_path(cx, cy, r + 1.0):
            continue
        if all(math.hypot(cx - a, cy - b) > r + rb + 0.5 for a, b, rb in centres):  # Poisson-disc
            centres.append((cx, cy, r))
    for cx, cy, r in centres:
        g = float(sc.ground_exact(np.array([cx]), np.array([cy]))[0])
        sc.veg.append(VegCluster(cx, cy, r, g - 0.2, g + rng.uniform(0.5, 1.5)))
    return sc


@dataclass(frozen=True)
class SequenceConfig:
    map: MapSpec
    lidar: LidarSpec
    n_scans: int
    speed: float
    rough: float = 0.0
    veg_clusters: int = 0
    rate_hz: float = 10.0


def sequence_config(name: str) -> SequenceConfig:
    """The sequence workloads: "sequence" (64-beam, 256 x 256 x 64 @ 0.2 m) and
    "high_speed" (128-beam, 512 x 512 x 64 @ 0.1 m)."""
    if name == "sequence":
        return SequenceConfig(MapSpec(256, 256, 64, 0.2), LidarSpec(64, 2048, 16.6), 20, 4.5)
    if name == "high_speed":
        return SequenceConfig(MapSpec(512, 512, 64, 0.1), LidarSpec(128, 2048, 22.5), 40, 12.0,
                              rough=0.15, veg_clusters=60)
    raise ValueError(name)


def _path_y(x):
    return 0.557 * np.sin(2.0 * np.pi * x / 40.0)


def _trajectory_pose(scene: Scene, speed: float, t: float, x_start: float = 0.0, yaw0: float = 0.0):
    """Vehicle position, yaw and pitch at time t along the sinusoidal path."""
    x = x_start + speed * t
    y = float(_path_y(x))
    dy = 0.557 * 2.0 * np.pi / 40.0 * math.cos(2.0 * np.pi * x / 40.0)
    yaw = yaw0 + math.atan(dy)
    pitch = math.radians(5.0) * math.sin(2.0 * np.pi * t / 2.0)
    # rotate the path by yaw0 about the start point so trajectories differ per map
    c, s = math.cos(yaw0), math.sin(yaw0)
    X = x_start + c * (x - x_start) - s * y
    Y = s * (x - x_start) + c * y
    z = float(scene.ground_exact(np.array([X]), np.array([Y]))[0])
    return np.array([X, Y, z]), yaw, pitch


def make_sequence_scene(cfg: SequenceConfig, rng, yaw0: float = 0.0, extent: float = 110.0) -> Scene:
    route = cfg.speed * cfg.n_scans / cfg.rate_hz
    ext = extent
    sc = random_scene(rng, (-25.0, route + 25.0), (-25.0, 25.0), rough=cfg.rough,
                      veg_clusters=cfg.veg_clusters, raster=0.1 if cfg.rough > 0 else 0.2,
                      path=(lambda x: float(_path_y(x))) if yaw0 == 0.0 else None)
    sc.build_raster(-ext, route + ext, -ext - route, ext + route)
    return sc


def _sequence_chunk(args):
    name, seed, steps = args
    cfg = sequence_config(name)
    rng = np.random.default_rng(seed)
    sc = make_sequence_scene(cfg, rng)
    out = []
    for step in steps:
        t = step / cfg.rate_hz
        veh, yaw, pitch = _trajectory_pose(sc, cfg.speed, t)
        T = pose_matrix(veh, yaw, pitch)
        srng = np.random.default_rng([seed, 1, step])
        out.append(scan_from_pose(sc, cfg.lidar, T, veh, srng, t=t))
    return out


def sequence_scans(name: str, n_scans: int | None = None, seed: int | None = None,
                   stride: int = 1, workers: int = 0):
    """Scans 0, stride, 2*stride, ... of the sequence workload `name`
    ("sequence" or "high_speed").

    workers > 1 casts the scans in a spawn-started process pool (each worker
    rebuilds the same seeded scene; the scans are identical)."""
    cfg = sequence_config(name)
    seed = SEEDS[name] if seed is None else seed
    n = cfg.n_scans if n_scans is None else n_scans
    steps = [i * stride for i in range(n)]
    if workers and workers > 1 and n > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        w = min(workers, n)
        chunks = [steps[i::w] for i in range(w)]
        with ProcessPoolExecutor(max_workers=w, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_sequence_chunk, [(name, seed, c) for c in chunks]))
        by_step = {}
        for c, part in zip(chunks, parts):
            for st, scan in zip(c, part):
                by_step[st] = scan
        return cfg, [by_step[st] for st in steps]
    return cfg, _sequence_chunk((name, seed, steps))


def _batched_map(args):
    """Scene, trajectory and n_steps scans of one map of the batched workload."""
    seed, m, n_steps, lo, hi = args
    cfg = SequenceConfig(MapSpec(256, 256, 64, 0.2), LidarSpec(128, 2048, 22.5), n_steps, 4.5)
    r = np.random.default_rng([seed, 0, m])
    yaw0 = float(r.uniform(0, 2 * np.pi))
    sc = make_sequence_scene(cfg, r, yaw0=yaw0, extent=70.0)
    out = []
    for s in range(n_steps):
        rs = np.random.default_rng([seed, 1, m, s])
        size = int(math.floor(math.exp(rs.uniform(math.log(lo), math.log(hi)))))
        subset = np.sort(rs.choice(cfg.lidar.n, size=size, replace=False))
        t = s / cfg.rate_hz
        veh, yaw, pitch = _trajectory_pose(sc, cfg.speed, t, yaw0=yaw0)
        T = pose_matrix(veh, yaw, pitch)
        out.append(scan_from_pose(sc, cfg.lidar, T, veh, rs, subset=subset, t=t))
    return out


def batched_scans(n_maps: int = 64, n_steps: int = 1, seed: int | None = None,
                  lo: int = 8192, hi: int = 262144, workers: int = 0):
    """Per step, a list of n_maps scans of log-uniform size (the batched workload).

    workers > 1 generates maps in a spawn-started process pool (the result
    is the same as with one process)."""
    cfg = SequenceConfig(MapSpec(256, 256, 64, 0.2), LidarSpec(128, 2048, 22.5), n_steps, 4.5)
    seed = SEEDS["batched"] if seed is None else seed
    jobs = [(seed, m, n_steps, lo, hi) for m in range(n_maps)]
    if workers and workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            per_map = list(ex.map(_batched_map, jobs))
    else:
        per_map = [_batched_map(j) for j in jobs]
    steps = [[per_map[m][s] for m in range(n_maps)] for s in range(n_steps)]
    return cfg, steps


SERVED_MAPS = (MapSpec(128, 128, 32, 0.2), MapSpec(256, 256, 64, 0.2), MapSpec(512, 512, 64, 0.1))
SERVED_LIDARS = (LidarSpec(16, 1024, 15.0), LidarSpec(64, 2048, 16.6), LidarSpec(128, 2048, 22.5))


SERVED_CASTS = 8  # lidar casts per robot, spread over its stream


def _served_robot(args):
    """One served robot: its map and sensor, its own trajectory over the
    whole stream (speed and route seeded per robot), its arrivals, and the
    lidar casts that give each arrival its points."""
    seed, i, duration_s, casts, rate_hz = args
    r = np.random.default_rng([seed, 0, i])
    ms = SERVED_MAPS[int(r.integers(0, 3))]
    ld = SERVED_LIDARS[int(r.integers(0, 3))]
    speed = float(r.uniform(2.0, 12.0))
    rough = 0.1 if ms.res < 0.2 else 0.0
    # the robot's route is speed * duration metres long; features line it
    # with the density of the sequence workload (30 boxes, 10 ditches per
    # 60 m x 50 m)
    route = speed * duration_s
    area = (route + 50.0) * 50.0
    sc = random_scene(r, (-25.0, route + 25.0), (-25.0, 25.0), rough=rough,
                      veg_clusters=int(round(area / 1500.0)) if rough > 0 else 0,
                      n_boxes=int(round(30 * area / 3000.0)), n_ditches=int(round(10 * area / 3000.0)),
                      raster=0.2, path=lambda x: float(_path_y(x)))
    # arrivals: exponential inter-arrival times with mean 1 / rate_hz
    ra = np.random.default_rng([seed, 2, i])
    times = []
    t = float(ra.uniform(0, 1.0 / rate_hz))
    while t < duration_s:
        times.append(t)
        t += float(ra.exponential(1.0 / rate_hz))
    # casts at the middle of equal spans of the stream; an arrival takes the
    # cast of its span, re-posed to its own pose on the trajectory
    span = duration_s / casts
    cast_scans = []
    for j in range(casts):
        tc = (j + 0.5) * span
        veh, yaw, pitch = _trajectory_pose(sc, speed, tc)
        sc.build_raster(veh[0] - ld.max_cast - 2.0, veh[0] + ld.max_cast + 2.0,
                        veh[1] - ld.max_cast - 2.0, veh[1] + ld.max_cast + 2.0)
        T = pose_matrix(veh, yaw, pitch)
        cast_scans.append(scan_from_pose(sc, ld, T, veh, np.random.default_rng([seed, 1, i, j]), t=tc))
        sc._grid = None
    arrivals = []
    for k, t in enumerate(times):
        veh, yaw, pitch = _trajectory_pose(sc, speed, t)
        arrivals.append((t, k, min(casts - 1, int(t / span)), pose_matrix(veh, yaw, pitch), veh))
    return dict(map=ms, lidar=ld, speed=speed, casts=cast_scans, arrivals=arrivals)


def served_stream(n_robots: int = 32, duration_s: float = 60.0, casts: int = SERVED_CASTS, rate_hz: float = 10.0,
                  seed: int | None = None, workers: int = 0):
    """The served workload: robots with their maps, sensors and trajectories,
    and the time-ordered arrivals of all robots.

    Returns (robots, arrivals). robots[i] = dict(map=MapSpec, lidar=LidarSpec,
    speed=m/s, casts=[Scan] * casts). arrivals = list of (t_s, robot, k,
    cast, T_ws, vehicle_xyz), sorted by t: robot's k-th scan arrives at t_s
    with the pose of its own trajectory at that time; its points are
    robots[robot]["casts"][cast].points (sensor frame). workers > 1 builds
    robots in a spawn-started process pool (same result)."""
    seed = SEEDS["served"] if seed is None else seed
    jobs = [(seed, i, duration_s, casts, rate_hz) for i in range(n_robots)]
    if workers and workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            robots = list(ex.map(_served_robot, jobs))
    else:
        robots = [_served_robot(j) for j in jobs]
    arr = []
    for i, rb in enumerate(robots):
        for t, k, c, T, veh in rb.pop("arrivals"):
            arr.append((t, i, k, c, T, veh))
    arr.sort(key=lambda a: (a[0], a[1]))
    return robots, arr


WORKLOADS = {
    "single_scan": dict(name="plain single scan: 16-beam, 16,384+2,000 pts, map 128x128x32 @ 0.2 m",
                        map=MapSpec(128, 128, 32, 0.2)),
    "sequence": dict(name="plain sequence: 64-beam, 131,072 pts/scan x 20 scans, map 256x256x64 @ 0.2 m, "
                          "shift every scan", map=MapSpec(256, 256, 64, 0.2)),
    "high_speed": dict(name="plain high-speed: 128-beam, 262,144 pts/scan x 40 scans at 12 m/s, "
                            "map 512x512x64 @ 0.1 m", map=MapSpec(512, 512, 64, 0.1)),
    "batched": dict(name="batched: 64 maps 256x256x64 @ 0.2 m, log-uniform 8,192-262,144 pts/scan",
                    map=MapSpec(256, 256, 64, 0.2)),
    "served": dict(name="served: 32 robots, 10 Hz Poisson arrivals, mixed sensors and maps", map=None),
}
