"""Autotuner for the launch shapes (gvom_tuning).

The segment walk's speed depends on the segment length (shorter segments
balance warps better but cost more set-up), on the block shape of its
persistent grid and on whether one fused kernel both lists and walks the
segments; the best choice depends on the map, the sensor and the GPU.
The extraction's speed depends on the pixel pass's tile edge (halo work
against blocks in flight) and on the column pass's bulk-copy chunk shape
(columns per chunk against stages in flight); tune_extract searches those.
The tuner times each candidate on the caller's own workload, keeps the
fastest, and remembers it in a JSON table (GVOM_TUNE_CACHE, default
~/.cache/gvom/tuning.json) under a key naming the device and the workload,
so later runs skip the search. Results never depend on the tuning, only time.
"""
from __future__ import annotations

import json
import os
import statistics
import time

# walk shapes (seg_len, march_block, march_blocks_per_sm) for batches, and
# with fused_ingest for single maps
WALK_CANDIDATES = [(L, blk, 0) for L in (8, 12, 16, 24, 32, 48, 64) for blk in (128, 256)]
CANDIDATES = [c + (f,) for c in WALK_CANDIDATES for f in (0, 1)]


def cache_path() -> str:
    return os.environ.get("GVOM_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gvom", "tuning.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(table: dict) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def workload_key(kind: str, dims, res: float, points: int) -> str:
    import torch
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    bucket = 1 << max(0, int(points).bit_length() - 1)  # power-of-two bucket of the point count
    return f"{dev}|{kind}|{'x'.join(str(int(d)) for d in dims)}@{res:g}|~{bucket}"


def search(run, candidates=CANDIDATES, repeats: int = 3):
    """run(candidate) -> seconds of one timed repetition; returns (best, table)."""
    times = {}
    for c in candidates:
        run(c)  # warm-up (first launch, scratch growth)
        times[c] = statistics.median(run(c) for _ in range(repeats))
    best = min(times, key=times.get)
    return best, {"/".join(str(x) for x in c): round(t * 1e6, 2) for c, t in times.items()}


def tuned(key: str, run, candidates=CANDIDATES, repeats: int = 3, refresh: bool = False):
    """The cached best candidate for key, or a fresh search (then cached)."""
    table = _load()
    if not refresh and key in table and len(table[key]["best"]) == len(candidates[0]):
        c = table[key]["best"]
        return tuple(c), table[key]
    t0 = time.perf_counter()
    best, times = search(run, candidates, repeats)
    entry = {"best": list(best), "us": times, "search_s": round(time.perf_counter() - t0, 2)}
    table[key] = entry
    _store(table)
    return best, entry


def tune_map(vmap, scans_dev, poses, vehicles, flush=None, refresh: bool = False, repeats: int = 3):
    """Tunes one VoxelMap's ingest on a few of its own scans (CUDA tensors)."""
    import torch
    stream = torch.cuda.current_stream()

    def run(c):
        apply_walk(vmap, c)
        tot = 0.0
        for pts, T, v in zip(scans_dev, poses, vehicles):
            vmap.shift(vmap.origin_for_pose(v))
            if flush is not None:
                flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vmap.ingest(pts, T)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1) * 1e-3
        return tot

    key = workload_key("map", vmap.shape, vmap.cfg.res, int(statistics.median(int(p.shape[0]) for p in scans_dev)))
    best, entry = tuned(key, run, repeats=repeats, refresh=refresh)
    apply_walk(vmap, best)
    return best, entry


def apply_walk(vmap, c):
    """Sets a walk candidate (seg_len, march_block, blocks_per_sm[, fused_ingest])."""
    vmap.set_tuning(c[0], c[1], c[2], fused_ingest=c[3] if len(c) > 3 else 0)


def extract_candidates(vmap):
    """Pixel tile edges and column chunk shapes to try for one map: the
    built-in rule and tiles whose rows with both halos are one, two or three
    warps wide (plus 16), times the four chunk shapes."""
    R = max(vmap.cfg.neg_max_px, vmap.cfg.slope_n // 2)
    tiles = {0, 16}
    for w in (32, 64, 96):
        t = w - 2 * R
        if 4 <= t <= 64:
            tiles.add(t)
    return [(t, c) for t in sorted(tiles) for c in (0, 1, 2, 3)]


def tune_extract(vmap, outs, flush=None, refresh: bool = False, repeats: int = 3):
    """Tunes one VoxelMap's extraction shapes (pixel tile edge, column chunk
    shape) on its current state, with the caller's output buffers."""
    import torch
    from paper_2109_13176_gb300 import GvomError
    stream = torch.cuda.current_stream()
    cands = []
    for c in extract_candidates(vmap):
        try:
            vmap.set_extract_tuning(*c)
            cands.append(c)
        except GvomError:
            pass  # does not fit shared memory for this map

    def run(c):
        vmap.set_extract_tuning(*c)
        if flush is not None:
            flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vmap.extract_maps(outs)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    cfg = vmap.cfg
    key = workload_key(f"extract-r{max(cfg.neg_max_px, cfg.slope_n // 2)}", vmap.shape, cfg.res, 0)
    best, entry = tuned(key, run, candidates=cands, repeats=repeats, refresh=refresh)
    vmap.set_extract_tuning(*best)
    return best, entry


def tune_batch(batch, maps, step_inputs, flush=None, refresh: bool = False, repeats: int = 2):
    """Tunes a MapBatch on its own steps: step_inputs = [(vehicles, scans, poses), ...]."""
    import torch
    stream = torch.cuda.current_stream()

    def run(c):
        batch.set_tuning(*c)
        tot = 0.0
        for vs, scans, Ts in step_inputs:
            if flush is not None:
                flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.step(maps, vs, scans, Ts)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1) * 1e-3
        return tot

    pts = sum(int(p.shape[0]) for p in step_inputs[0][1])
    key = workload_key(f"batch{len(maps)}", maps[0].shape, maps[0].cfg.res, pts)
    best, entry = tuned(key, run, candidates=WALK_CANDIDATES, repeats=repeats, refresh=refresh)
    batch.set_tuning(*best)
    return best, entry
