"""Autotuner for the launch tuning of libvox (vox_set_tuning).

The outputs never depend on the tuning (integer-exact method); only the speed
does. The tuner times every candidate on the caller's own workload with CUDA
events (after a warm-up, L2 flushed between repetitions), keeps the fastest,
and caches it in a JSON file keyed by the GPU name and a workload class, so a
later run with a similar workload reuses it without measuring.

Tuned knobs (see include/vox.h, vox_tuning):
  run_len      voxels per thread run in the generation kernel (16, 32 or 64)
  volume_path  bricks when the workspace allows (auto), per-voxel atomics, or
               per-voxel atomics merged across the warp
  ctas_per_sm  persistent CTAs per SM (0 = occupancy maximum, or fewer)
  list_runs    a list alone: thread runs across segment ends (0), 32-bit runs
               cut at them (1), or warp slices stored by TMA bulk copies (2)
"""

from __future__ import annotations

import json
import math
import os

from . import vox

CANDIDATES = [
    {"run_len": r, "volume_path": vp, "ctas_per_sm": c, "list_runs": 0}
    for r in (32, 64, 16)
    for vp in (vox.VOLUME_AUTO, vox.VOLUME_ATOMIC, vox.VOLUME_ATOMIC_WARP)
    for c in (0, 2)
] + [{"run_len": r, "volume_path": vox.VOLUME_AUTO, "ctas_per_sm": 0, "list_runs": 1} for r in (32, 64)] + [
    {"run_len": 32, "volume_path": vox.VOLUME_AUTO, "ctas_per_sm": c, "list_runs": 2} for c in (0, 4)]


def default_cache_path() -> str:
    return os.environ.get("VOX_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "vox_tuning.json"))


def workload_class(n_segments: int, total_voxels: int, dims, flags: int) -> str:
    """Coarse class of a workload: rounded-log2 buckets of the segment count, of the
    mean voxels per segment and of the volume size, plus the output flags."""
    w, h, d = (int(v) for v in dims)
    mean_len = total_voxels / max(1, n_segments)
    b = lambda x: int(round(math.log2(max(1.0, float(x)))))
    return f"n{b(n_segments)}-len{b(mean_len)}-vol{b(w * h * d)}-w32{int(w % 32 == 0)}-f{int(flags)}"


def load_cache(path: str | None = None) -> dict:
    path = path or default_cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or default_cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(params: dict) -> None:
    vox.vox_set_tuning(params.get("run_len", 0), params.get("volume_path", 0), params.get("ctas_per_sm", 0),
                       params.get("list_runs", 0))


def measure(run, reps: int = 5, flush_bytes: int = 256 << 20) -> float:
    """Mean milliseconds of `run()` (enqueues work on the current stream)."""
    import torch

    flush = torch.empty(flush_bytes // 4, dtype=torch.int32, device="cuda")
    run()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return sum(ts) / len(ts)


def tune(run, candidates=None, reps: int = 5) -> tuple[dict, dict]:
    """Time `run` under every candidate tuning; returns (best, {name: ms}).
    The tuning in force on return is the best one."""
    candidates = candidates or CANDIDATES
    timings = {}
    best, best_ms = None, float("inf")
    for c in candidates:
        apply(c)
        ms = measure(run, reps)
        timings[json.dumps(c, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = c, ms
    apply(best)
    return best, timings


def get_or_tune(run, n_segments: int, total_voxels: int, dims, flags: int, cache_path: str | None = None,
                reps: int = 5) -> dict:
    """Cached tuning for this GPU and workload class, measuring on a miss."""
    import torch

    key = f"{torch.cuda.get_device_name()}|{workload_class(n_segments, total_voxels, dims, flags)}"
    cache = load_cache(cache_path)
    if key in cache:
        params = cache[key]["params"]
        apply(params)
        return {"params": params, "key": key, "cached": True}
    best, timings = tune(run, reps=reps)
    cache[key] = {"params": best, "timings_ms": timings}
    save_cache(cache, cache_path)
    return {"params": best, "key": key, "cached": False, "timings_ms": timings}
