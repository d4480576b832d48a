"""Seeded synthetic inputs shaped like the paper's workloads (Section 5, items 1-3
of the varied parameters; Tables 2-4), plus the batched-scene and request-stream
workloads used for the batched and serving forms.

This module only draws endpoints. It holds none of the voxelization arithmetic:
no step count, no rounding, no packing. The oracle and the CUDA path both consume
the arrays it returns, byte for byte.

Every generator takes an explicit seed and uses numpy's PCG64 (``default_rng``).
Segments are returned as a C-contiguous ``int32[S, 6]`` array with rows
``(x0, y0, z0, x1, y1, z1)``; dims are ``(w, h, d)`` in voxels.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEGMENT_DTYPE = np.int32


def _fit_starts(rng: np.random.Generator, delta: np.ndarray, edge: int) -> np.ndarray:
    """Starts uniform per axis so that start and start+delta both lie in [0, edge)."""
    lo = np.maximum(0, -delta)
    hi = (edge - 1) - np.maximum(0, delta)
    # integers(lo, hi + 1) draws uniformly from the closed range [lo, hi]
    return rng.integers(lo, hi + 1).astype(np.int64)


def _segments_from_major(rng: np.random.Generator, major_len: np.ndarray, edge: int) -> np.ndarray:
    """Segments whose largest |delta| is ``major_len`` (per row): the major axis and
    its sign are uniform, the two other deltas uniform in [-major_len, major_len],
    and the start is placed uniformly so that both endpoints fit the volume."""
    s = major_len.shape[0]
    major_len = major_len.astype(np.int64)
    axis = rng.integers(0, 3, size=s)
    sign = rng.integers(0, 2, size=s) * 2 - 1
    delta = np.empty((s, 3), dtype=np.int64)
    for a in range(3):
        delta[:, a] = rng.integers(-major_len, major_len + 1)
    delta[np.arange(s), axis] = sign * major_len
    start = np.empty((s, 3), dtype=np.int64)
    for a in range(3):
        start[:, a] = _fit_starts(rng, delta[:, a], edge)
    out = np.empty((s, 6), dtype=SEGMENT_DTYPE)
    out[:, :3] = start
    out[:, 3:] = start + delta
    return out


def uniform_segments(rng: np.random.Generator, n: int, dims) -> np.ndarray:
    """n segments with all six coordinates uniform in their axis range."""
    w, h, d = (int(v) for v in dims)
    out = np.empty((n, 6), dtype=SEGMENT_DTYPE)
    for col, edge in enumerate((w, h, d, w, h, d)):
        out[:, col] = rng.integers(0, edge, size=n)
    return out


@dataclass
class Workload:
    """One scene: segments plus the volume they live in."""

    name: str
    segs: np.ndarray  # int32 [S, 6]
    dims: tuple  # (w, h, d)
    note: str = ""

    @property
    def n(self) -> int:
        return int(self.segs.shape[0])


def config1(seed: int = 0) -> Workload:
    """4096 segments, all endpoint coordinates uniform in [0, 255], 256^3 volume."""
    rng = np.random.default_rng(seed)
    dims = (256, 256, 256)
    return Workload("uniform-4096seg-256cube", uniform_segments(rng, 4096, dims), dims,
                    "Table 3 shape at 4096 segments of random length")


def config2(seed: int = 1, n_fixed: int = 1 << 20, include_long: bool = True) -> Workload:
    """Fixed-length batch (Table 3 shape): ``n_fixed`` segments whose major |delta|
    is 63 (64 voxels each) in a 1024^3 volume, followed by one 1023-step segment
    (Table 2 shape, the single-segment case)."""
    rng = np.random.default_rng(seed)
    edge = 1024
    segs = _segments_from_major(rng, np.full(n_fixed, 63, dtype=np.int64), edge)
    if include_long:
        long_seg = _segments_from_major(rng, np.array([1023], dtype=np.int64), edge)
        segs = np.ascontiguousarray(np.concatenate([segs, long_seg], axis=0))
    return Workload(f"fixed64-{n_fixed}seg+1x1023-1024cube", segs, (edge,) * 3,
                    "Table 3 shape (equal lengths) plus a Table 2 single segment")


def single_long_segment(seed: int = 1, n_fixed: int = 1 << 20) -> Workload:
    """The single 1023-step segment of config2 on its own (same bytes)."""
    w = config2(seed, n_fixed)
    return Workload("single-1023step-1024cube", np.ascontiguousarray(w.segs[-1:]), w.dims,
                    "Table 2 shape: one segment")


def config3(seed: int = 2, n: int = 4 << 20, edge: int = 4096) -> Workload:
    """Arbitrary-length batch (Table 4 shape): major |delta| = floor(exp(u ln 4097)) - 1,
    u uniform in [0, 1), so lengths are log-uniform over [0, 4095]; 4096^3 volume."""
    rng = np.random.default_rng(seed)
    u = rng.random(n)
    major = np.floor(np.exp(u * math.log(edge + 1))).astype(np.int64) - 1
    major = np.clip(major, 0, edge - 1)
    segs = _segments_from_major(rng, major, edge)
    return Workload(f"loguniform-{n}seg-{edge}cube", segs, (edge,) * 3,
                    "Table 4 shape (arbitrary lengths)")


def config4(seed: int = 3, n_scenes: int = 256, s_lo: float = 1e3, s_hi: float = 1e5):
    """Batched uneven scenes: volume edge uniform in {64,128,256,512}, segment count
    log-uniform in [s_lo, s_hi], endpoints uniform in each volume."""
    rng = np.random.default_rng(seed)
    edges = rng.choice(np.array([64, 128, 256, 512]), size=n_scenes)
    counts = np.floor(np.exp(rng.uniform(math.log(s_lo), math.log(s_hi), size=n_scenes))).astype(np.int64)
    scenes = []
    for k in range(n_scenes):
        dims = (int(edges[k]),) * 3
        scenes.append(Workload(f"scene{k}", uniform_segments(rng, int(counts[k]), dims), dims))
    return scenes


@dataclass
class Request:
    rid: int
    arrival_s: float
    n_segments: int
    edge: int
    seed: int

    def workload(self) -> Workload:
        rng = np.random.default_rng(self.seed)
        dims = (self.edge,) * 3
        return Workload(f"req{self.rid}", uniform_segments(rng, self.n_segments, dims), dims)


def config5(seed: int = 4, rate_hz: float = 2000.0, duration_s: float = 10.0,
            s_lo: float = 1e3, s_hi: float = 1e6, max_requests: int | None = None):
    """Poisson request stream: exponential inter-arrival times with mean 1/rate_hz;
    each request is a scene with a log-uniform segment count in [s_lo, s_hi] and a
    volume edge uniform in {128, 256, 512, 1024}. Segments are drawn lazily from a
    per-request seed (``Request.workload``)."""
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    rid = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s or (max_requests is not None and rid >= max_requests):
            break
        n = int(math.floor(math.exp(rng.uniform(math.log(s_lo), math.log(s_hi)))))
        edge = int(rng.choice(np.array([128, 256, 512, 1024])))
        reqs.append(Request(rid, t, n, edge, int(rng.integers(0, 2**63 - 1))))
        rid += 1
    return reqs


def sweep_single(n_voxels: int, seed: int = 5, edge: int = 1 << 21) -> Workload:
    """Table 2 sweep point: one segment with n_voxels voxels (major |delta| = n_voxels-1)."""
    rng = np.random.default_rng(seed)
    segs = _segments_from_major(rng, np.array([n_voxels - 1], dtype=np.int64), edge)
    return Workload(f"single-{n_voxels}vox", segs, (edge,) * 3)


# Lengths of the three sweeps of Section 5 (Tables 2-4), in voxels.
E1_LENGTHS = (1000, 2000, 5000, 10000, 20000, 50000, 100000, 200000, 500000, 1000000)
E2_LENGTHS = (20, 50, 100, 1000, 2000, 5000, 10000, 20000, 50000, 100000, 200000)
E3_TOTAL = 10**9


def sweep_fixed(length: int, n: int = 1024, seed: int = 6, edge: int = 1 << 21) -> Workload:
    """Table 3 sweep point: n segments of `length` voxels each (major |delta| =
    length - 1), random directions, inside an edge^3 volume."""
    rng = np.random.default_rng(seed + length)
    segs = _segments_from_major(rng, np.full(n, length - 1, dtype=np.int64), edge)
    return Workload(f"fixed-{n}x{length}vox", segs, (edge,) * 3)


def giga_lengths(rng: np.random.Generator, n: int, total: int, edge: int) -> np.ndarray:
    """n pairwise different segment lengths (voxels) summing to exactly `total`,
    each at most edge: weights uniform in [0.1, 1) scaled to the total, the
    rounding remainder spread one voxel at a time over the longest segments."""
    if total < n * (n + 1) // 2 or total > n * edge:
        raise ValueError("total out of reach")
    while True:
        wts = rng.uniform(0.1, 1.0, size=n)
        lengths = np.floor(wts / wts.sum() * total).astype(np.int64)
        rest = total - int(lengths.sum())
        order = np.argsort(-lengths, kind="stable")
        lengths[order[:rest]] += 1
        if len(np.unique(lengths)) == n and lengths.min() >= 1 and lengths.max() <= edge:
            return lengths


def sweep_giga(total: int = E3_TOTAL, n: int = 1024, seed: int = 7, edge: int = 1 << 21) -> Workload:
    """Table 4 shape: n segments of pairwise different, arbitrary lengths whose
    voxel counts sum to `total` (one giga-voxel by default)."""
    rng = np.random.default_rng(seed)
    lengths = giga_lengths(rng, n, total, edge)
    segs = _segments_from_major(rng, lengths - 1, edge)
    return Workload(f"arbitrary-{n}seg-{total}vox", segs, (edge,) * 3)
