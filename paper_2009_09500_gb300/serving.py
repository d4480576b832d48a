"""Continuous-batching request loop for voxelization requests.

Each request is a scene (segments + volume extent) whose result is an occupancy
volume kept resident on the device. Requests arrive over time (a Poisson stream
in the benchmark); the loop admits them first-come first-served while their
device bytes fit the free device memory (a live probe, under an optional cap)
and an in-flight slot is free, packs the admitted requests into one batch, and
launches the batch with vox_generate_batched on one of several streams. Batches launched while earlier
ones still run overlap on the device, and requests that arrive meanwhile join
the next batch as slots and memory free up (continuous batching). Latency is
completion minus arrival, on the host clock.

The scheduler (admission, slots, bookkeeping) is plain Python and takes its
launcher, memory probe and clock as arguments, so that it can be exercised on
the CPU with fakes; the default launcher runs libvox on the GPU, and the
default probe (gpu_free_bytes) reads the device's free memory. A request's
voxel count, used for the throughput figure, comes back from the device with
its batch (the scan's per-scene voxel bases); the host does none of the
method's arithmetic.
"""

from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class ServeRequest:
    rid: int
    arrival_s: float
    n: int
    dims: tuple
    segs_host: object = None      # pinned CPU int32 [n, 6] tensor (default launcher)
    voxels: int = 0               # total voxels, reported by the device with the batch
    admitted_s: float = math.nan
    done_s: float = math.nan
    status: int = -1
    batch_id: int = -1
    result: object = None         # the resident volume (device int32 tensor), if kept

    @property
    def mask_bytes(self) -> int:
        w, h, d = self.dims
        return 4 * ((w * h * d + 31) // 32)

    @property
    def piece_capacity(self) -> int:
        """Room for brick pieces, from the request's size alone: a segment of a
        volume of edge E crosses at most about E/64 brick faces per axis in
        256 x 64 x 64 bricks (fewer with the uniform endpoints served here), so
        2 + E/32 pieces per segment is ample; pieces beyond the room fall back
        to per-voxel atomics on the device, with the same result."""
        return self.n * (2 + max(self.dims) // 32) + 1024

    @property
    def device_bytes(self) -> int:
        """Volume + segments + workspace share (with brick pieces) of this request."""
        return self.mask_bytes + 24 * self.n + 16 * self.n + 8 * self.piece_capacity + 256

    @property
    def latency_ms(self) -> float:
        return 1000.0 * (self.done_s - self.arrival_s)


class Admission:
    """First-come first-served admission: take requests from the head of the
    queue while they fit the free device memory and the batch limits. With a
    memory probe (free bytes now, the in-flight batches' memory already taken)
    a request is admitted while it fits the probe's free bytes less a reserve,
    and within the cap `budget_bytes` of bytes in flight; a request larger than
    the cap can never run and is rejected."""

    def __init__(self, budget_bytes: int, max_batch_requests: int = 64, max_batch_segments: int = 1 << 24,
                 mem_probe=None, reserve_bytes: int = 1 << 30):
        self.budget_bytes = int(budget_bytes)
        self.max_batch_requests = int(max_batch_requests)
        self.max_batch_segments = int(max_batch_segments)
        self.mem_probe = mem_probe
        self.reserve_bytes = int(reserve_bytes)

    def limit(self, bytes_in_use: int) -> int:
        """Bytes in flight allowed now: the cap, and what the device has free."""
        if self.mem_probe is None:
            return self.budget_bytes
        free = int(self.mem_probe())
        return min(self.budget_bytes, bytes_in_use + max(0, free - self.reserve_bytes))

    def take(self, queue: collections.deque, bytes_in_use: int):
        batch, rejected = [], []
        used = bytes_in_use
        segs = 0
        limit = self.limit(bytes_in_use)
        while queue and len(batch) < self.max_batch_requests:
            r = queue[0]
            if r.device_bytes > self.budget_bytes:
                rejected.append(queue.popleft())
                continue
            if used + r.device_bytes > limit or (batch and segs + r.n > self.max_batch_segments):
                break  # head of line waits for memory (keeps arrival order)
            batch.append(queue.popleft())
            used += r.device_bytes
            segs += r.n
        return batch, rejected


@dataclass
class InFlight:
    bid: int
    reqs: list
    handle: object      # launcher's handle (completion test + buffers kept alive)
    bytes: int
    slot: int
    launched_s: float


@dataclass
class ServeStats:
    completed: int = 0
    rejected: int = 0
    failed: int = 0
    batches: int = 0
    voxels: int = 0
    wall_s: float = 0.0
    max_bytes_in_use: int = 0
    max_inflight: int = 0
    latencies_ms: list = field(default_factory=list)

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.array([math.nan])
        return {
            "completed": self.completed, "rejected": self.rejected, "failed": self.failed,
            "batches": self.batches, "mean_batch": self.completed / max(1, self.batches),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(np.mean(lat)), "voxels": self.voxels,
            "voxels_per_s": self.voxels / self.wall_s if self.wall_s > 0 else 0.0,
            "wall_s": self.wall_s, "max_bytes_in_use": self.max_bytes_in_use, "max_inflight": self.max_inflight,
        }


class Server:
    """The request loop. ``launcher(reqs, slot) -> handle`` starts a batch;
    ``handle.done() -> bool`` polls it; ``handle.finish() -> status`` collects it
    (and may attach results to the requests)."""

    def __init__(self, launcher, budget_bytes: int, max_inflight: int = 4, max_batch_requests: int = 64,
                 max_batch_segments: int = 1 << 24, clock=time.perf_counter, idle_sleep_s: float = 20e-6,
                 mem_probe=None, reserve_bytes: int = 1 << 30):
        self.launcher = launcher
        self.admission = Admission(budget_bytes, max_batch_requests, max_batch_segments, mem_probe, reserve_bytes)
        self.max_inflight = int(max_inflight)
        self.clock = clock
        self.idle_sleep_s = idle_sleep_s

    def run(self, requests, time_limit_s: float = 600.0) -> ServeStats:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        queue = collections.deque()
        inflight = []
        free_slots = list(range(self.max_inflight))
        stats = ServeStats()
        bytes_in_use = 0
        bid = 0
        t0 = self.clock()
        first_arrival = pending[0].arrival_s if pending else 0.0
        last_done = first_arrival
        while pending or queue or inflight:
            now = self.clock() - t0
            if now > time_limit_s:
                raise TimeoutError("serving loop exceeded its time limit")
            progressed = False
            while pending and pending[0].arrival_s <= now:
                queue.append(pending.popleft())
                progressed = True
            # completions
            for b in list(inflight):
                if b.handle.done():
                    st = b.handle.finish()
                    t = self.clock() - t0
                    for r in b.reqs:
                        r.done_s = t
                        r.status = st
                        if st == 0:
                            stats.completed += 1
                            stats.voxels += r.voxels
                            stats.latencies_ms.append(r.latency_ms)
                        else:
                            stats.failed += 1
                    last_done = max(last_done, t)
                    bytes_in_use -= b.bytes
                    free_slots.append(b.slot)
                    inflight.remove(b)
                    progressed = True
            # admission + launch (continuous batching)
            if queue and free_slots:
                batch, rejected = self.admission.take(queue, bytes_in_use)
                for r in rejected:
                    r.status = -2
                    stats.rejected += 1
                if batch:
                    slot = free_slots.pop(0)
                    t = self.clock() - t0
                    for r in batch:
                        r.admitted_s = t
                        r.batch_id = bid
                    nbytes = sum(r.device_bytes for r in batch)
                    handle = self.launcher(batch, slot)
                    inflight.append(InFlight(bid, batch, handle, nbytes, slot, t))
                    bytes_in_use += nbytes
                    stats.batches += 1
                    stats.max_bytes_in_use = max(stats.max_bytes_in_use, bytes_in_use)
                    stats.max_inflight = max(stats.max_inflight, len(inflight))
                    bid += 1
                    progressed = True
            if not progressed and self.idle_sleep_s > 0:
                time.sleep(self.idle_sleep_s)
        stats.wall_s = max(1e-9, last_done - first_arrival)
        return stats


# ------------------------------------------------------------- GPU launcher
class _Handle:
    def __init__(self, event, keep, reqs, keep_results):
        self.event = event
        self.keep = keep
        self.reqs = reqs
        self.keep_results = keep_results

    def done(self) -> bool:
        return self.event.query()

    def finish(self) -> int:
        status = int(self.keep["status"].item())
        if status == 0:
            base = self.keep["base"].cpu().numpy()  # per-scene voxel bases from the device scan
            for k, r in enumerate(self.reqs):
                r.voxels = int(base[k + 1] - base[k])
        if self.keep_results and status == 0:
            for r, m in zip(self.reqs, self.keep["masks"]):
                r.result = m
        self.keep = None
        return status


class GpuLauncher:
    """Launches a batch with vox_generate_batched_ex (volumes only,
    VOX_OUT_FRESH; by bricks when every request's width is a multiple of 32, the
    piece room estimated from the requests' voxel counts) on one of ``slots``
    streams: segments copied from pinned host memory, new volumes written whole
    by the launch, one scene table, one workspace, one completion event."""

    def __init__(self, slots: int, device="cuda", keep_results: bool = False):
        import torch

        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.keep_results = keep_results

    def __call__(self, reqs, slot):
        import torch

        from . import batching, vox

        stream = self.streams[slot]
        n_total = sum(r.n for r in reqs)
        with torch.cuda.stream(stream):
            segs = torch.empty((max(n_total, 1), 6), dtype=torch.int32, device=self.device)
            off = 0
            for r in reqs:
                if r.n:
                    segs[off:off + r.n].copy_(r.segs_host, non_blocking=True)
                off += r.n
            # fresh volumes: cleared by the batched launch (one kernel), not one fill per request
            masks = [torch.empty((r.mask_bytes // 4,), dtype=torch.int32, device=self.device) for r in reqs]
            table = batching.scene_table_bytes([r.n for r in reqs], [r.dims for r in reqs],
                                               [m.data_ptr() for m in masks])
            scenes = torch.frombuffer(bytearray(table), dtype=torch.uint8).pin_memory().to(self.device,
                                                                                         non_blocking=True)
            per_scene = [vox.vox_scene_bricks(r.dims) for r in reqs]
            total_bricks = sum(per_scene) if n_total and all(b > 0 for b in per_scene) else 0
            ws = torch.empty(vox.vox_workspace_size_batched_volume(n_total, len(reqs), total_bricks,
                                                                   sum(r.piece_capacity for r in reqs)),
                             dtype=torch.uint8, device=self.device)
            status = torch.zeros(1, dtype=torch.int32, device=self.device)
            base = torch.empty(len(reqs) + 1, dtype=torch.int64, device=self.device)
            st = vox.load().vox_generate_batched_ex(
                vox._ptr(segs), n_total, vox._ptr(scenes), len(reqs), total_bricks, None, 0,
                vox.OUT_BITMASK | vox.OUT_FRESH, vox._ptr(base), vox._ptr(ws), ws.numel(), vox._ptr(status),
                vox._stream(stream))
            if st != vox.OK:
                raise vox.VoxError(st, "vox_generate_batched_ex")
            ev = torch.cuda.Event()
            ev.record(stream)
        keep = {"segs": segs, "masks": masks, "scenes": scenes, "ws": ws, "status": status, "base": base}
        return _Handle(ev, keep, reqs, self.keep_results)


def make_requests(stream_reqs, pool_size: int = 256, seed: int = 11):
    """Turn a workloads.config5 arrival stream into ServeRequests with pinned
    host payloads. Payloads come from a pool of `pool_size` scenes drawn with the
    stream's own sizes (request i carries pool[i % pool_size]), so that a long
    stream does not need one fresh host buffer per request."""
    import torch

    pool = {}
    out = []
    for i, rq in enumerate(stream_reqs):
        key = i % pool_size
        if key not in pool:
            w = rq.workload()
            pool[key] = (torch.from_numpy(w.segs).pin_memory(), tuple(w.dims))
        segs, dims = pool[key]
        out.append(ServeRequest(rid=i, arrival_s=rq.arrival_s, n=int(segs.shape[0]), dims=dims, segs_host=segs))
    return out


def gpu_free_bytes(device=None) -> int:
    """Free device memory now: the driver's free bytes plus the bytes torch's
    caching allocator holds but does not use (free for the next allocation)."""
    import torch

    free, _ = torch.cuda.mem_get_info(device)
    return int(free + torch.cuda.memory_reserved(device) - torch.cuda.memory_allocated(device))
