"""Batched scenes: many independent voxelization problems in one launch
sequence (vox_generate_batched), optionally captured once in a CUDA graph and
replayed.

Section 5 of the paper ends on this point: single-segment calls waste the GPU on
call and copy overheads, and throughput comes from voxelizing many segments per
kernel call. Here a batch concatenates the scenes' segments, keeps one device
scene table, one list for the whole batch (scene k at [base[k], base[k+1])) and
one volume per scene. All device memory is allocated by torch; the work runs in
libvox's kernels.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import vox


class SceneRecord(ctypes.Structure):
    """Host image of vox_scene (include/vox.h), 40 bytes."""

    _fields_ = [("seg_begin", ctypes.c_int64), ("n", ctypes.c_int64), ("dims", vox.Dims),
                ("reserved", ctypes.c_int32), ("mask", ctypes.c_void_p)]


assert ctypes.sizeof(SceneRecord) == 40


def scene_table_bytes(seg_counts, dims_list, mask_ptrs) -> bytes:
    """Pack a vox_scene array: contiguous scenes in order."""
    n = len(seg_counts)
    arr = (SceneRecord * n)()
    begin = 0
    for k in range(n):
        arr[k].seg_begin = begin
        arr[k].n = int(seg_counts[k])
        w, h, d = (int(v) for v in dims_list[k])
        arr[k].dims = vox.Dims(w, h, d)
        arr[k].reserved = 0
        arr[k].mask = int(mask_ptrs[k]) if mask_ptrs[k] else None
        begin += int(seg_counts[k])
    return bytes(arr)


@dataclass
class Batch:
    """A batch resident on the device: segments, scene table, list, volumes, workspace."""

    segs: object          # int32 [n_total, 6] (cuda)
    scenes: object        # uint8 [40 * n_scenes] (cuda), the vox_scene table
    n_scenes: int
    dims: list
    seg_counts: list
    masks: list           # int32 volume tensors (cuda), one per scene
    lst: object           # int32 / int64 list for the whole batch, or None
    scene_base: object    # int64 [n_scenes + 1] (cuda)
    ws: object
    status: object
    flags: int
    V: int
    total_bricks: int = 0  # > 0: the volumes by bricks (workspace sized for them)
    pieces: int = 0

    def run(self, stream=None):
        """Enqueue the batched launch sequence on `stream` (asynchronous)."""
        st = vox.load().vox_generate_batched_ex(
            vox._ptr(self.segs), self.segs.shape[0], vox._ptr(self.scenes), self.n_scenes, self.total_bricks,
            vox._ptr(self.lst), self.lst.numel() if self.lst is not None else 0, self.flags,
            vox._ptr(self.scene_base), vox._ptr(self.ws), self.ws.numel(), vox._ptr(self.status),
            vox._stream(stream))
        if st != vox.OK:
            raise vox.VoxError(st, "vox_generate_batched_ex")

    def clear_volumes(self):
        for m in self.masks:
            m.zero_()

    def scene_list(self, k: int):
        """View of scene k's voxels in the batch list (after a synchronised run)."""
        b = self.scene_base.cpu().numpy()
        return self.lst[int(b[k]):int(b[k + 1])]


def make_batch(workloads_list, flags=vox.OUT_LIST32 | vox.OUT_BITMASK, device="cuda", bricks=True) -> Batch:
    """Upload scenes (workloads.Workload objects) as one batch. The list is sized
    exactly by the device's plan of the batch (vox_plan_batched: the scan's
    voxel total and, with ``bricks`` and every scene's width a multiple of 32,
    the brick pieces that size the workspace); the launch recounts and checks
    the capacity."""
    import torch

    segs_np = np.ascontiguousarray(np.concatenate([w.segs for w in workloads_list], axis=0), dtype=np.int32)
    seg_counts = [w.n for w in workloads_list]
    dims = [tuple(w.dims) for w in workloads_list]
    masks = []
    if flags & vox.OUT_BITMASK:  # fresh volumes are cleared by the launch itself
        alloc = torch.empty if flags & vox.OUT_FRESH else torch.zeros
        masks = [alloc(vox.vox_mask_words(dm), dtype=torch.int32, device=device) for dm in dims]
    ptrs = [m.data_ptr() for m in masks] if masks else [0] * len(dims)
    table = scene_table_bytes(seg_counts, dims, ptrs)
    scenes = torch.frombuffer(bytearray(table), dtype=torch.uint8).to(device)
    n_scenes = len(workloads_list)
    d_segs = torch.from_numpy(segs_np).to(device)
    status = torch.zeros(1, dtype=torch.int32, device=device)
    per_scene = [vox.vox_scene_bricks(dm) for dm in dims]
    total_bricks = sum(per_scene) if (bricks and flags & vox.OUT_BITMASK and len(segs_np) and
                                      all(b > 0 for b in per_scene)) else 0
    ws = torch.empty(vox.vox_workspace_size_batched_volume(len(segs_np), n_scenes, total_bricks, 0),
                     dtype=torch.uint8, device=device)
    V, pieces = vox.vox_plan_batched(d_segs, scenes, n_scenes, total_bricks, ws, status)
    if total_bricks:
        size = vox.vox_workspace_size_batched_volume(len(segs_np), n_scenes, total_bricks, pieces)
    else:
        size = vox.vox_workspace_size_batched(len(segs_np), n_scenes)
    ws = torch.empty(size, dtype=torch.uint8, device=device)
    lst = None
    if flags & vox.OUT_LIST64:
        lst = torch.empty(max(V, 1), dtype=torch.int64, device=device)
    elif flags & vox.OUT_LIST32:
        lst = torch.empty(max(V, 1), dtype=torch.int32, device=device)
    return Batch(segs=d_segs, scenes=scenes, n_scenes=n_scenes, dims=dims, seg_counts=seg_counts, masks=masks,
                 lst=lst, scene_base=torch.zeros(n_scenes + 1, dtype=torch.int64, device=device), ws=ws,
                 status=status, flags=flags, V=V, total_bricks=total_bricks, pieces=pieces)


class GraphRunner:
    """Capture a launch sequence once (torch.cuda.CUDAGraph) and replay it."""

    def __init__(self, fn, warmup: int = 1):
        import torch

        self.stream = torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            for _ in range(warmup):
                fn(self.stream)
        torch.cuda.current_stream().wait_stream(self.stream)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            fn(self.stream)
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()


class PlainScenes:
    """The same scenes, one vox_generate per scene (the plain per-scene launch),
    with per-scene workspaces sized for the brick volume path."""

    def __init__(self, batch: Batch, device="cuda"):
        import torch

        self.batch = batch
        self.items = []
        segs = batch.segs
        begin = 0
        for k in range(batch.n_scenes):
            n = batch.seg_counts[k]
            s = segs[begin:begin + n].clone()  # own, 16-byte aligned copy
            dims = batch.dims[k]
            ws0 = torch.empty(vox.vox_workspace_size_volume(n, dims, 0), dtype=torch.uint8, device=device)
            V, P = vox.vox_plan(s, dims, ws0, batch.status) if n else (0, 0)
            ws = torch.empty(vox.vox_workspace_size_volume(n, dims, P), dtype=torch.uint8, device=device)
            lst = None
            if batch.lst is not None:
                lst = torch.empty(max(V, 1), dtype=batch.lst.dtype, device=device)
            mask = batch.masks[k] if batch.masks else None
            self.items.append((s, dims, ws, lst, mask, V))
            begin += n

    def run(self, stream=None):
        b = self.batch
        for s, dims, ws, lst, mask, V in self.items:
            if s.shape[0] == 0:
                continue
            vox.vox_generate(s, dims, ws, b.status, lst, mask, b.flags, stream, capacity=V)


class SceneStep:
    """One scene's whole step -- count + scan, the list, a fresh volume -- on
    resident device buffers, captured once as a CUDA graph, on two streams: the
    brick binning's counting pass (vox_count_bins) runs beside the count + scan
    (they read only the segments and write disjoint workspace parts), then the
    list follows the scan on one stream and the volume follows both on the other
    (the two calls share only read-only workspace parts), so the list kernel and
    the volume's binning overlap on the device.

    segs: int32 [n, 6] on the device; list_flag: vox.OUT_LIST32, vox.OUT_LIST64
    or 0 (no list); volume: build the occupancy volume too."""

    def __init__(self, segs, dims, list_flag=vox.OUT_LIST32, volume=True, device="cuda"):
        import torch

        self.segs = segs
        self.dims = tuple(int(v) for v in dims)
        self.list_flag = int(list_flag)
        self.volume = bool(volume)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        n = int(segs.shape[0])
        ws = torch.empty(vox.vox_workspace_size_volume(n, self.dims, 0), dtype=torch.uint8, device=device)
        self.V, self.P = vox.vox_plan(segs, self.dims, ws, self.status) if n else (0, 0)
        self.ws = torch.empty(vox.vox_workspace_size_volume(n, self.dims, self.P), dtype=torch.uint8, device=device)
        self.lst = None
        if self.list_flag:
            dt = torch.int64 if self.list_flag == vox.OUT_LIST64 else torch.int32
            self.lst = torch.empty(max(self.V, 1), dtype=dt, device=device)
        self.mask = torch.empty(vox.vox_mask_words(self.dims), dtype=torch.int32, device=device) if volume else None
        self.plain_ws_bytes = vox.vox_workspace_size(n)  # count + scan only
        self.bricks = bool(volume and n and self.P > 0)
        self.side = torch.cuda.Stream(device=device)
        self.graph = GraphRunner(self.launch)

    def launch(self, s):
        """Enqueue the step on stream `s` (the volume on a second stream, joined back)."""
        import torch

        if self.segs.shape[0] == 0 or not self.volume:
            vox.vox_count(self.segs, self.dims, self.ws, self.status, None, None, s)
            if self.volume:
                vox.vox_generate_from_scan(self.segs, self.dims, self.ws, self.status, None, self.mask,
                                           vox.OUT_BITMASK | vox.OUT_FRESH, s)
            if self.list_flag and self.segs.shape[0]:
                vox.vox_generate_from_scan(self.segs, self.dims, self.ws, self.status, self.lst, None, self.list_flag,
                                           s, capacity=self.V)
            return
        start = torch.cuda.Event()
        start.record(s)
        self.side.wait_event(start)
        if self.bricks:  # the binning's count beside the count + scan
            vox.vox_count_bins(self.segs, self.dims, self.ws, self.side)
            vox.vox_count(self.segs, self.dims, self.ws, self.status, None, None, s, ws_bytes=self.plain_ws_bytes)
        else:
            vox.vox_count(self.segs, self.dims, self.ws, self.status, None, None, s)
        counted = torch.cuda.Event()
        counted.record(s)
        self.side.wait_event(counted)  # a count error keeps the volume from being written
        vox.vox_generate_from_scan(self.segs, self.dims, self.ws, self.status, None, self.mask,
                                   vox.OUT_BITMASK | vox.OUT_FRESH, self.side)
        if self.list_flag:
            vox.vox_generate_from_scan(self.segs, self.dims, self.ws, self.status, self.lst, None, self.list_flag, s,
                                       capacity=self.V)
        done = torch.cuda.Event()
        done.record(self.side)
        s.wait_event(done)

    def replay(self):
        """Replay the captured step on the current stream (asynchronous)."""
        self.graph.replay()
