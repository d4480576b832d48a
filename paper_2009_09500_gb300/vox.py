"""Python binding of libvox (include/vox.h): argument marshalling only.

Every step of the voxelization runs in the CUDA kernels of ``libvox.so``; this
module turns torch tensors into pointers, picks the current CUDA stream, and
raises on a non-OK status. There is no CPU fallback: if the library is missing
the import of a function fails loudly.

Names follow the C ABI: ``vox_count``, ``vox_generate``,
``vox_generate_from_scan``, ``vox_generate_host``, ``vox_workspace_size``,
``vox_mask_words``, ``vox_strerror``.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK = 0
ERR_INVALID_ARG = 1
ERR_OUT_OF_BOUNDS = 2
ERR_PACK_WIDTH = 3
ERR_CAPACITY = 4
ERR_TIMEOUT = 5
ERR_CUDA = 6
ERR_WORKSPACE = 7
ERR_ALIGNMENT = 8

OUT_LIST32 = 1
OUT_LIST64 = 2
OUT_BITMASK = 4
OUT_FRESH = 8
OUT_BRICKED = 16

EXPORTED = (
    "vox_workspace_size", "vox_count", "vox_generate", "vox_generate_from_scan",
    "vox_host_arena_size", "vox_generate_host", "vox_strerror", "vox_mask_words",
    "vox_debug_set_scan_stall", "vox_scan_tile_segments", "vox_generate_noalloc",
    "vox_workspace_size_volume", "vox_plan", "vox_workspace_size_batched", "vox_generate_batched",
    "vox_set_tuning", "vox_get_tuning", "vox_host_arena_size_volume",
    "vox_mask_words_bricked", "vox_brick_shape", "vox_unbrick",
    "vox_euclid_workspace_size", "vox_euclid_generate", "vox_euclid_plan", "vox_euclid_workspace_size_volume",
    "vox_count_bins", "vox_scene_bricks", "vox_workspace_size_batched_volume", "vox_generate_batched_ex",
    "vox_plan_batched", "vox_probe_red_or", "vox_probe_red_or_ops",
)

VOLUME_AUTO = 0
VOLUME_ATOMIC = 1
VOLUME_ATOMIC_WARP = 2


class Tuning(ctypes.Structure):
    _fields_ = [("run_len", ctypes.c_int32), ("volume_path", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("list_runs", ctypes.c_int32)]
NOALLOC_MAX_SEGMENTS = 2000000


class Dims(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32), ("d", ctypes.c_int32)]


class VoxError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__(f"{where}: {strerror(status)} (status {status})")


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libvox.so (never builds implicitly; call build.build_library())."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _build.LIB
    try:  # load torch's CUDA runtime first so that libvox shares it (same current device)
        import torch  # noqa: F401
    except ImportError:
        pass
    if not os.path.exists(path):
        raise RuntimeError(f"libvox.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
    lib.vox_workspace_size.argtypes = [i64]
    lib.vox_workspace_size.restype = sz
    lib.vox_count.argtypes = [vp, i64, Dims, vp, vp, vp, sz, vp, vp]
    lib.vox_count.restype = i32
    lib.vox_count_bins.argtypes = [vp, i64, Dims, vp, sz, vp]
    lib.vox_count_bins.restype = i32
    for name in ("vox_generate", "vox_generate_from_scan"):
        f = getattr(lib, name)
        f.argtypes = [vp, i64, Dims, vp, i64, vp, i32, vp, sz, vp, vp]
        f.restype = i32
    lib.vox_host_arena_size.argtypes = [i64, Dims, i32, i64]
    lib.vox_host_arena_size.restype = sz
    lib.vox_host_arena_size_volume.argtypes = [i64, Dims, i32, i64, i64]
    lib.vox_host_arena_size_volume.restype = sz
    lib.vox_mask_words_bricked.argtypes = [Dims]
    lib.vox_mask_words_bricked.restype = i64
    lib.vox_brick_shape.argtypes = [Dims, vp]
    lib.vox_brick_shape.restype = i32
    lib.vox_unbrick.argtypes = [vp, Dims, vp, vp, vp]
    lib.vox_unbrick.restype = i32
    lib.vox_euclid_workspace_size.argtypes = [i64]
    lib.vox_euclid_workspace_size.restype = sz
    lib.vox_euclid_generate.argtypes = [vp, i64, Dims, vp, i64, vp, i32, vp, vp, sz, vp, vp]
    lib.vox_euclid_generate.restype = i32
    lib.vox_euclid_plan.argtypes = [vp, i64, Dims, vp, sz, vp, vp, vp, vp, vp]
    lib.vox_euclid_workspace_size_volume.argtypes = [i64, Dims, i64]
    lib.vox_euclid_workspace_size_volume.restype = sz
    lib.vox_euclid_plan.restype = i32
    lib.vox_generate_host.argtypes = [vp, i64, Dims, vp, i64, vp, i32, vp, sz, vp, vp]
    lib.vox_generate_host.restype = i32
    lib.vox_strerror.argtypes = [i32]
    lib.vox_strerror.restype = ctypes.c_char_p
    lib.vox_mask_words.argtypes = [Dims]
    lib.vox_mask_words.restype = i64
    lib.vox_debug_set_scan_stall.argtypes = [i64, i64]
    lib.vox_debug_set_scan_stall.restype = None
    lib.vox_scan_tile_segments.argtypes = []
    lib.vox_scan_tile_segments.restype = i64
    lib.vox_workspace_size_volume.argtypes = [i64, Dims, i64]
    lib.vox_workspace_size_volume.restype = sz
    lib.vox_plan.argtypes = [vp, i64, Dims, vp, sz, vp, vp, vp, vp]
    lib.vox_plan.restype = i32
    lib.vox_workspace_size_batched.argtypes = [i64, ctypes.c_int32]
    lib.vox_workspace_size_batched.restype = sz
    lib.vox_generate_batched.argtypes = [vp, i64, vp, ctypes.c_int32, vp, i64, i32, vp, vp, sz, vp, vp]
    lib.vox_generate_batched.restype = i32
    lib.vox_scene_bricks.argtypes = [Dims]
    lib.vox_scene_bricks.restype = i64
    lib.vox_workspace_size_batched_volume.argtypes = [i64, ctypes.c_int32, i64, i64]
    lib.vox_workspace_size_batched_volume.restype = sz
    lib.vox_generate_batched_ex.argtypes = [vp, i64, vp, ctypes.c_int32, i64, vp, i64, i32, vp, vp, sz, vp, vp]
    lib.vox_generate_batched_ex.restype = i32
    lib.vox_plan_batched.argtypes = [vp, i64, vp, ctypes.c_int32, i64, vp, sz, vp, vp, vp, vp]
    lib.vox_plan_batched.restype = i32
    lib.vox_set_tuning.argtypes = [vp]
    lib.vox_set_tuning.restype = None
    lib.vox_get_tuning.argtypes = [vp]
    lib.vox_get_tuning.restype = None
    lib.vox_generate_noalloc.argtypes = [vp, i64, Dims, vp, i64, vp, i32, vp, vp]
    lib.vox_generate_noalloc.restype = i32
    lib.vox_probe_red_or.argtypes = [vp, i64, i64, ctypes.c_uint32, vp]
    lib.vox_probe_red_or.restype = i32
    lib.vox_probe_red_or_ops.argtypes = [i64]
    lib.vox_probe_red_or_ops.restype = i64
    if path == _build.LIB:
        _lib = lib
    return lib


def strerror(status: int) -> str:
    return load().vox_strerror(int(status)).decode()


def _dims(dims) -> Dims:
    w, h, d = (int(v) for v in dims)
    return Dims(w, h, d)


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(int(t.data_ptr()))


def _stream(stream) -> ctypes.c_void_p:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _check(st: int, where: str):
    if st != OK:
        raise VoxError(st, where)


def vox_workspace_size(n: int) -> int:
    return int(load().vox_workspace_size(int(n)))


def vox_workspace_size_volume(n: int, dims, piece_capacity: int) -> int:
    return int(load().vox_workspace_size_volume(int(n), _dims(dims), int(piece_capacity)))


def vox_plan(segs, dims, ws, status, stream=None):
    """Synchronous: returns (V, pieces) for these segments (pieces = 0 when the
    volume cannot use bricks). ``ws`` must hold vox_workspace_size_volume(n, dims, 0)."""
    _check_segs(segs)
    V = ctypes.c_int64(0)
    P = ctypes.c_int64(0)
    st = load().vox_plan(_ptr(segs), segs.shape[0], _dims(dims), _ptr(ws), ws.numel() * ws.element_size(),
                         _ptr(status), ctypes.byref(V), ctypes.byref(P), _stream(stream))
    _check(st, "vox_plan")
    return int(V.value), int(P.value)


def vox_workspace_size_batched(n_total: int, n_scenes: int) -> int:
    return int(load().vox_workspace_size_batched(int(n_total), int(n_scenes)))


def vox_scene_bricks(dims) -> int:
    return int(load().vox_scene_bricks(_dims(dims)))


def vox_workspace_size_batched_volume(n_total: int, n_scenes: int, total_bricks: int, piece_capacity: int) -> int:
    return int(load().vox_workspace_size_batched_volume(int(n_total), int(n_scenes), int(total_bricks),
                                                        int(piece_capacity)))


def vox_plan_batched(segs, scenes, n_scenes: int, total_bricks: int, ws, status, stream=None):
    """Synchronous: (total voxels, brick pieces) of a batch."""
    v, pc = ctypes.c_int64(0), ctypes.c_int64(0)
    st = load().vox_plan_batched(_ptr(segs), segs.shape[0], _ptr(scenes), int(n_scenes), int(total_bricks), _ptr(ws),
                                 ws.numel() * ws.element_size(), _ptr(status), ctypes.byref(v), ctypes.byref(pc),
                                 _stream(stream))
    _check(st, "vox_plan_batched")
    return int(v.value), int(pc.value)


def vox_set_tuning(run_len: int = 0, volume_path: int = 0, ctas_per_sm: int = 0, list_runs: int = 0) -> None:
    t = Tuning(int(run_len), int(volume_path), int(ctas_per_sm), int(list_runs))
    load().vox_set_tuning(ctypes.byref(t))


def vox_reset_tuning() -> None:
    load().vox_set_tuning(None)


def vox_get_tuning() -> dict:
    t = Tuning()
    load().vox_get_tuning(ctypes.byref(t))
    return {"run_len": t.run_len, "volume_path": t.volume_path, "ctas_per_sm": t.ctas_per_sm, "list_runs": t.list_runs}


def vox_mask_words(dims) -> int:
    return int(load().vox_mask_words(_dims(dims)))


def vox_strerror(status: int) -> str:
    return strerror(status)


def vox_scan_tile_segments() -> int:
    return int(load().vox_scan_tile_segments())


def vox_debug_set_scan_stall(tile: int, wait_ns: int = 0) -> None:
    load().vox_debug_set_scan_stall(int(tile), int(wait_ns))


def _check_segs(segs):
    import torch

    if not (segs.is_cuda and segs.dtype == torch.int32 and segs.dim() == 2 and segs.shape[1] == 6
            and segs.is_contiguous()):
        raise ValueError("segments must be a contiguous CUDA int32 tensor of shape [n, 6]")


def vox_count(segs, dims, ws, status, counts=None, offsets=None, stream=None, ws_bytes=None) -> None:
    """Launch the count + scan on ``stream``; raises on host-side errors only
    (device errors land in ``status``). ``ws_bytes`` (default: all of ``ws``) set
    to vox_workspace_size(n) leaves the brick binning's count to vox_count_bins."""
    _check_segs(segs)
    nbytes = ws.numel() * ws.element_size() if ws_bytes is None else int(ws_bytes)
    st = load().vox_count(_ptr(segs), segs.shape[0], _dims(dims), _ptr(counts), _ptr(offsets),
                          _ptr(ws), nbytes, _ptr(status), _stream(stream))
    _check(st, "vox_count")


def vox_count_bins(segs, dims, ws, stream=None) -> None:
    """The brick binning's counting pass alone (asynchronous)."""
    _check_segs(segs)
    st = load().vox_count_bins(_ptr(segs), segs.shape[0], _dims(dims), _ptr(ws), ws.numel() * ws.element_size(),
                               _stream(stream))
    _check(st, "vox_count_bins")


def _gen(fn, segs, dims, ws, status, list_out=None, mask=None, flags=None, stream=None, capacity=None):
    import torch

    _check_segs(segs)
    if flags is None:
        flags = 0
        if list_out is not None:
            flags |= OUT_LIST64 if list_out.dtype in (torch.int64, torch.uint64) else OUT_LIST32
        if mask is not None:
            flags |= OUT_BITMASK
    cap = int(capacity if capacity is not None else (list_out.numel() if list_out is not None else 0))
    st = fn(_ptr(segs), segs.shape[0], _dims(dims), _ptr(list_out), cap, _ptr(mask), int(flags),
            _ptr(ws), ws.numel() * ws.element_size(), _ptr(status), _stream(stream))
    return st


def vox_generate(segs, dims, ws, status, list_out=None, mask=None, flags=None, stream=None, capacity=None):
    """Count, scan and generate on ``stream`` (asynchronous). ``list_out``: int32
    tensor for the 32-bit list or int64 for the 64-bit list; ``mask``: int32
    tensor of vox_mask_words(dims) words, OR-ed into."""
    st = _gen(load().vox_generate, segs, dims, ws, status, list_out, mask, flags, stream, capacity)
    _check(st, "vox_generate")


def vox_generate_from_scan(segs, dims, ws, status, list_out=None, mask=None, flags=None, stream=None,
                           capacity=None):
    st = _gen(load().vox_generate_from_scan, segs, dims, ws, status, list_out, mask, flags, stream, capacity)
    _check(st, "vox_generate_from_scan")


def vox_generate_noalloc(segs, dims, status, list_out=None, mask=None, flags=None, stream=None, capacity=None):
    """vox_generate for callers that cannot allocate device memory: the scratch
    is the library's static device array, so a call takes at most
    NOALLOC_MAX_SEGMENTS segments (more raise VoxError with VOX_ERR_WORKSPACE,
    naming the limit, before anything is launched). The path is vox_generate's
    with a workspace of vox_workspace_size(n) bytes (volume by per-voxel
    atomics; VOX_OUT_BRICKED is refused with VOX_ERR_WORKSPACE). Calls that
    overlap on the GPU share that array and race."""
    import torch

    _check_segs(segs)
    if segs.shape[0] > NOALLOC_MAX_SEGMENTS:
        err = VoxError(ERR_WORKSPACE, "vox_generate_noalloc")
        err.args = (f"vox_generate_noalloc: {segs.shape[0]} segments exceed the static scratch's limit of "
                    f"{NOALLOC_MAX_SEGMENTS} segments per call (status {ERR_WORKSPACE})",)
        raise err
    if flags is None:
        flags = 0
        if list_out is not None:
            flags |= OUT_LIST64 if list_out.dtype in (torch.int64, torch.uint64) else OUT_LIST32
        if mask is not None:
            flags |= OUT_BITMASK
    cap = int(capacity if capacity is not None else (list_out.numel() if list_out is not None else 0))
    st = load().vox_generate_noalloc(_ptr(segs), segs.shape[0], _dims(dims), _ptr(list_out), cap, _ptr(mask),
                                     int(flags), _ptr(status), _stream(stream))
    _check(st, "vox_generate_noalloc")


def vox_probe_red_or(buf, ops: int, seed: int = 1, stream=None) -> int:
    """Issue about `ops` red.or reductions at pseudo-random words of the device
    int32 tensor `buf` (measurement helper, asynchronous); returns the exact count."""
    lib = load()
    st = lib.vox_probe_red_or(_ptr(buf), buf.numel(), int(ops), int(seed) & 0xffffffff, _stream(stream))
    _check(st, "vox_probe_red_or")
    return int(lib.vox_probe_red_or_ops(int(ops)))


def vox_probe_red_or_ops(ops: int) -> int:
    """The exact number of reductions vox_probe_red_or issues for `ops`."""
    return int(load().vox_probe_red_or_ops(int(ops)))


def vox_host_arena_size(n: int, dims, flags: int, capacity: int) -> int:
    return int(load().vox_host_arena_size(int(n), _dims(dims), int(flags), int(capacity)))


def vox_mask_words_bricked(dims) -> int:
    return int(load().vox_mask_words_bricked(_dims(dims)))


def vox_brick_shape(dims):
    """((B0, B1, B2), (nb0, nb1, nb2)) of the brick-major layout for dims."""
    out = (ctypes.c_int32 * 6)()
    st = load().vox_brick_shape(_dims(dims), out)
    if st != OK:
        raise VoxError(st, "vox_brick_shape")
    return tuple(out[:3]), tuple(out[3:])


def vox_unbrick(bricked, dims, mask, stream=None, status=None):
    """Brick-major volume (device int32 tensor) -> row-major volume `mask`."""
    st = load().vox_unbrick(_ptr(bricked), _dims(dims), _ptr(mask), _ptr(status), _stream(stream))
    if st != OK:
        raise VoxError(st, "vox_unbrick")


def vox_euclid_workspace_size(n: int) -> int:
    return int(load().vox_euclid_workspace_size(int(n)))


def vox_euclid_workspace_size_volume(n: int, dims, piece_capacity: int) -> int:
    return int(load().vox_euclid_workspace_size_volume(int(n), _dims(dims), int(piece_capacity)))


def vox_euclid_plan(segs, dims, ws, status, stream=None, with_pieces=False):
    """(total voxels, total samples[, brick pieces]) of the Euclidean-N variant
    (synchronous)."""
    v, s, pc = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    st = load().vox_euclid_plan(_ptr(segs), segs.shape[0], _dims(dims), _ptr(ws), ws.numel(), _ptr(status),
                                ctypes.byref(v), ctypes.byref(s), ctypes.byref(pc), _stream(stream))
    if st != OK:
        raise VoxError(st, "vox_euclid_plan")
    if with_pieces:
        return int(v.value), int(s.value), int(pc.value)
    return int(v.value), int(s.value)


def vox_euclid_generate(segs, dims, ws, status, list_out=None, mask=None, flags=None, offsets=None, stream=None,
                        capacity=None):
    """The Euclidean-N variant: compacted list and/or volume (asynchronous).
    offsets: device int64 [n + 1] receiving each segment's first list position."""
    import torch

    if flags is None:
        flags = 0
        if list_out is not None:
            flags |= OUT_LIST64 if list_out.dtype in (torch.int64, torch.uint64) else OUT_LIST32
        if mask is not None:
            flags |= OUT_BITMASK
    cap = (list_out.numel() if list_out is not None else 0) if capacity is None else int(capacity)
    st = load().vox_euclid_generate(_ptr(segs), segs.shape[0], _dims(dims), _ptr(list_out), cap, _ptr(mask),
                                    int(flags), _ptr(offsets), _ptr(ws), ws.numel(), _ptr(status), _stream(stream))
    if st != OK:
        raise VoxError(st, "vox_euclid_generate")


def vox_host_arena_size_volume(n: int, dims, flags: int, capacity: int, piece_capacity: int) -> int:
    return int(load().vox_host_arena_size_volume(int(n), _dims(dims), int(flags), int(capacity),
                                                 int(piece_capacity)))


def vox_generate_host(h_segs, dims, arena, h_list=None, h_mask=None, flags=None, stream=None):
    """Synchronous host-buffer variant: copies in, generates, copies out.
    h_segs / h_list / h_mask are CPU tensors (pinned for speed). Returns V."""
    import torch

    if not (h_segs.dtype == torch.int32 and h_segs.dim() == 2 and h_segs.shape[1] == 6
            and h_segs.is_contiguous() and not h_segs.is_cuda):
        raise ValueError("h_segs must be a contiguous CPU int32 tensor of shape [n, 6]")
    if flags is None:
        flags = 0
        if h_list is not None:
            flags |= OUT_LIST64 if h_list.dtype in (torch.int64, torch.uint64) else OUT_LIST32
        if h_mask is not None:
            flags |= OUT_BITMASK
    cap = h_list.numel() if h_list is not None else 0
    total = ctypes.c_int64(0)
    st = load().vox_generate_host(_ptr(h_segs), h_segs.shape[0], _dims(dims), _ptr(h_list), cap, _ptr(h_mask),
                                  int(flags), _ptr(arena), arena.numel() * arena.element_size(),
                                  ctypes.byref(total), _stream(stream))
    _check(st, "vox_generate_host")
    return int(total.value)


# ------------------------------------------------------------------ conveniences
class Voxelizer:
    """Owns a reusable workspace and status word on one device (torch-allocated),
    and allocates outputs on request. Thin: every call goes to the C ABI."""

    def __init__(self, max_segments: int, device=None):
        import torch

        self.device = torch.device(device or "cuda")
        self.max_segments = int(max_segments)
        self.ws = torch.empty(vox_workspace_size(self.max_segments), dtype=torch.uint8, device=self.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def _fit(self, n: int):
        if n > self.max_segments:
            import torch

            self.max_segments = n
            self.ws = torch.empty(vox_workspace_size(n), dtype=torch.uint8, device=self.device)

    def count(self, segs, dims, stream=None):
        """Returns (counts int32[n], offsets int64[n+1]) as device tensors."""
        import torch

        n = segs.shape[0]
        self._fit(n)
        counts = torch.empty(n, dtype=torch.int32, device=self.device)
        offsets = torch.empty(n + 1, dtype=torch.int64, device=self.device)
        vox_count(segs, dims, self.ws, self.status, counts, offsets, stream)
        return counts, offsets

    def total(self, segs, dims) -> int:
        _, off = self.count(segs, dims)
        self.raise_status()
        return int(off[-1].item())

    def generate(self, segs, dims, list_out=None, mask=None, flags=None, stream=None):
        self._fit(segs.shape[0])
        vox_generate(segs, dims, self.ws, self.status, list_out, mask, flags, stream)

    def raise_status(self):
        st = int(self.status.item())
        if st != OK:
            raise VoxError(st, "device")


def segments_tensor(segs_np: np.ndarray, device="cuda"):
    import torch

    a = np.ascontiguousarray(segs_np, dtype=np.int32)
    return torch.from_numpy(a).to(device)
