"""The oracle over disjoint parts of a large workload, in worker processes.

Full-size parity on the largest workloads (billions of voxels, an 8 GiB volume)
is out of reach of one single-threaded oracle call within a test's time, so the
unchanged oracle functions run on disjoint parts in parallel: contiguous
segment ranges for lists (a range's voxels are a contiguous part of the list,
starting at the oracle's own offset of its first segment), z-slabs for volumes
(oracle.bitmask_zslab), whole scenes or requests for batches. Each worker
compares its part element by element with the matching part of the CUDA path's
output, which the test process copies from the device into a host buffer the
worker can read (shared memory, or the pickled array when shared memory is too
small), and returns the number of mismatches and the first ones.

Workers are started with the spawn method: none inherits the test process's
CUDA context. Nothing here feeds the CUDA path; the device data only flows
toward the comparison.
"""

from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import shared_memory

import numpy as np

_cache = {}


def _init():
    import oracle

    oracle.get()


class Buf:
    """A host array that workers can read: in shared memory when there is room
    for it in /dev/shm, else carried by value (pickled)."""

    def __init__(self, arr: np.ndarray, shared: bool):
        arr = np.ascontiguousarray(arr)
        self.dtype, self.shape = arr.dtype.str, arr.shape
        self.shm = None
        self.arr = None
        if shared and arr.nbytes > 0:
            self.shm = shared_memory.SharedMemory(create=True, size=arr.nbytes)
            np.ndarray(arr.shape, arr.dtype, buffer=self.shm.buf)[...] = arr
            self.name = self.shm.name
        else:
            self.arr = arr
            self.name = None

    def __getstate__(self):
        return {"dtype": self.dtype, "shape": self.shape, "name": self.name, "arr": self.arr}

    def __setstate__(self, st):
        self.dtype, self.shape, self.name, self.arr = st["dtype"], st["shape"], st["name"], st["arr"]
        self.shm = None

    def view(self) -> np.ndarray:
        if self.arr is not None:
            return self.arr
        if self.name is None:
            return np.zeros(self.shape, np.dtype(self.dtype))
        shm = _cache.get(self.name)
        if shm is None:
            # spawned workers share the test process's resource tracker, which
            # already knows the segment; the test process unlinks it
            shm = shared_memory.SharedMemory(name=self.name)
            _cache[self.name] = shm
        return np.ndarray(self.shape, np.dtype(self.dtype), buffer=shm.buf)

    def release(self):
        if self.shm is not None:
            self.shm.close()
            self.shm.unlink()
            self.shm = None


def _forget(name):
    shm = _cache.pop(name, None)
    if shm is not None:
        shm.close()


def _mismatch(got: np.ndarray, want: np.ndarray, base: int = 0) -> dict:
    if got.shape == want.shape and np.array_equal(got, want):
        return {"bad": 0}
    if got.shape != want.shape:
        return {"bad": -1, "why": f"shape {got.shape} != {want.shape}"}
    bad = np.flatnonzero(got != want)
    return {"bad": int(len(bad)), "first": [int(base + i) for i in bad[:8]],
            "got": [int(v) for v in got[bad[:8]]], "want": [int(v) for v in want[bad[:8]]]}


# ------------------------------------------------------------------ worker jobs
def job_list(segs: Buf, s0: int, s1: int, wide: bool, dev_part: Buf, base: int) -> dict:
    """Oracle list of segments [s0, s1) against the device's list part."""
    import oracle

    O = oracle.get()
    part = segs.view()[s0:s1]
    want = O.list64(part) if wide else O.list32(part)
    got = dev_part.view()
    got = got.view(np.uint64) if wide else got.view(np.uint32)
    out = _mismatch(got, want, base)
    del got
    _forget(dev_part.name)
    return out


def job_zslab(segs: Buf, dims, z0: int, z1: int, dev_parts) -> dict:
    """Oracle z-slab [z0, z1) of the volume against one or more device copies of
    the same slab (e.g. the brick-built and the atomic volume)."""
    import oracle

    O = oracle.get()
    want = O.bitmask_zslab(segs.view(), dims, z0, z1)
    out = {"words": int(want.shape[0]), "nonzero": int(np.count_nonzero(want)), "parts": []}
    for b in dev_parts:
        got = b.view().view(np.uint32)
        out["parts"].append(_mismatch(got, want, 0))
        del got
        _forget(b.name)
    return out


def job_scene(segs: Buf, s0: int, s1: int, dims, flags_list: int, dev_list: Buf | None, dev_mask: Buf | None) -> dict:
    """One scene (segments [s0, s1) of a batch in volume `dims`): its list part
    and its volume against the oracle. flags_list: 0, 32 or 64."""
    import oracle

    O = oracle.get()
    part = segs.view()[s0:s1]
    out = {}
    if dev_list is not None:
        want = O.list64(part) if flags_list == 64 else O.list32(part)
        got = dev_list.view().view(want.dtype)
        out["list"] = _mismatch(got, want)
        del got
        _forget(dev_list.name)
    if dev_mask is not None:
        want = O.bitmask(part, dims)
        got = dev_mask.view().view(np.uint32)
        out["mask"] = _mismatch(got, want)
        del got
        _forget(dev_mask.name)
    return out


# ------------------------------------------------------------------ the pool
def shm_room() -> int:
    """Bytes free in /dev/shm (0 when there is none)."""
    try:
        st = os.statvfs("/dev/shm")
        return st.f_bavail * st.f_frsize
    except OSError:
        return 0


class OraclePool:
    """Spawn-started worker pool running the oracle; jobs in flight are bounded
    so that the host buffers they hold stay within `max_bytes_in_flight`."""

    def __init__(self, workers: int | None = None, max_bytes_in_flight: int = 24 << 30):
        self.workers = workers or max(1, min(16, os.cpu_count() or 1))
        self.ex = ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"), initializer=_init)
        self.max_bytes = max_bytes_in_flight
        self.pending = []  # (future, bufs, nbytes, tag)
        self.results = []
        self.bytes = 0
        self._room = shm_room()
        self._shared_bytes = 0

    def buf(self, arr: np.ndarray) -> Buf:
        # shared memory while /dev/shm has room (with a margin), else by value
        shared = self._shared_bytes + arr.nbytes < 0.8 * self._room
        b = Buf(arr, shared)
        if b.shm is not None:
            self._shared_bytes += arr.nbytes
        return b

    def _release(self, bufs):
        for b in bufs:
            if b.shm is not None:
                self._shared_bytes -= int(np.prod(b.shape)) * np.dtype(b.dtype).itemsize
            b.release()

    def _drain(self, keep_bytes: int):
        while self.pending and self.bytes > keep_bytes:
            fut, bufs, nbytes, tag = self.pending.pop(0)
            self.results.append((tag, fut.result()))
            self._release(bufs)
            self.bytes -= nbytes

    def submit(self, tag, fn, *args, bufs=()):
        """Run fn(*args) in a worker; `bufs` (device copies owned by this job)
        are released when the job is done."""
        nbytes = sum(int(np.prod(b.shape)) * np.dtype(b.dtype).itemsize for b in bufs)
        self._drain(self.max_bytes - nbytes)
        self.pending.append((self.ex.submit(fn, *args), list(bufs), nbytes, tag))
        self.bytes += nbytes

    def finish(self):
        self._drain(-1)
        out, self.results = self.results, []
        return out

    def close(self):
        try:
            self.finish()
        finally:
            self.ex.shutdown(wait=True, cancel_futures=True)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
