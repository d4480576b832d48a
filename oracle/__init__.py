"""CPU oracle for parametric 3D segment voxelization (Section 3, Eq. (2)-(3), Fig. 3).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` are the only callers. The product path
(the CUDA library and its binding) never imports this package.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, compiled with gcc
into ``liboracle.so`` next to it). This module only marshals numpy arrays.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_OUT_OF_BOUNDS = 2
ERR_PACK_WIDTH = 3

_lib = None


def build(src: str = _SRC, out: str = _LIB, extra_flags=()) -> str:
    """Compile the oracle with gcc (-O2, no vector intrinsics, portable C)."""
    cmd = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", *extra_flags, "-o", out, src]
    subprocess.run(cmd, check=True)
    return out


def _needs_build() -> bool:
    return (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)


def load(path: str | None = None):
    """Load (building first if stale) and return the ctypes handle."""
    global _lib
    if path is None:
        if _lib is not None:
            return _lib
        if _needs_build():
            build()
        path = _LIB
    lib = ctypes.CDLL(path)
    p = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.oracle_steps.argtypes = [p]
    lib.oracle_steps.restype = i64
    lib.oracle_voxel.argtypes = [p, i64, p]
    lib.oracle_voxel.restype = None
    lib.oracle_validate.argtypes = [p, i64, p, ctypes.c_int]
    lib.oracle_validate.restype = ctypes.c_int
    lib.oracle_count.argtypes = [p, i64, p]
    lib.oracle_count.restype = None
    lib.oracle_offsets.argtypes = [p, i64, p]
    lib.oracle_offsets.restype = None
    for name in ("oracle_list32", "oracle_list64"):
        getattr(lib, name).argtypes = [p, i64, p, i64]
        getattr(lib, name).restype = i64
    lib.oracle_bitmask.argtypes = [p, i64, p, p, i64]
    lib.oracle_bitmask.restype = i64
    lib.oracle_bitmask_zslab.argtypes = [p, i64, p, i64, i64, p, i64]
    lib.oracle_bitmask_zslab.restype = i64
    lib.oracle_voxels_xyz.argtypes = [p, i64, i64, p, i64]
    lib.oracle_voxels_xyz.restype = i64
    lib.oracle_sectors_touched.argtypes = [p, i64]
    lib.oracle_sectors_touched.restype = i64
    lib.oracle_popcount.argtypes = [p, i64]
    lib.oracle_popcount.restype = i64
    lib.oracle_isqrt.argtypes = [i64]
    lib.oracle_isqrt.restype = i64
    lib.oracle_euclid_steps.argtypes = [p]
    lib.oracle_euclid_steps.restype = i64
    lib.oracle_euclid_voxel.argtypes = [p, i64, p]
    lib.oracle_euclid_voxel.restype = None
    lib.oracle_euclid_count.argtypes = [p, i64, p]
    lib.oracle_euclid_count.restype = i64
    for name in ("oracle_euclid_list32", "oracle_euclid_list64"):
        getattr(lib, name).argtypes = [p, i64, p, i64]
        getattr(lib, name).restype = i64
    lib.oracle_euclid_bitmask.argtypes = [p, i64, p, p, i64]
    lib.oracle_euclid_bitmask.restype = i64
    if path == _LIB:
        _lib = lib
    return lib


class Oracle:
    """numpy-level view of one compiled oracle library (the default one, or a
    separately compiled copy, e.g. with a planted mistake in a mutation test)."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    @staticmethod
    def _segs(segs) -> np.ndarray:
        a = np.ascontiguousarray(segs, dtype=np.int32)
        if a.ndim != 2 or a.shape[1] != 6:
            raise ValueError("segments must be int32[S, 6]")
        return a

    @staticmethod
    def _ptr(a: np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)

    def steps(self, seg) -> int:
        a = self._segs(np.asarray(seg).reshape(1, 6))
        return int(self.lib.oracle_steps(self._ptr(a)))

    def voxel(self, seg, k: int):
        a = self._segs(np.asarray(seg).reshape(1, 6))
        out = np.zeros(3, dtype=np.int64)
        self.lib.oracle_voxel(self._ptr(a), int(k), self._ptr(out))
        return tuple(int(v) for v in out)

    def validate(self, segs, dims, want_list32: bool = False) -> int:
        a = self._segs(segs)
        d = np.ascontiguousarray(dims, dtype=np.int32)
        return int(self.lib.oracle_validate(self._ptr(a), a.shape[0], self._ptr(d), int(want_list32)))

    def count(self, segs) -> np.ndarray:
        a = self._segs(segs)
        out = np.zeros(a.shape[0], dtype=np.int32)
        self.lib.oracle_count(self._ptr(a), a.shape[0], self._ptr(out))
        return out

    def offsets(self, counts) -> np.ndarray:
        c = np.ascontiguousarray(counts, dtype=np.int32)
        out = np.zeros(c.shape[0] + 1, dtype=np.int64)
        self.lib.oracle_offsets(self._ptr(c), c.shape[0], self._ptr(out))
        return out

    def total(self, segs) -> int:
        return int(self.offsets(self.count(segs))[-1])

    def list32(self, segs) -> np.ndarray:
        a = self._segs(segs)
        v = self.total(a)
        out = np.zeros(v, dtype=np.uint32)
        got = self.lib.oracle_list32(self._ptr(a), a.shape[0], self._ptr(out), v)
        assert got == v, "list length differs from the voxel count"
        return out

    def list64(self, segs) -> np.ndarray:
        a = self._segs(segs)
        v = self.total(a)
        out = np.zeros(v, dtype=np.uint64)
        got = self.lib.oracle_list64(self._ptr(a), a.shape[0], self._ptr(out), v)
        assert got == v, "list length differs from the voxel count"
        return out

    @staticmethod
    def mask_words(dims) -> int:
        w, h, d = (int(x) for x in dims)
        return (w * h * d + 31) // 32

    def bitmask(self, segs, dims, mask: np.ndarray | None = None) -> np.ndarray:
        a = self._segs(segs)
        d = np.ascontiguousarray(dims, dtype=np.int32)
        if mask is None:
            mask = np.zeros(self.mask_words(dims), dtype=np.uint32)
        assert mask.dtype == np.uint32 and mask.flags.c_contiguous
        got = self.lib.oracle_bitmask(self._ptr(a), a.shape[0], self._ptr(d), self._ptr(mask), mask.shape[0])
        assert got >= 0, "a voxel fell outside the volume"
        return mask

    def slab_words(self, dims, z0: int, z1: int) -> int:
        w, h, _ = (int(x) for x in dims)
        return (w * h * (z1 - z0) + 31) // 32

    def bitmask_zslab(self, segs, dims, z0: int, z1: int, slab: np.ndarray | None = None) -> np.ndarray:
        """The volume's voxels with z in [z0, z1), OR-ed into a w x h x (z1 - z0)
        slab (bit x + w (y + h (z - z0))); with z0 w h a multiple of 32 its words
        are the whole volume's words from z0 w h / 32 on."""
        a = self._segs(segs)
        d = np.ascontiguousarray(dims, dtype=np.int32)
        if slab is None:
            slab = np.zeros(self.slab_words(dims, z0, z1), dtype=np.uint32)
        assert slab.dtype == np.uint32 and slab.flags.c_contiguous
        got = self.lib.oracle_bitmask_zslab(self._ptr(a), a.shape[0], self._ptr(d), int(z0), int(z1),
                                            self._ptr(slab), slab.shape[0])
        assert got >= 0, "a voxel fell outside the slab"
        return slab

    def voxels_xyz(self, segs, s_begin: int = 0, s_end: int | None = None) -> np.ndarray:
        a = self._segs(segs)
        if s_end is None:
            s_end = a.shape[0]
        v = int(self.count(a[s_begin:s_end]).astype(np.int64).sum())
        out = np.zeros((v, 3), dtype=np.int64)
        got = self.lib.oracle_voxels_xyz(self._ptr(a), s_begin, s_end, self._ptr(out), v)
        assert got == v, "voxel sequence length differs from the voxel count"
        return out

    def sectors_touched(self, mask: np.ndarray) -> int:
        m = np.ascontiguousarray(mask, dtype=np.uint32)
        return int(self.lib.oracle_sectors_touched(self._ptr(m), m.shape[0]))

    def popcount(self, mask: np.ndarray) -> int:
        m = np.ascontiguousarray(mask, dtype=np.uint32)
        return int(self.lib.oracle_popcount(self._ptr(m), m.shape[0]))

    # ---- the Euclidean-N variant (Eq. (1)-(2) read literally, repeats removed)
    def isqrt(self, x: int) -> int:
        return int(self.lib.oracle_isqrt(int(x)))

    def euclid_steps(self, seg) -> int:
        a = self._segs(np.asarray(seg).reshape(1, 6))
        return int(self.lib.oracle_euclid_steps(self._ptr(a)))

    def euclid_voxel(self, seg, k: int):
        a = self._segs(np.asarray(seg).reshape(1, 6))
        out = np.zeros(3, dtype=np.int64)
        self.lib.oracle_euclid_voxel(self._ptr(a), int(k), self._ptr(out))
        return tuple(int(v) for v in out)

    def euclid_count(self, segs) -> np.ndarray:
        a = self._segs(segs)
        out = np.zeros(a.shape[0], dtype=np.int64)
        self.lib.oracle_euclid_count(self._ptr(a), a.shape[0], self._ptr(out))
        return out

    def euclid_list32(self, segs) -> np.ndarray:
        a = self._segs(segs)
        v = int(self.lib.oracle_euclid_count(self._ptr(a), a.shape[0], None))
        out = np.zeros(v, dtype=np.uint32)
        assert self.lib.oracle_euclid_list32(self._ptr(a), a.shape[0], self._ptr(out), v) == v
        return out

    def euclid_list64(self, segs) -> np.ndarray:
        a = self._segs(segs)
        v = int(self.lib.oracle_euclid_count(self._ptr(a), a.shape[0], None))
        out = np.zeros(v, dtype=np.uint64)
        assert self.lib.oracle_euclid_list64(self._ptr(a), a.shape[0], self._ptr(out), v) == v
        return out

    def euclid_bitmask(self, segs, dims, mask: np.ndarray | None = None) -> np.ndarray:
        a = self._segs(segs)
        d = np.ascontiguousarray(dims, dtype=np.int32)
        if mask is None:
            mask = np.zeros(self.mask_words(dims), dtype=np.uint32)
        got = self.lib.oracle_euclid_bitmask(self._ptr(a), a.shape[0], self._ptr(d), self._ptr(mask), mask.shape[0])
        assert got >= 0, "a voxel fell outside the volume"
        return mask


_default = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default
