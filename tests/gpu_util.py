"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare with the oracle. Oracle outputs are computed here on the CPU from the
same input bytes; nothing the CUDA path produces feeds the oracle."""

from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2009_09500_gb300 import vox

SENTINEL32 = -0x21524111  # 0xDEADBEEF as int32
SENTINEL64 = -0x2152411021524111


def run_gpu(segs_np, dims, flags, capacity=None, extra=64, mask_init=None, use_from_scan=False, pieces=None,
            mask_words=None):
    """vox_count then vox_generate (or vox_generate_from_scan) on cuda:0.
    The list gets ``extra`` sentinel elements past the capacity the call is told
    about, to catch writes beyond it. ``pieces``: None for the plain workspace
    (per-voxel atomic volume), "plan" to size the brick workspace with vox_plan,
    or an explicit piece capacity."""
    segs = torch.from_numpy(np.ascontiguousarray(segs_np, dtype=np.int32)).cuda()
    n = segs.shape[0]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    planned = None
    if pieces is None:
        ws = torch.empty(vox.vox_workspace_size(n), dtype=torch.uint8, device="cuda")
    else:
        ws = torch.empty(vox.vox_workspace_size_volume(n, dims, 0), dtype=torch.uint8, device="cuda")
        if n:
            planned = vox.vox_plan(segs, dims, ws, status)
        cap = planned[1] if pieces == "plan" else int(pieces)
        ws = torch.empty(vox.vox_workspace_size_volume(n, dims, cap), dtype=torch.uint8, device="cuda")
    counts = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    offsets = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    vox.vox_count(segs, dims, ws, status, counts[:n] if n else None, offsets)
    torch.cuda.synchronize()
    count_status = int(status.item())
    V = int(offsets[-1].item())
    if capacity is None:
        capacity = V
    res = {"count_status": count_status, "V": V, "counts": counts[:n].cpu().numpy(),
           "offsets": offsets.cpu().numpy(), "capacity": capacity, "planned": planned}
    list_t = None
    if flags & vox.OUT_LIST64:
        list_t = torch.full((capacity + extra,), SENTINEL64, dtype=torch.int64, device="cuda")
    elif flags & vox.OUT_LIST32:
        list_t = torch.full((capacity + extra,), SENTINEL32, dtype=torch.int32, device="cuda")
    mask_t = None
    if flags & vox.OUT_BITMASK:
        words = vox.vox_mask_words(dims) if mask_words is None else mask_words
        if mask_init is None:
            mask_t = torch.zeros(words, dtype=torch.int32, device="cuda")
        else:
            mask_t = torch.from_numpy(mask_init.view(np.int32).copy()).cuda()
    fn = vox.vox_generate_from_scan if use_from_scan else vox.vox_generate
    fn(segs, dims, ws, status, list_t, mask_t, flags=flags, capacity=capacity)
    torch.cuda.synchronize()
    res["status"] = int(status.item())
    if list_t is not None:
        res["list_full"] = list_t.cpu().numpy()
    if mask_t is not None:
        res["mask"] = mask_t.cpu().numpy().view(np.uint32)
    return res


def oracle_list(O, segs, flags):
    return O.list64(segs) if flags & vox.OUT_LIST64 else O.list32(segs)


def assert_list_equal(got_full, want, V, extra=64):
    got = got_full[:V]
    if got.dtype == np.int32:
        got = got.view(np.uint32)
    elif got.dtype == np.int64:
        got = got.view(np.uint64)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{len(bad)} list mismatches, first at {bad[:8]}: got {got[bad[:8]]}, want {want[bad[:8]]}")
    tail = got_full[V:]
    sentinel = SENTINEL64 if got_full.dtype == np.int64 else SENTINEL32
    assert (tail == sentinel).all(), "write past the end of the list"


def sparse_mask_from_list64(l64: np.ndarray, dims):
    """Nonzero words of the volume holding the voxels of an oracle 64-bit list:
    (sorted word indices, OR of their bits)."""
    w, h, _ = (int(v) for v in dims)
    m = np.uint64((1 << 21) - 1)
    x = (l64 & m).astype(np.int64)
    y = ((l64 >> np.uint64(21)) & m).astype(np.int64)
    z = ((l64 >> np.uint64(42)) & m).astype(np.int64)
    lin = x + w * (y + h * z)
    word = lin >> 5
    bit = (np.int64(1) << (lin & 31)).astype(np.uint32)
    order = np.argsort(word, kind="stable")
    word, bit = word[order], bit[order]
    starts = np.flatnonzero(np.concatenate([[True], word[1:] != word[:-1]]))
    return word[starts], np.bitwise_or.reduceat(bit, starts)


def check_mask_sparse(mask_t: torch.Tensor, words: np.ndarray, bits: np.ndarray):
    """The device volume has exactly these nonzero words with these bits."""
    idx = torch.from_numpy(words).cuda()
    got = mask_t[idx].cpu().numpy().view(np.uint32)
    assert np.array_equal(got, bits), f"{int((got != bits).sum())} volume words differ"
    nnz = int(torch.count_nonzero(mask_t).item())
    assert nnz == len(words), f"{nnz} nonzero words on the device, {len(words)} expected"


def get_oracle():
    return oracle.get()


def brick_pieces_expected(O, segs, dims, max_len=64):
    """Number of brick pieces from the oracle's voxels and the documented brick
    shape: every maximal run of a segment's voxels inside one brick, cut into
    parts of at most max_len voxels. Brick shape: B0 = the largest 32 * 2^k not
    above min(w, 256), then the largest power-of-two rows B1 x B2 (B1 = 2 B2 or
    B2) with B0/32 * B1 * B2 <= 32768 words."""
    w = int(dims[0])
    b0 = 32
    while 2 * b0 <= min(w, 256):
        b0 *= 2
    rows = 32768 // (b0 // 32)
    p2 = 1
    while (2 * p2) ** 2 <= rows:
        p2 *= 2
    b1 = 2 * p2 if 2 * p2 * p2 <= rows else p2
    B = np.array([b0, b1, p2])
    xyz = O.voxels_xyz(segs)
    counts = O.count(segs).astype(np.int64)
    starts = np.zeros(len(xyz), dtype=bool)
    starts[np.concatenate([[0], np.cumsum(counts)[:-1]])] = True
    bc = xyz // B
    first = starts.copy()
    first[1:] |= np.any(bc[1:] != bc[:-1], axis=1)
    runs = np.diff(np.concatenate([np.flatnonzero(first), [len(xyz)]]))
    return int(((runs + max_len - 1) // max_len).sum())


def bricked_from_row_major(mask_u32: np.ndarray, dims) -> np.ndarray:
    """The brick-major layout of a row-major volume, rearranged with numpy from
    the layout documented for VOX_OUT_BRICKED (brick (bx, by, bz) at index
    bx + nb0 (by + nb1 bz), x fastest inside a brick, edge bricks zero-padded)."""
    (b0, b1, b2), (n0, n1, n2) = vox.vox_brick_shape(dims)
    w, h, d = (int(v) for v in dims)
    bits = np.unpackbits(mask_u32.view(np.uint8), bitorder="little")[: w * h * d].reshape(d, h, w)
    pad = np.zeros((n2 * b2, n1 * b1, n0 * b0), dtype=np.uint8)
    pad[:d, :h, :w] = bits
    bricks = pad.reshape(n2, b2, n1, b1, n0, b0).transpose(0, 2, 4, 1, 3, 5)
    return np.packbits(np.ascontiguousarray(bricks).reshape(-1), bitorder="little").view(np.uint32)
