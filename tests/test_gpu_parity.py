"""CUDA path against the oracle, element by element, through the C ABI.

Bit-exact for every output (lists, volume words, counts, offsets): the method is
integer-only, so the tolerance is zero. Sizes span several scan tiles (2048
segments), several generation windows (256 segments) and ragged tails; the
full-size workloads run in the launch configuration that bench.py times.
"""

import numpy as np
import pytest
import torch

from gpu_util import (assert_list_equal, brick_pieces_expected, bricked_from_row_major, check_mask_sparse,
                      get_oracle, oracle_list, run_gpu, sparse_mask_from_list64)
from paper_2009_09500_gb300 import vox, workloads

pytestmark = pytest.mark.gpu

L32, L64, BM, FR = vox.OUT_LIST32, vox.OUT_LIST64, vox.OUT_BITMASK, vox.OUT_FRESH


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2009_09500_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build_library()
    vox.load()


def full_check(segs, dims, flags, **kw):
    O = get_oracle()
    r = run_gpu(segs, dims, flags, **kw)
    assert r["count_status"] == 0 and r["status"] == 0, (r["count_status"], r["status"])
    counts = O.count(segs)
    off = O.offsets(counts)
    assert np.array_equal(r["counts"], counts)
    assert np.array_equal(r["offsets"], off)
    assert r["V"] == off[-1]
    if flags & (L32 | L64):
        assert_list_equal(r["list_full"], oracle_list(O, segs, flags), r["V"])
    if flags & BM:
        fresh = (flags & FR) or kw.get("mask_init") is None
        want = O.bitmask(segs, dims, None if fresh else kw["mask_init"].copy())
        assert np.array_equal(r["mask"], want), f"{int((r['mask'] != want).sum())} volume words differ"
    return r


# ------------------------------------------------------------ paper-shaped workloads
def test_config1_list32_and_mask():
    w = workloads.config1()
    full_check(w.segs, w.dims, L32 | BM)


def test_config1_each_output_alone():
    w = workloads.config1()
    for flags in (L32, L64, BM, L64 | BM):
        full_check(w.segs, w.dims, flags)


def test_config2_full_size_list32_and_mask():
    """1M fixed 64-voxel segments + one 1023-step segment, 1024^3 volume: the
    benchmarked workload, whole outputs compared."""
    w = workloads.config2()
    full_check(w.segs, w.dims, L32 | BM)


def test_config2_single_long_segment():
    w = workloads.single_long_segment()
    full_check(w.segs, w.dims, L32 | BM)
    full_check(w.segs, w.dims, L64)


def test_config3_prefix_list64_and_sparse_mask():
    """Log-uniform lengths in a 4096^3 volume (8 GiB of bits, beyond 2^32):
    whole list and every nonzero volume word compared."""
    w = workloads.config3(n=60000)
    O = get_oracle()
    segs = torch.from_numpy(w.segs).cuda()
    n = segs.shape[0]
    ws = torch.empty(vox.vox_workspace_size(n), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    want = O.list64(w.segs)
    V = len(want)
    lst = torch.empty(V, dtype=torch.int64, device="cuda")
    mask = torch.zeros(vox.vox_mask_words(w.dims), dtype=torch.int32, device="cuda")
    vox.vox_generate(segs, w.dims, ws, status, lst, mask)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(lst.cpu().numpy().view(np.uint64), want)
    words, bits = sparse_mask_from_list64(want, w.dims)
    check_mask_sparse(mask, words, bits)


# --------------------------------------------------------------------- edge cases
def test_empty_input():
    r = run_gpu(np.zeros((0, 6), np.int32), (8, 8, 8), L32 | BM)
    assert r["status"] == 0 and r["V"] == 0
    assert (r["mask"] == 0).all()


def test_degenerate_segments_back_to_back():
    """5000 one-voxel segments: more segments than a staged window holds."""
    rng = np.random.default_rng(1)
    p = rng.integers(0, 32, size=(5000, 3)).astype(np.int32)
    segs = np.concatenate([p, p], axis=1)
    full_check(segs, (32, 32, 32), L32 | BM)
    full_check(segs, (32, 32, 32), L64)


@pytest.mark.parametrize("n", [1, 2, 3, 1023, 1024, 1025, 2047, 2048, 2049, 4097, 6143, 10001])
def test_ragged_sizes(n):
    rng = np.random.default_rng(n)
    segs = workloads.uniform_segments(rng, n, (64, 48, 40))
    full_check(segs, (64, 48, 40), L32 | BM)


def test_mixed_lengths_and_windows():
    """Short and long segments interleaved so that windows end mid-run and runs
    cross many segment boundaries."""
    rng = np.random.default_rng(5)
    parts = []
    for _ in range(40):
        k = int(rng.integers(1, 3000))
        L = int(rng.choice([0, 1, 2, 3, 7, 64, 500, 1023]))
        parts.append(workloads._segments_from_major(rng, np.full(k, L, np.int64), 1024))
    segs = np.ascontiguousarray(np.concatenate(parts))
    full_check(segs, (1024, 1024, 1024), L32 | BM)


def test_ties_and_directions():
    segs = []
    for N in (2, 4, 6, 10, 64, 1000):
        m = N // 2
        for sx in (1, -1):
            for sy in (1, -1):
                for sz in (1, -1):
                    S = np.array([N if sx < 0 else 0, m if sy < 0 else 0, m if sz < 0 else 0])
                    E = S + np.array([sx * N, sy * m, sz * m])
                    segs.append(np.concatenate([S, E]))
                    segs.append(np.concatenate([E, S]))
                    segs.append(np.concatenate([S[[1, 0, 2]], E[[1, 0, 2]]]))
                    segs.append(np.concatenate([S[[2, 1, 0]], E[[2, 1, 0]]]))
    full_check(np.array(segs, dtype=np.int32), (1024, 1024, 1024), L32 | BM)


def test_long_segments_wide_division():
    """N above 46340: entry numerators 2kA + N above 2^32 when a run enters mid-segment."""
    rng = np.random.default_rng(8)
    edge = 1 << 21
    dims = (edge, 16, 8)
    segs = []
    for _ in range(6):
        x0, x1 = (0, edge - 1) if rng.random() < 0.5 else (edge - 1, 0)
        segs.append([x0, int(rng.integers(0, 16)), int(rng.integers(0, 8)), x1, int(rng.integers(0, 16)),
                     int(rng.integers(0, 8))])
    segs.append([5, 0, 0, 5 + 70001, 15, 7])
    segs = np.array(segs, dtype=np.int32)
    full_check(segs, dims, L64 | BM)


def test_longest_near_diagonal_segments():
    """N = 2^21 - 1 (the longest segment the packing allows) with minor |d| near N,
    near N/2 and small: minor axes carry on almost every step and the biased
    remainders reach the top of the 32-bit range; runs enter deep inside."""
    M = (1 << 21) - 1
    edge = 1 << 21
    segs = np.array([
        [0, 0, 0, M, M - 1, M - 2],
        [M, 0, M, 0, M - 1, 1],
        [0, M, 0, M, M // 2, M // 2 + 1],
        [5, 7, M, M, 8, 3],
    ], dtype=np.int32)
    full_check(segs, (edge, edge, edge), L64)


def test_volume_not_word_aligned():
    rng = np.random.default_rng(6)
    dims = (13, 7, 5)
    segs = workloads.uniform_segments(rng, 3000, dims)
    full_check(segs, dims, L32 | BM)


def test_mask_is_ored_into():
    rng = np.random.default_rng(7)
    dims = (64, 64, 64)
    segs = workloads.uniform_segments(rng, 500, dims)
    init = rng.integers(0, 2**32, size=vox.vox_mask_words(dims), dtype=np.uint64).astype(np.uint32)
    init[::3] = 0
    full_check(segs, dims, BM, mask_init=init)


def test_from_scan_matches():
    w = workloads.config1()
    full_check(w.segs, w.dims, L32 | BM, use_from_scan=True)


def test_capacity_exact_and_too_small():
    w = workloads.config1()
    O = get_oracle()
    V = O.total(w.segs)
    full_check(w.segs, w.dims, L32, capacity=V)
    r = run_gpu(w.segs, w.dims, L32 | BM, capacity=V - 1)
    assert r["status"] == vox.ERR_CAPACITY
    assert (r["list_full"] == -0x21524111).all(), "nothing may be written on a capacity error"
    assert (r["mask"] == 0).all()


def test_out_of_bounds_endpoint_writes_nothing():
    w = workloads.config1()
    segs = w.segs.copy()
    segs[1234, 4] = 256  # y1 outside [0, 256)
    r = run_gpu(segs, w.dims, L32 | BM)
    assert r["count_status"] == vox.ERR_OUT_OF_BOUNDS and r["status"] == vox.ERR_OUT_OF_BOUNDS
    assert (r["list_full"] == -0x21524111).all()
    assert (r["mask"] == 0).all()
    segs = w.segs.copy()
    segs[7, 0] = -1
    r = run_gpu(segs, w.dims, L32)
    assert r["status"] == vox.ERR_OUT_OF_BOUNDS


def test_host_side_errors_launch_nothing():
    segs = torch.zeros((4, 6), dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size(4), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lst = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(vox.VoxError) as e:
        vox.vox_generate(segs, (2048, 8, 8), ws, st, lst)
    assert e.value.status == vox.ERR_PACK_WIDTH
    with pytest.raises(vox.VoxError) as e:
        vox.vox_generate(segs, (0, 8, 8), ws, st, lst)
    assert e.value.status == vox.ERR_INVALID_ARG
    with pytest.raises(vox.VoxError) as e:
        vox.vox_generate(segs, (8, 8, 8), ws[:64], st, lst)
    assert e.value.status == vox.ERR_WORKSPACE
    big = torch.zeros((5, 6), dtype=torch.int32, device="cuda")
    with pytest.raises(vox.VoxError) as e:
        vox.vox_generate(big[1:], (8, 8, 8), ws, st, lst)  # 24-byte offset: not 16-byte aligned
    assert e.value.status == vox.ERR_ALIGNMENT


def test_scan_wait_is_bounded():
    """Fault injection on the host side of the GPU: one scan tile withholds its
    prefix; the look-back of the next tile gives up after 50 ms and reports
    VOX_ERR_TIMEOUT; the context stays usable and the next call is correct."""
    rng = np.random.default_rng(9)
    dims = (64, 64, 64)
    segs = workloads.uniform_segments(rng, 3 * vox.vox_scan_tile_segments() + 17, dims)
    try:
        vox.vox_debug_set_scan_stall(1, 50_000_000)
        r = run_gpu(segs, dims, L32 | BM)
        assert r["count_status"] == vox.ERR_TIMEOUT
        assert r["status"] == vox.ERR_TIMEOUT
        assert (r["mask"] == 0).all()
    finally:
        vox.vox_debug_set_scan_stall(-1, 0)
    full_check(segs, dims, L32 | BM)


def test_generate_host_matches():
    w = workloads.config1()
    O = get_oracle()
    V = O.total(w.segs)
    h_segs = torch.from_numpy(w.segs).pin_memory()
    h_list = torch.empty(V, dtype=torch.int32).pin_memory()
    h_mask = torch.full((vox.vox_mask_words(w.dims),), 7, dtype=torch.int32).pin_memory()
    flags = L32 | BM
    arena = torch.empty(vox.vox_host_arena_size(w.n, w.dims, flags, V), dtype=torch.uint8, device="cuda")
    got_V = vox.vox_generate_host(h_segs, w.dims, arena, h_list, h_mask)
    assert got_V == V
    assert np.array_equal(h_list.numpy().view(np.uint32), O.list32(w.segs))
    assert np.array_equal(h_mask.numpy().view(np.uint32), O.bitmask(w.segs, w.dims))


def brick_piece_count(segs, dims):
    """Pieces of the brick volume, from vox_plan on the device (sizing only)."""
    d = torch.from_numpy(np.ascontiguousarray(segs)).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size_volume(len(segs), dims, 0), dtype=torch.uint8, device="cuda")
    return vox.vox_plan(d, dims, ws, st)[1]


@pytest.mark.parametrize("which,flags,pieces", [
    ("config1", L32 | BM, "plan"), ("config1", BM, "plan"), ("config1", L64 | BM, "plan"),
    ("config1", L32 | BM, 50),       # too few pieces: atomics on the device, same result
    ("config2", L32 | BM, "plan"),   # the benchmarked e2e call
])
def test_generate_host_volume_arena_matches(which, flags, pieces):
    """The host-buffer call with a brick-sized arena: brick-built volume, list copy
    overlapped on a second stream; host outputs against the oracle, whole, over
    stale host buffers."""
    w = getattr(workloads, which)()
    O = get_oracle()
    V = O.total(w.segs)
    P = brick_piece_count(w.segs, w.dims) if pieces == "plan" else pieces
    h_segs = torch.from_numpy(w.segs).pin_memory()
    h_list = None
    if flags & (L32 | L64):
        h_list = torch.full((V,), -1, dtype=torch.int64 if flags & L64 else torch.int32).pin_memory()
    h_mask = torch.full((vox.vox_mask_words(w.dims),), -1, dtype=torch.int32).pin_memory()
    arena = torch.empty(vox.vox_host_arena_size_volume(w.n, w.dims, flags, V, P), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        assert vox.vox_generate_host(h_segs, w.dims, arena, h_list, h_mask, flags) == V
        if h_list is not None:
            want = O.list64(w.segs) if flags & L64 else O.list32(w.segs)
            assert np.array_equal(h_list.numpy().view(want.dtype), want)
        assert np.array_equal(h_mask.numpy().view(np.uint32), O.bitmask(w.segs, w.dims))
        h_mask.fill_(-1)


def test_repeated_calls_are_stable():
    w = workloads.config2(n_fixed=30000)
    r1 = run_gpu(w.segs, w.dims, L32 | BM)
    r2 = run_gpu(w.segs, w.dims, L32 | BM)
    assert np.array_equal(r1["list_full"], r2["list_full"])
    assert np.array_equal(r1["mask"], r2["mask"])


# ------------------------------------------------------- volume by brick ownership
@pytest.mark.parametrize("flags", [BM, L32 | BM, L64 | BM])
def test_bricks_config1(flags):
    w = workloads.config1()
    r = full_check(w.segs, w.dims, flags, pieces="plan")
    V, P = r["planned"]
    assert V == r["V"] and P == brick_pieces_expected(get_oracle(), w.segs, w.dims)


def test_bricks_config2_full_size():
    """The benchmarked workload with the brick-built volume, whole outputs compared."""
    w = workloads.config2()
    r = full_check(w.segs, w.dims, L32 | BM, pieces="plan")
    assert r["planned"][1] > w.n


@pytest.mark.parametrize("dims", [(64, 64, 64), (96, 40, 17), (32, 7, 5), (128, 128, 64), (256, 8, 300)])
def test_bricks_volume_shapes(dims):
    rng = np.random.default_rng(sum(dims))
    segs = workloads.uniform_segments(rng, 3000, dims)
    r = full_check(segs, dims, BM, pieces="plan")
    assert r["planned"][1] == brick_pieces_expected(get_oracle(), segs, dims)


def test_bricks_fallback_when_pieces_do_not_fit():
    """Too small a piece capacity: the call falls back to atomics on the device,
    same bits."""
    w = workloads.config1()
    full_check(w.segs, w.dims, L32 | BM, pieces=100)


def test_bricks_width_not_multiple_of_32_uses_atomics():
    rng = np.random.default_rng(15)
    dims = (13, 7, 5)
    segs = workloads.uniform_segments(rng, 2000, dims)
    r = full_check(segs, dims, BM, pieces="plan")
    assert r["planned"][1] == 0


def test_bricks_or_into_and_degenerate():
    rng = np.random.default_rng(16)
    dims = (64, 64, 64)
    p0 = rng.integers(0, 64, size=(3000, 3)).astype(np.int32)
    segs = np.concatenate([np.concatenate([p0, p0], axis=1), workloads.uniform_segments(rng, 500, dims)])
    init = rng.integers(0, 2**32, size=vox.vox_mask_words(dims), dtype=np.uint64).astype(np.uint32)
    init[::2] = 0
    full_check(segs, dims, BM, pieces="plan", mask_init=init)


def test_bricks_config3_prefix_sparse():
    w = workloads.config3(n=60000)
    O = get_oracle()
    segs = torch.from_numpy(w.segs).cuda()
    n = w.n
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size_volume(n, w.dims, 0), dtype=torch.uint8, device="cuda")
    V, P = vox.vox_plan(segs, w.dims, ws, status)
    ws = torch.empty(vox.vox_workspace_size_volume(n, w.dims, P), dtype=torch.uint8, device="cuda")
    mask = torch.zeros(vox.vox_mask_words(w.dims), dtype=torch.int32, device="cuda")
    vox.vox_generate(segs, w.dims, ws, status, None, mask)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    words, bits = sparse_mask_from_list64(O.list64(w.segs), w.dims)
    check_mask_sparse(mask, words, bits)


def test_bricks_generation_repeated_after_one_count():
    """vox_count once, then the volume pass twice (fresh volumes): both exact.
    The brick pass resets its own tickets, so it can run again on the counts."""
    w = workloads.config1()
    O = get_oracle()
    segs = torch.from_numpy(w.segs).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size_volume(w.n, w.dims, 0), dtype=torch.uint8, device="cuda")
    V, P = vox.vox_plan(segs, w.dims, ws, status)
    ws = torch.empty(vox.vox_workspace_size_volume(w.n, w.dims, P), dtype=torch.uint8, device="cuda")
    vox.vox_count(segs, w.dims, ws, status)
    want = O.bitmask(w.segs, w.dims)
    for _ in range(2):
        mask = torch.zeros(vox.vox_mask_words(w.dims), dtype=torch.int32, device="cuda")
        vox.vox_generate_from_scan(segs, w.dims, ws, status, None, mask, BM)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert np.array_equal(mask.cpu().numpy().view(np.uint32), want)


# ------------------------------------------- fresh volumes (VOX_OUT_FRESH): overwritten
def garbage_mask(rng, dims):
    return rng.integers(0, 2**32, size=vox.vox_mask_words(dims), dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("dims,pieces", [
    ((256, 256, 256), "plan"),   # bricks, TMA tensor store
    ((128, 128, 64), "plan"),    # bricks, TMA, B0 = 128
    ((96, 40, 17), "plan"),      # bricks, plain-store merge (B0 = 64), edge bricks
    ((32, 7, 5), "plan"),        # one ragged brick
    ((13, 7, 5), "plan"),        # w % 32 != 0: cleared, then atomics
    ((64, 64, 64), None),        # plain workspace: cleared, then atomics
    ((256, 256, 256), 100),      # pieces do not fit: bricks cleared, gated atomics
])
def test_fresh_volume_overwrites(dims, pieces):
    rng = np.random.default_rng(sum(dims) + (7 if pieces is None else 0))
    segs = workloads.uniform_segments(rng, 3000, dims)
    full_check(segs, dims, BM | FR, pieces=pieces, mask_init=garbage_mask(rng, dims))
    full_check(segs, dims, L32 | BM | FR, pieces=pieces, mask_init=garbage_mask(rng, dims), use_from_scan=True)


def test_fresh_volume_with_no_segments_is_cleared():
    dims = (64, 32, 16)
    rng = np.random.default_rng(71)
    r = run_gpu(np.zeros((0, 6), np.int32), dims, BM | FR, mask_init=garbage_mask(rng, dims))
    assert r["status"] == 0 and (r["mask"] == 0).all()


def test_fresh_volume_atomic_tuning():
    rng = np.random.default_rng(72)
    dims = (256, 128, 64)
    segs = workloads.uniform_segments(rng, 4000, dims)
    vox.vox_set_tuning(0, vox.VOLUME_ATOMIC, 0)
    try:
        full_check(segs, dims, L32 | BM | FR, pieces="plan", mask_init=garbage_mask(rng, dims))
    finally:
        vox.vox_set_tuning(0, 0, 0)


def test_fresh_config2_full_size():
    """The benchmarked call: list32 and a fresh brick-built volume over a volume
    full of stale bits, whole outputs compared."""
    w = workloads.config2()
    rng = np.random.default_rng(73)
    full_check(w.segs, w.dims, L32 | BM | FR, pieces="plan", mask_init=garbage_mask(rng, w.dims),
               use_from_scan=True)


def test_fresh_device_error_leaves_volume_unchanged_or_cleared():
    w = workloads.config1()
    segs = w.segs.copy()
    segs[99, 2] = 300  # z0 outside [0, 256)
    rng = np.random.default_rng(74)
    init = garbage_mask(rng, w.dims)
    r = run_gpu(segs, w.dims, BM | FR, mask_init=init)
    assert r["status"] == vox.ERR_OUT_OF_BOUNDS
    assert (r["mask"] == init).all() or (r["mask"] == 0).all()


def test_fresh_without_bitmask_is_rejected():
    segs = torch.zeros((4, 6), dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size(4), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lst = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(vox.VoxError) as e:
        vox.vox_generate(segs, (8, 8, 8), ws, st, lst, flags=L32 | FR)
    assert e.value.status == vox.ERR_INVALID_ARG


# --------------------------------------------- brick-major volumes (VOX_OUT_BRICKED)
BR = vox.OUT_BRICKED


@pytest.mark.parametrize("dims,flags", [
    ((256, 256, 256), BM | BR),
    ((256, 256, 256), L32 | BM | BR),
    ((96, 40, 17), BM | BR),       # one padded brick of 64 x 128 x 128
    ((32, 7, 5), BM | BR),
    ((128, 128, 64), L64 | BM | BR),
])
def test_bricked_volume_matches_layout(dims, flags):
    """Brick-major volume against the oracle's volume rearranged by the
    documented layout, over a buffer of stale bits; vox_unbrick back to the
    oracle's row-major volume."""
    rng = np.random.default_rng(sum(dims) + flags)
    segs = workloads.uniform_segments(rng, 3000, dims)
    O = get_oracle()
    words = vox.vox_mask_words_bricked(dims)
    init = rng.integers(0, 2**32, size=words, dtype=np.uint64).astype(np.uint32)
    r = run_gpu(segs, dims, flags, pieces="plan", mask_words=words, mask_init=init)
    assert r["status"] == 0
    want_rm = O.bitmask(segs, dims)
    assert np.array_equal(r["mask"], bricked_from_row_major(want_rm, dims))
    if flags & (L32 | L64):
        assert_list_equal(r["list_full"], oracle_list(O, segs, flags), r["V"])
    bricked = torch.from_numpy(r["mask"].view(np.int32).copy()).cuda()
    row = torch.full((vox.vox_mask_words(dims),), -1, dtype=torch.int32, device="cuda")
    vox.vox_unbrick(bricked, dims, row)
    torch.cuda.synchronize()
    assert np.array_equal(row.cpu().numpy().view(np.uint32), want_rm)


def test_bricked_config2_full_size():
    w = workloads.config2()
    O = get_oracle()
    words = vox.vox_mask_words_bricked(w.dims)
    assert words == vox.vox_mask_words(w.dims)  # 1024^3: bricks tile the volume exactly
    r = run_gpu(w.segs, w.dims, L32 | BM | BR, pieces="plan", mask_words=words, use_from_scan=True)
    assert r["status"] == 0
    assert np.array_equal(r["mask"], bricked_from_row_major(O.bitmask(w.segs, w.dims), w.dims))


def test_bricked_errors_and_empty():
    rng = np.random.default_rng(81)
    dims = (256, 64, 64)
    segs = workloads.uniform_segments(rng, 500, dims)
    words = vox.vox_mask_words_bricked(dims)
    # plain workspace (no brick arrays): refused on the host, nothing launched
    with pytest.raises(vox.VoxError) as e:
        run_gpu(segs, dims, BM | BR, mask_words=words)
    assert e.value.status == vox.ERR_WORKSPACE
    # pieces beyond the workspace's capacity: reported on the device
    r = run_gpu(segs, dims, BM | BR, pieces=10, mask_words=words)
    assert r["status"] == vox.ERR_WORKSPACE
    # the layout needs w % 32 == 0; bricked needs the volume flag
    assert vox.vox_mask_words_bricked((13, 7, 5)) == 0
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    d = torch.from_numpy(segs).cuda()
    ws = torch.empty(vox.vox_workspace_size_volume(500, dims, 4000), dtype=torch.uint8, device="cuda")
    lst = torch.empty(100000, dtype=torch.int32, device="cuda")
    with pytest.raises(vox.VoxError) as e:
        vox.vox_generate(d, dims, ws, st, lst, None, flags=L32 | BR)
    assert e.value.status == vox.ERR_INVALID_ARG
    # no segments: the whole brick-major buffer is cleared
    r = run_gpu(np.zeros((0, 6), np.int32), dims, BM | BR, mask_words=words,
                mask_init=np.full(words, 0xFFFFFFFF, np.uint32), pieces=1)
    assert r["status"] == 0 and (r["mask"] == 0).all()


# ------------------------------------- per-voxel atomics merged across the warp
@pytest.mark.parametrize("dims,n,mode", [
    ((256, 256, 256), 4096, "zero"),   # the 4096-segment workload's shape
    ((13, 7, 5), 3000, "zero"),        # rows not word aligned, words shared by many lanes
    ((64, 64, 64), 20000, "or"),       # dense: lanes often hold equal words; OR into stale bits
    ((1024, 16, 8), 500, "zero"),      # long flat segments: runs that cross segment ends
])
def test_warp_merged_atomics(dims, n, mode):
    """The volume alone by per-voxel atomics merged across the warp
    (VOX_VOLUME_ATOMIC_WARP), against the oracle, for every run length."""
    rng = np.random.default_rng(sum(dims) + n)
    segs = workloads.uniform_segments(rng, n, dims)
    init = None
    if mode == "or":
        init = rng.integers(0, 2**32, size=vox.vox_mask_words(dims), dtype=np.uint64).astype(np.uint32)
        init[::2] = 0
    try:
        for r in (16, 32, 64):
            vox.vox_set_tuning(r, vox.VOLUME_ATOMIC_WARP, 0)
            full_check(segs, dims, BM, pieces="plan", mask_init=None if init is None else init.copy())
            full_check(segs, dims, BM | FR, pieces="plan", mask_init=garbage_mask(rng, dims))
    finally:
        vox.vox_reset_tuning()


def test_warp_merged_atomics_config3_prefix():
    """64-bit bit indices (4096^3 volume), long segments: the sparse volume."""
    w = workloads.config3(n=60000)
    O = get_oracle()
    segs = torch.from_numpy(w.segs).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size(w.n), dtype=torch.uint8, device="cuda")
    mask = torch.zeros(vox.vox_mask_words(w.dims), dtype=torch.int32, device="cuda")
    try:
        vox.vox_set_tuning(32, vox.VOLUME_ATOMIC_WARP, 0)
        vox.vox_generate(segs, w.dims, ws, status, None, mask)
        torch.cuda.synchronize()
    finally:
        vox.vox_reset_tuning()
    assert int(status.item()) == 0
    words, bits = sparse_mask_from_list64(O.list64(w.segs), w.dims)
    check_mask_sparse(mask, words, bits)
    del mask
    torch.cuda.empty_cache()
