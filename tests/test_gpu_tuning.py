"""Every launch tuning gives the same bits (GPU), and the tuner picks one."""

import numpy as np
import pytest
import torch

from gpu_util import get_oracle
from paper_2009_09500_gb300 import autotune, vox, workloads

pytestmark = pytest.mark.gpu


def test_all_candidates_bit_exact_and_tuner(tmp_path):
    from paper_2009_09500_gb300 import build

    build.build_library()
    w = workloads.config2(n_fixed=40000)
    O = get_oracle()
    want_list = O.list32(w.segs)
    want_mask = O.bitmask(w.segs, w.dims)
    segs = torch.from_numpy(w.segs).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size_volume(w.n, w.dims, 0), dtype=torch.uint8, device="cuda")
    V, P = vox.vox_plan(segs, w.dims, ws, st)
    ws = torch.empty(vox.vox_workspace_size_volume(w.n, w.dims, P), dtype=torch.uint8, device="cuda")
    lst = torch.empty(V, dtype=torch.int32, device="cuda")
    mask = torch.zeros(vox.vox_mask_words(w.dims), dtype=torch.int32, device="cuda")
    try:
        for c in autotune.CANDIDATES:
            autotune.apply(c)
            lst.zero_()
            mask.zero_()
            vox.vox_generate(segs, w.dims, ws, st, lst, mask)
            torch.cuda.synchronize()
            assert int(st.item()) == 0
            assert np.array_equal(lst.cpu().numpy().view(np.uint32), want_list), c
            assert np.array_equal(mask.cpu().numpy().view(np.uint32), want_mask), c
        run = lambda: vox.vox_generate(segs, w.dims, ws, st, lst, mask)
        res = autotune.get_or_tune(run, w.n, V, w.dims, vox.OUT_LIST32 | vox.OUT_BITMASK,
                                   cache_path=str(tmp_path / "c.json"), reps=2)
        assert res["params"] in autotune.CANDIDATES and not res["cached"]
        res2 = autotune.get_or_tune(run, w.n, V, w.dims, vox.OUT_LIST32 | vox.OUT_BITMASK,
                                    cache_path=str(tmp_path / "c.json"))
        assert res2["cached"] and res2["params"] == res["params"]
    finally:
        vox.vox_reset_tuning()


@pytest.mark.parametrize("run_len", [16, 32, 64])
def test_segment_cut_runs_bit_exact(run_len):
    """32-bit list with runs cut at segment ends (list_runs = 1): lengths 1..128,
    one-voxel segments, long segments that fill several passes of a window, and
    uniform random segments, interleaved; the whole list against the oracle."""
    from paper_2009_09500_gb300 import build

    build.build_library()
    rng = np.random.default_rng(12)
    parts = [
        workloads._segments_from_major(rng, rng.integers(0, 128, 20000), 1024),
        workloads._segments_from_major(rng, np.zeros(3000, np.int64), 1024),
        workloads._segments_from_major(rng, rng.integers(900, 1024, 40), 1024),
        workloads.config1().segs,
    ]
    segs_np = np.concatenate(parts)
    segs_np = segs_np[rng.permutation(segs_np.shape[0])]
    dims = (1024, 1024, 1024)
    O = get_oracle()
    want = O.list32(segs_np)
    segs = torch.from_numpy(np.ascontiguousarray(segs_np)).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size(segs.shape[0]), dtype=torch.uint8, device="cuda")
    lst = torch.full((len(want) + 64,), -1, dtype=torch.int32, device="cuda")
    try:
        for list_runs in (1, 0):
            vox.vox_set_tuning(run_len, 0, 0, list_runs)
            lst.fill_(-1)
            vox.vox_generate(segs, dims, ws, st, lst, None, vox.OUT_LIST32, capacity=len(want))
            torch.cuda.synchronize()
            assert int(st.item()) == 0
            got = lst.cpu().numpy().view(np.uint32)
            assert np.array_equal(got[:len(want)], want), (run_len, list_runs)
            assert (got[len(want):] == np.uint32(0xffffffff)).all(), "written past the list"
    finally:
        vox.vox_reset_tuning()


@pytest.mark.parametrize("wide", [False, True])
def test_warp_slice_list_bit_exact(wide):
    """Lists alone by warp slices (list_runs = 2), 32- and 64-bit: lengths up to
    the volume edge, runs of one-voxel segments (slices spanning many windows of
    32 segments), long segments spanning many slices, a ragged list end; the
    whole list against the oracle, nothing written past it; a capacity error
    writes nothing."""
    from paper_2009_09500_gb300 import build

    build.build_library()
    rng = np.random.default_rng(14 + wide)
    edge = 4096 if wide else 1024
    parts = [
        workloads._segments_from_major(rng, rng.integers(0, edge, 6000), edge),
        workloads._segments_from_major(rng, np.zeros(5000, np.int64), edge),
        workloads._segments_from_major(rng, rng.integers(0, 40, 20000), edge),
        workloads._segments_from_major(rng, np.full(30, edge - 1, np.int64), edge),
    ]
    segs_np = np.concatenate(parts)
    segs_np = segs_np[rng.permutation(segs_np.shape[0])]
    dims = (edge, edge, edge)
    O = get_oracle()
    if O.total(segs_np) % 4 == 0:  # a ragged end: the last slice's tail by plain stores
        segs_np = np.concatenate([segs_np, segs_np[:1] * 0])
    want = O.list64(segs_np) if wide else O.list32(segs_np)
    V = len(want)
    assert V % 4 != 0
    segs = torch.from_numpy(np.ascontiguousarray(segs_np)).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size(segs.shape[0]), dtype=torch.uint8, device="cuda")
    dt = torch.int64 if wide else torch.int32
    lst = torch.full((V + 64,), -1, dtype=dt, device="cuda")
    flag = vox.OUT_LIST64 if wide else vox.OUT_LIST32
    try:
        vox.vox_set_tuning(32, 0, 0, 2)
        for _ in range(2):  # twice: the chunk counter is reset per launch
            lst.fill_(-1)
            vox.vox_generate(segs, dims, ws, st, lst, None, flag, capacity=V)
            torch.cuda.synchronize()
            assert int(st.item()) == 0
            got = lst.cpu().numpy().view(want.dtype)
            assert np.array_equal(got[:V], want)
            assert (got[V:] == np.array(-1, dtype=np.int64).astype(want.dtype)).all(), "written past the list"
        lst.fill_(-1)
        vox.vox_generate(segs, dims, ws, st, lst, None, flag, capacity=V - 1)
        torch.cuda.synchronize()
        assert int(st.item()) == vox.ERR_CAPACITY
        assert (lst.cpu().numpy() == -1).all(), "nothing may be written on a capacity error"
    finally:
        vox.vox_reset_tuning()


def _seg_along_x(x0, y, z, length):
    """A segment of `length` voxels along x."""
    return [x0, y, z, x0 + length - 1, y, z]


@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("case", ["one_short", "few_long_ragged", "whole_slices", "long_then_tiny"])
def test_warp_slice_list_few_segment_ends(case, wide):
    """Lists by warp slices where slices have few segment ends (the lanes walk in
    step, crossing segment ends in place): one 100-voxel segment (one slice, most
    lanes without voxels), a few long segments ending mid-slice, a list of whole
    slices exactly (5 x 1056 voxels), long segments followed by one-voxel ones (a
    slice's window ending inside it); the whole list against the oracle, nothing
    written past it."""
    from paper_2009_09500_gb300 import build

    build.build_library()
    edge = 4096 if wide else 1024
    rng = np.random.default_rng(41)
    if case == "one_short":
        segs_np = np.array([_seg_along_x(3, 5, 7, 100)], np.int32)
    elif case == "few_long_ragged":
        segs_np = workloads._segments_from_major(rng, np.array([edge - 1, 777, edge // 2 + 3, 1234 % edge]), edge)
    elif case == "whole_slices":
        segs_np = np.array([_seg_along_x(0, 1, 2, 1000), _seg_along_x(0, 3, 4, 1000), _seg_along_x(0, 5, 6, 1000),
                            _seg_along_x(0, 7, 8, 1000), _seg_along_x(0, 9, 10, 1000), _seg_along_x(0, 11, 12, 280)],
                           np.int32)
        assert int(np.abs(segs_np[:, 3] - segs_np[:, 0]).sum() + len(segs_np)) == 5 * 1056
    else:
        longs = workloads._segments_from_major(rng, np.full(40, edge - 1, np.int64), edge)
        tiny = workloads._segments_from_major(rng, np.zeros(3000, np.int64), edge)
        segs_np = np.concatenate([longs, tiny, longs[:3]])
    segs_np = np.ascontiguousarray(segs_np.astype(np.int32))
    dims = (edge, edge, edge)
    O = get_oracle()
    want = O.list64(segs_np) if wide else O.list32(segs_np)
    V = len(want)
    segs = torch.from_numpy(segs_np).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size(segs.shape[0]), dtype=torch.uint8, device="cuda")
    dt = torch.int64 if wide else torch.int32
    lst = torch.full((V + 64,), -1, dtype=dt, device="cuda")
    try:
        vox.vox_set_tuning(32, 0, 0, 2)
        vox.vox_generate(segs, dims, ws, st, lst, None, vox.OUT_LIST64 if wide else vox.OUT_LIST32, capacity=V)
        torch.cuda.synchronize()
    finally:
        vox.vox_reset_tuning()
    assert int(st.item()) == 0
    got = lst.cpu().numpy().view(want.dtype)
    assert np.array_equal(got[:V], want)
    assert (got[V:] == np.array(-1, dtype=np.int64).astype(want.dtype)).all(), "written past the list"
