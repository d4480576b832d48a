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
