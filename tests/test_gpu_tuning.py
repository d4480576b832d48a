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
