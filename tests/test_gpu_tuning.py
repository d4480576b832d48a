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
