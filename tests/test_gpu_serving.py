"""The serving loop on the GPU: requests arriving while others run are batched
together; each request's resident volume must be the same alone and in the mix,
bit for bit, and equal to the oracle's."""

import numpy as np
import pytest
import torch

from gpu_util import get_oracle
from paper_2009_09500_gb300 import serving, vox, workloads

pytestmark = pytest.mark.gpu


def test_served_volumes_equal_alone_and_oracle():
    from paper_2009_09500_gb300 import build

    build.build_library()
    stream = workloads.config5(seed=21, rate_hz=20000.0, duration_s=0.004, s_lo=200, s_hi=5000)
    for r in stream:  # smaller volumes for the oracle
        r.edge = min(r.edge, 256)
    reqs = serving.make_requests(stream, pool_size=len(stream))
    assert len(reqs) >= 40
    launcher = serving.GpuLauncher(slots=3, keep_results=True)
    srv = serving.Server(launcher, budget_bytes=64 << 20, max_inflight=3, max_batch_requests=8)
    st = srv.run(reqs)
    assert st.completed == len(reqs) and st.failed == 0 and st.rejected == 0
    assert st.batches < len(reqs), "requests were batched"
    O = get_oracle()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for r in reqs:
        segs_np = r.segs_host.numpy()
        got = r.result.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, O.bitmask(segs_np, r.dims)), f"request {r.rid} differs from the oracle"
        # the same request alone through the plain entry point
        segs = torch.from_numpy(segs_np).cuda()
        ws = torch.empty(vox.vox_workspace_size(r.n), dtype=torch.uint8, device="cuda")
        alone = torch.zeros(vox.vox_mask_words(r.dims), dtype=torch.int32, device="cuda")
        vox.vox_generate(segs, r.dims, ws, status, None, alone)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert np.array_equal(alone.cpu().numpy().view(np.uint32), got), f"request {r.rid}: alone != in the mix"
