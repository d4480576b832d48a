"""The sweeps of Section 5 (Tables 2-4) through the C ABI against the oracle:
64-bit lists in a 2^21-edge volume. Whole lists where the oracle finishes in
seconds; at the largest sizes (2e8 and 1e9 voxels) counts and offsets in full
and the list slices of sampled segments, each against the oracle run on that
segment alone (bit-exact)."""

import numpy as np
import pytest
import torch

from gpu_util import assert_list_equal, get_oracle, run_gpu
from paper_2009_09500_gb300 import vox, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2009_09500_gb300 import build

    build.build_library()
    vox.load()


@pytest.mark.parametrize("length", workloads.E1_LENGTHS)
def test_e1_single_segment_full(length):
    w = workloads.sweep_single(length)
    O = get_oracle()
    r = run_gpu(w.segs, w.dims, vox.OUT_LIST64)
    assert r["status"] == 0 and r["V"] == length
    assert_list_equal(r["list_full"], O.list64(w.segs), r["V"])


@pytest.mark.parametrize("length", [20, 50, 100, 1000, 2000])
def test_e2_equal_length_full(length):
    w = workloads.sweep_fixed(length)
    O = get_oracle()
    r = run_gpu(w.segs, w.dims, vox.OUT_LIST64)
    assert r["status"] == 0 and r["V"] == 1024 * length
    assert_list_equal(r["list_full"], O.list64(w.segs), r["V"])


def sampled_check(w, n_sample, seed):
    """One vox_generate call on the whole workload; counts and offsets compared
    in full, then the list slices of sampled segments (plus the first and the
    last) against the oracle on each segment alone."""
    O = get_oracle()
    n = w.n
    counts = O.count(w.segs).astype(np.int64)
    off = O.offsets(counts)
    V = int(off[-1])
    segs = torch.from_numpy(w.segs).cuda()
    ws = torch.empty(vox.vox_workspace_size(n), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_counts = torch.empty(n, dtype=torch.int32, device="cuda")
    d_off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    vox.vox_count(segs, w.dims, ws, status, d_counts, d_off)
    lst = torch.empty(V + 16, dtype=torch.int64, device="cuda")
    lst[V:] = -1
    vox.vox_generate(segs, w.dims, ws, status, lst, None, vox.OUT_LIST64, capacity=V)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(d_counts.cpu().numpy(), counts)
    assert np.array_equal(d_off.cpu().numpy(), off)
    assert bool((lst[V:] == -1).all()), "write past the end of the list"
    rng = np.random.default_rng(seed)
    pick = sorted(set(rng.choice(n, size=n_sample, replace=False).tolist()) | {0, n - 1})
    for s in pick:
        got = lst[int(off[s]):int(off[s + 1])].cpu().numpy().view(np.uint64)
        want = O.list64(np.ascontiguousarray(w.segs[s:s + 1]))
        assert np.array_equal(got, want), f"segment {s}"
    return V


def test_e2_equal_length_200000_sampled():
    assert sampled_check(workloads.sweep_fixed(200000), 12, 1) == 1024 * 200000


def test_e3_arbitrary_lengths_one_giga_voxel_sampled():
    assert sampled_check(workloads.sweep_giga(), 6, 2) == workloads.E3_TOTAL
