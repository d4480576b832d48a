"""Full-size parity on the largest workloads, element by element against the
oracle: every list element and every volume word, with the oracle run on
disjoint parts in spawn-started worker processes (tests/oracle_par.py).

  * 4M log-uniform segments in a 4096^3 volume (Table 4 shape): counts and
    offsets, the whole 64-bit list (2.07e9 voxels, 16.5 GB), the 8 GiB volume
    built by per-voxel atomics (OR into zeros) and by bricks (fresh, over stale
    bits), each checked z-slab by z-slab (no stray bit anywhere);
  * 1.1M segments of 2000 voxels (V = 2.2e9 > 2^31): the whole list and volume;
  * all 256 scenes of the batched workload: every scene's list part and volume;
  * served requests of the request-stream workload's full sizes (1e5..1e6
    segments, 1024^3 volumes): every request's resident volume, alone and in
    the mix.

Bit-exact (tolerance zero): the method is integer-only.
"""

import numpy as np
import pytest
import torch

import oracle_par as OP
from gpu_util import get_oracle
from paper_2009_09500_gb300 import batching, serving, vox, workloads

pytestmark = pytest.mark.gpu

L32, L64, BM, FR = vox.OUT_LIST32, vox.OUT_LIST64, vox.OUT_BITMASK, vox.OUT_FRESH
LIST_CHUNK_VOXELS = 32 << 20
SLAB_Z = 256


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2009_09500_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build_library()
    vox.load()


@pytest.fixture(scope="module")
def pool():
    with OP.OraclePool(max_bytes_in_flight=16 << 30) as p:
        yield p


def submit_list(pool, segs_buf, off, dev_list, wide, tag=""):
    """Every list element: contiguous segment ranges of about LIST_CHUNK_VOXELS
    voxels, each against the oracle's list of those segments."""
    n = len(off) - 1
    s0 = 0
    while s0 < n:
        s1 = int(np.searchsorted(off, off[s0] + LIST_CHUNK_VOXELS, side="left"))
        s1 = min(n, max(s1, s0 + 1))
        part = dev_list[int(off[s0]):int(off[s1])].cpu().numpy()
        b = pool.buf(part)
        del part
        pool.submit((tag, "list", s0, s1), OP.job_list, segs_buf, s0, s1, wide, b, int(off[s0]), bufs=[b])
        s0 = s1


def submit_slabs(pool, segs_buf, dims, dev_masks, tag=""):
    """Every volume word, z-slab by z-slab, for each device volume given."""
    w, h, d = (int(v) for v in dims)
    assert (w * h) % 32 == 0
    per_plane = w * h // 32
    for z0 in range(0, d, SLAB_Z):
        z1 = min(d, z0 + SLAB_Z)
        parts = []
        for m in dev_masks:
            part = m[z0 * per_plane:z1 * per_plane].cpu().numpy()
            parts.append(pool.buf(part))
            del part
        pool.submit((tag, "slab", z0, z1), OP.job_zslab, segs_buf, dims, z0, z1, parts, bufs=parts)


def assert_clean(results, expect_jobs=None):
    bad = []
    nonzero = 0
    for tag, r in results:
        if tag[1] == "list":
            if r["bad"]:
                bad.append((tag, r))
        elif tag[1] == "slab":
            nonzero += r["nonzero"]
            for i, p in enumerate(r["parts"]):
                if p["bad"]:
                    bad.append((tag, i, p))
        else:
            for k, p in r.items():
                if p["bad"]:
                    bad.append((tag, k, p))
    assert not bad, f"{len(bad)} parts differ from the oracle, first: {bad[:3]}"
    if expect_jobs is not None:
        assert len(results) == expect_jobs
    return nonzero


def assert_same_list_by_warp_slices(segs, dims, ws, status, lst):
    """The list alone by warp slices (launch tuning 32,0,0,2: the one the
    benchmark's tuner picks for long segments) equals, element by element, the
    list `lst` that the oracle checks in full."""
    lst2 = torch.empty_like(lst)
    try:
        vox.vox_set_tuning(32, 0, 0, 2)
        vox.vox_generate(segs, dims, ws, status, lst2, None, L64, capacity=lst.numel())
        torch.cuda.synchronize()
    finally:
        vox.vox_reset_tuning()
    assert int(status.item()) == 0
    assert torch.equal(lst2, lst), "the warp-slice list differs"
    del lst2
    torch.cuda.empty_cache()


def test_config3_full_size_exact(pool):
    """4M log-uniform segments, 4096^3: whole list64 and both 8 GiB volumes."""
    w = workloads.config3()
    O = get_oracle()
    n = w.n
    counts = O.count(w.segs)
    off = O.offsets(counts)
    V = int(off[-1])
    assert V == 2_065_164_092
    segs = torch.from_numpy(w.segs).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size(n), dtype=torch.uint8, device="cuda")
    d_counts = torch.empty(n, dtype=torch.int32, device="cuda")
    d_off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    vox.vox_count(segs, w.dims, ws, status, d_counts, d_off)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(d_counts.cpu().numpy(), counts)
    assert np.array_equal(d_off.cpu().numpy(), off)
    del d_counts, d_off
    words = vox.vox_mask_words(w.dims)
    # the list and the volume by per-voxel atomics (plain workspace), OR-ed into zeros
    lst = torch.empty(V, dtype=torch.int64, device="cuda")
    mask_atomic = torch.zeros(words, dtype=torch.int32, device="cuda")
    vox.vox_generate(segs, w.dims, ws, status, lst, mask_atomic)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert_same_list_by_warp_slices(segs, w.dims, ws, status, lst)
    # the fresh volume by bricks (the benchmarked path) over stale bits
    ws0 = torch.empty(vox.vox_workspace_size_volume(n, w.dims, 0), dtype=torch.uint8, device="cuda")
    V2, P = vox.vox_plan(segs, w.dims, ws0, status)
    del ws0
    assert V2 == V and P > n
    wsb = torch.empty(vox.vox_workspace_size_volume(n, w.dims, P), dtype=torch.uint8, device="cuda")
    mask_brick = torch.full((words,), -1, dtype=torch.int32, device="cuda")
    vox.vox_generate(segs, w.dims, wsb, status, None, mask_brick, BM | FR)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    del wsb
    segs_buf = pool.buf(w.segs)
    try:
        submit_list(pool, segs_buf, off, lst, True, "c3")
        submit_slabs(pool, segs_buf, w.dims, [mask_atomic, mask_brick], "c3")
        results = pool.finish()
    finally:
        segs_buf.release()
    nonzero = assert_clean(results)
    assert nonzero == int(torch.count_nonzero(mask_brick).item())
    del lst, mask_atomic, mask_brick
    torch.cuda.empty_cache()


def test_total_beyond_2_to_31_exact(pool):
    """1.1M segments of 2000 voxels in 4096^3: V = 2.2e9 > 2^31, so totals,
    offsets and voxel ids need 64 bits; whole list64 and whole volume."""
    rng = np.random.default_rng(31)
    n = 1_100_000
    segs_np = workloads._segments_from_major(rng, np.full(n, 1999, np.int64), 4096)
    dims = (4096, 4096, 4096)
    O = get_oracle()
    off = O.offsets(O.count(segs_np))
    V = int(off[-1])
    assert V == n * 2000 and V > (1 << 31)
    segs = torch.from_numpy(segs_np).cuda()
    ws = torch.empty(vox.vox_workspace_size(n), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    vox.vox_count(segs, dims, ws, status, None, d_off)
    lst = torch.empty(V, dtype=torch.int64, device="cuda")
    mask = torch.zeros(vox.vox_mask_words(dims), dtype=torch.int32, device="cuda")
    vox.vox_generate(segs, dims, ws, status, lst, mask)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(d_off.cpu().numpy(), off)
    assert_same_list_by_warp_slices(segs, dims, ws, status, lst)
    segs_buf = pool.buf(segs_np)
    try:
        submit_list(pool, segs_buf, off, lst, True, "2^31")
        submit_slabs(pool, segs_buf, dims, [mask], "2^31")
        results = pool.finish()
    finally:
        segs_buf.release()
    assert_clean(results)
    del lst, mask
    torch.cuda.empty_cache()


def test_batched_config4_all_scenes_exact(pool):
    """The 256-scene batch (uneven scenes, volumes by bricks, one launch
    sequence): every scene's list part and volume."""
    scenes = workloads.config4()
    b = batching.make_batch(scenes)
    assert b.total_bricks > 0
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0, vox.strerror(int(b.status.item()))
    # the same batch under the launch tuning its tuner picks (the list by warp
    # slices): outputs equal to these, which the oracle checks in full below
    lst_ref = b.lst.clone()
    masks_ref = [m.clone() for m in b.masks]
    try:
        vox.vox_set_tuning(32, 0, 0, 2)
        b.run()
        torch.cuda.synchronize()
    finally:
        vox.vox_reset_tuning()
    assert int(b.status.item()) == 0, vox.strerror(int(b.status.item()))
    assert torch.equal(b.lst, lst_ref), "the batched list by warp slices differs"
    assert all(torch.equal(m, r) for m, r in zip(b.masks, masks_ref))
    del lst_ref, masks_ref
    O = get_oracle()
    base = b.scene_base.cpu().numpy()
    per_scene = np.array([O.total(s.segs) for s in scenes])
    assert np.array_equal(np.diff(base), per_scene) and base[0] == 0 and base[-1] == b.V
    segs_np = np.ascontiguousarray(np.concatenate([s.segs for s in scenes]))
    segs_buf = pool.buf(segs_np)
    try:
        s0 = 0
        for k, s in enumerate(scenes):
            lb = pool.buf(b.lst[int(base[k]):int(base[k + 1])].cpu().numpy())
            mb = pool.buf(b.masks[k].cpu().numpy())
            pool.submit(("c4", "scene", k), OP.job_scene, segs_buf, s0, s0 + s.n, s.dims, 32, lb, mb,
                        bufs=[lb, mb])
            s0 += s.n
        results = pool.finish()
    finally:
        segs_buf.release()
    assert_clean(results, expect_jobs=len(scenes))


def test_served_full_size_requests_exact(pool):
    """Requests of the request stream's full sizes (1e5..1e6 segments, 1024^3
    and smaller volumes) through the continuous-batching loop: every resident
    volume against the oracle (slab by slab) and against the same request run
    alone."""
    stream = workloads.config5(seed=23, rate_hz=4000.0, duration_s=0.0035, s_lo=1e5, s_hi=1e6)
    for i, r in enumerate(stream):  # the first three at the largest volume
        if i < 3:
            r.edge = 1024
    reqs = serving.make_requests(stream, pool_size=len(stream))
    assert len(reqs) >= 6
    assert max(r.n for r in reqs) >= 500_000 and sum(r.dims[0] == 1024 for r in reqs) >= 3
    launcher = serving.GpuLauncher(slots=3, keep_results=True)
    srv = serving.Server(launcher, budget_bytes=48 << 30, max_inflight=3, max_batch_requests=4)
    st = srv.run(reqs)
    assert st.completed == len(reqs) and st.failed == 0 and st.rejected == 0
    assert st.batches < len(reqs), "requests were batched"
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for r in reqs:
        segs_np = r.segs_host.numpy()
        segs = torch.from_numpy(segs_np).cuda()
        ws = torch.empty(vox.vox_workspace_size(r.n), dtype=torch.uint8, device="cuda")
        alone = torch.zeros(vox.vox_mask_words(r.dims), dtype=torch.int32, device="cuda")
        vox.vox_generate(segs, r.dims, ws, status, None, alone)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(alone, r.result), f"request {r.rid}: alone != in the mix"
        del segs, ws, alone
        segs_buf = pool.buf(segs_np)
        try:
            submit_slabs(pool, segs_buf, r.dims, [r.result], f"req{r.rid}")
            results = pool.finish()
        finally:
            segs_buf.release()
        assert_clean(results)
        r.result = None
    torch.cuda.empty_cache()
