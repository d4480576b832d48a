"""Batched scenes through vox_generate_batched, against the oracle scene by
scene, against per-scene plain launches, and replayed from a CUDA graph
(bit-exact everywhere: integer outputs)."""

import numpy as np
import pytest
import torch

from gpu_util import get_oracle
from paper_2009_09500_gb300 import batching, vox, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2009_09500_gb300 import build

    build.build_library()
    vox.load()


def check_scenes(batch, scenes, sample=None):
    O = get_oracle()
    torch.cuda.synchronize()
    assert int(batch.status.item()) == 0, vox.strerror(int(batch.status.item()))
    base = batch.scene_base.cpu().numpy()
    counts = np.concatenate([O.count(w.segs) for w in scenes]).astype(np.int64)
    per_scene = np.array([O.total(w.segs) for w in scenes])
    assert np.array_equal(np.diff(base), per_scene)
    assert base[-1] == counts.sum() == batch.V
    lst = batch.lst.cpu().numpy() if batch.lst is not None else None
    ks = range(len(scenes)) if sample is None else sample
    for k in ks:
        w = scenes[k]
        if lst is not None:
            got = lst[base[k]:base[k + 1]]
            want = O.list64(w.segs) if batch.flags & vox.OUT_LIST64 else O.list32(w.segs)
            assert np.array_equal(got.view(want.dtype), want), f"scene {k} list"
        if batch.masks:
            if batch.masks[k] is None:
                continue
            got = batch.masks[k].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, O.bitmask(w.segs, w.dims)), f"scene {k} volume"


def small_scenes(n=24, seed=40):
    return workloads.config4(seed=seed, n_scenes=n, s_lo=50, s_hi=3000)


def test_batched_small_list32_and_volumes():
    scenes = small_scenes()
    b = batching.make_batch(scenes)
    b.run()
    check_scenes(b, scenes)


def test_batched_list64_only_and_volume_only():
    scenes = small_scenes(12, seed=41)
    b = batching.make_batch(scenes, flags=vox.OUT_LIST64)
    b.run()
    check_scenes(b, scenes)
    b = batching.make_batch(scenes, flags=vox.OUT_BITMASK)
    b.run()
    check_scenes(b, scenes)


def test_batched_with_empty_and_odd_scenes():
    rng = np.random.default_rng(42)
    scenes = []
    for k, dims in enumerate([(64, 64, 64), (13, 7, 5), (96, 40, 17), (32, 32, 32), (128, 8, 300)]):
        n = [0, 500, 1, 2049, 333][k]
        scenes.append(workloads.Workload(f"s{k}", workloads.uniform_segments(rng, n, dims), dims))
    b = batching.make_batch(scenes)
    b.run()
    check_scenes(b, scenes)


def test_batched_equals_plain_and_graph_replay():
    scenes = small_scenes(32, seed=43)
    b = batching.make_batch(scenes)
    b.run()
    torch.cuda.synchronize()
    ref_list = b.lst.cpu().numpy().copy()
    ref_masks = [m.cpu().numpy().copy() for m in b.masks]
    # plain per-scene launches into fresh volumes
    b.clear_volumes()
    plain = batching.PlainScenes(b)
    plain.run()
    torch.cuda.synchronize()
    base = b.scene_base.cpu().numpy()
    for k, (s, dims, ws, lst, mask, V) in enumerate(plain.items):
        assert np.array_equal(lst[:V].cpu().numpy(), ref_list[base[k]:base[k + 1]])
        assert np.array_equal(mask.cpu().numpy(), ref_masks[k])
    # captured once, replayed twice into cleared volumes
    g = batching.GraphRunner(b.run)
    for _ in range(2):
        b.clear_volumes()
        b.lst.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(b.status.item()) == 0
        assert np.array_equal(b.lst.cpu().numpy(), ref_list)
        for k, m in enumerate(b.masks):
            assert np.array_equal(m.cpu().numpy(), ref_masks[k])


def test_batched_bad_scene_table_writes_nothing():
    scenes = small_scenes(4, seed=44)
    b = batching.make_batch(scenes)
    table = bytearray(b.scenes.cpu().numpy().tobytes())
    rec = batching.SceneRecord.from_buffer(table, 2 * 40)
    rec.seg_begin += 1  # a gap between scene 1 and scene 2
    b.scenes.copy_(torch.frombuffer(table, dtype=torch.uint8))
    b.lst.fill_(-7)
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == vox.ERR_INVALID_ARG
    assert (b.lst.cpu().numpy() == -7).all()
    assert all(int(m.abs().sum().item()) == 0 for m in b.masks)


def test_batched_list32_rejects_wide_scene():
    rng = np.random.default_rng(45)
    dims = (2048, 8, 8)
    scenes = [workloads.Workload("wide", workloads.uniform_segments(rng, 100, dims), dims)]
    b = batching.make_batch(scenes, flags=vox.OUT_LIST32)
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == vox.ERR_PACK_WIDTH


def test_batched_fresh_volumes_overwrite_stale_bits():
    """VOX_OUT_FRESH: every scene's volume is cleared on the device first, so
    stale bits vanish; a scene without a volume is skipped."""
    scenes = small_scenes(10, seed=44)
    b = batching.make_batch(scenes, flags=vox.OUT_LIST32 | vox.OUT_BITMASK | vox.OUT_FRESH)
    for m in b.masks:
        m.fill_(-1)
    b.run()
    check_scenes(b, scenes)
    # drop scene 3's volume from the table: its (stale) buffer stays as it is
    ptrs = [m.data_ptr() for m in b.masks]
    ptrs[3] = 0
    table = batching.scene_table_bytes(b.seg_counts, b.dims, ptrs)
    b.scenes.copy_(torch.frombuffer(bytearray(table), dtype=torch.uint8))
    for m in b.masks:
        m.fill_(-1)
    b.run()
    torch.cuda.synchronize()
    assert bool((b.masks[3] == -1).all())
    b.masks[3] = None
    check_scenes(b, scenes)


@pytest.mark.parametrize("which", ["config1", "config2"])
def test_scene_step_graph_matches_oracle(which):
    """batching.SceneStep (count, then list and fresh volume on two streams, one
    CUDA graph), replayed twice over stale outputs: list and volume against the
    oracle, whole."""
    O = get_oracle()
    w = getattr(workloads, which)()
    segs = torch.from_numpy(w.segs).cuda()
    st = batching.SceneStep(segs, w.dims, vox.OUT_LIST32, volume=True)
    for _ in range(2):
        st.lst.fill_(-1)
        st.mask.fill_(-1)
        st.replay()
        torch.cuda.synchronize()
        assert int(st.status.item()) == 0
        assert np.array_equal(st.lst.cpu().numpy().view(np.uint32), O.list32(w.segs))
        assert np.array_equal(st.mask.cpu().numpy().view(np.uint32), O.bitmask(w.segs, w.dims))


def test_scene_step_list64_only_and_empty():
    O = get_oracle()
    w = workloads.config1()
    segs = torch.from_numpy(w.segs).cuda()
    st = batching.SceneStep(segs, w.dims, vox.OUT_LIST64, volume=False)
    st.replay()
    torch.cuda.synchronize()
    assert np.array_equal(st.lst.cpu().numpy().view(np.uint64), O.list64(w.segs))
    empty = batching.SceneStep(torch.zeros((0, 6), dtype=torch.int32, device="cuda"), (64, 64, 64), 0, volume=True)
    empty.mask.fill_(-1)
    empty.replay()
    torch.cuda.synchronize()
    assert int(empty.status.item()) == 0 and bool((empty.mask == 0).all())


def test_count_bins_beside_the_scan():
    """vox_count on the count + scan part of the workspace and vox_count_bins on
    a second stream, then the volume: the oracle's volume; a workspace without
    the brick arrays is refused."""
    O = get_oracle()
    w = workloads.config1()
    segs = torch.from_numpy(w.segs).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_workspace_size_volume(w.n, w.dims, 0), dtype=torch.uint8, device="cuda")
    V, P = vox.vox_plan(segs, w.dims, ws, st)
    ws = torch.empty(vox.vox_workspace_size_volume(w.n, w.dims, P), dtype=torch.uint8, device="cuda")
    mask = torch.full((vox.vox_mask_words(w.dims),), -1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    vox.vox_count_bins(segs, w.dims, ws, side)
    vox.vox_count(segs, w.dims, ws, st, ws_bytes=vox.vox_workspace_size(w.n))
    torch.cuda.current_stream().wait_stream(side)
    vox.vox_generate_from_scan(segs, w.dims, ws, st, None, mask, vox.OUT_BITMASK | vox.OUT_FRESH)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(mask.cpu().numpy().view(np.uint32), O.bitmask(w.segs, w.dims))
    small = torch.empty(vox.vox_workspace_size(w.n), dtype=torch.uint8, device="cuda")
    with pytest.raises(vox.VoxError) as e:
        vox.vox_count_bins(segs, w.dims, small)
    assert e.value.status == vox.ERR_WORKSPACE


def test_batched_bricks_and_atomics_agree_with_oracle():
    """The same scenes with the volumes by bricks (the default when every width
    is a multiple of 32) and by atomics (bricks=False)."""
    scenes = small_scenes(16, seed=46)
    b = batching.make_batch(scenes)
    assert b.total_bricks > 0 and b.pieces > 0
    b.run()
    check_scenes(b, scenes)
    a = batching.make_batch(scenes, bricks=False)
    assert a.total_bricks == 0
    a.run()
    check_scenes(a, scenes)


def test_batched_bricks_pieces_do_not_fit():
    """A brick workspace with room for 10 pieces: the batched atomics take over on
    the device, same volumes (OR-into and fresh)."""
    scenes = small_scenes(8, seed=47)
    for flags in (vox.OUT_BITMASK, vox.OUT_LIST32 | vox.OUT_BITMASK | vox.OUT_FRESH):
        b = batching.make_batch(scenes, flags=flags)
        b.ws = torch.empty(vox.vox_workspace_size_batched_volume(int(b.segs.shape[0]), b.n_scenes, b.total_bricks, 10),
                           dtype=torch.uint8, device="cuda")
        for m in b.masks:
            m.fill_(-1 if flags & vox.OUT_FRESH else 0)
        b.run()
        check_scenes(b, scenes)


def test_batched_bricks_wrong_total_is_refused_on_the_device():
    scenes = small_scenes(4, seed=48)
    b = batching.make_batch(scenes)
    b.total_bricks += 1
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == vox.ERR_INVALID_ARG


@pytest.mark.parametrize("volume_path", [vox.VOLUME_ATOMIC, vox.VOLUME_ATOMIC_WARP])
def test_batched_atomic_volume_paths(volume_path):
    """The batched volumes by per-voxel atomics (per-lane merging, and merged
    across the warp), every scene against the oracle."""
    scenes = small_scenes(20, seed=47)
    b = batching.make_batch(scenes, flags=vox.OUT_BITMASK)
    try:
        vox.vox_set_tuning(32, volume_path, 0)
        b.run()
        check_scenes(b, scenes)
    finally:
        vox.vox_reset_tuning()
