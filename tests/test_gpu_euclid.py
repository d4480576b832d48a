"""The Euclidean-N variant (Eq. (1)-(2) read literally, repeated voxels dropped)
through the C ABI against the oracle, bit-exact: compacted lists, per-segment
offsets, volumes, totals from the plan, errors."""

import numpy as np
import pytest
import torch

from gpu_util import get_oracle
from paper_2009_09500_gb300 import vox, workloads

pytestmark = pytest.mark.gpu

L32, L64, BM, FR = vox.OUT_LIST32, vox.OUT_LIST64, vox.OUT_BITMASK, vox.OUT_FRESH
SENT = -0x21524111


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2009_09500_gb300 import build

    build.build_library()
    vox.load()


def run_euclid(segs_np, dims, flags, capacity=None, mask_init=None, extra=64, pieces=None, offsets=True):
    """pieces: None for the plain workspace (volume by atomics), "plan" for a
    brick workspace sized by the plan, or an explicit piece capacity."""
    O = get_oracle()
    segs = torch.from_numpy(np.ascontiguousarray(segs_np, dtype=np.int32)).cuda()
    n = segs.shape[0]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    if pieces is None:
        ws = torch.empty(vox.vox_euclid_workspace_size(n), dtype=torch.uint8, device="cuda")
    else:
        ws = torch.empty(vox.vox_euclid_workspace_size_volume(n, dims, 0), dtype=torch.uint8, device="cuda")
        P = vox.vox_euclid_plan(segs, dims, ws, status, with_pieces=True)[2] if n else 0
        cap_p = P if pieces == "plan" else int(pieces)
        ws = torch.empty(vox.vox_euclid_workspace_size_volume(n, dims, cap_p), dtype=torch.uint8, device="cuda")
    Vd, Vs = vox.vox_euclid_plan(segs, dims, ws, status) if n else (0, 0)
    counts = O.euclid_count(segs_np) if n else np.zeros(0, np.int64)
    assert Vd == int(counts.sum())
    assert Vs == sum(O.euclid_steps(s) + 1 for s in np.asarray(segs_np).tolist())
    cap = Vd if capacity is None else capacity
    lst = None
    if flags & (L32 | L64):
        lst = torch.full((cap + extra,), SENT, dtype=torch.int64 if flags & L64 else torch.int32, device="cuda")
    mask = None
    if flags & BM:
        words = vox.vox_mask_words(dims)
        mask = (torch.zeros(words, dtype=torch.int32, device="cuda") if mask_init is None
                else torch.from_numpy(mask_init.view(np.int32).copy()).cuda())
    offs = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda") if offsets else None
    vox.vox_euclid_generate(segs, dims, ws, status, lst, mask, flags, offs, capacity=cap)
    torch.cuda.synchronize()
    return {"status": int(status.item()), "Vd": Vd, "counts": counts,
            "offsets": None if offs is None else offs.cpu().numpy(),
            "list": None if lst is None else lst.cpu().numpy(), "mask": None if mask is None else mask.cpu().numpy().view(np.uint32)}


def check(segs, dims, flags, **kw):
    O = get_oracle()
    r = run_euclid(segs, dims, flags, **kw)
    assert r["status"] == 0, vox.strerror(r["status"])
    Vd = r["Vd"]
    if r["offsets"] is not None:
        assert np.array_equal(r["offsets"], np.concatenate([[0], np.cumsum(r["counts"])]))
    if flags & (L32 | L64):
        want = O.euclid_list64(segs) if flags & L64 else O.euclid_list32(segs)
        got = r["list"][:Vd].view(want.dtype)
        if not np.array_equal(got, want):
            bad = np.flatnonzero(got != want)
            raise AssertionError(f"{len(bad)} list mismatches, first at {bad[:5]}")
        assert (r["list"][Vd:] == SENT).all(), "write past the end of the list"
    if flags & BM:
        init = kw.get("mask_init")
        want = O.euclid_bitmask(segs, dims, None if (init is None or flags & FR) else init.copy())
        assert np.array_equal(r["mask"], want)
    return r


def test_config1_list32_and_volume():
    w = workloads.config1()
    check(w.segs, w.dims, L32 | BM)


def test_config1_each_output():
    w = workloads.config1()
    for flags in (L32, L64, BM, L64 | BM):
        check(w.segs, w.dims, flags)


def test_config2_full_size():
    w = workloads.config2()
    r = check(w.segs, w.dims, L32 | BM)
    assert r["Vd"] > workloads.config2().n * 64  # repeats dropped, extra voxels kept


@pytest.mark.parametrize("n", [1, 2, 3, 2047, 2048, 2049, 5000])
def test_ragged_sizes(n):
    rng = np.random.default_rng(n)
    dims = (300, 200, 100)
    check(workloads.uniform_segments(rng, n, dims), dims, L64 | BM)


def test_degenerate_and_axis_aligned():
    rng = np.random.default_rng(9)
    p = rng.integers(0, 64, size=(500, 3)).astype(np.int32)
    segs = np.concatenate([np.concatenate([p, p], 1), workloads.uniform_segments(rng, 500, (64, 64, 64))])
    e = p.copy()
    e[:, 0] = 63 - p[:, 0]
    segs = np.concatenate([segs, np.concatenate([p, e], 1)]).astype(np.int32)
    check(segs, (64, 64, 64), L32 | BM)


def test_long_segments_wide_entry():
    """|E - S| up to about 3.6e6 (N above 46340: entry numerators above 2^32), runs
    that start deep inside a segment."""
    rng = np.random.default_rng(10)
    edge = 1 << 21
    segs = rng.integers(0, edge, size=(6, 6)).astype(np.int32)
    segs[0] = [0, 0, 0, edge - 1, edge - 1, edge - 1]
    check(segs, (edge, edge, edge), L64)


def test_capacity_too_small_writes_nothing():
    w = workloads.config1()
    O = get_oracle()
    Vd = int(O.euclid_count(w.segs).sum())
    r = run_euclid(w.segs, w.dims, L32 | BM, capacity=Vd - 1)
    assert r["status"] == vox.ERR_CAPACITY
    assert (r["list"] == SENT).all() and (r["mask"] == 0).all()


def test_fresh_volume_and_out_of_bounds():
    w = workloads.config1()
    rng = np.random.default_rng(11)
    init = rng.integers(0, 2**32, size=vox.vox_mask_words(w.dims), dtype=np.uint64).astype(np.uint32)
    check(w.segs, w.dims, BM | FR, mask_init=init)
    bad = w.segs.copy()
    bad[5, 3] = 256
    segs = torch.from_numpy(bad).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(vox.vox_euclid_workspace_size(w.n), dtype=torch.uint8, device="cuda")
    with pytest.raises(vox.VoxError) as e:
        vox.vox_euclid_plan(segs, w.dims, ws, st)
    assert e.value.status == vox.ERR_OUT_OF_BOUNDS


def test_empty_input():
    r = run_euclid(np.zeros((0, 6), np.int32), (8, 8, 8), L32)
    assert r["status"] == 0 and r["offsets"][0] == 0


# ------------------------------------------------- the variant's volume by bricks
@pytest.mark.parametrize("which,flags,pieces", [
    ("config1", L32 | BM, "plan"), ("config1", BM, "plan"), ("config1", L64 | BM | FR, "plan"),
    ("config1", L32 | BM, 100),       # pieces do not fit: atomics on the device
    ("config1", BM | FR, 100),
])
def test_bricks_volume(which, flags, pieces):
    w = getattr(workloads, which)()
    rng = np.random.default_rng(12)
    init = rng.integers(0, 2**32, size=vox.vox_mask_words(w.dims), dtype=np.uint64).astype(np.uint32)
    check(w.segs, w.dims, flags, pieces=pieces, mask_init=init)


@pytest.mark.parametrize("dims", [(96, 40, 17), (32, 7, 5), (128, 128, 64)])
def test_bricks_volume_shapes(dims):
    rng = np.random.default_rng(sum(dims))
    check(workloads.uniform_segments(rng, 3000, dims), dims, L32 | BM, pieces="plan")


def test_bricks_config2_full_size():
    w = workloads.config2()
    rng = np.random.default_rng(13)
    init = rng.integers(0, 2**32, size=vox.vox_mask_words(w.dims), dtype=np.uint64).astype(np.uint32)
    check(w.segs, w.dims, L32 | BM | FR, pieces="plan", mask_init=init)


def test_bricks_volume_only_with_offsets_and_capacity_error():
    w = workloads.config1()
    check(w.segs, w.dims, BM, pieces="plan")  # offsets from a list-free write pass
    O = get_oracle()
    Vd = int(O.euclid_count(w.segs).sum())
    r = run_euclid(w.segs, w.dims, L32 | BM, capacity=Vd - 1, pieces="plan")
    assert r["status"] == vox.ERR_CAPACITY
    assert (r["list"] == SENT).all() and (r["mask"] == 0).all()


def test_long_runs_many_row_flushes():
    """About 2.4e8 samples in 2000 long segments: runs of about 230 samples (the
    run slots are fixed by n), so each lane's row fills and is flushed several times
    per run and a warp's 32 runs lie in one or two segments; whole 64-bit list and
    segment offsets against the oracle."""
    rng = np.random.default_rng(12)
    edge = 1 << 21
    segs = workloads._segments_from_major(rng, np.full(2000, 99_999, np.int64), edge).astype(np.int32)
    r = check(segs, (edge, edge, edge), L64)
    assert r["Vd"] > 2000 * 100_000
