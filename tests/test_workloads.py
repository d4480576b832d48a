"""The seeded sweep inputs have the shapes the paper's Section 5 states (no
voxel arithmetic here: lengths are max |delta| + 1 of the drawn endpoints)."""

import numpy as np

from paper_2009_09500_gb300 import workloads


def lengths(w):
    d = np.abs(w.segs[:, 3:].astype(np.int64) - w.segs[:, :3])
    return d.max(axis=1) + 1


def inside(w):
    return bool((w.segs >= 0).all() and (w.segs < np.array(w.dims * 2)).all())


def test_e1_single_segment_lengths():
    for L in workloads.E1_LENGTHS:
        w = workloads.sweep_single(L)
        assert w.n == 1 and lengths(w)[0] == L and inside(w)


def test_e2_equal_lengths():
    for L in (20, 1000, 200000):
        w = workloads.sweep_fixed(L)
        assert w.n == 1024 and (lengths(w) == L).all() and inside(w)


def test_e3_one_giga_voxel_of_different_lengths():
    w = workloads.sweep_giga()
    ln = lengths(w)
    assert w.n == 1024 and int(ln.sum()) == workloads.E3_TOTAL
    assert len(np.unique(ln)) == 1024 and inside(w)
    assert w.segs.dtype == np.int32 and w.segs.flags.c_contiguous


def test_seeded_inputs_repeat():
    a, b = workloads.sweep_giga(), workloads.sweep_giga()
    assert np.array_equal(a.segs, b.segs)
    assert np.array_equal(workloads.config2(n_fixed=1000).segs, workloads.config2(n_fixed=1000).segs)
