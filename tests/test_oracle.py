"""The oracle against its pins (CPU only)."""

import numpy as np
import pytest

import oracle_pins as P
from paper_2009_09500_gb300 import workloads


def test_hand_voxels(orc):
    P.pin_hand_voxels(orc)


def test_hand_packing(orc):
    P.pin_hand_packing(orc)


def test_brute_force_all_pairs_5cube(orc):
    P.pin_brute_force(orc, P.all_pairs(5))


def test_brute_force_random_12cube(orc):
    rng = np.random.default_rng(11)
    P.pin_brute_force(orc, P.random_pairs(rng, 1500, 12))


def test_brute_force_flat_and_long(orc):
    # longer, flatter boxes: one long axis, small minors
    rng = np.random.default_rng(12)
    segs = []
    for _ in range(300):
        L = int(rng.integers(1, 60))
        a = int(rng.integers(0, 3))
        s = rng.integers(0, 4, size=3)
        e = s + rng.integers(-3, 4, size=3)
        s[a], e[a] = (0, L) if rng.random() < 0.5 else (L, 0)
        lo = np.minimum(s, e).min()
        segs.append(np.concatenate([s - min(lo, 0), e - min(lo, 0)]))
    P.pin_brute_force(orc, np.array(segs, dtype=np.int32))


def test_closed_forms(orc):
    P.pin_closed_forms(orc)


def test_carry_recurrence(orc):
    rng = np.random.default_rng(13)
    P.pin_carry_recurrence(orc, P.random_pairs(rng, 400, 300))


def test_scan(orc):
    P.pin_scan(orc)


def test_validate(orc):
    P.pin_validate(orc)


def test_invariants_config1(orc):
    w = workloads.config1()
    assert orc.validate(w.segs, w.dims, want_list32=True) == 0
    P.pin_invariants(orc, w.segs, w.dims)


def test_invariants_config2_prefix(orc):
    w = workloads.config2(n_fixed=20000)
    assert orc.validate(w.segs, w.dims, want_list32=True) == 0
    c = orc.count(w.segs)
    assert (c[:-1] == 64).all() and c[-1] == 1024
    P.pin_invariants(orc, w.segs, w.dims)


def test_invariants_config3_prefix(orc):
    w = workloads.config3(n=3000)
    assert orc.validate(w.segs, w.dims) == 0
    P.pin_invariants(orc, w.segs, w.dims)


def test_invariants_edge_cases(orc):
    segs = np.array([
        [0, 0, 0, 0, 0, 0],
        [3, 3, 3, 3, 3, 3],
        [0, 0, 0, 1, 0, 0],
        [1, 1, 1, 0, 0, 0],
        [0, 5, 0, 5, 0, 0],
        [9, 0, 9, 0, 9, 0],
        [0, 0, 0, 9, 1, 0],
        [9, 9, 9, 0, 8, 9],
    ], dtype=np.int32)
    P.pin_invariants(orc, segs, (10, 10, 10))
    P.pin_invariants(orc, np.zeros((0, 6), dtype=np.int32))


def test_outputs_agree_config1(orc):
    w = workloads.config1()
    P.pin_outputs_agree(orc, w.segs, w.dims)


def test_outputs_agree_odd_volume(orc):
    # a volume whose size is not a multiple of 32 bits, and rows not word aligned
    rng = np.random.default_rng(14)
    dims = (13, 7, 5)
    segs = workloads.uniform_segments(rng, 200, dims)
    P.pin_outputs_agree(orc, segs, dims)


def test_zslab_config1(orc):
    """Slabs of the 256^3 volume, cut at word-aligned and ragged planes, with
    segments crossing the cuts."""
    w = workloads.config1()
    P.pin_zslab(orc, w.segs[:600], w.dims, [0, 1, 37, 64, 128, 129, 255, 256])


def test_zslab_odd_volume(orc):
    rng = np.random.default_rng(17)
    dims = (13, 7, 21)
    segs = workloads.uniform_segments(rng, 400, dims)
    P.pin_zslab(orc, segs, dims, [0, 3, 4, 10, 20, 21])
    # an empty slab
    assert not orc.bitmask_zslab(segs, dims, 5, 5).any()


def test_zslab_words_align_with_the_whole_volume(orc):
    """With z0 w h a multiple of 32 the slab's words are the volume's words."""
    rng = np.random.default_rng(18)
    dims = (64, 16, 48)
    segs = workloads.uniform_segments(rng, 500, dims)
    full = orc.bitmask(segs, dims)
    per_plane = 64 * 16 // 32
    for z0, z1 in ((0, 16), (16, 40), (40, 48)):
        assert np.array_equal(orc.bitmask_zslab(segs, dims, z0, z1), full[z0 * per_plane:z1 * per_plane])


def test_generator_shapes():
    w2 = workloads.config2(n_fixed=4096)
    d = (w2.segs[:, 3:].astype(np.int64) - w2.segs[:, :3])
    assert (np.abs(d[:-1]).max(1) == 63).all() and np.abs(d[-1]).max() == 1023
    assert (w2.segs >= 0).all() and (w2.segs < 1024).all()
    w3 = workloads.config3(n=20000)
    d3 = np.abs(w3.segs[:, 3:].astype(np.int64) - w3.segs[:, :3]).max(1)
    assert d3.min() == 0 and d3.max() <= 4095 and (w3.segs < 4096).all() and (w3.segs >= 0).all()
    # log-uniform lengths: median near sqrt(4097) - 1
    assert 40 < np.median(d3) < 90
    sc = workloads.config4(n_scenes=16)
    for s in sc:
        assert s.dims[0] in (64, 128, 256, 512) and 1000 <= s.n <= 100000
        assert (s.segs < s.dims[0]).all()
    reqs = workloads.config5(duration_s=0.05)
    assert 50 < len(reqs) < 200
    assert all(1000 <= r.n_segments <= 1000000 for r in reqs)


def test_euclidean_length_gives_repeats():
    """Reading check for Eq. (1): with N = int(|E - S|) (Euclidean) the samples of
    the space diagonal (0,0,0)->(3,3,0) land twice in one voxel, which the target
    set of Section 2 (two neighbours per voxel) excludes; the Chebyshev N does not."""
    from fractions import Fraction
    import math

    S, E = (0, 0, 0), (3, 3, 0)
    n_euc = int(math.sqrt(sum((e - s) ** 2 for s, e in zip(S, E))))
    pts = []
    for k in range(n_euc + 1):
        pts.append(tuple(P._nearest_from_fraction(S[a], Fraction((E[a] - S[a]) * k, n_euc), 1) for a in range(3)))
    assert len(set(pts)) < len(pts)


# ---------------------------------------------- the Euclidean-N variant (Eq. (1)-(2))
def test_euclid_hand(orc):
    P.pin_euclid_hand(orc)


def test_euclid_isqrt(orc):
    P.pin_euclid_isqrt(orc)


def test_euclid_brute_force_all_pairs_4cube(orc):
    P.pin_euclid_brute_force(orc, P.all_pairs(4))


def test_euclid_brute_force_random(orc):
    rng = np.random.default_rng(31)
    P.pin_euclid_brute_force(orc, P.random_pairs(rng, 800, 14))


def test_euclid_closed_forms(orc):
    P.pin_euclid_closed_forms(orc)


def test_euclid_invariants(orc):
    P.pin_euclid_invariants(orc, workloads.config1().segs[:600])
    rng = np.random.default_rng(32)
    P.pin_euclid_invariants(orc, workloads.uniform_segments(rng, 300, (2048, 64, 3000)))


def test_euclid_volume(orc):
    rng = np.random.default_rng(33)
    dims = (40, 23, 17)
    P.pin_euclid_volume(orc, workloads.uniform_segments(rng, 400, dims), dims)
