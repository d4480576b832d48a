"""Pins for the oracle: checks that fix what a voxelization of a segment must be,
each written independently of the oracle's own rounding formula.

Every ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError on a
mismatch, so the same pins run against the real oracle (tests/test_oracle.py) and
against copies with a planted mistake (tests/test_oracle_mutants.py), where at
least one pin must fail.

Sources of truth (Section 3 of the paper, Eq. (2)-(3), Fig. 3, and the target
set of Section 2: every voxel but the two ends has exactly two neighbours, centred
as close as possible to the segment):
  * hand-worked examples in tests/golden/ (derived on paper, not by code);
  * brute force: for each k, the lattice point of the bounding box nearest to the
    exact point G_k = S + (E - S) k / N, found by exhaustive search;
  * the nearest-point inequality |v - G_k| <= 1/2 per axis with the tie rule;
  * closed forms: axis-aligned lines, diagonals, half slopes, exact rationals;
  * structure: N + 1 voxels, both endpoints, major axis advancing one per step,
    26-connected and thin, inside the bounding box;
  * a second formulation (the incremental carry recurrence started at k = 0);
  * the exclusive scan against a running sum; the volume against the voxel set.
"""

from __future__ import annotations

import itertools
import math
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------- golden files
def parse_hand_voxels():
    cases = []
    with open(os.path.join(GOLDEN, "hand_voxels.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            seg_s, vox_s = line.split(":")
            seg = [int(v) for v in seg_s.split()]
            vox = [tuple(int(v) for v in t.split()) for t in vox_s.split(";")]
            cases.append((seg, vox))
    return cases


def parse_hand_packing():
    packs, masks = [], []
    with open(os.path.join(GOLDEN, "hand_packing.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, rest = line.split(None, 1)
            if kind == "pack":
                xyz_s, vals = rest.split(":")
                xyz = tuple(int(v) for v in xyz_s.split())
                p32, p64 = (int(v) for v in vals.split())
                packs.append((xyz, p32, p64))
            elif kind == "mask":
                dims_s, segs_s, bits_s = rest.split("|")
                dims = tuple(int(v) for v in dims_s.split())
                segs = [[int(v) for v in t.split()] for t in segs_s.split(";")]
                bits = [int(v) for v in bits_s.split()]
                masks.append((dims, segs, bits))
    return packs, masks


def pin_hand_voxels(O):
    for seg, vox in parse_hand_voxels():
        got = O.voxels_xyz(np.array([seg], dtype=np.int32))
        assert [tuple(r) for r in got.tolist()] == vox, (seg, got.tolist(), vox)
        assert int(O.count(np.array([seg], dtype=np.int32))[0]) == len(vox)


def pin_hand_packing(O):
    packs, masks = parse_hand_packing()
    for (x, y, z), p32, p64 in packs:
        seg = np.array([[x, y, z, x, y, z]], dtype=np.int32)
        assert int(O.list32(seg)[0]) == p32, ((x, y, z), int(O.list32(seg)[0]), p32)
        assert int(O.list64(seg)[0]) == p64, ((x, y, z), int(O.list64(seg)[0]), p64)
    for dims, segs, bits in masks:
        m = O.bitmask(np.array(segs, dtype=np.int32), dims)
        expected = np.zeros(O.mask_words(dims), dtype=np.uint32)
        for b in bits:
            expected[b // 32] |= np.uint32(1 << (b % 32))
        assert np.array_equal(m, expected), (dims, segs, m, expected)


# ----------------------------------------------------------------- brute force
def brute_force_voxels(seg):
    """Exhaustive nearest-lattice search, independent of any rounding formula.

    N = max |d_a|. For each k, every lattice point v of the segment's bounding box
    is scored by its squared distance to G_k = S + d k / N, scaled by N^2 to stay in
    integers: sum_a (N (v_a - S_a) - k d_a)^2. The minimum wins; on a tie the point
    farther from S (larger sum |v_a - S_a|) wins, and the winner must be unique."""
    S = np.array(seg[:3], dtype=np.int64)
    E = np.array(seg[3:], dtype=np.int64)
    d = E - S
    N = int(np.abs(d).max())
    if N == 0:
        return [tuple(int(v) for v in S)]
    lo, hi = np.minimum(S, E), np.maximum(S, E)
    axes = [np.arange(lo[a], hi[a] + 1) for a in range(3)]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    out = []
    for k in range(N + 1):
        dev = N * (grid - S) - k * d
        dist2 = (dev * dev).sum(1)
        cand = grid[dist2 == dist2.min()]
        far = np.abs(cand - S).sum(1)
        cand = cand[far == far.max()]
        assert len(cand) == 1, (seg, k, cand)
        out.append(tuple(int(v) for v in cand[0]))
    return out


def pin_brute_force(O, segs):
    segs = np.asarray(segs, dtype=np.int32)
    counts = O.count(segs).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(counts)])
    xyz = O.voxels_xyz(segs)
    for s in range(len(segs)):
        want = brute_force_voxels(segs[s].tolist())
        got = [tuple(r) for r in xyz[off[s]:off[s + 1]].tolist()]
        assert got == want, (segs[s].tolist(), got, want)


def all_pairs(edge):
    pts = list(itertools.product(range(edge), repeat=3))
    return np.array([list(p) + list(q) for p in pts for q in pts], dtype=np.int32)


def random_pairs(rng, n, edge):
    return rng.integers(0, edge, size=(n, 6)).astype(np.int32)


# --------------------------------------------------- structure and nearest-point
def pin_invariants(O, segs, dims=None):
    segs = np.asarray(segs, dtype=np.int32)
    s64 = segs.astype(np.int64)
    S, E = s64[:, :3], s64[:, 3:]
    d = E - S
    N = np.abs(d).max(1)
    counts = O.count(segs).astype(np.int64)
    assert np.array_equal(counts, N + 1), "count must be max|d| + 1"
    off = O.offsets(counts.astype(np.int32))
    assert off[0] == 0 and np.array_equal(np.diff(off), counts), "exclusive scan"
    xyz = O.voxels_xyz(segs)
    assert len(xyz) == off[-1]
    if len(segs) == 0:
        return
    assert np.array_equal(xyz[off[:-1]], S), "first voxel is S"
    assert np.array_equal(xyz[off[1:] - 1], E), "last voxel is E"
    seg_of = np.repeat(np.arange(len(segs)), counts)
    k = np.arange(len(xyz)) - off[:-1][seg_of]
    Ns = N[seg_of][:, None]
    # nearest lattice point per axis: 2 |N (v - S) - k d| <= N, i.e. |v - G_k| <= 1/2
    dev = Ns * (xyz - S[seg_of]) - k[:, None] * d[seg_of]
    assert (2 * np.abs(dev) <= Ns).all(), "voxel is not the nearest lattice point"
    tie = (2 * np.abs(dev) == Ns) & (Ns > 0)
    # on a tie the voxel sits on the side of G_k away from S, i.e. along d
    assert (np.sign(dev[tie]) == np.sign(d[seg_of][tie])).all(), "tie not away from S"
    lo, hi = np.minimum(S, E)[seg_of], np.maximum(S, E)[seg_of]
    assert ((xyz >= lo) & (xyz <= hi)).all(), "outside the bounding box"
    if dims is not None:
        assert ((xyz >= 0) & (xyz < np.asarray(dims)[None, :])).all()
    starts = np.zeros(len(xyz), dtype=bool)
    starts[off[:-1]] = True
    inner = ~starts[1:]
    step = (xyz[1:] - xyz[:-1])[inner]
    dsg = np.sign(d[seg_of[:-1][inner]])
    assert ((step == 0) | (step == dsg)).all(), "axis step must be 0 or sign(d)"
    assert (np.abs(step).max(1) == 1).all(), "consecutive voxels are 26-neighbours"
    major = np.abs(d[seg_of[:-1][inner]]) == N[seg_of[:-1][inner]][:, None]
    assert (step[major] == dsg[major]).all(), "major axis advances one voxel per step"
    # thin (Section 2): voxels two steps apart are not neighbours
    inner2 = ~(starts[1:-1] | starts[2:])
    if inner2.any():
        jump = np.abs(xyz[2:] - xyz[:-2])[inner2].max(1)
        assert (jump == 2).all(), "voxel k+2 must not touch voxel k"


# ---------------------------------------------------------------- closed forms
def _nearest_from_fraction(s, f: Fraction, d_sign: int) -> int:
    """s + the integer nearest to f; at exactly one half, the one farther from s."""
    fl = f.numerator // f.denominator
    frac = f - fl
    if frac > Fraction(1, 2):
        return s + fl + 1
    if frac < Fraction(1, 2):
        return s + fl
    return s + (fl + 1 if d_sign > 0 else fl)


def pin_closed_forms(O):
    # axis-aligned lines, both directions, short to the largest supported length
    for axis in range(3):
        for sign in (1, -1):
            for L in (1, 2, 63, 1023, (1 << 21) - 1):
                S = [0, 0, 0]
                if sign < 0:
                    S[axis] = L
                E = list(S)
                E[axis] = S[axis] + sign * L
                seg = S + E
                assert O.steps(seg) == L
                for k in sorted({0, 1, L // 2, L - 1, L}):
                    want = list(S)
                    want[axis] = S[axis] + sign * k
                    assert O.voxel(seg, k) == tuple(want), (seg, k)
    # 45-degree diagonals on two or three axes: every axis with |d| = N moves each step
    for dvec in ((5, 5, 0), (7, -7, 7), (-300, 0, 300), (1 << 20, 1 << 20, -(1 << 20))):
        S = [max(0, -v) for v in dvec]
        seg = S + [S[a] + dvec[a] for a in range(3)]
        N = max(abs(v) for v in dvec)
        for k in sorted({0, 1, N // 3, N - 1, N}):
            want = tuple(S[a] + (k if dvec[a] > 0 else -k if dvec[a] < 0 else 0) for a in range(3))
            assert O.voxel(seg, k) == want, (seg, k)
    # half slope: |d| = N/2 with N even gives distance floor((k + 1) / 2) from S
    for N in (2, 4, 10, 64, 4094):
        m = N // 2
        seg = [0, m, 0, N, 0, m]  # d = (N, -m, m)
        for k in range(0, N + 1, max(1, N // 16)):
            q = (k + 1) // 2
            assert O.voxel(seg, k) == (k, m - q, q), (seg, k)
    # degenerate segment
    assert O.voxel([7, 8, 9, 7, 8, 9], 0) == (7, 8, 9)
    assert O.steps([7, 8, 9, 7, 8, 9]) == 0
    # exact rationals on large random segments (independent nearest-integer rule)
    rng = np.random.default_rng(1234)
    for _ in range(300):
        edge = int(rng.choice([17, 1024, 4096, 1 << 21]))
        seg = rng.integers(0, edge, size=6).tolist()
        N = O.steps(seg)
        ks = {0, N} | set(int(v) for v in rng.integers(0, N + 1, size=8))
        for k in ks:
            want = []
            for a in range(3):
                da = seg[3 + a] - seg[a]
                if N == 0:
                    want.append(seg[a])
                else:
                    want.append(_nearest_from_fraction(seg[a], Fraction(da * k, N), 1 if da > 0 else -1))
            assert O.voxel(seg, k) == tuple(want), (seg, k)


# --------------------------------------------------- second formulation (carry)
def carry_recurrence_voxels(seg):
    """Integer-only incremental form started at k = 0: per axis keep a remainder r
    (initially N); each step adds 2|d|, and each time r reaches 2N it gives back 2N
    and the coordinate moves one voxel in the direction of d."""
    S = seg[:3]
    d = [seg[3 + a] - seg[a] for a in range(3)]
    N = max(abs(v) for v in d)
    v = list(S)
    r = [N, N, N]
    out = [tuple(v)]
    for _ in range(N):
        for a in range(3):
            r[a] += 2 * abs(d[a])
            if r[a] >= 2 * N:
                r[a] -= 2 * N
                v[a] += 1 if d[a] > 0 else -1
        out.append(tuple(v))
    return out


def pin_carry_recurrence(O, segs):
    segs = np.asarray(segs, dtype=np.int32)
    counts = O.count(segs).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(counts)])
    xyz = O.voxels_xyz(segs)
    for s in range(len(segs)):
        got = [tuple(r) for r in xyz[off[s]:off[s + 1]].tolist()]
        assert got == carry_recurrence_voxels(segs[s].tolist()), segs[s].tolist()


# ------------------------------------------------------------------------ scan
def pin_scan(O):
    rng = np.random.default_rng(7)
    for n in (0, 1, 2, 1000, 4097):
        counts = rng.integers(1, 5000, size=n).astype(np.int32)
        off = O.offsets(counts)
        run = 0
        for s in range(n):
            assert off[s] == run
            run += int(counts[s])
        assert off[n] == run
    # totals beyond 2^31 and 2^32 (int64 offsets)
    counts = np.full(5000, (1 << 21) + 1, dtype=np.int32)
    off = O.offsets(counts)
    assert int(off[-1]) == 5000 * ((1 << 21) + 1) > (1 << 32)
    assert int(off[4321]) == 4321 * ((1 << 21) + 1)


# ------------------------------------------------------- lists and the volume
def pin_outputs_agree(O, segs, dims):
    """The packed lists decode to the voxel sequence; the volume holds exactly
    the set of those voxels; the sector count matches a direct count."""
    segs = np.asarray(segs, dtype=np.int32)
    xyz = O.voxels_xyz(segs)
    l64 = O.list64(segs)
    dec64 = np.stack([(l64 >> np.uint64(s)) & np.uint64((1 << 21) - 1) for s in (0, 21, 42)], 1)
    assert np.array_equal(dec64.astype(np.int64), xyz)
    if max(dims) <= 1024:
        l32 = O.list32(segs)
        dec32 = np.stack([(l32 >> np.uint32(s)) & np.uint32(1023) for s in (0, 10, 20)], 1)
        assert np.array_equal(dec32.astype(np.int64), xyz)
    w, h, dd = dims
    m = O.bitmask(segs, dims)
    lin = np.unique(xyz[:, 0] + w * (xyz[:, 1] + h * xyz[:, 2]))
    bits = np.unpackbits(m.view(np.uint8), bitorder="little")
    assert np.array_equal(np.flatnonzero(bits), lin)
    assert O.popcount(m) == len(lin)
    assert O.sectors_touched(m) == len(np.unique(lin // 256))
    # OR-ing again changes nothing (idempotent), and OR-ing into a filled volume keeps it
    m2 = O.bitmask(segs, dims, m.copy())
    assert np.array_equal(m2, m)


def pin_zslab(O, segs, dims, cuts):
    """A z-slab [z0, z1) of the volume holds exactly the voxels of the voxel
    sequence with z0 <= z < z1, at bit x + w (y + h (z - z0)), and nothing else;
    the slabs between consecutive `cuts` together hold every voxel once."""
    segs = np.asarray(segs, dtype=np.int32)
    w, h, _ = (int(v) for v in dims)
    xyz = O.voxels_xyz(segs)
    covered = 0
    for z0, z1 in zip(cuts[:-1], cuts[1:]):
        sel = (xyz[:, 2] >= z0) & (xyz[:, 2] < z1)
        want = np.unique(xyz[sel, 0] + w * (xyz[sel, 1] + h * (xyz[sel, 2] - z0)))
        slab = O.bitmask_zslab(segs, dims, z0, z1)
        assert slab.shape[0] == (w * h * (z1 - z0) + 31) // 32
        got = np.flatnonzero(np.unpackbits(slab.view(np.uint8), bitorder="little"))
        assert np.array_equal(got, want), (z0, z1)
        covered += int(sel.sum())
    assert covered == len(xyz)


# ------------------------------------------------------------------ validation
def pin_validate(O):
    ok = np.array([[0, 0, 0, 9, 9, 9]], dtype=np.int32)
    assert O.validate(ok, (10, 10, 10)) == 0
    assert O.validate(ok, (10, 10, 9)) == 2          # z1 = 9 outside [0, 9)
    assert O.validate(np.array([[0, -1, 0, 1, 1, 1]], dtype=np.int32), (10, 10, 10)) == 2
    assert O.validate(ok, (0, 10, 10)) == 1
    assert O.validate(ok, (1 << 21, 10, 10)) == 0
    assert O.validate(ok, ((1 << 21) + 1, 10, 10)) == 1
    assert O.validate(ok, (1025, 10, 10), want_list32=True) == 3
    assert O.validate(ok, (1024, 10, 10), want_list32=True) == 0
    assert O.validate(np.zeros((0, 6), dtype=np.int32), (1, 1, 1)) == 0


ALL_FAST_PINS = (pin_hand_voxels, pin_hand_packing, pin_closed_forms, pin_scan, pin_validate)


# ------------------------------------------- the Euclidean-N variant (Eq. (1)-(2))
def parse_hand_euclid():
    cases = []
    with open(os.path.join(GOLDEN, "hand_euclid.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            seg_s, vox_s = line.split(":")
            cases.append(([int(v) for v in seg_s.split()], [tuple(int(v) for v in t.split()) for t in vox_s.split(";")]))
    return cases


def unpack64(l64):
    m = np.uint64((1 << 21) - 1)
    return np.stack([(l64 & m), (l64 >> np.uint64(21)) & m, (l64 >> np.uint64(42)) & m], 1).astype(np.int64)


def euclid_xyz(O, seg):
    return [tuple(r) for r in unpack64(O.euclid_list64(np.array([seg], dtype=np.int32))).tolist()]


def pin_euclid_hand(O):
    for seg, vox in parse_hand_euclid():
        assert euclid_xyz(O, seg) == vox, (seg, euclid_xyz(O, seg), vox)
        assert int(O.euclid_count(np.array([seg], dtype=np.int32))[0]) == len(vox)


def pin_euclid_isqrt(O):
    """N = int(|d|) against Python's integer square root, on squares, their
    neighbours and random values up to 3 (2^21 - 1)^2."""
    rng = np.random.default_rng(5)
    top = 3 * ((1 << 21) - 1) ** 2
    xs = [0, 1, 2, 3, 4, 5, 8, 9, 10, 15, 16, 17, top]
    for r in [2, 3, 46340, 46341, 1 << 20, (1 << 21) - 1, 3631212]:
        xs += [r * r - 1, r * r, r * r + 1]
    xs += [int(v) for v in rng.integers(0, top, size=2000)]
    for x in xs:
        assert O.isqrt(x) == math.isqrt(x), x
    for seg in rng.integers(0, 1 << 21, size=(200, 6)).tolist():
        d2 = sum((seg[3 + a] - seg[a]) ** 2 for a in range(3))
        assert O.euclid_steps(seg) == math.isqrt(d2)


def euclid_brute_force(seg):
    """Independent of any rounding formula: N = the largest integer with N^2 <=
    |d|^2 (by search); per sample k and axis, every coordinate between S and E is
    scored by |N (v - S) - k d| (the distance to G_k scaled by N), the smallest
    wins, a tie goes to the coordinate farther from S; repeats of the previous
    voxel are dropped."""
    S = [int(v) for v in seg[:3]]
    E = [int(v) for v in seg[3:]]
    d = [E[a] - S[a] for a in range(3)]
    d2 = sum(x * x for x in d)
    N = 0
    while (N + 1) * (N + 1) <= d2:
        N += 1
    if N == 0:
        return [tuple(S)]
    out = []
    for k in range(N + 1):
        v = []
        for a in range(3):
            lo, hi = min(S[a], E[a]), max(S[a], E[a])
            best = None
            for c in range(lo, hi + 1):
                key = (abs(N * (c - S[a]) - k * d[a]), -abs(c - S[a]))
                if best is None or key < best[0]:
                    best = (key, c)
            v.append(best[1])
        if not out or tuple(v) != out[-1]:
            out.append(tuple(v))
    return out


def pin_euclid_brute_force(O, segs):
    segs = np.asarray(segs, dtype=np.int32)
    counts = O.euclid_count(segs)
    xyz = unpack64(O.euclid_list64(segs))
    off = np.concatenate([[0], np.cumsum(counts)])
    for s in range(len(segs)):
        want = euclid_brute_force(segs[s].tolist())
        got = [tuple(r) for r in xyz[off[s]:off[s + 1]].tolist()]
        assert got == want, (segs[s].tolist(), got, want)


def pin_euclid_closed_forms(O):
    """Where |d| = max|d_a| (one non-zero axis) or all non-zero axes move together
    (pure diagonals), the variant's voxels are those of N = max|d|."""
    rng = np.random.default_rng(6)
    segs = []
    for _ in range(300):
        t = int(rng.integers(0, 2000))
        s = rng.integers(0, 4000, size=3)
        sign = rng.choice([-1, 1], size=3)
        for mask in ([1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1], [1, 0, 1], [1, 1, 1]):
            e = s + sign * t * np.array(mask)
            segs.append(np.concatenate([s, e]) + 2000)
    segs = np.array(segs, dtype=np.int32)
    assert np.array_equal(O.euclid_list64(segs), O.list64(segs))


def pin_euclid_invariants(O, segs):
    """Per segment: first voxel S, last E; between N_max + 1 and N + 1 voxels
    (N_max = max|d_a|, N = int(|d|)); every step moves each axis by 0 or one voxel
    toward E and at least one axis; no voxel twice."""
    segs = np.asarray(segs, dtype=np.int32)
    counts = O.euclid_count(segs)
    xyz = unpack64(O.euclid_list64(segs))
    off = np.concatenate([[0], np.cumsum(counts)])
    assert off[-1] == len(xyz)
    for s in range(len(segs)):
        S, E = segs[s, :3].astype(np.int64), segs[s, 3:].astype(np.int64)
        v = xyz[off[s]:off[s + 1]]
        nmax = int(np.abs(E - S).max())
        ne = math.isqrt(int(((E - S) ** 2).sum()))
        assert nmax + 1 <= len(v) <= ne + 1, (segs[s], len(v), nmax, ne)
        assert tuple(v[0]) == tuple(S) and tuple(v[-1]) == tuple(E)
        if len(v) > 1:
            step = np.diff(v, axis=0)
            assert (np.abs(step) <= 1).all() and (np.abs(step).sum(1) >= 1).all()
            assert ((step * np.sign(E - S)) >= 0).all()
        assert len(np.unique(v, axis=0)) == len(v)


def pin_euclid_volume(O, segs, dims):
    """The variant's volume holds exactly the distinct voxels of its list."""
    segs = np.asarray(segs, dtype=np.int32)
    xyz = unpack64(O.euclid_list64(segs))
    w, h, _ = dims
    lin = np.unique(xyz[:, 0] + w * (xyz[:, 1] + h * xyz[:, 2]))
    want = np.zeros(O.mask_words(dims), dtype=np.uint32)
    np.bitwise_or.at(want, lin // 32, (np.uint64(1) << (lin % 32).astype(np.uint64)).astype(np.uint32))
    assert np.array_equal(O.euclid_bitmask(segs, dims), want)
