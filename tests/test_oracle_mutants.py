"""Mutation check of the pins: plant one plausible mistake at a time in a copy of
the oracle's C source (on the CPU), compile it, and require that at least one pin
rejects it. A pin set that let any of these through would not pin the oracle."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import oracle_pins as P
from paper_2009_09500_gb300 import workloads

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, original text, planted text); each original must occur exactly once
MUTANTS = [
    ("round-down instead of nearest", "(2 * m + den) / (2 * (__int128)den)", "(2 * m) / (2 * (__int128)den)"),
    ("ties toward the start", "(2 * m + den) / (2 * (__int128)den)", "(2 * m + den - 1) / (2 * (__int128)den)"),
    ("sign of the step dropped", "return num < 0 ? s - (int64_t)q : s + (int64_t)q;", "return s + (int64_t)q;"),
    ("sum of |d| as N", "if (d > n) n = d;", "n += d;"),
    ("loop from k = 1 as printed in Fig. 3",
     "if (g < cap)\n                oracle_voxel(seg, k, xyz + 3 * g);",
     "if (k == 0) continue;\n            if (g < cap)\n                oracle_voxel(seg, k, xyz + 3 * g);"),
    ("32-bit list drops the start voxel",
     "if (g < cap) out[g] = pack32(v);",
     "if (k == 0) continue;\n            if (g < cap) out[g] = pack32(v);"),
    ("y and z swapped in the 32-bit word", "((uint32_t)v[1] << 10) | ((uint32_t)v[2] << 20)",
     "((uint32_t)v[2] << 10) | ((uint32_t)v[1] << 20)"),
    ("wrong 64-bit field width", "((uint64_t)v[1] << 21) | ((uint64_t)v[2] << 42)",
     "((uint64_t)v[1] << 20) | ((uint64_t)v[2] << 40)"),
    ("x and y transposed in the volume index", "(v[0] + w * (v[1] + h * v[2]))", "(v[1] + w * (v[0] + h * v[2]))"),
    ("volume stride uses depth", "int64_t w = dims[0], h = dims[1];", "int64_t w = dims[0], h = dims[2];"),
    ("inclusive instead of exclusive scan", "offsets[s] = run;\n        run += counts[s];",
     "run += counts[s];\n        offsets[s] = run;"),
    ("count without the start voxel", "(int32_t)(oracle_steps(segs + 6 * s) + 1)", "(int32_t)(oracle_steps(segs + 6 * s))"),
    ("upper bound inclusive", "v >= dims[c % 3]", "v > dims[c % 3]"),
    ("W taken from E instead of E - S", "(__int128)(E - S) * k", "(__int128)(E) * k"),
    ("bit order reversed in the word", "(uint32_t)1 << (lin % 32)", "(uint32_t)0x80000000u >> (lin % 32)"),
    ("Euclidean length rounded up", "    return oracle_isqrt(sq);", "    return oracle_isqrt(sq) + (oracle_isqrt(sq) * oracle_isqrt(sq) < sq);"),
    ("square root digit step dropped", "            r = (r >> 1) + bit;", "            r = (r >> 1);"),
    ("repeated voxels kept", "if (k > 0 && v[0] == prev[0] && v[1] == prev[1] && v[2] == prev[2]) continue;",
     "if (0) continue;"),
    ("repeat test on x only", "if (k > 0 && v[0] == prev[0] && v[1] == prev[1] && v[2] == prev[2]) continue;",
     "if (k > 0 && v[0] == prev[0]) continue;"),
    ("variant uses N = max|d|", "    return oracle_isqrt(sq);", "    return oracle_steps(seg);"),
    ("slab offset dropped", "w * h * (v[2] - z0)", "w * h * v[2]"),
    ("slab search off by one", "            lo = mid + 1;", "            lo = mid + 1 + (mid == 0);"),
    ("slab search ignores the direction", "int rising = seg[5] >= seg[2];", "int rising = 1;"),
]


def _pins(O):
    """Run every pin; return the names of those that failed."""
    failed = []
    rng = np.random.default_rng(21)
    checks = [
        ("hand_voxels", lambda: P.pin_hand_voxels(O)),
        ("hand_packing", lambda: P.pin_hand_packing(O)),
        ("closed_forms", lambda: P.pin_closed_forms(O)),
        ("scan", lambda: P.pin_scan(O)),
        ("validate", lambda: P.pin_validate(O)),
        ("brute_force", lambda: P.pin_brute_force(O, P.all_pairs(3))),
        ("carry", lambda: P.pin_carry_recurrence(O, P.random_pairs(rng, 50, 40))),
        ("invariants", lambda: P.pin_invariants(O, workloads.config1().segs[:300], (256, 256, 256))),
        ("outputs", lambda: P.pin_outputs_agree(O, workloads.uniform_segments(rng, 50, (13, 7, 5)), (13, 7, 5))),
        ("euclid_hand", lambda: P.pin_euclid_hand(O)),
        ("euclid_isqrt", lambda: P.pin_euclid_isqrt(O)),
        ("euclid_brute_force", lambda: P.pin_euclid_brute_force(O, P.all_pairs(3))),
        ("euclid_invariants", lambda: P.pin_euclid_invariants(O, workloads.config1().segs[:100])),
        ("zslab", lambda: P.pin_zslab(O, workloads.uniform_segments(rng, 200, (40, 12, 24)), (40, 12, 24),
                                      [0, 5, 6, 13, 24])),
    ]
    for name, fn in checks:
        try:
            fn()
        except (AssertionError, ValueError, IndexError):
            failed.append(name)
    return failed


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    return tmp_path_factory.mktemp("oracle_mutants")


def test_unmutated_copy_passes(mutant_dir):
    out = str(mutant_dir / "liboracle_copy.so")
    oracle.build(SRC, out)
    assert _pins(oracle.Oracle(oracle.load(out))) == []


@pytest.mark.parametrize("idx", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(mutant_dir, idx):
    name, orig, planted = MUTANTS[idx]
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site not unique: {orig!r}"
    src = mutant_dir / f"mutant{idx}.c"
    src.write_text(text.replace(orig, planted))
    out = str(mutant_dir / f"liboracle_mutant{idx}.so")
    try:
        oracle.build(str(src), out)
    except subprocess.CalledProcessError:
        pytest.fail(f"mutant {name} does not compile")
    failed = _pins(oracle.Oracle(oracle.load(out)))
    assert failed, f"no pin caught the planted mistake: {name}"
