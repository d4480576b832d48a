"""The C-ABI library builds for sm_103a, loads on a machine without a GPU, and
exports every entry point that include/vox.h declares (no compute calls)."""

import os
import re
import subprocess

import pytest

from paper_2009_09500_gb300 import build, vox

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vox.h")


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(vox_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return vox.load()


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("vox_count", "vox_generate", "vox_workspace_size", "vox_strerror", "vox_generate_host"):
        assert must in names
    assert set(names) == set(vox.EXPORTED), (names, vox.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in declared_functions():
        assert name in exported, name


def test_host_only_queries(lib):
    assert vox.vox_workspace_size(0) > 0
    assert vox.vox_workspace_size(1 << 20) >= 8 * (1 << 20)
    assert vox.vox_mask_words((1024, 1024, 1024)) == (1 << 30) // 32
    assert vox.vox_mask_words((13, 7, 5)) == (13 * 7 * 5 + 31) // 32
    assert vox.vox_mask_words((0, 7, 5)) == 0
    assert vox.vox_scan_tile_segments() == 2048
    assert vox.strerror(vox.ERR_TIMEOUT) == "bounded in-kernel wait expired"
    assert vox.strerror(12345) == "unknown status"
    arena = vox.vox_host_arena_size(1000, (256, 256, 256), vox.OUT_LIST32 | vox.OUT_BITMASK, 5000)
    assert arena >= 1000 * 24 + 5000 * 4 + (1 << 24) // 8


def test_library_is_sm103a_only():
    cmd = build.nvcc_command()
    assert "arch=compute_103a,code=sm_103a" in cmd
    assert not any("sm_90" in c or "sm_100" in c for c in cmd)


def test_binding_has_no_oracle_import():
    """The product path never reaches the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2009_09500_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_brick_shape_queries(lib):
    """The brick geometry follows the documented rule (host-only queries)."""
    assert vox.vox_brick_shape((1024, 1024, 1024)) == ((256, 64, 64), (4, 16, 16))
    assert vox.vox_mask_words_bricked((1024, 1024, 1024)) == (1 << 30) // 32
    assert vox.vox_brick_shape((96, 40, 17)) == ((64, 128, 128), (2, 1, 1))
    assert vox.vox_mask_words_bricked((96, 40, 17)) == 2 * 64 * 128 * 128 // 32
    assert vox.vox_brick_shape((32, 7, 5)) == ((32, 256, 128), (1, 1, 1))
    assert vox.vox_mask_words_bricked((13, 7, 5)) == 0
    with pytest.raises(vox.VoxError):
        vox.vox_brick_shape((13, 7, 5))
