"""Autotuner host logic (CPU): workload classes, the JSON cache, and the
process-wide tuning of the C ABI (host-only calls)."""

import json

from paper_2009_09500_gb300 import autotune, build, vox


def setup_module(_):
    build.build_library()
    vox.load()


def test_workload_class_buckets():
    a = autotune.workload_class(1 << 20, 64 << 20, (1024, 1024, 1024), 5)
    b = autotune.workload_class((1 << 20) + 1000, (64 << 20) + 5000, (1024, 1024, 1024), 5)
    c = autotune.workload_class(1 << 22, 1 << 31, (4096,) * 3, 4)
    assert a == b and a != c
    assert "w321" in a and "w320" in autotune.workload_class(10, 10, (13, 7, 5), 4)


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "t.json")
    assert autotune.load_cache(p) == {}
    autotune.save_cache({"gpu|cls": {"params": {"run_len": 16}}}, p)
    assert autotune.load_cache(p)["gpu|cls"]["params"]["run_len"] == 16
    json.loads(open(p).read())


def test_tuning_set_get_and_sanitised():
    try:
        vox.vox_set_tuning(16, vox.VOLUME_ATOMIC, 2, 1)
        assert vox.vox_get_tuning() == {"run_len": 16, "volume_path": 1, "ctas_per_sm": 2, "list_runs": 1}
        vox.vox_set_tuning(32, vox.VOLUME_ATOMIC_WARP, 0, 2)
        assert vox.vox_get_tuning() == {"run_len": 32, "volume_path": 2, "ctas_per_sm": 0, "list_runs": 2}
        vox.vox_set_tuning(7, 9, -3, 5)
        assert vox.vox_get_tuning() == {"run_len": 0, "volume_path": 0, "ctas_per_sm": 0, "list_runs": 0}
    finally:
        vox.vox_reset_tuning()
    assert vox.vox_get_tuning() == {"run_len": 0, "volume_path": 0, "ctas_per_sm": 0, "list_runs": 0}


def test_candidates_cover_the_knobs():
    keys = {(c["run_len"], c["volume_path"], c["ctas_per_sm"], c["list_runs"]) for c in autotune.CANDIDATES}
    assert {16, 32, 64} == {k[0] for k in keys} and {0, 1, 2} == {k[1] for k in keys} and len(keys) == 22
    assert {0, 1, 2} == {k[3] for k in keys}
