"""The parallel comparison harness of the full-size GPU tests, on the CPU: the
oracle's own outputs compare clean part by part, and a planted difference in
the compared copy (one list element, one volume bit) is found and located."""

import numpy as np

import oracle_par as OP
from paper_2009_09500_gb300 import workloads


def test_pool_finds_planted_differences(orc):
    w = workloads.config3(n=6000, edge=128)
    off = orc.offsets(orc.count(w.segs))
    lst = orc.list64(w.segs)
    vol = orc.bitmask(w.segs, w.dims)
    lst_bad = lst.copy()
    lst_bad[4321] ^= np.uint64(1)
    vol_bad = vol.copy()
    vol_bad[1000] ^= np.uint32(1 << 7)
    per_plane = 128 * 128 // 32
    with OP.OraclePool(workers=2) as pool:
        sb = pool.buf(w.segs)
        try:
            for data, tag in ((lst, "good"), (lst_bad, "bad")):
                for s0 in range(0, w.n, 2500):
                    s1 = min(w.n, s0 + 2500)
                    b = pool.buf(data[off[s0]:off[s1]])
                    pool.submit((tag, "list", s0), OP.job_list, sb, s0, s1, True, b, int(off[s0]), bufs=[b])
            for z0 in range(0, 128, 48):
                z1 = min(128, z0 + 48)
                parts = [pool.buf(vol[z0 * per_plane:z1 * per_plane]), pool.buf(vol_bad[z0 * per_plane:z1 * per_plane])]
                pool.submit(("v", "slab", z0), OP.job_zslab, sb, w.dims, z0, z1, parts, bufs=parts)
            res = pool.finish()
        finally:
            sb.release()
    lists = {(t[0], t[2]): r for t, r in res if t[1] == "list"}
    assert all(r["bad"] == 0 for (tag, _), r in lists.items() if tag == "good")
    bad = [r for (tag, _), r in lists.items() if tag == "bad" and r["bad"]]
    assert len(bad) == 1 and bad[0]["bad"] == 1 and bad[0]["first"] == [4321]
    slabs = [r for t, r in res if t[1] == "slab"]
    assert all(r["parts"][0]["bad"] == 0 for r in slabs)
    assert sum(r["parts"][1]["bad"] for r in slabs) == 1
    assert sum(r["nonzero"] for r in slabs) == int(np.count_nonzero(vol))


def test_by_value_when_shared_memory_is_short(orc):
    """Buffers carried by value (no shared memory) compare the same way."""
    w = workloads.config1()
    lst = orc.list32(w.segs[:500])
    with OP.OraclePool(workers=1) as pool:
        pool._room = 0
        sb = pool.buf(w.segs[:500])
        b = pool.buf(lst)
        assert sb.shm is None and b.shm is None
        pool.submit(("x", "list"), OP.job_list, sb, 0, 500, False, b, 0, bufs=[b])
        (tag, r), = pool.finish()
    assert r["bad"] == 0
