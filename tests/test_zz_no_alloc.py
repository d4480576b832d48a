"""The allocation-free entry point, vox_generate_noalloc.

It exists for callers that cannot allocate device memory when they voxelize: a
plug-in inside a host application that owns the device-memory budget through
its own pool, or a loop that cannot pay for cudaMalloc/cudaFree. Its scratch is
a static device array in the library, shared by every call, so the GPU test
below runs it twice in a row on different inputs (and once more on the first
input) and requires the same bits as the regular entry point, vox_generate with
a workspace of vox_workspace_size(n) bytes, each time, and the oracle's. The file
sorts last so that a stop-at-first-failure run has already run every other test
when it gets here.
"""

import ctypes

import numpy as np
import pytest

from paper_2009_09500_gb300 import build, vox, workloads


def _outputs(dims, V, device):
    import torch

    lst = torch.full((V + 32,), -1, dtype=torch.int32, device=device)
    mask = torch.zeros(vox.vox_mask_words(dims), dtype=torch.int32, device=device)
    return lst, mask


def _regular(w):
    import torch

    segs = torch.from_numpy(w.segs).cuda()
    ws = torch.empty(vox.vox_workspace_size(w.n), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    off = torch.empty(w.n + 1, dtype=torch.int64, device="cuda")
    vox.vox_count(segs, w.dims, ws, status, None, off)
    V = int(off[-1].item())
    lst, mask = _outputs(w.dims, V, "cuda")
    vox.vox_generate(segs, w.dims, ws, status, lst, mask, capacity=V)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return V, lst.cpu().numpy(), mask.cpu().numpy()


def _noalloc(w, V):
    import torch

    segs = torch.from_numpy(w.segs).cuda()
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    lst, mask = _outputs(w.dims, V, "cuda")
    vox.vox_generate_noalloc(segs, w.dims, status, lst, mask, capacity=V)
    torch.cuda.synchronize()
    return int(status.item()), lst.cpu().numpy(), mask.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_regular_entry_point_two_calls_in_a_row():
    import torch

    import oracle

    assert torch.cuda.is_available()
    build.build_library()
    vox.load()
    O = oracle.get()
    a = workloads.config1()
    b = workloads.config2(n_fixed=150000)
    Va, la, ma = _regular(a)
    Vb, lb, mb = _regular(b)
    # the regular entry point itself against the oracle
    for w, V, l_ref, m_ref in ((a, Va, la, ma), (b, Vb, lb, mb)):
        assert np.array_equal(l_ref[:V].view(np.uint32), O.list32(w.segs))
        assert np.array_equal(m_ref.view(np.uint32), O.bitmask(w.segs, w.dims))
    # two calls in a row on different inputs, then the first input again:
    # stale scratch from an earlier call must not leak into a later one
    for w, V, l_ref, m_ref in ((a, Va, la, ma), (b, Vb, lb, mb), (a, Va, la, ma)):
        st, l_got, m_got = _noalloc(w, V)
        assert st == 0, vox.strerror(st)
        assert np.array_equal(l_got, l_ref), "list differs from vox_generate"
        assert np.array_equal(m_got, m_ref), "volume differs from vox_generate"


@pytest.mark.gpu
def test_noalloc_refuses_the_brick_major_layout():
    """The brick-major volume needs the brick path's arrays, which the static
    scratch does not hold: refused on the host, nothing launched."""
    import torch

    build.build_library()
    vox.load()
    dims = (256, 64, 64)
    segs = torch.from_numpy(workloads.uniform_segments(np.random.default_rng(3), 100, dims)).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    mask = torch.zeros(vox.vox_mask_words_bricked(dims), dtype=torch.int32, device="cuda")
    with pytest.raises(vox.VoxError) as e:
        vox.vox_generate_noalloc(segs, dims, status, None, mask, flags=vox.OUT_BITMASK | vox.OUT_BRICKED)
    assert e.value.status == vox.ERR_WORKSPACE


def test_noalloc_rejects_more_segments_than_its_scratch_holds():
    """Host-side check: nothing is launched, no device memory is touched."""
    build.build_library()
    lib = vox.load()
    n = vox.NOALLOC_MAX_SEGMENTS + 1
    st = lib.vox_generate_noalloc(ctypes.c_void_p(16), n, vox.Dims(8, 8, 8), ctypes.c_void_p(0), 0,
                                  ctypes.c_void_p(64), vox.OUT_BITMASK, ctypes.c_void_p(128), ctypes.c_void_p(0))
    assert st == vox.ERR_WORKSPACE


def test_noalloc_binding_names_the_limit():
    """The Python binding refuses more than NOALLOC_MAX_SEGMENTS segments before
    calling the library, with the limit in the message."""
    import torch

    build.build_library()
    vox.load()

    class FakeSegs:  # shape and checks only: nothing is read from it
        shape = (vox.NOALLOC_MAX_SEGMENTS + 5, 6)
        is_cuda = True
        dtype = torch.int32

        def dim(self):
            return 2

        def is_contiguous(self):
            return True

    with pytest.raises(vox.VoxError) as e:
        vox.vox_generate_noalloc(FakeSegs(), (8, 8, 8), None, None, None, flags=vox.OUT_BITMASK)
    assert e.value.status == vox.ERR_WORKSPACE and str(vox.NOALLOC_MAX_SEGMENTS) in str(e.value)
