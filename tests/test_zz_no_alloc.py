"""wsr_bin_static: binning for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc once they run (a frame loop in a host
application that forbids device allocation after start-up, since an
allocation can synchronise the device; or a plug-in given only its input and
output buffers), so they cannot provide a workspace.  This entry point keeps
its scratch in a fixed device array inside the library.  The tests call it
through the C ABI several times in a row, on scenes and views of different
sizes, and check each result against wsr_bin (which uses a caller-provided
workspace): tile offsets and instance totals bit-exact, each tile's list equal
as a set (the order inside a tile is arbitrary by design), and the rendered
image equal within float rounding.  They also check that repeated calls change
neither the device's free memory nor torch's allocator statistics, and that
the device status output reports a list that was too small and, in the
deterministic mode, a tile too long to sort.  The file name makes pytest
collect it last.
"""
import ctypes

import numpy as np
import pytest

import wsr_scenes as ws

pytestmark = pytest.mark.gpu


def _case(seed, n, width, height, tile, deterministic=False):
    import torch

    from paper_2410_18931_gb300 import Gaussians, Renderer
    sc = ws.random_scene(n, seed, sh_degree=2, vd_opacity=True, clusters=8, box=1.5, log_scale_mu=-3.5)
    cam = ws.look_at((0.2, -0.1, -4.0), width=width, height=height).rounded()
    w = ws.default_weight(ws.LC)
    g = Gaussians.from_scene(sc)
    wpar = torch.tensor(w.as_array(), device="cuda")
    r = Renderer([cam], tile=tile, deterministic=deterministic)
    st = r.alloc_state(g.n)
    r.wsr_project(g, w.kind, wpar, st.records)
    r.wsr_bin_count(st.records, g.n, st.tile_offsets)
    total = r.wsr_bin_total()
    st.tile_list = torch.empty(total + 64, dtype=torch.int32, device="cuda")
    r.wsr_bin(st.records, g.n, st.tile_offsets, st.tile_list)
    assert r.wsr_check() == 0
    return r, g, w, wpar, st, total


def _bin_static(r, st, capacity, outputs=None):
    """One call through the C ABI; ``outputs`` (offsets, list, total, status) are reused when given."""
    import torch

    from paper_2410_18931_gb300 import _abi as A
    lib = A.load()
    if outputs is None:
        outputs = (torch.full_like(st.tile_offsets, -1),
                   torch.full((max(capacity, 1),), -1, dtype=torch.int32, device="cuda"),
                   torch.zeros(1, dtype=torch.int64, device="cuda"),
                   torch.full((1,), -1, dtype=torch.int32, device="cuda"))
    offsets, tile_list, total, dstatus = outputs
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = lib.wsr_bin_static(ctypes.c_void_p(st.records.data_ptr()), st.n, r.cams_c, r.n_cams,
                                ctypes.byref(r.tiles_c), ctypes.c_void_p(offsets.data_ptr()),
                                ctypes.c_void_p(tile_list.data_ptr()), capacity,
                                ctypes.c_void_p(total.data_ptr()), ctypes.c_void_p(dstatus.data_ptr()), stream)
    torch.cuda.synchronize()
    return status, offsets, tile_list, int(total.item()), int(dstatus.item())


def _segments(offsets, tile_list):
    off = offsets.cpu().numpy().astype(np.int64)
    lst = tile_list.cpu().numpy()
    return [np.sort(lst[off[t]:off[t + 1]]) for t in range(off.size - 1)]


@pytest.mark.parametrize("order", [(0, 1, 0), (1, 0, 1)])
def test_bin_static_matches_bin_on_consecutive_calls(order):
    cases = [dict(seed=3, n=60_000, width=640, height=360, tile=(16, 16)),
             dict(seed=4, n=20_000, width=200, height=120, tile=(8, 8))]
    for k in order:
        r, g, w, wpar, st, total = _case(**cases[k])
        status, offsets, tile_list, tot, dstatus = _bin_static(r, st, total + 64)
        assert status == 0 and dstatus == 0
        assert tot == total
        assert np.array_equal(offsets.cpu().numpy(), st.tile_offsets.cpu().numpy())
        for a, b in zip(_segments(offsets, tile_list), _segments(st.tile_offsets, st.tile_list)):
            assert np.array_equal(a, b)
        # the image rendered from either list agrees within float rounding
        import torch
        rgb_a = st.rgb.clone()
        r.wsr_render_fwd(st.records, g.n, st.tile_offsets, st.tile_list, w.kind, wpar, rgb_a, st.den)
        rgb_b = torch.empty_like(rgb_a)
        den_b = torch.empty_like(st.den)
        r.wsr_render_fwd(st.records, g.n, offsets, tile_list, w.kind, wpar, rgb_b, den_b)
        torch.cuda.synchronize()
        assert (rgb_a - rgb_b).abs().max().item() <= 2e-6


def test_bin_static_overflow_reports_true_total_and_stays_in_bounds():
    r, g, w, wpar, st, total = _case(seed=5, n=30_000, width=320, height=200, tile=(16, 16))
    from paper_2410_18931_gb300 import _abi as A
    cap = total // 2
    status, offsets, tile_list, tot, dstatus = _bin_static(r, st, cap)
    assert status == 0
    assert dstatus == A.WSR_ERR_CAPACITY
    assert tot == total
    off = offsets.cpu().numpy().astype(np.int64)
    assert off.max() <= cap and np.all(np.diff(off) >= 0)


def test_bin_static_rejects_too_many_tiles():
    import torch

    from paper_2410_18931_gb300 import _abi as A
    lib = A.load()
    cams, n = A.make_cameras([ws.look_at((0, 0, -5), width=4096, height=2160)])
    t8 = A.tiles(8, 8)      # 512 x 270 = 138,240 tiles > WSR_BIN_STATIC_MAX_TILES
    assert lib.wsr_num_tiles(cams, n, ctypes.byref(t8)) > A.WSR_BIN_STATIC_MAX_TILES
    dummy = torch.empty(16, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    status = lib.wsr_bin_static(p, 1, cams, n, ctypes.byref(t8), p, p, 4, None, None, None)
    assert status == A.WSR_ERR_UNSUPPORTED


def test_bin_static_in_the_deterministic_mode_gives_the_sorted_lists():
    """With wsr_tiles.deterministic = 1, wsr_bin_static sorts each tile's list
    by record index, exactly as wsr_bin does with a workspace: offsets and
    lists equal element by element."""
    import torch
    r, g, w, wpar, st, total = _case(37, 20_000, 200, 150, (16, 16), deterministic=True)
    status, offsets, tile_list, tot, dstatus = _bin_static(r, st, total + 64)
    assert status == 0 and dstatus == 0 and tot == total
    assert torch.equal(offsets, st.tile_offsets)
    assert torch.equal(tile_list[:total], st.tile_list[:total])
    off = offsets.cpu().numpy().astype(np.int64)
    lst = tile_list.cpu().numpy().astype(np.int64)
    for t in range(len(off) - 1):
        assert np.all(np.diff(lst[off[t]:off[t + 1]]) > 0), t


def test_bin_static_reports_a_tile_too_long_to_sort():
    """The deterministic mode sorts each tile's list in shared memory, up to
    WSR_DET_MAX_SEGMENT instances; 12,000 Gaussians stacked on one 16x16 tile
    exceed it, and the static entry's device status says so (WSR_ERR_UNSUPPORTED)
    while the call itself, which cannot know before its kernels run, returns
    WSR_OK.  A following call on an ordinary scene reports WSR_OK again: each
    call clears the array's status first."""
    import torch

    from paper_2410_18931_gb300 import Gaussians, Renderer
    from paper_2410_18931_gb300 import _abi as A
    sc = ws.random_scene(12_000, 8, sh_degree=0, vd_opacity=False, clusters=0, box=0.01, log_scale_mu=-5.0,
                         log_scale_sd=0.1)
    # 0.578 units at distance 4 is 8 pixels (fx = 55.4): the stack projects to a tile centre, 24 or 40
    sc.means[:, :2] += np.float32(0.578)
    cam = ws.look_at((0.0, 0.0, -4.0), width=64, height=64).rounded()
    w = ws.default_weight(ws.EXP)
    g = Gaussians.from_scene(sc)
    r = Renderer([cam], tile=(16, 16), deterministic=True)
    st = r.alloc_state(g.n)
    r.wsr_project(g, w.kind, torch.tensor(w.as_array(), device="cuda"), st.records)
    status, offsets, tile_list, tot, dstatus = _bin_static(r, st, 4 * sc.n)
    assert status == A.WSR_OK
    assert np.diff(offsets.cpu().numpy().astype(np.int64)).max() > A.WSR_DET_MAX_SEGMENT
    assert dstatus == A.WSR_ERR_UNSUPPORTED
    r2, g2, w2, wpar2, st2, total2 = _case(seed=9, n=5_000, width=160, height=96, tile=(16, 16), deterministic=True)
    status, _, _, tot2, dstatus = _bin_static(r2, st2, total2 + 16)
    assert status == A.WSR_OK and dstatus == A.WSR_OK and tot2 == total2


def test_bin_static_allocates_nothing():
    """After a first call (which may load the library's kernels), further
    calls leave the device's free memory (cudaMemGetInfo) and torch's
    allocator statistics exactly as they were: the call allocates nothing,
    neither through the CUDA runtime nor through torch.  Every buffer the
    calls use is created before the first measurement."""
    import torch
    r, g, w, wpar, st, total = _case(seed=11, n=40_000, width=480, height=270, tile=(16, 16))
    outputs = (torch.empty_like(st.tile_offsets), torch.empty(total + 64, dtype=torch.int32, device="cuda"),
               torch.empty(1, dtype=torch.int64, device="cuda"), torch.empty(1, dtype=torch.int32, device="cuda"))
    assert _bin_static(r, st, total + 64, outputs)[0] == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = {k: v for k, v in torch.cuda.memory_stats().items() if k.endswith(".current") or "alloc_count" in k}
    for _ in range(4):
        status, _, _, tot, dstatus = _bin_static(r, st, total + 64, outputs)
        assert status == 0 and dstatus == 0 and tot == total
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = {k: v for k, v in torch.cuda.memory_stats().items() if k.endswith(".current") or "alloc_count" in k}
    assert free1 == free0, (free0, free1)
    assert stats1 == stats0
