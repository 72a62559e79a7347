"""Sort-free tile binning (Sec. 4.1: no depth sort, each Gaussian listed in
every tile its footprint reaches), checked as sets against FP64 geometry from
the oracle's projection.

What is unique: the (Gaussian, tile) pairs where some pixel centre of the tile
has q <= 9 must all be listed (pairs within 1e-4 of the cutoff are ties and
may go either way).  What is free: the order inside a tile, and extra pairs
the kernel keeps for safety; each extra must still be near the footprint --
a pixel-centre column of the tile meets the ellipse's x-extent within the
tile's band of pixel-centre rows, widened by a small fraction of its size.
"""
import numpy as np
import pytest

import oracle
import wsr_scenes as ws

pytestmark = pytest.mark.gpu

CUT = 9.0


def _scene():
    rng = np.random.default_rng(71)
    base = ws.random_scene(2500, 72, sh_degree=1, vd_opacity=False, clusters=6, box=1.2, log_scale_mu=-3.6)
    needles = ws.random_scene(300, 73, sh_degree=1, vd_opacity=False, box=0.9)
    needles.log_scales[:, 0] = rng.uniform(np.log(0.2), np.log(1.2), 300).astype(np.float32)
    needles.log_scales[:, 1:] = np.float32(np.log(2e-3))
    big = ws.random_scene(8, 74, sh_degree=1, vd_opacity=False, box=0.6, log_scale_mu=-0.7, log_scale_sd=0.3)
    parts = (base, needles, big)
    return ws.Scene(*(np.concatenate([getattr(p, k) for p in parts]) for k in
                      ("means", "log_scales", "quats", "sh", "opacity", "lc_v")), 1, False)


def _truth(P, W, H, tw, th):
    """Per visible Gaussian: the set of tiles holding a pixel centre with
    q <= 9 (1 - 1e-4), and a function telling whether a tile is allowed."""
    must, allowed = {}, {}
    for i in np.flatnonzero(P["visible"]):
        mx, my = P["mean2d"][i]
        a, b, c = P["cov2d"][i]
        det = a * c - b * b
        A, B, C = c / det, -b / det, a / det                 # conic: q = A dx^2 + 2 B dx dy + C dy^2
        ex, ey = np.sqrt(CUT * a), np.sqrt(CUT * c)           # extents of q <= 9
        x0, x1 = max(int(np.ceil(mx - ex - 0.5)), 0), min(int(np.floor(mx + ex - 0.5)), W - 1)
        y0, y1 = max(int(np.ceil(my - ey - 0.5)), 0), min(int(np.floor(my + ey - 0.5)), H - 1)
        if x0 > x1 or y0 > y1:
            must[i] = set()
        else:
            dx = np.arange(x0, x1 + 1) + 0.5 - mx
            dy = np.arange(y0, y1 + 1) + 0.5 - my
            q = A * dx[None, :] ** 2 + 2 * B * dx[None, :] * dy[:, None] + C * dy[:, None] ** 2
            yy, xx = np.nonzero(q <= CUT * (1 - 1e-4))
            must[i] = set(zip(((yy + y0) // th).tolist(), ((xx + x0) // tw).tolist()))
        allowed[i] = (mx, my, A, B, C, ex, ey)
    return must, allowed


def _allowed(g, ty, tx, W, H, tw, th):
    mx, my, A, B, C, ex, ey = g
    # the kernel's footprint is q <= 9 (1 + 1e-4) + 1.4e-4 (it keeps every pixel centre whose FP32 q
    # reaches the cutoff); taken here as q <= CUT_K.  Near a row where the ellipse is tangent, that
    # widening moves the x-extent by about sqrt(9e-4 / A), more than a pixel fraction on big footprints.
    cut_k = CUT * 1.0002 + 5e-4
    ex, ey = ex * np.sqrt(cut_k / CUT), ey * np.sqrt(cut_k / CUT)
    # the tile's band of pixel-centre rows, inside the footprint's y-extent (the kernel pads
    # the extents by a relative 1e-4 and 0.01 pixel: rows that close are allowed too)
    sy = 1e-3 * ey + 0.02
    ya = max(ty * th + 0.5, my - ey - sy) - my
    yb = min(min(ty * th + th, H) - 0.5, my + ey + sy) - my
    if ya > yb + 1e-9:
        return False
    # x-extent of {q <= 9} over dy in [ya, yb]: for fixed dy, dx = (-B dy +- sqrt(B^2 dy^2 - A (C dy^2 - 9))) / A
    dys = np.linspace(ya, yb, 257)
    disc = np.maximum(B * B * dys ** 2 - A * (C * dys ** 2 - cut_k), 0.0)
    xl = np.min((-B * dys - np.sqrt(disc)) / A)
    xr = np.max((-B * dys + np.sqrt(disc)) / A)
    d = 5e-3 * ex + 0.05 + (yb - ya) / 256 * abs(B / A)       # margin plus the sampling step in dy
    cols = np.arange(tx * tw, min(tx * tw + tw, W)) + 0.5 - mx
    return bool(np.any((cols >= xl - d) & (cols <= xr + d)))


def _check_lists(sc, cam, w, tile, persistent=False):
    """Bins one view and checks its lists against the footprint geometry;
    returns the rendered image."""
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer
    g = Gaussians.from_scene(sc)
    r = Renderer([cam], tile=tile, persistent=persistent)
    st = r.forward(g, w.kind, torch.tensor(w.as_array(), device="cuda"))
    torch.cuda.synchronize()
    off = st.tile_offsets.cpu().numpy().astype(np.int64)
    lst = st.tile_list.cpu().numpy().astype(np.int64)
    tw, th = tile
    tiles_x = -(-cam.width // tw)
    assert len(off) - 1 == tiles_x * -(-cam.height // th)
    assert off[0] == 0 and np.all(np.diff(off) >= 0)
    listed = {}
    for t in np.flatnonzero(np.diff(off)):
        ids = lst[off[t]:off[t + 1]]
        assert len(np.unique(ids)) == len(ids), t                # no pair twice
        for i in ids.tolist():
            listed.setdefault(i, set()).add((t // tiles_x, t % tiles_x))
    P = oracle.project(sc, cam, w)
    must, allowed = _truth(P, cam.width, cam.height, tw, th)
    n_must = sum(len(s) for s in must.values())
    assert n_must > 5000
    for i, s in must.items():
        missing = s - listed.get(i, set())
        assert not missing, (i, sorted(missing)[:5])
    extra = 0
    for i, s in listed.items():
        assert i in allowed, i                                   # culled Gaussians are never listed
        for ty, tx in s - must.get(i, set()):
            assert _allowed(allowed[i], ty, tx, cam.width, cam.height, tw, th), (i, ty, tx)
            extra += 1
    assert extra <= 0.03 * n_must, (extra, n_must)
    return st.rgb.cpu().numpy()


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8), (16, 8)])
def test_tile_lists_hold_exactly_the_footprint_tiles(tile):
    cam = ws.look_at((0.3, -0.2, -3.6), width=200, height=150).rounded()
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.9, (0.1, 0.2, 0.1))
    _check_lists(_scene(), cam, w, tile)


@pytest.mark.parametrize("height", [1024, 1032])
def test_tile_lists_and_order_around_the_one_block_scan_limit(height):
    """The scan and the persistent schedule's tile order run in one block up
    to 32768 tiles and in three passes beyond: 8x8 tiles on 2048 x 1024
    (32768 tiles) and 2048 x 1032 (33024).  The lists hold the footprint
    tiles, and the persistent schedule (which walks the tile order) renders
    the image the one-block-per-tile schedule does."""
    cam = ws.look_at((0.3, -0.2, -2.2), width=2048, height=height).rounded()
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.9, (0.1, 0.2, 0.1))
    sc = _scene()
    a = _check_lists(sc, cam, w, (8, 8), persistent=True)
    b = _check_lists(sc, cam, w, (8, 8), persistent=False)
    assert np.abs(a - b).max() <= 2e-6


def test_tile_lists_of_several_uneven_views_in_one_call():
    """Three views of uneven, ragged sizes binned in one call: view v's tiles
    follow view v-1's, and its list entries are record indices v n + i."""
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer
    sc = _scene()
    cams = [ws.look_at((0.3, -0.2, -3.6), width=200, height=150).rounded(),
            ws.look_at((-1.2, 0.4, -3.2), width=67, height=45).rounded(),
            ws.look_at((2.0, 1.0, -2.8), width=130, height=97).rounded()]
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.9, (0.1, 0.2, 0.1))
    g = Gaussians.from_scene(sc)
    tw, th = 16, 16
    r = Renderer(cams, tile=(tw, th), persistent=True)
    st = r.forward(g, w.kind, torch.tensor(w.as_array(), device="cuda"))
    torch.cuda.synchronize()
    off = st.tile_offsets.cpu().numpy().astype(np.int64)
    lst = st.tile_list.cpu().numpy().astype(np.int64)
    n = sc.n
    t0 = 0
    for v, cam in enumerate(cams):
        tiles_x, tiles_y = -(-cam.width // tw), -(-cam.height // th)
        listed = {}
        for t in range(tiles_x * tiles_y):
            ids = lst[off[t0 + t]:off[t0 + t + 1]]
            assert len(np.unique(ids)) == len(ids)
            assert np.all(ids // n == v), (v, t)                 # only this view's records
            for i in (ids % n).tolist():
                listed.setdefault(i, set()).add((t // tiles_x, t % tiles_x))
        P = oracle.project(sc, cam, w)
        must, allowed = _truth(P, cam.width, cam.height, tw, th)
        n_must = sum(len(s) for s in must.values())
        assert n_must > 500, (v, n_must)
        for i, s in must.items():
            assert not (s - listed.get(i, set())), (v, i)
        extra = 0
        for i, s in listed.items():
            assert i in allowed, (v, i)
            for ty, tx in s - must.get(i, set()):
                assert _allowed(allowed[i], ty, tx, cam.width, cam.height, tw, th), (v, i, ty, tx)
                extra += 1
        assert extra <= 0.03 * n_must, (v, extra, n_must)
        t0 += tiles_x * tiles_y
    assert t0 == len(off) - 1


def test_device_total_inside_a_captured_graph():
    """wsr_bin's device total (total_dev) inside a captured CUDA graph: each
    replay writes the true instance count of that replay's records, with no
    host read in the graph, including a replay whose list overflows (the
    total then exceeds the capacity and tells the caller how far to grow)."""
    import torch

    from paper_2410_18931_gb300 import Gaussians, Renderer
    from paper_2410_18931_gb300 import _abi as A
    sc = _scene()
    cam = ws.look_at((0.1, -0.2, -3.0), width=200, height=150).rounded()
    w = ws.default_weight(ws.EXP)
    g = Gaussians.from_scene(sc)
    wpar = torch.tensor(w.as_array(), device="cuda")
    r = Renderer([cam], tile=(16, 16))
    st = r.alloc_state(g.n)
    r.wsr_project(g, w.kind, wpar, st.records)
    r.wsr_bin_count(st.records, g.n, st.tile_offsets)
    total = r.wsr_bin_total()
    tile_list = torch.empty(total + 16, dtype=torch.int32, device="cuda")
    total_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    records = st.records.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):                     # warm-up call outside the capture
        r.wsr_bin(records, g.n, st.tile_offsets, tile_list, stream=side, total_dev=total_dev)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        r.wsr_bin(records, g.n, st.tile_offsets, tile_list, total_dev=total_dev)
    total_dev.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert int(total_dev.item()) == total
    # the same graph on records with every Gaussian doubled in place: half the Gaussians moved onto
    # the other half's positions are binned twice as often where they overlap
    half = g.n // 2
    records.view(-1, 12)[half:2 * half] = records.view(-1, 12)[:half]
    total_dev.zero_()
    graph.replay()
    err = r.wsr_check()                               # read before the recount below clears it
    got = int(total_dev.item())
    r.wsr_bin_count(records, g.n, st.tile_offsets)
    expect = r.wsr_bin_total()
    assert got == expect and expect != total
    assert (err == A.WSR_ERR_CAPACITY) == (expect > tile_list.numel())


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8), (16, 8)])
def test_work_counts_of_the_render_kernels(tile):
    """wsr_count_pairs: the pairs with q <= 9 agree with the oracle's count (up
    to ties decided differently in FP32, far fewer than 0.1%); the forward's
    evaluated slots and the backward's walked pixels hold every pair and fit
    in the tile instances' pixels; the forward's slots come in whole warps
    (32 threads of PX x 2 pixels) and the backward's in rows of half a tile
    width or a whole one."""
    import torch

    from paper_2410_18931_gb300 import Gaussians, Renderer
    sc = _scene()
    cam = ws.look_at((0.1, -0.2, -3.0), width=200, height=150).rounded()
    w = ws.default_weight(ws.EXP)
    g = Gaussians.from_scene(sc)
    r = Renderer([cam], tile=tile)
    st = r.forward(g, w.kind, torch.tensor(w.as_array(), device="cuda"))
    pairs, fwd_slots, bwd_pixels = r.wsr_count_pairs(st)
    instances = r.wsr_bin_total()
    ref = oracle.render(sc, cam, w)["pairs"]
    assert abs(pairs - ref) <= 1e-3 * ref, (pairs, ref)
    cap = instances * tile[0] * tile[1]
    assert pairs <= fwd_slots <= cap and pairs <= bwd_pixels <= cap
    px = 1 if tile == (8, 8) else 2
    assert fwd_slots % (32 * px * 2 if tile != (8, 8) else 64) == 0
    assert bwd_pixels % (tile[0] // 2) == 0
