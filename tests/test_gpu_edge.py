"""Degenerate and extreme inputs of the method, CUDA path against the FP64
oracle: needle-like footprints (the FP64 conic recomputation), one Gaussian
covering the whole image, thousands of Gaussians stacked on one tile (many
chunks per tile, both schedules) and the maximum number of views per call."""
import numpy as np
import pytest

import oracle
import wsr_scenes as ws
from tests.gpu_util import TIE, GRAD_TOL, add_envelopes, assert_image_parity, grad_envelope, grad_excess

pytestmark = pytest.mark.gpu


def _concat(a, b):
    """Scene with the Gaussians of a followed by those of b (same SH layout)."""
    return ws.Scene(*(np.concatenate([getattr(a, k), getattr(b, k)]) for k in
                      ("means", "log_scales", "quats", "sh", "opacity", "lc_v")),
                    a.sh_degree, a.view_dependent_opacity)


def _check_forward(scene, cams, w, tile=(16, 16), persistent=False):
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer
    g = Gaussians.from_scene(scene)
    wpar = torch.tensor(w.as_array(), device="cuda")
    r = Renderer(cams, tile=tile, persistent=persistent)
    st = r.forward(g, w.kind, wpar)
    torch.cuda.synchronize()
    rgb = st.rgb.cpu().numpy()
    o = 0
    for cam in cams:
        m = cam.width * cam.height
        ref = oracle.render(scene, cam, w, amb_tau=TIE)
        assert_image_parity(rgb[o:o + m].reshape(cam.height, cam.width, 3), ref, what=(cam.width, cam.height))
        o += m
    return r, g, wpar, st


def _check_gradients(scene, cams, w, r, g, wpar, st, keys=("means", "log_scales", "quats", "sh", "opacity")):
    import torch
    rng = np.random.default_rng(11)
    Gs = [rng.normal(size=(c.height, c.width, 3)).astype(np.float32) for c in cams]
    G = torch.from_numpy(np.concatenate([x.reshape(-1, 3) for x in Gs])).cuda()
    out = r.backward(g, w.kind, wpar, st, G)
    torch.cuda.synchronize()
    env = None
    for cam, Gv in zip(cams, Gs):
        e = grad_envelope(scene, cam, w, Gv.astype(np.float64))
        env = e if env is None else add_envelopes(env, e)
    for k in keys:
        ex = grad_excess(out[k].cpu().numpy(), env, k)
        assert ex <= GRAD_TOL, (k, ex)
    return out


def test_needle_footprints_take_the_fp64_conic_and_match():
    """Long thin Gaussians seen obliquely: det(Sigma_2D) < 1e-3 a c, where the
    conic is recomputed in FP64; forward and gradients against the oracle."""
    rng = np.random.default_rng(21)
    needles = ws.random_scene(600, 22, sh_degree=1, vd_opacity=False, box=0.8)
    needles.log_scales[:, 0] = rng.uniform(np.log(0.5), np.log(1.5), 600).astype(np.float32)
    needles.log_scales[:, 1:] = np.float32(np.log(1e-3))
    back = ws.random_scene(2000, 23, sh_degree=1, vd_opacity=False, box=1.2, log_scale_mu=-3.3)
    sc = _concat(needles, back)
    cam = ws.look_at((0.4, 0.3, -3.5), width=256, height=192).rounded()
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.9, (0.1, 0.2, 0.1))
    P = oracle.project(sc, cam, w)
    a, b, c = P["cov2d"][:, 0], P["cov2d"][:, 1], P["cov2d"][:, 2]
    fp64 = P["visible"] & ((a * c - b * b) < 1e-3 * a * c)
    assert fp64.sum() >= 20, int(fp64.sum())           # the FP64 path is exercised
    r, g, wpar, st = _check_forward(sc, [cam], w)
    _check_gradients(sc, [cam], w, r, g, wpar, st)


def test_one_gaussian_covering_the_whole_image():
    big = ws.random_scene(1, 31, sh_degree=2, vd_opacity=True, box=0.1)
    big.means[:] = 0.0
    big.log_scales[:] = np.float32(np.log(4.0))         # far beyond the view at distance 4
    small = ws.random_scene(500, 32, sh_degree=2, vd_opacity=True, box=1.0, log_scale_mu=-3.0)
    sc = _concat(big, small)
    cam = ws.look_at((0.0, 0.0, -4.0), width=160, height=120).rounded()
    w = ws.WeightParams(ws.LC, 8.0, 0.0, 0.8, (0.2, 0.2, 0.2))
    P = oracle.project(sc, cam, w)
    assert P["rx"][0] > 160 and P["ry"][0] > 120         # its footprint holds every pixel
    for tile in [(16, 16), (32, 8)]:
        r, g, wpar, st = _check_forward(sc, [cam], w, tile=tile)
        _check_gradients(sc, [cam], w, r, g, wpar, st, keys=("means", "log_scales", "quats", "sh", "opacity",
                                                             "lc_v"))


@pytest.mark.parametrize("persistent", [False, True])
def test_thousands_of_gaussians_on_one_tile(persistent):
    """20,000 Gaussians of ~2-pixel footprints stacked where two 16x16 tiles
    meet (each tile holds ~20,000: 157 chunks of 128) next to a sparse
    background."""
    stack = ws.random_scene(20_000, 42, sh_degree=0, vd_opacity=False, box=0.01, log_scale_mu=-5.5,
                            log_scale_sd=0.2)
    stack.means[:] += np.array([0.05, 0.05, 0.0], np.float32)
    back = ws.random_scene(3000, 43, sh_degree=0, vd_opacity=False, box=1.0, log_scale_mu=-3.5)
    sc = _concat(stack, back)
    cam = ws.look_at((0.0, 0.0, -3.0), width=96, height=80).rounded()
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 1.0, (0.0, 0.0, 0.0))
    r, g, wpar, st = _check_forward(sc, [cam], w, persistent=persistent)
    counts = np.diff(st.tile_offsets.cpu().numpy().astype(np.int64))
    assert counts.max() >= 10_000, int(counts.max())    # many chunks in one tile
    _check_gradients(sc, [cam], w, r, g, wpar, st)


def test_thirty_two_views_in_one_call():
    sc = ws.random_scene(4000, 51, sh_degree=3, vd_opacity=True, clusters=8, box=1.2, log_scale_mu=-3.4)
    rng = np.random.default_rng(52)
    sizes = [(int(rng.integers(8, 70)), int(rng.integers(5, 50))) for _ in range(32)]
    cams = [c.rounded() for c in ws.sphere_cameras(32, 4.5, sizes)]
    w = ws.WeightParams(ws.LC, 9.0, 0.0, 0.7, (0.1, 0.3, 0.2))
    for persistent in (False, True):
        r, g, wpar, st = _check_forward(sc, cams, w, tile=(8, 8), persistent=persistent)
    _check_gradients(sc, cams, w, r, g, wpar, st, keys=("means", "log_scales", "quats", "sh", "opacity", "lc_v"))


@pytest.mark.parametrize("persistent", [False, True])
def test_degenerate_image_shapes(persistent):
    """Views of 1x1, one row, one column and a 17x3 strip in one call: ragged
    tiles in both directions, forward and gradients against the oracle."""
    sc = ws.random_scene(2000, 61, sh_degree=2, vd_opacity=True, box=1.0, log_scale_mu=-2.6)
    sizes = [(1, 1), (57, 1), (1, 43), (17, 3)]
    cams = [ws.look_at((0.3 * k, 0.2, -3.0), width=wd, height=ht).rounded() for k, (wd, ht) in enumerate(sizes)]
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.7, (0.2, 0.1, 0.3))
    for tile in [(16, 16), (8, 8)]:
        r, g, wpar, st = _check_forward(sc, cams, w, tile=tile, persistent=persistent)
    _check_gradients(sc, cams, w, r, g, wpar, st)
