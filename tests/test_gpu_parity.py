"""CUDA path against the FP64 oracle, element by element (needs a GPU).

Tolerances: forward max abs pixel error 1e-4 plus, for pixels holding a
Gaussian within its FP32 rounding window of the cutoff q = 9 (the oracle's
per-pair bound), the oracle's bound on what deciding those ties the other
way changes; in images of 10,000 pixels or more, at most 0.1% of the pixels
over 1e-4 before that allowance.  Gradients: max error / max magnitude 1e-3
per tensor plus each entry's tie bound.
"""
import numpy as np
import pytest

import oracle
import wsr_scenes as ws
from tests.gpu_util import (FWD_TOL, GRAD_TOL, TIE, add_envelopes, assert_image_parity, compare_image, gpu_render,
                            grad_envelope, grad_excess, rel_err)

pytestmark = pytest.mark.gpu

TILES = [(16, 16), (8, 8), (32, 8), (16, 8)]


def _oracle(scene, cam, weight):
    return oracle.render(scene, cam, weight, amb_tau=TIE)


@pytest.mark.parametrize("tile", TILES)
def test_workload1_forward_all_tiles(tile):
    """1k Gaussians, 128x128, EXP, degree 0: full image, every tile shape."""
    scene, cams, weight, _ = ws.workload(1)
    cam = cams[0].rounded()
    (rgb, den), = gpu_render(scene, [cam], weight, tile=tile)
    ref = _oracle(scene, cam, weight)
    assert_image_parity(rgb, ref, what=tile)
    assert np.abs(den - ref["den"]).max() <= 1e-3 * max(1.0, np.abs(ref["den"]).max())


@pytest.mark.parametrize("kind", [ws.DIR, ws.EXP, ws.LC])
@pytest.mark.parametrize("deg,vd", [(3, True), (1, False), (2, True), (0, True)])
def test_ragged_image_each_weight(kind, deg, vd):
    """20k clustered Gaussians on a 200x120 image (not a multiple of any
    tile side), SH degree 0-3, both opacity modes, each weight function."""
    sc = ws.random_scene(20_000, 7 + deg, sh_degree=deg, vd_opacity=vd, clusters=16, box=1.5,
                         log_scale_mu=-3.5, log_scale_sd=0.6)
    cam = ws.look_at((0.3, -0.2, -4.0), width=200, height=120).rounded()
    w = ws.WeightParams(kind, 0.1 if kind == ws.EXP else 4.5, 0.8, 0.7, (0.2, 0.1, 0.3))
    if kind == ws.DIR:
        w = ws.WeightParams(kind, 0.0, 0.0, 0.7, (0.2, 0.1, 0.3))
    ref = _oracle(sc, cam, w)
    for tile in [(16, 16), (32, 8)]:
        (rgb, _), = gpu_render(sc, [cam], w, tile=tile)
        assert_image_parity(rgb, ref, what=tile)


@pytest.mark.parametrize("kind", [ws.DIR, ws.EXP, ws.LC])
def test_workload2_full_size_forward(kind):
    """200k Gaussians, 32 clusters, SH degree 3, view-dependent opacity,
    1280x720: the whole image against the oracle, each weight function."""
    scene, cams, weight, _ = ws.workload(2, weight_kind=kind)
    cam = cams[0].rounded()
    (rgb, _), = gpu_render(scene, [cam], weight)
    ref = _oracle(scene, cam, weight)
    assert_image_parity(rgb, ref, what=kind)


def test_workload3_full_size_forward():
    """1M Gaussians, 64 clusters, SH degree 3, VD opacity, LC, 1920x1080:
    every pixel within 1e-4 plus its tie allowance, and at most 0.1% of the
    2,073,600 pixels over 1e-4 before it."""
    scene, cams, weight, _ = ws.workload(3)
    cam = cams[0].rounded()
    (rgb, _), = gpu_render(scene, [cam], weight)
    ref = _oracle(scene, cam, weight)
    st = assert_image_parity(rgb, ref, what="1M x 1080p")
    assert st["pixels"] == 1920 * 1080


def test_multiview_uneven_sizes():
    """Three views of different sizes in one call; each view against the oracle."""
    sc = ws.random_scene(30_000, 11, sh_degree=3, vd_opacity=True, clusters=8, box=2.0)
    cams = [c.rounded() for c in ws.sphere_cameras(3, 6.0, [(160, 90), (97, 131), (256, 144)])]
    w = ws.default_weight(ws.LC)
    views = gpu_render(sc, cams, w)
    for cam, (rgb, _) in zip(cams, views):
        ref = _oracle(sc, cam, w)
        assert_image_parity(rgb, ref, what=(cam.width, cam.height))


def test_reduced_precision_storage_matches_oracle_on_stored_values():
    """bf16 scales/quats and f16 SH/opacity: the kernel arithmetic against the
    oracle run on the stored (rounded) values."""
    sc = ws.random_scene(20_000, 12, sh_degree=3, vd_opacity=True, clusters=16, box=1.5, log_scale_mu=-3.5)
    q = ws.quantize_reduced(sc)
    cam = ws.look_at((0.0, 0.0, -4.0), width=160, height=120).rounded()
    w = ws.default_weight(ws.LC)
    (rgb, _), = gpu_render(q, [cam], w, reduced=True)
    ref = _oracle(q, cam, w)
    assert_image_parity(rgb, ref, what="reduced")


@pytest.mark.parametrize("n_views", [1, 3])
def test_reduced_precision_storage_gradients_match_oracle_on_stored_values(n_views):
    """bf16 scales/quats and f16 SH/opacity, backward over one view and over
    three: every gradient tensor (FP32, with respect to the stored values)
    against the oracle's analytic gradient on the stored (rounded) values."""
    import torch
    sc = ws.random_scene(3_000, 24, sh_degree=3, vd_opacity=True, clusters=6, box=1.2, log_scale_mu=-3.2,
                         log_scale_sd=0.5)
    q = ws.quantize_reduced(sc)
    cams = [ws.look_at((0.2, 0.1, -3.5), width=96, height=72).rounded(),
            ws.look_at((-1.5, 0.6, -3.0), width=70, height=50).rounded(),
            ws.look_at((1.8, -0.4, -2.9), width=88, height=61).rounded()][:n_views]
    w = ws.WeightParams(ws.LC, 4.8, 0.8, 0.6, (0.3, 0.2, 0.1))
    views, (r, g, wpar, st) = gpu_render(q, cams, w, reduced=True, want_state=True)
    rng = np.random.default_rng(6)
    Gs = [rng.normal(size=(c.height, c.width, 3)).astype(np.float32) for c in cams]
    G = np.concatenate([x.reshape(-1, 3) for x in Gs])
    out = r.backward(g, w.kind, wpar, st, torch.tensor(G, device="cuda"))
    torch.cuda.synchronize()
    env = None
    for c, Gv in zip(cams, Gs):
        e = grad_envelope(q, c, w, Gv.astype(np.float64))
        env = e if env is None else add_envelopes(env, e)
    for k in ("means", "log_scales", "quats", "sh", "opacity", "lc_v"):
        e = grad_excess(out[k].cpu().numpy(), env, k)
        assert e <= GRAD_TOL, (k, e)


def _grad_case(scene, cam, weight, tile=(16, 16)):
    import torch
    views, (r, g, wpar, st) = gpu_render(scene, [cam], weight, tile=tile, want_state=True)
    G = np.random.default_rng(5).normal(size=(cam.height, cam.width, 3)).astype(np.float32)
    out = r.backward(g, weight.kind, wpar, st, torch.tensor(G, device="cuda").reshape(-1, 3))
    torch.cuda.synchronize()
    out["records"] = st.records
    env = grad_envelope(scene, cam, weight, G.astype(np.float64))
    return out, env


@pytest.mark.parametrize("kind,deg,vd", [(ws.LC, 3, True), (ws.EXP, 3, True), (ws.DIR, 1, False),
                                         (ws.EXP, 2, False)])
def test_gradients_match_oracle(kind, deg, vd):
    sc = ws.random_scene(3_000, 20 + deg, sh_degree=deg, vd_opacity=vd, clusters=6, box=1.2,
                         log_scale_mu=-3.2, log_scale_sd=0.5)
    cam = ws.look_at((0.2, 0.1, -3.5), width=96, height=72).rounded()
    w = ws.WeightParams(kind, 0.1 if kind == ws.EXP else 4.8, 0.8, 0.6, (0.3, 0.2, 0.1))
    out, env = _grad_case(sc, cam, w)
    ref = env[1]
    tie_w = env[2]["wpar"] - ref["wpar"]
    for k in ("means", "log_scales", "quats", "sh", "opacity"):
        e = grad_excess(out[k].cpu().numpy(), env, k)
        assert e <= GRAD_TOL, (k, e)
    if kind == ws.LC:
        assert grad_excess(out["lc_v"].cpu().numpy(), env, "lc_v") <= GRAD_TOL
    gw = out["weight_params"].cpu().numpy()
    for k in range(6):
        if (kind == ws.DIR and k < 2) or (kind == ws.LC and k == 1):
            continue
        assert abs(gw[k] - ref["wpar"][k]) <= GRAD_TOL * max(abs(ref["wpar"][k]), 1e-3) + tie_w[k], \
            (k, gw[k], ref["wpar"][k], tie_w[k])


def test_lc_weight_at_zero_v_keeps_its_gradient():
    """LC (Eq. 10) with v_i = 0 exactly for a fifth of the Gaussians: they add
    nothing to Eq. 7 (w_i = 0) but are not culled, since dL/dv_i =
    max(0, 1 - d/sigma) dL/dw is not zero; every gradient tensor, lc_v's
    entries at v_i = 0 included, against the oracle."""
    sc = ws.random_scene(3_000, 27, sh_degree=2, vd_opacity=True, clusters=6, box=1.2,
                         log_scale_mu=-3.2, log_scale_sd=0.5)
    sc.lc_v[::5] = 0.0
    cam = ws.look_at((0.2, 0.1, -3.5), width=96, height=72).rounded()
    w = ws.WeightParams(ws.LC, 4.8, 0.8, 0.6, (0.3, 0.2, 0.1))
    out, env = _grad_case(sc, cam, w)
    for k in ("means", "log_scales", "quats", "sh", "opacity", "lc_v"):
        e = grad_excess(out[k].cpu().numpy(), env, k)
        assert e <= GRAD_TOL, (k, e)
    g0 = out["lc_v"].cpu().numpy()[::5]
    assert (np.abs(env[1]["lc_v"][::5]) > 0).sum() > 100
    assert (np.abs(g0) > 0).sum() > 100


def test_gradient_records_match_oracle():
    """The per-Gaussian 2D gradient records of the tile kernel alone."""
    sc = ws.random_scene(2_000, 31, sh_degree=2, vd_opacity=True, clusters=4, box=1.0, log_scale_mu=-3.0)
    cam = ws.look_at((0.0, 0.0, -3.0), width=80, height=64).rounded()
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.8, (0.1, 0.2, 0.3))
    out, env = _grad_case(sc, cam, w)
    gr = out["grad_records"].cpu().numpy().reshape(-1, 12).astype(np.float64)
    assert np.all(gr[:, 9:] == 0.0)
    gr = gr[:, :9]
    P = oracle.project(sc, cam, w)
    uw = P["u"] * P["w"]
    col = P["color"]
    # oracle g2d: dL/dc and dL/d(uw) at fixed c; the kernel: d/d(c uw) and d/d(uw) at fixed c uw
    conv = gr.copy()
    conv[:, 6:9] = gr[:, 6:9] * uw[:, None]
    conv[:, 5] = gr[:, 5] + (gr[:, 6:9] * col).sum(1)
    # the kernel stores moments of gq = dL/dq' in the frame of the render record's sum of squares
    # q' = r^2 + qd dx^2, r = qs dy + qw dx: {Sr, Sx, Srr, Srx, Sxx}.  In FP64, with the record's own
    # (qs, qw, qd) and v = (qw r + qd dx, qs r) = k Sigma_2D^{-1} d, they give dL/dmu = -2 sum gq v and
    # dL/d(a, b, c) of Sigma_2D = [[a, b], [b, c]] (b one variable) = -sum gq (vx^2, 2 vx vy, vy^2) / k
    rec = out["records"].cpu().numpy().reshape(-1, 12).astype(np.float64)
    qs, qw, qd = rec[:, 2], rec[:, 3], rec[:, 4]
    Sr, Sx, Srr, Srx, Sxx = (gr[:, k].copy() for k in range(5))
    kk = 0.5 / np.log(2.0)
    conv[:, 0] = -2.0 * (qw * Sr + qd * Sx)
    conv[:, 1] = -2.0 * qs * Sr
    conv[:, 2] = -(qw * qw * Srr + 2.0 * qw * qd * Srx + qd * qd * Sxx) / kk
    conv[:, 3] = -2.0 * qs * (qw * Srr + qd * Srx) / kk
    conv[:, 4] = -qs * qs * Srr / kk
    # the oracle gives dL/d(A, B, C) of the conic K = Sigma_2D^{-1} (q = A dx^2 + 2B dx dy + C dy^2):
    # dL/dSigma = -K G K, G = [[dA, dB/2], [dB/2, dC]]
    A, B, C = (P["conic"][:, k] for k in range(3))

    def to_sigma(g, A, B, C, sign=-1.0):
        g = g.copy()
        dA, dB, dC = g[:, 2], 0.5 * g[:, 3], g[:, 4]
        p00, p01 = A * dA + B * dB, A * dB + B * dC
        p10, p11 = B * dA + C * dB, B * dB + C * dC
        g[:, 2] = sign * (p00 * A + p01 * B)
        g[:, 3] = sign * ((p00 * B + p01 * C) + (p10 * A + p11 * B))
        g[:, 4] = sign * (p10 * B + p11 * C)
        return g

    # the map is linear in g: the mid value maps as is, the tie bound through |K| . |G| . |K|
    mid = to_sigma(env[1]["g2d"], A, B, C)
    bound = to_sigma(env[2]["g2d"] - env[1]["g2d"], np.abs(A), np.abs(B), np.abs(C), sign=1.0)
    env_s = ({"g2d": mid - bound}, {"g2d": mid}, {"g2d": mid + bound})
    for c, name in [((0, 2), "mean"), ((2, 5), "Sigma_2D"), ((5, 6), "uw"), ((6, 9), "color")]:
        part = tuple({"g2d": e["g2d"][:, c[0]:c[1]]} for e in env_s)
        err = grad_excess(conv[:, c[0]:c[1]], part, "g2d")
        assert err <= GRAD_TOL, (name, err)


def test_workload3_full_size_gradients():
    """1M Gaussians, 1920x1080, LC, L1 loss against the seeded target:
    every gradient tensor against the oracle's analytic gradient."""
    import torch
    scene, cams, weight, extra = ws.workload(3)
    cam = cams[0].rounded()
    views, (r, g, wpar, st) = gpu_render(scene, [cam], weight, want_state=True)
    target = ws.target_image(extra["target_seed"], cam.height, cam.width)
    tgt = torch.tensor(target, device="cuda").reshape(-1, 3)
    loss = torch.empty(1, device="cuda")
    G = torch.empty_like(st.rgb)
    r.loss_l1(st.rgb, tgt, loss, G)
    out = r.backward(g, weight.kind, wpar, st, G)
    torch.cuda.synchronize()
    Gn = G.cpu().numpy().astype(np.float64).reshape(cam.height, cam.width, 3)
    env = grad_envelope(scene, cam, weight, Gn)
    for k in ("means", "log_scales", "quats", "sh", "opacity", "lc_v"):
        e = grad_excess(out[k].cpu().numpy(), env, k)
        assert e <= GRAD_TOL, (k, e)


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

def test_empty_scene_is_background():
    sc = ws.random_scene(10, 1, sh_degree=1, vd_opacity=True).subset(np.arange(0))
    cam = ws.look_at((0.0, 0.0, -4.0), width=40, height=24).rounded()
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.5, (0.25, 0.5, 0.75))
    (rgb, den), = gpu_render(sc, [cam], w)
    assert np.abs(rgb - np.array([0.25, 0.5, 0.75])).max() < 1e-7
    assert np.all(den == np.float32(0.5))


def test_all_culled_behind_camera():
    sc = ws.random_scene(500, 2, sh_degree=0, vd_opacity=False, box=0.5)
    sc.means[:, 2] -= 10.0                     # camera at z = -4 looking along +z: all behind it
    cam = ws.look_at((0.0, 0.0, -4.0), width=48, height=32).rounded()
    w = ws.default_weight(ws.DIR, w_bg=1.0, c_bg=(0.1, 0.2, 0.3))
    (rgb, _), = gpu_render(sc, [cam], w)
    assert np.abs(rgb - np.array([0.1, 0.2, 0.3])).max() < 1e-7


def test_zero_opacity_gives_background_exactly():
    sc = ws.random_scene(2000, 3, sh_degree=2, vd_opacity=True, box=1.0, log_scale_mu=-3.0)
    sc.opacity[:] = 0.0
    cam = ws.look_at((0.0, 0.0, -3.0), width=64, height=48).rounded()
    w = ws.WeightParams(ws.LC, 10.0, 0.0, 0.9, (0.3, 0.6, 0.9))
    (rgb, den), = gpu_render(sc, [cam], w)
    assert np.abs(rgb - np.float32([0.3, 0.6, 0.9])).max() < 1e-6
    assert np.all(den == np.float32(0.9))


def test_single_gaussian_straddling_the_border():
    sc = ws.random_scene(1, 4, sh_degree=0, vd_opacity=False, box=0.1)
    sc.means[:] = [[0.55, -0.4, 0.0]]
    sc.log_scales[:] = -1.6
    cam = ws.look_at((0.0, 0.0, -2.0), width=50, height=30).rounded()
    w = ws.default_weight(ws.EXP)
    (rgb, _), = gpu_render(sc, [cam], w)
    ref = _oracle(sc, cam, w)
    assert_image_parity(rgb, ref)
    assert (np.abs(rgb - 0.0).max(axis=2) > 1e-3).sum() > 20      # it does reach the image


def test_permutation_changes_only_rounding():
    sc = ws.random_scene(20_000, 5, sh_degree=3, vd_opacity=True, clusters=8, box=1.5)
    cam = ws.look_at((0.0, 0.0, -4.0), width=128, height=96).rounded()
    w = ws.default_weight(ws.LC)
    (a, _), = gpu_render(sc, [cam], w)
    perm = np.random.default_rng(1).permutation(sc.n)
    (b, _), = gpu_render(sc.subset(perm), [cam], w)
    assert np.abs(a - b).max() < 2e-6


@pytest.mark.parametrize("persistent", [False, True])
def test_capacity_overflow_is_reported_and_recovered(persistent):
    """A tile list too small for the frame: the overflow is reported with the
    true total, nothing is written past the list, offsets stay clamped (the
    persistent schedule's tile order is built from them), and the renderer
    regrows the list and renders the full image."""
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer
    from paper_2410_18931_gb300 import _abi as A
    sc = ws.random_scene(5000, 6, sh_degree=1, vd_opacity=True, box=1.0, log_scale_mu=-2.5)
    cam = ws.look_at((0.0, 0.0, -3.0), width=96, height=64).rounded()
    w = ws.default_weight(ws.EXP)
    g = Gaussians.from_scene(sc)
    wpar = torch.tensor(w.as_array(), device="cuda")
    r = Renderer([cam], persistent=persistent)
    st = r.alloc_state(g.n)
    r.wsr_project(g, w.kind, wpar, st.records)
    r.wsr_bin_count(st.records, g.n, st.tile_offsets)
    total = r.wsr_bin_total()
    assert total > 1000
    small = torch.zeros(total // 3, dtype=torch.int32, device="cuda")
    guard = torch.full((4096,), -7, dtype=torch.int32, device="cuda")   # allocated right after
    r.wsr_bin(st.records, g.n, st.tile_offsets, small)
    assert r.wsr_check() == A.WSR_ERR_CAPACITY
    assert r.wsr_bin_total() == total
    offs = st.tile_offsets.cpu().numpy().astype(np.int64)
    assert offs.max() <= small.numel() and np.all(np.diff(offs) >= 0)
    assert (guard.cpu().numpy() == -7).all()
    assert r.wsr_check() == A.WSR_OK                                    # cleared
    # the Renderer grows the list and renders the full image
    r2 = Renderer([cam], persistent=persistent)
    r2.capacity = total // 3
    st2 = r2.forward(g, w.kind, wpar)
    ref = _oracle(sc, cam, w)
    assert_image_parity(st2.rgb.cpu().numpy().reshape(cam.height, cam.width, 3), ref)
    assert r2.capacity >= total


def test_autograd_function_matches_raw_backward():
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer, render
    sc = ws.random_scene(3000, 8, sh_degree=3, vd_opacity=True, clusters=4, box=1.0, log_scale_mu=-3.0)
    cam = ws.look_at((0.0, 0.0, -3.0), width=64, height=48).rounded()
    w = ws.default_weight(ws.LC)
    g = Gaussians.from_scene(sc)
    params = [t.clone().requires_grad_(True) for t in (g.means, g.log_scales, g.quats, g.sh, g.opacity, g.lc_v)]
    wpar = torch.tensor(w.as_array(), device="cuda", requires_grad=True)
    gg = Gaussians(*params, g.sh_degree, g.view_dependent)
    r = Renderer([cam])
    img = render(r, w.kind, gg, wpar)
    R = torch.randn_like(img)
    (img * R).sum().backward()
    st = r.forward(g, w.kind, wpar.detach())
    raw = r.backward(g, w.kind, wpar.detach(), st, R)
    # same computation; only the order of the float atomics differs
    for p, k in zip(params, ("means", "log_scales", "quats", "sh", "opacity", "lc_v")):
        assert rel_err(p.grad.cpu().numpy(), raw[k].cpu().numpy()) < 1e-5, k
    assert rel_err(wpar.grad.cpu().numpy(), raw["weight_params"].cpu().numpy()) < 1e-5


@pytest.mark.parametrize("pixels", [1, 33 * 17, 1920 * 1080 + 7])
def test_l1_loss_kernel(pixels):
    """Mean absolute error and its sign gradient, vectorised body plus the
    scalar tail (3 * pixels is 3, 1683 and 6,220,821: tails of 3, 3 and 1),
    with exact ties where the gradient is zero."""
    import torch
    from paper_2410_18931_gb300 import Renderer
    cam = ws.look_at((0.0, 0.0, -3.0), width=33, height=17)
    r = Renderer([cam])
    gen = torch.Generator(device="cuda").manual_seed(pixels)
    a = torch.rand(pixels, 3, device="cuda", generator=gen)
    b = torch.rand(pixels, 3, device="cuda", generator=gen)
    b.view(-1)[::5] = a.view(-1)[::5]
    loss = torch.empty(1, device="cuda")
    g = torch.empty_like(a)
    r.loss_l1(a, b, loss, g)
    ref = (a.double() - b.double()).abs().mean()
    # FP32 summation: the longest chain of additions (a thread's strided terms,
    # the warp and block trees, one atomic per block) stays under 700 terms
    assert abs(loss.item() - ref.item()) <= 700 * 2.0 ** -24 * ref.item() + 1e-9
    assert torch.equal(g, torch.sign(a - b) / a.numel())


def test_workload3_subset_gradients_match_fp64_finite_differences():
    """The 1M x 1920x1080 workload's first 1,000 visible Gaussians: GPU
    gradients of the linear loss <R, C> against central finite differences
    of the FP64 oracle's forward, for sampled entries of every parameter
    tensor and for sigma, w_B and c_B.  An entry is skipped when the set of
    pairs with q <= 9 changes between +h and -h; the tolerance is 1e-3 of the
    tensor's largest GPU gradient plus the oracle's tie bound at that entry."""
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer
    scene, cams, w, _ = ws.workload(3)
    cam = cams[0].rounded()
    w = w.rounded()
    vis = np.nonzero(oracle.project(scene, cam, w)["visible"])[0][:1000]
    sc = scene.subset(vis)
    rng = np.random.default_rng(7)
    R = rng.normal(size=(cam.height, cam.width, 3)).astype(np.float32)
    g = Gaussians.from_scene(sc)
    wpar = torch.tensor(w.as_array(), device="cuda")
    r = Renderer([cam])
    st = r.forward(g, w.kind, wpar)
    out = r.backward(g, w.kind, wpar, st, torch.from_numpy(R.reshape(-1, 3)).cuda())
    torch.cuda.synchronize()
    lo, mid, hi = grad_envelope(sc, cam, w, R.astype(np.float64))
    Rd = R.astype(np.float64)

    def loss_pairs(s, wp):
        o = oracle.render(s, cam, wp)
        return float((o["rgb"] * Rd).sum()), o["pairs"]

    checked = 0
    # steps per tensor: small against the footprint (means move ~0.003 px), far above float32 rounding;
    # the parameters are float32, so the difference quotient uses the step actually taken
    steps = dict(means=1e-5, log_scales=1e-4, quats=1e-4, sh=1e-3, opacity=1e-3, lc_v=1e-3)
    for name, hstep in steps.items():
        gpu = out[name].cpu().numpy().astype(np.float64).reshape(-1)
        slack = (np.asarray(hi[name]) - np.asarray(mid[name])).reshape(-1)      # the entry's tie bound
        scale = np.abs(gpu).max()
        flat = getattr(sc, name).reshape(-1)
        for k in rng.choice(flat.size, 12, replace=False):
            x0 = flat[k]
            xp, xm = np.float32(x0 + hstep), np.float32(x0 - hstep)
            flat[k] = xp
            lp, pp = loss_pairs(sc, w)
            flat[k] = xm
            lm, pm = loss_pairs(sc, w)
            flat[k] = x0
            if pp != pm:
                continue
            fd = (lp - lm) / (float(xp) - float(xm))
            assert abs(gpu[k] - fd) <= GRAD_TOL * scale + slack[k], (name, k, gpu[k], fd, scale)
            checked += 1
    gw = out["weight_params"].cpu().numpy().astype(np.float64)
    base = [w.sigma, w.beta, w.w_bg, *w.c_bg]
    for k in (0, 2, 3, 4, 5):             # sigma, w_B, c_B (beta is unused by the LC weight)
        h = 1e-4 * max(1.0, abs(base[k]))
        vals = list(base)
        vals[k] = base[k] + h
        lp, pp = loss_pairs(sc, ws.WeightParams(w.kind, vals[0], vals[1], vals[2], tuple(vals[3:])))
        vals[k] = base[k] - h
        lm, pm = loss_pairs(sc, ws.WeightParams(w.kind, vals[0], vals[1], vals[2], tuple(vals[3:])))
        if pp != pm:
            continue
        fd = (lp - lm) / (2 * h)
        tie = hi["wpar"][k] - mid["wpar"][k]
        assert abs(gw[k] - fd) <= 1e-3 * max(abs(fd), 1e-3) + tie, (k, gw[k], fd)
        checked += 1
    assert checked >= 50
