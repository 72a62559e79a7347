"""Pins of the FP64 oracle against things other than itself (CPU only).

* an independent NumPy brute force built on library routines (scipy rotation,
  scipy spherical harmonics, complex-step Jacobian, numpy inverse);
* closed forms: a single isotropic Gaussian on the optical axis, and the
  two-Gaussian toy of Fig. 3 (Sec. 4.2) under each weight function;
* invariants of Eq. 7: permutation, zero opacity, uniform colour, equal depth;
* the real SH basis against scipy and by quadrature (orthonormality);
* the analytic gradient against central finite differences.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import wsr_scenes as ws
from tests import brute_force as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQRT4PI = 2.0 * math.sqrt(math.pi)   # 1 / Y_00


def _scene(means, log_scales, quats, sh, opacity, lc_v, deg, vd):
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float64))
    return ws.Scene(f(means), f(log_scales), f(quats), f(sh), f(opacity), f(lc_v), deg, vd)


def tiny_scene(seed, deg, vd, n=40, box=1.2, ls=-2.2):
    """Small random scene plus Gaussians that exercise the edge cases: one
    behind the camera, one in front of it but inside the near plane (culled),
    one far off-screen to the side with a footprint that reaches into the
    image (Jacobian clamp), one huge and close."""
    sc = ws.random_scene(n, seed, sh_degree=deg, vd_opacity=vd, clusters=0, box=box,
                         log_scale_mu=ls, log_scale_sd=0.4)
    K = (deg + 1) ** 2
    extra_means = np.array([[0.05, -0.05, -2.9],  # t_z = 0.1: in front, inside the near plane 0.2
                            [0.1, 0.0, -3.1],    # behind / at the camera (camera at z=-3)
                            [0.3, -2.2, -0.6],   # above the image: t_y/t_z beyond the clamp
                            [2.6, 0.2, -0.5],    # off to the side: t_x/t_z beyond the clamp
                            [-0.1, 0.1, -2.2]])  # close to the camera: large footprint
    extra_ls = np.array([[-2.3, -2.4, -2.2], [-2.0, -2.0, -2.0], [-0.9, -0.6, -0.8], [-0.6, -1.0, -0.8],
                         [-2.5, -2.2, -2.4]])
    m = extra_means.shape[0]
    rng = np.random.default_rng(seed + 100)
    q = rng.normal(size=(m, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sh = rng.normal(0, 0.3, size=(m, K, 3))
    op = (np.abs(rng.normal(0.5, 0.2, size=(m, K))) if vd else rng.normal(size=m))
    return _scene(np.concatenate([sc.means, extra_means]), np.concatenate([sc.log_scales, extra_ls]),
                  np.concatenate([sc.quats, q]), np.concatenate([sc.sh, sh]),
                  np.concatenate([sc.opacity, op]), np.concatenate([sc.lc_v, rng.uniform(0.05, 0.15, m)]),
                  deg, vd)


def tiny_cam(w=40, h=30):
    """Camera with unequal focal lengths and an off-centre principal point, so
    that a mix-up of x and y intrinsics changes the result."""
    c = ws.look_at((0.0, 0.0, -3.0), width=w, height=h)
    c.fy = c.fx * 1.15
    c.cx = 0.47 * w
    c.cy = 0.54 * h
    return c


WEIGHTS = [ws.WeightParams(ws.DIR, 0.0, 0.0, 1.0, (0.0, 0.0, 0.0)),
           ws.WeightParams(ws.EXP, 0.1, 0.8, 0.7, (0.2, 0.1, 0.3)),
           ws.WeightParams(ws.LC, 3.6, 0.0, 0.5, (0.3, 0.3, 0.1))]


# --------------------------------------------------------------------------
# spherical harmonics
# --------------------------------------------------------------------------

def _unit(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_sh_basis_matches_scipy():
    d = _unit(300, 1)
    Y = oracle.sh_basis(d, 3)
    Yref = bf.real_sh(3, d)
    assert np.abs(Y - Yref).max() < 1e-13


def test_sh_basis_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi is exact for these degrees.
    x, wts = np.polynomial.legendre.leggauss(10)
    phi = np.arange(20) * 2 * np.pi / 20
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wts[:, None] * np.full(20, 2 * np.pi / 20)[None, :]).reshape(-1)
    Y = oracle.sh_basis(d, 3)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_degree0_is_constant():
    Y = oracle.sh_basis(_unit(50, 2), 0)
    assert np.allclose(Y, 1.0 / SQRT4PI, rtol=0, atol=1e-15)


def test_sh_gradient_tangential_matches_fd():
    d = _unit(40, 3)
    Y, dY = oracle.sh_basis(d, 3, with_grad=True)
    rng = np.random.default_rng(4)
    h = 1e-6
    for i in range(d.shape[0]):
        e = rng.normal(size=3)
        e -= d[i] * (d[i] @ e)
        e /= np.linalg.norm(e)
        yp = oracle.sh_basis((d[i] + h * e) / np.linalg.norm(d[i] + h * e), 3)[0]
        ym = oracle.sh_basis((d[i] - h * e) / np.linalg.norm(d[i] - h * e), 3)[0]
        fd = (yp - ym) / (2 * h)
        an = dY[i] @ e          # tangential direction: radial part drops out
        assert np.abs(fd - an).max() < 1e-7


# --------------------------------------------------------------------------
# projection and the sum against the brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("deg,vd", [(0, False), (1, True), (3, True), (2, False)])
def test_projection_matches_brute_force(deg, vd):
    sc = tiny_scene(10 + deg, deg, vd)
    cam = tiny_cam()
    w = WEIGHTS[2]
    P = oracle.project(sc, cam, w)
    B = bf.project(sc, cam, w)
    assert (P["visible"] == B["visible"]).all()
    assert not P["visible"].all()          # the near-plane case is present
    v = P["visible"]
    for key in ("mean2d", "cov2d", "conic", "color", "u", "w"):
        a, b = P[key][v], B[key][v]
        scale = max(1.0, np.abs(b).max())
        assert np.abs(a - b).max() <= 1e-11 * scale, key


@pytest.mark.parametrize("deg,vd", [(3, True), (2, False)])
def test_off_axis_camera_matches_brute_force(deg, vd):
    """A camera off every axis, so its rotation is not symmetric: the camera
    centre -R^t T, the view directions of the SH and the world-to-camera
    transform all differ from their transposed forms."""
    sc = tiny_scene(60 + deg, deg, vd, n=60)
    cam = ws.look_at((1.3, -0.9, -2.5), width=36, height=28)
    cam.fy = cam.fx * 1.1
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    assert np.abs(R - R.T).max() > 0.1
    w = WEIGHTS[1]
    P = oracle.project(sc, cam, w)
    B = bf.project(sc, cam, w)
    assert (P["visible"] == B["visible"]).all()
    v = P["visible"]
    for key in ("mean2d", "cov2d", "conic", "color", "u", "w"):
        a, b = P[key][v], B[key][v]
        assert np.abs(a - b).max() <= 1e-11 * max(1.0, np.abs(b).max()), key
    o = oracle.render(sc, cam, w, threads=2)
    b = bf.render(sc, cam, w)
    assert np.abs(o["rgb"] - b["rgb"]).max() < 1e-12
    assert o["pairs"] > 300


@pytest.mark.parametrize("wi", [0, 1, 2])
@pytest.mark.parametrize("deg,vd", [(0, False), (3, True), (1, False)])
def test_render_matches_brute_force(wi, deg, vd):
    sc = tiny_scene(20 + 3 * deg + wi, deg, vd)
    cam = tiny_cam()
    w = WEIGHTS[wi]
    o = oracle.render(sc, cam, w, threads=3)
    b = bf.render(sc, cam, w)
    assert np.abs(o["rgb"] - b["rgb"]).max() < 1e-12
    assert np.abs(o["den"] - b["den"]).max() < 1e-12
    # the scene really puts Gaussians on the image
    assert o["pairs"] > 500


def test_render_pixels_matches_full_render():
    sc = tiny_scene(5, 3, True)
    cam = tiny_cam()
    w = WEIGHTS[1]
    full = oracle.render(sc, cam, w, threads=2)
    xy = np.array([[x, y] for y in range(0, 30, 3) for x in range(0, 40, 4)], np.int32)
    pix = oracle.render_pixels(sc, cam, w, xy, threads=2)
    ref = full["rgb"][xy[:, 1], xy[:, 0]]
    assert np.abs(pix["rgb"] - ref).max() < 1e-13
    assert np.abs(pix["den"] - full["den"][xy[:, 1], xy[:, 0]]).max() < 1e-13


def test_thread_count_does_not_change_result():
    sc = tiny_scene(6, 2, True)
    cam = tiny_cam()
    a = oracle.render(sc, cam, WEIGHTS[2], threads=1)
    b = oracle.render(sc, cam, WEIGHTS[2], threads=7)
    assert np.array_equal(a["rgb"], b["rgb"])


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def _single(s, o_logit, colour, delta, weight, W=64, H=64):
    sc = _scene([[0.0, 0.0, 0.0]], [[math.log(s)] * 3], [[0.3, -0.5, 0.7, 0.2]],
                [[[(c - 0.5) * SQRT4PI for c in colour]]], [o_logit], [0.1], 0, False)
    cam = ws.look_at((0.0, 0.0, -delta), width=W, height=H)
    return sc, cam


@pytest.mark.parametrize("wi", [0, 1, 2])
def test_single_isotropic_gaussian_closed_form(wi):
    """One isotropic Gaussian on the optical axis: Sigma_2D = ((f s/delta)^2 + 0.3) I."""
    s, delta, logit, colour = 0.15, 3.0, 0.4, (0.9, 0.3, 0.6)
    w = WEIGHTS[wi]
    sc, cam = _single(s, logit, colour, delta, w)
    out = oracle.render(sc, cam, w)
    f = cam.fx
    var = (f * s / delta) ** 2 + 0.3
    u = 1.0 / (1.0 + math.exp(-logit))
    if wi == 0:
        wd = 1.0
    elif wi == 1:
        wd = math.exp(-w.sigma * delta ** w.beta)
    else:
        wd = max(0.0, 1 - delta / w.sigma) * 0.1
    assert wd > 0
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    q = ((xs + 0.5 - cam.cx) ** 2 + (ys + 0.5 - cam.cy) ** 2) / var
    g = np.where(q <= 9.0, np.exp(-0.5 * q), 0.0)
    a = u * wd * g
    exp_rgb = (np.asarray(w.c_bg) * w.w_bg + a[..., None] * np.asarray(colour)) / (w.w_bg + a)[..., None]
    assert np.abs(out["rgb"] - exp_rgb).max() < 1e-13
    assert np.abs(out["den"] - (w.w_bg + a)).max() < 1e-13
    # the footprint is a disc of radius 3 sqrt(var)
    assert out["pairs"] == int((q <= 9.0).sum())


def test_fig3_two_gaussian_toy():
    """Fig. 3 (Sec. 4.2): two opaque (alpha = 1) Gaussians, red in front of
    blue, no background.  DIR mixes them evenly (purple); EXP and LC favour the
    nearer one by w(d1) : w(d2)."""
    with open(os.path.join(GOLDEN, "fig3_two_gaussians.json")) as fh:
        gold = json.load(fh)
    d1, d2 = gold["depths"]
    red, blue = gold["colours"]
    for name, spec in gold["weights"].items():
        w = ws.WeightParams(spec["kind"], spec.get("sigma", 0.0), spec.get("beta", 0.0), 0.0, (0, 0, 0))
        cam = ws.look_at((0.0, 0.0, -d2), width=33, height=33)   # odd size: centre pixel at q = 0
        sc = _scene([[0.0, 0.0, d1 - d2], [0.0, 0.0, 0.0]], [[-2.0] * 3, [-1.5] * 3],
                    [[1, 0, 0, 0], [1, 0, 0, 0]],
                    [[[(c - 0.5) * SQRT4PI for c in red]], [[(c - 0.5) * SQRT4PI for c in blue]]],
                    [[SQRT4PI], [SQRT4PI]], [spec.get("v", 0.1)] * 2, 0, True)
        out = oracle.render(sc, cam, w)
        centre = out["rgb"][16, 16]
        if "expected" in spec:
            assert np.abs(centre - np.asarray(spec["expected"])).max() < 1e-12, name
        wd = {0: lambda d: 1.0,
              1: lambda d: math.exp(-w.sigma * d ** w.beta),
              2: lambda d: max(0.0, 1 - d / w.sigma) * spec.get("v", 0.1)}[spec["kind"]]
        w1, w2 = wd(d1), wd(d2)
        exp_c = (np.asarray(red) * w1 + np.asarray(blue) * w2) / (w1 + w2)
        assert np.abs(centre - exp_c).max() < 1e-12, name
        if spec["kind"] != 0:
            assert centre[0] > centre[2]      # the nearer (red) Gaussian dominates


# --------------------------------------------------------------------------
# invariants of Eq. 7
# --------------------------------------------------------------------------

def test_permutation_invariance():
    sc = tiny_scene(30, 3, True)
    cam = tiny_cam()
    perm = np.random.default_rng(0).permutation(sc.n)
    for w in WEIGHTS:
        a = oracle.render(sc, cam, w)["rgb"]
        b = oracle.render(sc.subset(perm), cam, w)["rgb"]
        assert np.abs(a - b).max() < 1e-13


def test_zero_opacity_gives_background():
    sc = tiny_scene(31, 2, True)
    sc.opacity[:] = 0.0
    cam = tiny_cam()
    for w in WEIGHTS:
        out = oracle.render(sc, cam, w)
        assert np.abs(out["rgb"] - np.asarray(w.c_bg)).max() < 1e-15   # c_B w_B / w_B
        assert np.abs(out["den"] - w.w_bg).max() == 0.0


def test_uniform_colour():
    sc = tiny_scene(32, 0, True)
    c = np.array([0.25, 0.5, 0.75])
    sc.sh[:, 0, :] = (c - 0.5) * SQRT4PI
    cam = tiny_cam()
    for w in WEIGHTS:
        w2 = ws.WeightParams(w.kind, w.sigma, w.beta, w.w_bg, tuple(c))
        out = oracle.render(sc, cam, w2)
        assert np.abs(out["rgb"] - c).max() < 1e-13
        w0 = ws.WeightParams(w.kind, w.sigma, w.beta, 0.0, (0.0, 0.0, 0.0))
        out0 = oracle.render(sc, cam, w0)
        m = np.abs(out0["den"]) > 1e-9
        assert np.abs(out0["rgb"][m] - c).max() < 1e-12


def test_equal_depth_reduces_to_dir():
    """With every Gaussian at the same depth, w(d) is one constant w and
    Eq. 7 under EXP or LC equals DIR with background weight w_B / w."""
    sc = tiny_scene(33, 3, True)
    sc.means[:, 2] = 0.0                      # camera at z = -3 looking along +z: depth 3
    sc.lc_v[:] = 0.1
    cam = tiny_cam()
    for w in WEIGHTS[1:]:
        wd = math.exp(-w.sigma * 3.0 ** w.beta) if w.kind == ws.EXP else (1 - 3.0 / w.sigma) * 0.1
        a = oracle.render(sc, cam, w)["rgb"]
        d = oracle.render(sc, cam, ws.WeightParams(ws.DIR, 0, 0, w.w_bg / wd, w.c_bg))["rgb"]
        assert np.abs(a - d).max() < 1e-12


def test_lc_zero_beyond_sigma():
    """LC (Eq. 10): a Gaussian farther than sigma gets weight 0."""
    sc = tiny_scene(34, 1, True)
    cam = tiny_cam()
    w = ws.WeightParams(ws.LC, 0.5, 0.0, 1.0, (0.1, 0.2, 0.3))   # every depth > 0.5
    P = oracle.project(sc, cam, w)
    assert (P["w"][P["visible"]] == 0.0).all()
    out = oracle.render(sc, cam, w)
    assert np.abs(out["rgb"] - np.asarray(w.c_bg)).max() < 1e-15


# --------------------------------------------------------------------------
# analytic gradient against central finite differences
# --------------------------------------------------------------------------

def _loss_and_pairs(sc, cam, w, R):
    out = oracle.render(sc, cam, w, threads=1)
    return float((out["rgb"] * R).sum()), out["pairs"]


def _fd_check(sc, cam, w, seed, max_comp=None):
    rng = np.random.default_rng(seed)
    R = rng.normal(size=(cam.height, cam.width, 3))
    an = oracle.grad(sc, cam, w, R, threads=2)
    arrays = {"means": sc.means, "log_scales": sc.log_scales, "quats": sc.quats,
              "sh": sc.sh, "opacity": sc.opacity, "lc_v": sc.lc_v}
    worst = {}
    for name, A in arrays.items():
        flat = A.reshape(-1)
        g = an[name].reshape(-1)
        idx = np.arange(flat.size)
        if max_comp is not None and flat.size > max_comp:
            idx = rng.choice(flat.size, max_comp, replace=False)
        fd = np.full(flat.size, np.nan)
        for k in idx:
            x0 = flat[k]
            h = 1e-6 * max(1.0, abs(x0))
            flat[k] = x0 + h
            lp, pp = _loss_and_pairs(sc, cam, w, R)
            flat[k] = x0 - h
            lm, pm = _loss_and_pairs(sc, cam, w, R)
            flat[k] = x0
            if pp != pm:
                continue            # the set of pairs changed: cutoff crossed
            fd[k] = (lp - lm) / (2 * h)
        ok = ~np.isnan(fd)
        err = np.abs(fd[ok] - g[ok]).max() if ok.any() else 0.0
        scale = max(np.abs(g).max(), 1e-12)
        worst[name] = err / scale
    # global parameters: sigma, beta, w_B, c_B
    base = [w.sigma, w.beta, w.w_bg, *w.c_bg]
    for k in range(6):
        if (w.kind == ws.DIR and k < 2) or (w.kind == ws.LC and k == 1):
            assert an["wpar"][k] == 0.0
            continue
        h = 1e-6 * max(1.0, abs(base[k]))
        vals = list(base)
        vals[k] = base[k] + h
        lp, pp = _loss_and_pairs(sc, cam, ws.WeightParams(w.kind, vals[0], vals[1], vals[2], tuple(vals[3:])), R)
        vals[k] = base[k] - h
        lm, pm = _loss_and_pairs(sc, cam, ws.WeightParams(w.kind, vals[0], vals[1], vals[2], tuple(vals[3:])), R)
        fd = (lp - lm) / (2 * h)
        worst[f"wpar{k}"] = abs(fd - an["wpar"][k]) / max(abs(an["wpar"][k]), 1e-3)
    return worst, an


@pytest.mark.parametrize("wi,deg,vd", [(2, 3, True), (1, 3, True), (0, 1, False), (1, 2, False)])
def test_gradient_matches_finite_differences(wi, deg, vd):
    sc = tiny_scene(40 + wi + deg, deg, vd, n=14)
    cam = tiny_cam(32, 24)
    worst, an = _fd_check(sc, cam, WEIGHTS[wi], seed=wi + 7)
    for name, e in worst.items():
        assert e < 2e-6, (name, e, worst)
    # the clamped off-screen Gaussian and the culled one are part of the test
    P = oracle.project(sc, cam, WEIGHTS[wi])
    assert not P["visible"][-4] and not P["visible"][-5]
    assert 0.0 < P["t"][-5, 2] <= cam.znear           # in front of the camera, inside the near plane
    lx, ly = 1.3 * 0.5 * cam.width / cam.fx, 1.3 * 0.5 * cam.height / cam.fy
    t = P["t"]
    assert abs(t[-3, 1] / t[-3, 2]) > ly and abs(t[-2, 0] / t[-2, 2]) > lx
    assert np.abs(an["means"][-3]).max() > 0   # both clamped Gaussians contribute
    assert np.abs(an["means"][-2]).max() > 0


def test_gradient_2d_records_match_finite_differences_of_projection_outputs():
    """dL/d(uw) and dL/dc of the per-Gaussian 2D record, checked by scaling
    one Gaussian's opacity (LC v_i scales u w linearly)."""
    sc = tiny_scene(50, 2, True, n=12)
    cam = tiny_cam(32, 24)
    w = WEIGHTS[2]
    R = np.random.default_rng(1).normal(size=(cam.height, cam.width, 3))
    an = oracle.grad(sc, cam, w, R)
    P = oracle.project(sc, cam, w)
    for i in np.nonzero(P["visible"] & (P["w"] > 0))[0][:6]:
        v0 = sc.lc_v[i]
        h = 1e-6
        sc.lc_v[i] = v0 * (1 + h)
        lp, _ = _loss_and_pairs(sc, cam, w, R)
        sc.lc_v[i] = v0 * (1 - h)
        lm, _ = _loss_and_pairs(sc, cam, w, R)
        sc.lc_v[i] = v0
        uw = P["u"][i] * P["w"][i]
        fd = (lp - lm) / (2 * h * uw)            # d/d(uw) since uw scales by (1 +- h)
        assert abs(fd - an["g2d"][i, 5]) < 1e-6 * max(1.0, abs(fd))


def test_lc_weight_at_zero_v_keeps_its_gradient():
    """LC (Eq. 10) with v_i = 0 exactly, in front of sigma: w_i = 0, so the
    Gaussian adds nothing to Eq. 7, but dL/dv_i = max(0, 1 - d/sigma) dL/dw is
    not zero; the analytic gradient equals central finite differences in v_i
    (C is linear in v_i around 0 through a_i = u w g)."""
    sc = tiny_scene(51, 1, True, n=12)
    cam = tiny_cam(32, 24)
    w = WEIGHTS[2]
    P = oracle.project(sc, cam, w)
    zero = np.nonzero(P["visible"] & (P["depth"] < w.sigma))[0][:3]
    assert len(zero) == 3
    sc.lc_v[zero] = 0.0
    R = np.random.default_rng(4).normal(size=(cam.height, cam.width, 3))
    an = oracle.grad(sc, cam, w, R)
    for i in zero:
        h = 1e-6
        sc.lc_v[i] = h
        lp, _ = _loss_and_pairs(sc, cam, w, R)
        sc.lc_v[i] = -h
        lm, _ = _loss_and_pairs(sc, cam, w, R)
        sc.lc_v[i] = 0.0
        fd = (lp - lm) / (2 * h)
        assert abs(fd) > 1e-6, fd
        assert abs(fd - an["lc_v"][i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, an["lc_v"][i])


def test_row_window_equals_rows_of_the_full_image():
    """A window of rows of the same camera (the same Jacobian clamp) is the
    corresponding rows of the full image, and its gradient is the gradient
    of a loss on those rows only."""
    sc = tiny_scene(60, 3, True)
    cam = tiny_cam()
    w = WEIGHTS[2]
    full = oracle.render(sc, cam, w, amb_tau=0.02)
    win = oracle.render(sc, cam, w, rows=(7, 19), amb_tau=0.02)
    assert np.array_equal(win["rgb"], full["rgb"][7:19])
    assert np.array_equal(win["amb"], full["amb"][7:19])
    R = np.random.default_rng(2).normal(size=(cam.height, cam.width, 3))
    R[:7] = 0.0
    R[19:] = 0.0
    gf = oracle.grad(sc, cam, w, R)
    gw = oracle.grad(sc, cam, w, R[7:19], rows=(7, 19))
    for k in ("means", "log_scales", "quats", "sh", "opacity", "lc_v", "wpar"):
        assert np.abs(gf[k] - gw[k]).max() <= 1e-12 * max(1.0, np.abs(gf[k]).max()), k


def test_tie_bound_covers_a_shifted_cutoff():
    """The per-pixel tie bound is an upper bound on what deciding the pairs
    within tau of q = 9 the other way changes: rendering with the cutoff moved
    to 9 + tau (or 9 - tau) stays within it."""
    sc = tiny_scene(61, 3, True, n=60, ls=-2.5)
    cam = tiny_cam(48, 36)
    for w in WEIGHTS:
        for tau in (0.02, 0.3):
            base = oracle.render(sc, cam, w, amb_tau=tau)
            assert (base["amb"] > 0).any()
            for cut in (9.0 + tau, 9.0 - tau):
                moved = oracle.render(sc, cam, w, cutoff=cut)
                d = np.abs(moved["rgb"] - base["rgb"]).max(axis=2)
                assert np.all(d <= base["amb"] + 1e-12), (w.kind, tau, cut)


# --------------------------------------------------------------------------
# cutoff ties: the bounds used when an FP32 renderer is compared with Eq. 7
# --------------------------------------------------------------------------

@pytest.mark.parametrize("wi,deg,vd", [(0, 0, False), (1, 3, True), (2, 1, False), (2, 3, True)])
def test_tie_bounds_cover_any_decision_of_the_ties(wi, deg, vd):
    """Pairs within tau of q = 9 decided at random (a seeded hash per pair),
    independently in the forward sums and in the gradient's sums: every pixel
    stays within its allowance, and every gradient entry (each parameter
    tensor, sigma, beta, w_B, c_B, the 2D records) within its tie bound."""
    sc = tiny_scene(3 + wi, deg, vd, n=300, ls=-2.6)
    cam = tiny_cam(64, 48)
    w = WEIGHTS[wi]
    tau = 0.05
    G = np.random.default_rng(1 + wi).normal(size=(cam.height, cam.width, 3))
    base = oracle.render(sc, cam, w, amb_tau=tau)
    ref = oracle.grad(sc, cam, w, G, tie=tau)
    assert (base["amb"] > 0).sum() > 50
    for sf, sg in [(1, 2), (3, 0), (0, 4), (5, 5), (11, 13)]:
        with oracle.tie_flips(sf, sg, tau):
            r = oracle.render(sc, cam, w)
            g = oracle.grad(sc, cam, w, G)
        d = np.abs(r["rgb"] - base["rgb"]).max(axis=2)
        assert np.all(d <= base["amb"] * (1 + 1e-9) + 1e-13), (sf, (d - base["amb"]).max())
        for k in ("means", "log_scales", "quats", "sh", "opacity", "lc_v", "wpar", "g2d"):
            ex = np.abs(g[k] - ref[k]) - ref["tie"][k] * (1 + 1e-9)
            assert ex.max() <= 1e-12 * max(1.0, np.abs(ref[k]).max()), (sf, sg, k, ex.max())


def test_tie_bound_is_zero_without_ties():
    """A window that holds no pair gives no allowance and no gradient bound."""
    sc = tiny_scene(62, 2, True, n=40)
    cam = tiny_cam()
    w = WEIGHTS[1]
    G = np.random.default_rng(3).normal(size=(cam.height, cam.width, 3))
    r = oracle.render(sc, cam, w, amb_tau=1e-13)
    g = oracle.grad(sc, cam, w, G, tie=1e-13)
    assert np.all(r["amb"] == 0) and np.all(r["tie_mass"] == 0)
    for k, b in g["tie"].items():
        assert np.all(b == 0), k


def _ellipse_pixels(P, idx_all, nang):
    """Pixel centres nearest to nang points on each Gaussian's q = 9 ellipse."""
    a, b, c = (P["cov2d"][idx_all, k] for k in range(3))
    l00 = np.sqrt(a)
    l10 = b / l00
    l11 = np.sqrt(c - l10 * l10)
    th = np.linspace(0.0, 2.0 * np.pi, nang, endpoint=False)
    ct, st = np.cos(th)[None, :], np.sin(th)[None, :]
    dx = 3.0 * l00[:, None] * ct
    dy = 3.0 * (l10[:, None] * ct + l11[:, None] * st)
    x = np.floor(P["mean2d"][idx_all, 0][:, None] + dx) + 0.5
    y = np.floor(P["mean2d"][idx_all, 1][:, None] + dy) + 0.5
    return np.repeat(idx_all, nang), np.stack([x.reshape(-1), y.reshape(-1)], axis=1)


def _restated_ratios(sc, cam, w, tile, nang=12):
    """Each rounding source of the FP32 test in isolation, against the part
    of the window that bounds it, and the whole test against the window."""
    from tests import fp32_restatement as R32
    P = oracle.project(sc, cam, w)
    vis32, rec, rows = R32.records(sc, cam)
    vis = np.nonzero(P["visible"] & vis32)[0]
    idx, xy = _ellipse_pixels(P, vis, nang)
    t = oracle.tie_width(sc, cam, w, idx, xy)
    T = dict(zip(oracle.TIE_TERMS, t["terms"].T))
    assert np.all(t["tau"] > 0) and np.allclose(t["terms"].sum(1), t["tau"], rtol=1e-12)
    px, py = xy[:, 0], xy[:, 1]
    q = t["q"]
    # the mean alone: the exact conic at the float32 mean
    mu = rec[idx, :2].astype(np.float64)
    A, B, C = (P["conic"][idx, k] for k in range(3))
    dxm, dym = px - mu[:, 0], py - mu[:, 1]
    q_mean = A * dxm * dxm + 2 * B * dxm * dym + C * dym * dym
    # the rows alone: Sigma = T T^t + 0.3 I formed exactly from the float32 rows, at the exact mean
    r = rows[idx].astype(np.float64)
    a = (r[:, :3] ** 2).sum(1) + 0.3
    c = (r[:, 3:] ** 2).sum(1) + 0.3
    b = (r[:, :3] * r[:, 3:]).sum(1)
    dx, dy = px - P["mean2d"][idx, 0], py - P["mean2d"][idx, 1]
    q_rows = (c * dx * dx - 2 * b * dx * dy + a * dy * dy) / (a * c - b * b)
    # the rest of the record (sums, qs/qw/qd, threshold): the float32 record's form at the exact mean
    rec_exact_mu = rec[idx].astype(np.float64)
    rec_exact_mu[:, :2] = P["mean2d"][idx]
    q_form = R32.q_record(rec_exact_mu, px, py)
    # the evaluation alone: the float32 test against the same record evaluated exactly
    q_eval = R32.q_at(rec[idx], px, py, tile)
    q_rec = R32.q_record(rec[idx].astype(np.float64), px, py)
    with np.errstate(divide="ignore", invalid="ignore"):      # a zero term gives inf (the check fails)
        return dict(mean=np.abs(q_mean - q) / T["mean"],
                    rows=np.abs(q_rows - q) / T["rows"],
                    record=np.abs(q_form - q_rows) / (T["sums"] + T["record"] + T["threshold"]),
                    evaluation=np.abs(q_eval - q_rec) / T["evaluation"],
                    total=np.abs(q_eval - q) / t["tau"])


def test_tie_model_covers_an_fp32_restatement():
    """The FP32 rounding model behind the tie windows against a float32
    restatement of the record and the per-pixel test (every operation
    rounded to float32), at pixel centres next to each Gaussian's q = 9
    ellipse: each rounding source alone (the mean; the rows of T; the sums,
    qs, qw, qd and the threshold; the evaluation at the pixel) stays within
    the part of the window that bounds it, and the whole test within the
    window, on scenes with Gaussians inside the near plane, beyond the
    Jacobian clamp and close to the camera, a slice of the 1M-Gaussian 1080p
    workload, and needles (some formed in FP64).  The window is not vacuous:
    the worst rounding seen reaches a twentieth of it."""
    worst = 0.0
    cases = [(tiny_scene(3, 0, False, n=400, ls=-2.6), tiny_cam(64, 48), WEIGHTS[0], 16),
             (tiny_scene(4, 3, True, n=400, ls=-2.6), tiny_cam(64, 48), WEIGHTS[1], 32)]
    scene, cams, w3, _ = ws.workload(3)
    cases.append((scene.subset(np.arange(6000)), cams[0].rounded(), w3, 16))
    nd = ws.random_scene(2000, 5, sh_degree=0, vd_opacity=False, clusters=0, box=1.0, log_scale_mu=-3.0,
                         log_scale_sd=0.3)
    nd.log_scales[:, 0] = -0.5
    cases.append((nd, ws.look_at((0.3, 0.2, -3.0), width=320, height=240).rounded(), ws.default_weight(ws.DIR), 16))
    for sc, cam, w, tile in cases:
        ratios = _restated_ratios(sc, cam, w, tile)
        for k, v in ratios.items():
            assert np.all(np.isfinite(v)) and v.max() <= 1.0, (k, v.max())
        worst = max(worst, float(ratios["total"].max()))
    assert worst >= 0.05, worst
