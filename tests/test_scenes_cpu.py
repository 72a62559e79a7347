"""The seeded input generators (``wsr_scenes``), which both the oracle and
the CUDA path read: the same seed gives the same scene, the draws follow the
stated recipe, the cameras are the stated pinholes, the five workloads have
their stated shapes, and reduced storage rounds as bf16 / f16 do."""
import math

import numpy as np
import pytest

import wsr_scenes as ws

Y00 = 0.5 / math.sqrt(math.pi)        # the degree-0 real spherical harmonic


def test_random_scene_is_seeded():
    a = ws.random_scene(500, 11, sh_degree=2, vd_opacity=True, clusters=4)
    b = ws.random_scene(500, 11, sh_degree=2, vd_opacity=True, clusters=4)
    c = ws.random_scene(500, 12, sh_degree=2, vd_opacity=True, clusters=4)
    for k in a.arrays():
        assert np.array_equal(a.arrays()[k], b.arrays()[k]), k
        assert a.arrays()[k].dtype == np.float32, k
    assert not np.array_equal(a.means, c.means)


@pytest.mark.parametrize("vd", [True, False])
def test_random_scene_follows_its_recipe(vd):
    n = 40_000
    sc = ws.random_scene(n, 3, sh_degree=3, vd_opacity=vd, clusters=0, box=2.0, log_scale_mu=-3.5,
                         log_scale_sd=0.6, sh_rest_sd=0.2, opa_rest_sd=0.05, lc_v_range=(0.05, 0.15))
    assert sc.means.shape == (n, 3) and sc.sh.shape == (n, 16, 3)
    assert np.abs(sc.means).max() <= 2.0
    assert abs(sc.means.mean()) < 0.03
    ls = sc.log_scales.astype(np.float64)
    assert abs(ls.mean() + 3.5) < 0.01 and abs(ls.std() - 0.6) < 0.01
    assert np.allclose(np.linalg.norm(sc.quats.astype(np.float64), axis=1), 1.0, atol=1e-6)
    dc = sc.sh[:, 0, :].astype(np.float64) * Y00 + 0.5       # the colour DC contribution + 0.5: U[0, 1]
    assert dc.min() >= -1e-6 and dc.max() <= 1 + 1e-6 and abs(dc.mean() - 0.5) < 0.01
    assert abs(sc.sh[:, 1:, :].std() - 0.2) < 0.005
    if vd:
        u = sc.opacity[:, 0].astype(np.float64) * Y00          # DC opacity contribution: sigmoid(N(0, 1))
        assert u.min() > 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01
        assert abs(sc.opacity[:, 1:].std() - 0.05) < 0.002
    else:
        assert sc.opacity.shape == (n,) and abs(sc.opacity.std() - 1.0) < 0.02
    assert sc.lc_v.min() >= 0.05 and sc.lc_v.max() <= 0.15


def test_clustered_means_lie_around_their_centres():
    sc = ws.random_scene(20_000, 5, sh_degree=0, vd_opacity=False, clusters=1, cluster_sigma=0.3, box=1.0)
    m = sc.means.astype(np.float64)
    assert np.abs(m.std(axis=0) - 0.3).max() < 0.01               # one cluster: its spread alone


def test_look_at_is_the_stated_pinhole():
    pos = np.array([1.3, -0.9, -2.5])
    cam = ws.look_at(pos, width=160, height=90)
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    T = np.asarray(cam.T, np.float64)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and abs(np.linalg.det(R) - 1.0) < 1e-12
    assert np.allclose(-R.T @ T, pos, atol=1e-12)                 # camera centre
    t = R @ np.zeros(3) + T                                       # the target (origin) on the optical axis
    assert abs(t[0]) < 1e-12 and abs(t[1]) < 1e-12 and t[2] > 0
    assert abs(cam.fx - 45.0 / math.tan(math.radians(30.0))) < 1e-9 and cam.fx == cam.fy
    assert (cam.cx, cam.cy) == (80.0, 45.0)
    up = R.T @ np.array([0.0, -1.0, 0.0])                         # camera y points down
    assert up[1] > 0


def test_ring_and_sphere_cameras_sit_on_their_radius():
    for c in ws.ring_cameras(5, 4.0, 64, 48):
        R = np.asarray(c.R, np.float64).reshape(3, 3)
        centre = -R.T @ np.asarray(c.T, np.float64)
        assert abs(np.linalg.norm(centre) - 4.0) < 1e-12 and abs(centre[1]) < 1e-12
    c0 = ws.ring_cameras(3, 5.0, 64, 48)[0]
    assert np.allclose(-np.asarray(c0.R).reshape(3, 3).T @ np.asarray(c0.T), [0, 0, -5.0], atol=1e-12)
    for c in ws.sphere_cameras(9, 6.0, [(32, 24)] * 9):
        R = np.asarray(c.R, np.float64).reshape(3, 3)
        assert abs(np.linalg.norm(-R.T @ np.asarray(c.T, np.float64)) - 6.0) < 1e-12


def test_the_five_workloads_have_their_stated_shapes():
    sc, cams, w, extra = ws.workload(1)
    assert sc.n == 1000 and sc.sh_degree == 0 and not sc.view_dependent_opacity
    assert [(c.width, c.height) for c in cams] == [(128, 128)]
    assert w.kind == ws.EXP and w.c_bg == (0.0, 0.0, 0.0) and w.w_bg == 1.0
    sc, cams, w, _ = ws.workload(2, n_override=100)
    assert sc.sh_degree == 3 and sc.view_dependent_opacity and w.kind == ws.LC
    assert [(c.width, c.height) for c in cams] == [(1280, 720)]
    sc, cams, w, extra = ws.workload(3, n_override=100)
    assert [(c.width, c.height) for c in cams] == [(1920, 1080)] and extra["target_seed"] == 3
    _, cams, _, _ = ws.workload(4, n_override=100)
    sizes = sorted((c.width, c.height) for c in cams)
    assert sizes == sorted([(640, 360)] * 4 + [(1280, 720)] * 4 + [(1920, 1080)] * 4 + [(2560, 1440)] * 4)
    _, cams, _, _ = ws.workload(5, n_override=100)
    assert [(c.width, c.height) for c in cams] == [(3840, 2160)] * 8
    with pytest.raises(ValueError):
        ws.workload(6)


def test_reduced_storage_rounds_as_bf16_and_f16():
    torch = pytest.importorskip("torch")
    sc = ws.random_scene(3000, 9, sh_degree=3, vd_opacity=True, clusters=4)
    q = ws.quantize_reduced(sc)
    for k in ("log_scales", "quats"):
        want = torch.from_numpy(getattr(sc, k)).to(torch.bfloat16).float().numpy()
        assert np.array_equal(getattr(q, k), want), k
        assert np.all((getattr(q, k).view(np.uint32) & 0xFFFF) == 0), k
    for k in ("sh", "opacity"):
        want = torch.from_numpy(getattr(sc, k)).to(torch.float16).float().numpy()
        assert np.array_equal(getattr(q, k), want), k
    assert np.array_equal(q.means, sc.means) and np.array_equal(q.lc_v, sc.lc_v)
    assert np.array_equal(ws.bf16_bits(q.quats).astype(np.uint32) << 16, q.quats.view(np.uint32))


def test_target_image_is_seeded_and_in_range():
    a, b = ws.target_image(3, 30, 40), ws.target_image(3, 30, 40)
    assert a.shape == (30, 40, 3) and a.dtype == np.float32 and np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() < 1.0 and abs(a.mean() - 0.5) < 0.02
    assert not np.array_equal(a, ws.target_image(4, 30, 40))
