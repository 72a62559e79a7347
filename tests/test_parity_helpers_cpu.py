"""The comparison helpers the GPU parity tests rely on, checked on the CPU
with the oracle standing in for the GPU: an exact copy passes, a planted
error beyond the tolerance fails, and only errors inside the cutoff-tie
allowance are forgiven."""
import numpy as np

import oracle
import wsr_scenes as ws
from tests.gpu_util import (FWD_TOL, GRAD_TOL, TIE, assert_image_parity, compare_image, grad_envelope, grad_excess,
                            image_stats, rel_err)


def _small():
    sc = ws.random_scene(400, 21, sh_degree=1, vd_opacity=True, clusters=4, box=1.0, log_scale_mu=-2.8)
    cam = ws.look_at((0.2, -0.1, -3.0), width=48, height=36).rounded()
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.7, (0.2, 0.1, 0.3)).rounded()
    return sc, cam, w


def test_compare_image_forgives_only_the_tie_allowance():
    sc, cam, w = _small()
    ref = oracle.render(sc, cam, w, amb_tau=TIE)
    exact = ref["rgb"].astype(np.float32)
    excess, raw, n_amb = compare_image(exact, ref)
    assert excess <= 1e-6 and raw <= 1e-6 and n_amb > 0
    # an error of 3x the tolerance on a pixel with no tie allowance is caught
    free = np.argwhere(ref["amb"] == 0)
    y, x = free[len(free) // 2]
    bad = exact.copy()
    bad[y, x, 0] += 3 * FWD_TOL
    assert compare_image(bad, ref)[0] > FWD_TOL
    # the same error on a pixel whose tie allowance covers it is forgiven
    tied = np.argwhere(ref["amb"] > 4 * FWD_TOL)
    assert len(tied) > 0                               # the scene has such pixels
    y, x = tied[0]
    ok = exact.copy()
    ok[y, x, 1] += 3 * FWD_TOL
    assert compare_image(ok, ref)[0] <= FWD_TOL


def test_grad_excess_measures_the_distance_outside_the_envelope():
    sc, cam, w = _small()
    G = np.random.default_rng(3).normal(size=(cam.height, cam.width, 3))
    env = grad_envelope(sc, cam, w, G)
    mid = env[1]
    for key in ("means", "log_scales", "quats", "sh", "opacity"):
        assert grad_excess(mid[key], env, key) == 0.0, key
        scale = np.abs(mid[key]).max()
        bad = mid[key].copy().reshape(-1)
        j = int(np.argmax(np.abs(bad)))
        bad[j] += 3 * GRAD_TOL * scale                 # 3x the bar on the largest entry
        assert grad_excess(bad, env, key) > GRAD_TOL, key
    assert rel_err(mid["means"], mid["means"]) == 0.0


def test_binning_acceptance_helpers():
    """The binning test's helpers: every required (Gaussian, tile) pair is also
    an allowed one, and a tile well away from a footprint is not allowed."""
    from tests.test_gpu_bin import _allowed, _truth
    sc, cam, w = _small()
    P = oracle.project(sc, cam, w)
    for tw, th in ((16, 16), (8, 8), (32, 8)):
        must, allowed = _truth(P, cam.width, cam.height, tw, th)
        assert sum(len(s) for s in must.values()) > 50
        for i, s in must.items():
            for ty, tx in s:
                assert _allowed(allowed[i], ty, tx, cam.width, cam.height, tw, th), (i, ty, tx)
        # a Gaussian whose footprint lies in one tile: the tiles two away are not allowed
        tiles_x, tiles_y = -(-cam.width // tw), -(-cam.height // th)
        checked = 0
        for i, s in must.items():
            if len(s) != 1:
                continue
            ty, tx = next(iter(s))
            for dy, dx in ((2, 0), (-2, 0), (0, 2), (0, -2)):
                if 0 <= ty + dy < tiles_y and 0 <= tx + dx < tiles_x:
                    assert not _allowed(allowed[i], ty + dy, tx + dx, cam.width, cam.height, tw, th)
                    checked += 1
        assert checked > 0


def test_raw_rule_counts_pixels_that_need_the_allowance():
    """In an image of 12,000 pixels, 12 pixels (0.1%) over the tolerance
    before their allowance pass and 13 fail, even though every one of them
    lies within its allowance; images under 10,000 pixels are held to the
    allowance alone."""
    import pytest
    ref = {"rgb": np.zeros((120, 100, 3)), "amb": np.full((120, 100), 1e-3)}
    gpu = np.zeros((120, 100, 3), np.float32)
    flat = gpu.reshape(-1, 3)
    flat[:12, 0] = 5e-4
    st = assert_image_parity(gpu, ref)
    assert st["pixels_over_tol_raw"] == 12 and st["pixels_using_allowance"] == 12
    flat[12, 1] = 5e-4
    with pytest.raises(AssertionError):
        assert_image_parity(gpu, ref)
    small = {"rgb": ref["rgb"][:50], "amb": ref["amb"][:50]}
    assert image_stats(gpu[:50], small)["pixels_over_tol_raw"] == 13
    assert_image_parity(gpu[:50], small)
    # beyond the allowance fails whatever the size
    flat[0, 2] = 2e-3
    with pytest.raises(AssertionError):
        assert_image_parity(gpu[:50], small)
