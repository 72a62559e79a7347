"""Pins of the FP64 training-step oracle (``oracle/train.py``): the 3DGS loss
of Sec. 4.4 (L1 + 0.2 D-SSIM) and Adam, each checked against something other
than its own formula: a library filter, the adjoint identity, closed forms,
brute force and finite differences, and torch's Adam."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import train as T


def _rng(seed):
    return np.random.default_rng(seed)


def test_window_is_normalised_separable_gaussian():
    w = T.ssim_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w, w.T, rtol=0, atol=0)
    # rank one: every row is a multiple of the centre row
    assert np.linalg.matrix_rank(w, tol=1e-14) == 1
    # centre tap of the 1-D factor: 1 / sum_k exp(-k^2 / 4.5), k = -5..5
    g0 = 1.0 / sum(np.exp(-k * k / 4.5) for k in range(-5, 6))
    assert abs(w[5, 5] - g0 * g0) < 1e-15
    # ratio of neighbouring taps exp(-(2k+1)/4.5)
    assert abs(w[5, 6] / w[5, 5] - np.exp(-1.0 / 4.5)) < 1e-13


def test_filter_matches_scipy_zero_padded_correlation():
    ndimage = pytest.importorskip("scipy.ndimage")
    img = _rng(1).random((19, 23))
    win = _rng(2).random((11, 11))          # not symmetric: catches a flipped window
    ref = ndimage.correlate(img, win, mode="constant", cval=0.0)
    np.testing.assert_allclose(T.filter2d(img, win), ref, rtol=1e-13, atol=1e-13)


def test_filter_adjoint_identity():
    r = _rng(3)
    win = r.random((11, 11))
    x, g = r.random((17, 13)), r.random((17, 13))
    lhs = float((T.filter2d(x, win) * g).sum())
    rhs = float((x * T.filter2d_adjoint(g, win)).sum())
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_ssim_of_an_image_with_itself_is_one():
    x = _rng(4).random((20, 16))
    np.testing.assert_allclose(T.ssim_map(x, x), 1.0, rtol=0, atol=1e-13)
    out = T.loss_3dgs([np.stack([x] * 3, -1)], [np.stack([x] * 3, -1)])
    assert abs(out["loss"]) < 1e-13 and abs(out["ssim"] - 1.0) < 1e-13


def test_ssim_of_constant_images_closed_form_with_zero_padding():
    """Constant images a, b: with S the window mass inside the image at a
    pixel, mu_x = aS, E[x^2] = a^2 S, s_xx = a^2 S(1 - S), s_xy = ab S(1 - S),
    which gives SSIM in closed form; S = 1 in the interior."""
    a, b, H, W = 0.7, 0.2, 24, 30
    g = np.exp(-(np.arange(11) - 5.0) ** 2 / 4.5)
    g /= g.sum()

    def mass(i, n):          # mass of the 1-D window inside [0, n) at i
        return sum(g[k] for k in range(11) if 0 <= i + k - 5 < n)

    S = np.array([[mass(i, H) * mass(j, W) for j in range(W)] for i in range(H)])
    c1, c2 = 1e-4, 9e-4
    ref = ((2 * a * b * S * S + c1) * (2 * a * b * S * (1 - S) + c2)
           / (((a * a + b * b) * S * S + c1) * ((a * a + b * b) * S * (1 - S) + c2)))
    got = T.ssim_map(np.full((H, W), a), np.full((H, W), b))
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)
    interior = (2 * a * b + c1) / (a * a + b * b + c1)
    assert abs(got[12, 15] - interior) < 1e-12


def test_ssim_map_brute_force_per_pixel():
    """Per pixel: weighted local means, variances and covariance of the pixels
    under the window (weights of taps outside the image multiply zeros)."""
    r = _rng(5)
    x, y = r.random((7, 9)), r.random((7, 9))
    win = T.ssim_window()
    got = T.ssim_map(x, y, win)
    for i in range(7):
        for j in range(9):
            mx = my = exx = eyy = exy = 0.0
            for a in range(11):
                for b in range(11):
                    ii, jj = i + a - 5, j + b - 5
                    if 0 <= ii < 7 and 0 <= jj < 9:
                        w = win[a, b]
                        mx += w * x[ii, jj]
                        my += w * y[ii, jj]
                        exx += w * x[ii, jj] ** 2
                        eyy += w * y[ii, jj] ** 2
                        exy += w * x[ii, jj] * y[ii, jj]
            num = (2 * mx * my + 1e-4) * (2 * (exy - mx * my) + 9e-4)
            den = (mx ** 2 + my ** 2 + 1e-4) * ((exx - mx ** 2) + (eyy - my ** 2) + 9e-4)
            assert abs(got[i, j] - num / den) < 1e-12
    np.testing.assert_allclose(T.ssim_map(y, x, win), got, rtol=1e-13)


def test_l1_part_and_lambda():
    r = _rng(6)
    x, y = r.random((8, 6, 3)), r.random((8, 6, 3))
    out0 = T.loss_3dgs([x], [y], lam=0.0)
    assert abs(out0["loss"] - np.abs(x - y).mean()) < 1e-15
    np.testing.assert_allclose(out0["grad"][0], np.sign(x - y) / x.size, rtol=0, atol=0)
    out1 = T.loss_3dgs([x], [y], lam=1.0, with_grad=False)
    assert abs(out1["loss"] - (1.0 - out1["ssim"])) < 1e-15
    # two views: the means run over all their elements together
    x2, y2 = r.random((5, 11, 3)), r.random((5, 11, 3))
    both = T.loss_3dgs([x, x2], [y, y2], with_grad=False)
    l1 = (np.abs(x - y).sum() + np.abs(x2 - y2).sum()) / (x.size + x2.size)
    assert abs(both["l1"] - l1) < 1e-15


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_loss_gradient_finite_differences(lam):
    r = _rng(7)
    x = r.random((13, 12, 3))
    y = r.random((13, 12, 3))
    views_x = [x, r.random((6, 17, 3))]
    views_y = [y, r.random((6, 17, 3))]
    out = T.loss_3dgs(views_x, views_y, lam=lam)
    h = 1e-6
    for v, (i, j, c) in [(0, (0, 0, 0)), (0, (6, 5, 1)), (0, (12, 11, 2)), (0, (3, 10, 0)), (1, (5, 16, 1)),
                         (1, (2, 0, 2))]:
        xp = [a.copy() for a in views_x]
        xm = [a.copy() for a in views_x]
        xp[v][i, j, c] += h
        xm[v][i, j, c] -= h
        fd = (T.loss_3dgs(xp, views_y, lam=lam, with_grad=False)["loss"]
              - T.loss_3dgs(xm, views_y, lam=lam, with_grad=False)["loss"]) / (2 * h)
        an = out["grad"][v][i, j, c]
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-4), (v, i, j, c, fd, an)


def test_adam_matches_torch_adam_float64():
    torch = pytest.importorskip("torch")
    r = _rng(8)
    p0 = r.standard_normal(50)
    grads = [r.standard_normal(50) * 10.0 ** r.uniform(-4, 1, 50) for _ in range(6)]
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0, np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = T.adam_step(p, g, m, v, t, 3e-3, eps=1e-15)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_adam_constant_gradient_steps_by_lr():
    """With a constant gradient the bias-corrected moments are exact, so
    every step moves each coordinate by lr * g / (|g| + eps)."""
    g = np.array([2.0, -0.5, 1e-3, 0.0])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 8):
        q, m, v = T.adam_step(p, g, m, v, t, 0.01, eps=1e-8)
        np.testing.assert_allclose(q - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
        p = q
