"""FP64 oracle of the training step around the renderer: the 3DGS rendering
loss the paper trains with, and the Adam update.

TEST INFRASTRUCTURE ONLY (as the rest of ``oracle/``): the tests, the smoke
check and the benchmark's CPU-baseline leg are the only callers; nothing here
is imported by the CUDA library or its binding.

* Loss (Sec. 4.4, "Loss function"): the paper keeps the 3DGS rendering loss,
  L = (1 - lambda) * L1 + lambda * D-SSIM with lambda = 0.2.  Readings (the
  paper states only the above): L1 is the mean absolute error over every
  pixel and channel of every view; D-SSIM = 1 - SSIM, SSIM being the mean of
  the SSIM map (Wang et al. 2004) over every pixel and channel of every view,
  each channel filtered separately with the normalised 11 x 11 Gaussian
  window of standard deviation 1.5, zero padding outside the image (the window
  is not renormalised at the border), C1 = 0.01^2 and C2 = 0.03^2 (the SSIM
  paper's K1, K2 for a dynamic range of 1).
* Adam (Kingma & Ba 2015, Algorithm 1): the paper trains in PyTorch as 3DGS
  does, with Adam; the update is
      m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
      theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Everything is plain numpy in float64, written from those definitions: the
window filter is the shifted sum of its 121 taps; the gradient is the chain
rule through the SSIM map, with the filter's adjoint written out separately.
"""
from __future__ import annotations

import numpy as np

SSIM_WINDOW = 11
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
DSSIM_LAMBDA = 0.2


def ssim_window(size: int = SSIM_WINDOW, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """The separable Gaussian window, normalised to sum 1: outer(g, g) with
    g[k] proportional to exp(-(k - size//2)^2 / (2 sigma^2))."""
    k = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-k * k / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def filter2d(img: np.ndarray, win: np.ndarray) -> np.ndarray:
    """out[i, j] = sum_{a, b} win[a, b] * img[i + a - r, j + b - r], with img
    taken as zero outside its bounds (r = size // 2)."""
    H, W = img.shape
    r = win.shape[0] // 2
    pad = np.zeros((H + 2 * r, W + 2 * r))
    pad[r:r + H, r:r + W] = img
    out = np.zeros((H, W))
    for a in range(win.shape[0]):
        for b in range(win.shape[1]):
            out += win[a, b] * pad[a:a + H, b:b + W]
    return out


def filter2d_adjoint(g: np.ndarray, win: np.ndarray) -> np.ndarray:
    """Adjoint of ``filter2d``: each output gradient g[i, j] goes back to the
    pixels (i + a - r, j + b - r) it was filtered from, weighted by win[a, b];
    contributions that fall outside the image are dropped."""
    H, W = g.shape
    r = win.shape[0] // 2
    acc = np.zeros((H + 2 * r, W + 2 * r))
    for a in range(win.shape[0]):
        for b in range(win.shape[1]):
            acc[a:a + H, b:b + W] += win[a, b] * g
    return acc[r:r + H, r:r + W]


def ssim_stats(x: np.ndarray, y: np.ndarray, win: np.ndarray):
    """Local weighted statistics of one channel: mu_x, mu_y, E[x^2], E[y^2], E[xy]."""
    return (filter2d(x, win), filter2d(y, win), filter2d(x * x, win), filter2d(y * y, win),
            filter2d(x * y, win))


def ssim_map(x: np.ndarray, y: np.ndarray, win: np.ndarray | None = None) -> np.ndarray:
    """SSIM map of one channel:
    ((2 mu_x mu_y + C1)(2 s_xy + C2)) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
    with s_xx = E[x^2] - mu_x^2, s_yy likewise, s_xy = E[xy] - mu_x mu_y."""
    win = ssim_window() if win is None else win
    mx, my, exx, eyy, exy = ssim_stats(x, y, win)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    a1, a2 = 2.0 * mx * my + SSIM_C1, 2.0 * sxy + SSIM_C2
    b1, b2 = mx * mx + my * my + SSIM_C1, sxx + syy + SSIM_C2
    return (a1 * a2) / (b1 * b2)


def _ssim_map_grad(x, y, win, gs):
    """d(sum gs * ssim_map)/dx for one channel.  Chain rule through the five
    statistics, then the filter's adjoint back to the pixels."""
    mx, my, exx, eyy, exy = ssim_stats(x, y, win)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    a1, a2 = 2.0 * mx * my + SSIM_C1, 2.0 * sxy + SSIM_C2
    b1, b2 = mx * mx + my * my + SSIM_C1, sxx + syy + SSIM_C2
    s = (a1 * a2) / (b1 * b2)
    # partials of s in terms of (mu_x, E[x^2], E[xy]); mu_x enters a1, a2 (via
    # s_xy), b1 and b2 (via s_xx)
    d_mx = (2.0 * my * a2 - 2.0 * my * a1) / (b1 * b2) - s * (2.0 * mx / b1 - 2.0 * mx / b2)
    d_exx = -s / b2
    d_exy = 2.0 * a1 / (b1 * b2)
    return (filter2d_adjoint(gs * d_mx, win) + 2.0 * x * filter2d_adjoint(gs * d_exx, win)
            + y * filter2d_adjoint(gs * d_exy, win))


def loss_3dgs(images, targets, lam: float = DSSIM_LAMBDA, with_grad: bool = True):
    """The rendering loss of Sec. 4.4 over a list of views.

    images, targets: lists of [H_v, W_v, 3] arrays (any float type; used as
    float64).  Returns dict(loss, l1, ssim, grad=[H_v, W_v, 3] per view):
    loss = (1 - lam) * l1 + lam * (1 - ssim), l1 and ssim the means over all
    pixels and channels of all views.  d|d|/dd is taken as 0 at d = 0.
    """
    xs = [np.asarray(a, np.float64) for a in images]
    ys = [np.asarray(b, np.float64) for b in targets]
    count = float(sum(a.size for a in xs))
    win = ssim_window()
    l1 = sum(float(np.abs(a - b).sum()) for a, b in zip(xs, ys)) / count
    ssim_sum = 0.0
    grads = []
    for a, b in zip(xs, ys):
        ga = np.zeros_like(a)
        for ch in range(a.shape[2]):
            ssim_sum += float(ssim_map(a[..., ch], b[..., ch], win).sum())
            if with_grad:
                gs = np.full(a.shape[:2], -lam / count)     # d loss / d ssim_map
                ga[..., ch] = _ssim_map_grad(a[..., ch], b[..., ch], win, gs)
        if with_grad:
            ga += (1.0 - lam) * np.sign(a - b) / count
        grads.append(ga)
    ssim = ssim_sum / count
    out = dict(loss=(1.0 - lam) * l1 + lam * (1.0 - ssim), l1=l1, ssim=ssim)
    if with_grad:
        out["grad"] = grads
    return out


def adam_step(param, grad, m, v, t: int, lr, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at 1-based step t.
    lr may be a scalar or an array broadcast against param.  Returns
    (param, m, v) as new float64 arrays."""
    p = np.asarray(param, np.float64)
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - np.asarray(lr, np.float64) * m_hat / (np.sqrt(v_hat) + eps), m, v
