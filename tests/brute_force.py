"""Independent NumPy brute force of WSR (Eq. 7), used to pin the FP64 oracle.

Every Gaussian is tested against every pixel (no footprint loop), and the
projection is assembled from library routines rather than hand-written
formulas:

* rotation from the quaternion: ``scipy.spatial.transform.Rotation``;
* the affine Jacobian J of Eq. 5: complex-step differentiation of the pinhole
  map (x, y, z) -> (fx x / z + cx, fy y / z + cy), evaluated at the point whose
  x/z and y/z are clamped to 1.3 tan(fov) (3DGS pre-processing);
* conic: ``numpy.linalg.inv``;
* spherical harmonics: ``scipy.special.sph_harm_y`` turned into the real basis
  with the Condon-Shortley phase (m > 0: sqrt(2) Re Y_l^m, m < 0:
  sqrt(2) Im Y_l^|m|).

Only tiny scenes (tens of Gaussians, tens of pixels per side) are meant to go
through here.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y


def real_sh(deg: int, dirs: np.ndarray) -> np.ndarray:
    """Real SH basis [M, (deg+1)^2] at unit directions [M, 3], index l^2 + l + m."""
    d = np.asarray(dirs, np.float64).reshape(-1, 3)
    theta = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    phi = np.arctan2(d[:, 1], d[:, 0])
    out = np.zeros((d.shape[0], (deg + 1) ** 2))
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            y = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                v = np.sqrt(2.0) * y.real
            elif m < 0:
                v = np.sqrt(2.0) * y.imag
            else:
                v = y.real
            out[:, l * l + l + m] = v
    return out


def _pinhole(t, cam):
    return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])


def jacobian(t, cam) -> np.ndarray:
    """2x3 Jacobian of the pinhole map at the clamped point (complex step)."""
    t = np.asarray(t, np.float64)
    lx = 1.3 * 0.5 * cam.width / cam.fx
    ly = 1.3 * 0.5 * cam.height / cam.fy
    tc = np.array([np.clip(t[0] / t[2], -lx, lx) * t[2],
                   np.clip(t[1] / t[2], -ly, ly) * t[2], t[2]])
    h = 1e-30
    J = np.zeros((2, 3))
    for k in range(3):
        z = tc.astype(np.complex128)
        z[k] += 1j * h
        J[:, k] = _pinhole(z, cam).imag / h
    return J


def project(scene, cam, weight):
    """Per-Gaussian quantities, one Gaussian at a time."""
    n = scene.n
    R = np.asarray(cam.R, np.float64)
    T = np.asarray(cam.T, np.float64)
    centre = -R.T @ T
    K = (scene.sh_degree + 1) ** 2
    out = dict(visible=np.zeros(n, bool), mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)),
               cov2d=np.zeros((n, 3)), color=np.zeros((n, 3)), u=np.zeros(n), w=np.zeros(n),
               depth=np.zeros(n))
    q = scene.quats.astype(np.float64)
    rot = Rotation.from_quat(np.concatenate([q[:, 1:4], q[:, :1]], axis=1)).as_matrix()
    for i in range(n):
        p = scene.means[i].astype(np.float64)
        t = R @ p + T
        out["depth"][i] = t[2]
        if not t[2] > cam.znear:
            continue
        out["visible"][i] = True
        s = np.exp(scene.log_scales[i].astype(np.float64))
        sig3 = rot[i] @ np.diag(s * s) @ rot[i].T
        J = jacobian(t, cam)
        sig2 = J @ R @ sig3 @ R.T @ J.T + 0.3 * np.eye(2)
        con = np.linalg.inv(sig2)
        out["cov2d"][i] = [sig2[0, 0], sig2[0, 1], sig2[1, 1]]
        out["conic"][i] = [con[0, 0], con[0, 1], con[1, 1]]
        out["mean2d"][i] = _pinhole(t, cam)
        v = p - centre
        Y = real_sh(scene.sh_degree, v / np.linalg.norm(v))[0]
        H = scene.sh[i].astype(np.float64).reshape(K, 3)
        out["color"][i] = np.maximum(Y @ H + 0.5, 0.0)
        if scene.view_dependent_opacity:
            out["u"][i] = Y @ scene.opacity[i].astype(np.float64)
        else:
            out["u"][i] = 1.0 / (1.0 + np.exp(-float(scene.opacity[i])))
        d = t[2]
        if weight.kind == 0:
            out["w"][i] = 1.0
        elif weight.kind == 1:
            out["w"][i] = np.exp(-weight.sigma * d ** weight.beta)
        else:
            out["w"][i] = max(0.0, 1.0 - d / weight.sigma) * float(scene.lc_v[i])
    return out


def render(scene, cam, weight):
    """Eq. 7 at every pixel, every Gaussian tested at every pixel."""
    P = project(scene, cam, weight)
    H, W = cam.height, cam.width
    xs = np.arange(W) + 0.5
    ys = np.arange(H) + 0.5
    X, Yg = np.meshgrid(xs, ys)
    num = np.zeros((H, W, 3))
    den = np.zeros((H, W))
    for i in np.nonzero(P["visible"])[0]:
        dx = X - P["mean2d"][i, 0]
        dy = Yg - P["mean2d"][i, 1]
        A, B, C = P["conic"][i]
        q = A * dx * dx + 2 * B * dx * dy + C * dy * dy
        a = np.where(q <= 9.0, P["u"][i] * P["w"][i] * np.exp(-0.5 * q), 0.0)
        num += a[..., None] * P["color"][i]
        den += a
    D = weight.w_bg + den
    rgb = (np.asarray(weight.c_bg, np.float64) * weight.w_bg + num) / D[..., None]
    return dict(rgb=rgb, den=D, proj=P)
