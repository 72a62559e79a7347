"""A float32 restatement of how an FP32 renderer decides the footprint test.

Test infrastructure for the oracle's cutoff-tie model (``oracle.tie_width``):
it forms, with numpy float32 arithmetic (every operation rounded to float32),
the quantities the model bounds -- the projected mean, T = J W R S, the 2D
covariance Sigma_2D = T T^t + 0.3 I with its determinant as
|r0 x r1|^2 + 0.3 (a0 + c0) + 0.09 (in FP64 from the float32 rows when
det < 1e-3 a c), the conic as the sum of squares
q' = (qs dy + qw dx)^2 + qd dx^2 prescaled by k = log2(e)/2 -- and evaluates
q' at a pixel from a tile origin, as (tile origin offset) + (offset within
the tile).  Written from Sec. 3 (Eqs. 3, 5) and the 3DGS pre-processing the
paper keeps (0.3 dilation, Jacobian clamp at 1.3 tan(fov), near plane 0.2);
it shares nothing with the CUDA library or the oracle.
"""
from __future__ import annotations

import numpy as np

F = np.float32
K_HALF_LOG2E = F(0.5 / np.log(2.0))          # k = log2(e) / 2
Q_MAX = F(9.0) * K_HALF_LOG2E                # 9 k in float32


def _rot(q):
    w, x, y, z = (q[:, k] for k in range(4))
    two = F(2.0)
    one = F(1.0)
    return np.stack([
        one - two * (y * y + z * z), two * (x * y - w * z), two * (x * z + w * y),
        two * (x * y + w * z), one - two * (x * x + z * z), two * (y * z - w * x),
        two * (x * z - w * y), two * (y * z + w * x), one - two * (x * x + y * y)], axis=1)


def records(scene, cam):
    """Per Gaussian: visible [n], the float32 record [n, 5] (mu_x, mu_y, qs,
    qw, qd) and the float32 rows of T [n, 6] it was formed from."""
    p = scene.means.astype(F)
    W = np.asarray(cam.R, np.float64).astype(F).reshape(3, 3)
    T = np.asarray(cam.T, np.float64).astype(F)
    fx, fy, cx, cy = F(cam.fx), F(cam.fy), F(cam.cx), F(cam.cy)
    t = [W[r, 0] * p[:, 0] + W[r, 1] * p[:, 1] + W[r, 2] * p[:, 2] + T[r] for r in range(3)]
    tx, ty, tz = t
    visible = tz > F(cam.znear)
    qr = scene.quats.astype(F)
    inv = F(1.0) / np.sqrt(qr[:, 0] * qr[:, 0] + qr[:, 1] * qr[:, 1] + qr[:, 2] * qr[:, 2] + qr[:, 3] * qr[:, 3])
    R = _rot(qr * inv[:, None])
    s = np.exp(scene.log_scales.astype(F))
    # M = W R diag(s), row-major [n, 9]
    M = np.stack([(W[r, 0] * R[:, c] + W[r, 1] * R[:, 3 + c] + W[r, 2] * R[:, 6 + c]) * s[:, c]
                  for r in range(3) for c in range(3)], axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        iz = F(1.0) / tz
        ux, uy = tx * iz, ty * iz
        limx = F(1.3 * 0.5 * cam.width / float(cam.fx))
        limy = F(1.3 * 0.5 * cam.height / float(cam.fy))
        rxc, ryc = np.clip(ux, -limx, limx), np.clip(uy, -limy, limy)
        J00, J02 = fx * iz, -fx * rxc * iz
        J11, J12 = fy * iz, -fy * ryc * iz
        r0 = np.stack([J00 * M[:, k] + J02 * M[:, 6 + k] for k in range(3)], axis=1)
        r1 = np.stack([J11 * M[:, 3 + k] + J12 * M[:, 6 + k] for k in range(3)], axis=1)
        a0 = r0[:, 0] * r0[:, 0] + r0[:, 1] * r0[:, 1] + r0[:, 2] * r0[:, 2]
        c0 = r1[:, 0] * r1[:, 0] + r1[:, 1] * r1[:, 1] + r1[:, 2] * r1[:, 2]
        b0 = r0[:, 0] * r1[:, 0] + r0[:, 1] * r1[:, 1] + r0[:, 2] * r1[:, 2]
        x0 = r0[:, 1] * r1[:, 2] - r0[:, 2] * r1[:, 1]
        x1 = r0[:, 2] * r1[:, 0] - r0[:, 0] * r1[:, 2]
        x2 = r0[:, 0] * r1[:, 1] - r0[:, 1] * r1[:, 0]
        d3 = F(0.3)
        a, c = a0 + d3, c0 + d3
        det = (x0 * x0 + x1 * x1 + x2 * x2) + d3 * (a0 + c0) + d3 * d3
        idet = F(1.0) / det
        qs = np.sqrt(K_HALF_LOG2E * a * idet)
        qw = -(b0 / a) * qs
        qd = K_HALF_LOG2E / a
        # strongly anisotropic: the conic in FP64 from the float32 rows
        thin = det < F(1e-3) * a * c
        if thin.any():
            p0, q0 = r0[thin].astype(np.float64), r1[thin].astype(np.float64)
            ad = (p0 * p0).sum(1) + 0.3
            cd = (q0 * q0).sum(1) + 0.3
            bd = (p0 * q0).sum(1)
            dd = (np.cross(p0, q0) ** 2).sum(1) + 0.3 * (ad - 0.3 + cd - 0.3) + 0.09
            kd = float(K_HALF_LOG2E)
            qsd = np.sqrt(kd * ad / dd)
            qs[thin] = qsd.astype(F)
            qw[thin] = (-(bd / ad) * qsd).astype(F)
            qd[thin] = (kd / ad).astype(F)
        mx = fx * tx / tz + cx
        my = fy * ty / tz + cy
    return visible, np.stack([mx, my, qs, qw, qd], axis=1).astype(F), np.concatenate([r0, r1], axis=1)


def q_record(rec, px, py):
    """q of the float32 record evaluated exactly (FP64) at the pixel, on the
    scale of the FP32 threshold: 9 q' / (9 k)_FP32."""
    r = rec.astype(np.float64)
    dx, dy = px - r[:, 0], py - r[:, 1]
    qp = (r[:, 2] * dy + r[:, 3] * dx) ** 2 + r[:, 4] * dx * dx
    return 9.0 * qp / float(Q_MAX)


def q_at(rec, px, py, tile=16):
    """q as the FP32 test sees it (9 q' / (9 k)_FP32) at the pixel centres
    (px, py) (x + 0.5, y + 0.5), for record rows ``rec`` [m, 5]: q' formed
    from the offset of the pixel's tile origin and the offset within the tile."""
    mx, my, qs, qw, qd = (rec[:, k] for k in range(5))
    xo = np.floor((px - 0.5) / tile) * tile
    yo = np.floor((py - 0.5) / tile) * tile
    gx = (xo.astype(F) + F(0.5)) - mx
    gy = (yo.astype(F) + F(0.5)) - my
    ox = (px - 0.5 - xo).astype(F)
    oy = (py - 0.5 - yo).astype(F)
    r = (qs * gy + qw * gx) + qs * oy + qw * ox
    P = qd * gx * gx + ox * (F(2.0) * qd * gx + ox * qd)
    qp = r * r + P
    return 9.0 * qp.astype(np.float64) / float(Q_MAX)
