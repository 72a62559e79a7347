"""The oracle's FP32 rounding model of the cutoff test against the GPU's own
records (needs a GPU).

The tie windows that the parity tests forgive come from a model of how far
an FP32 renderer's q can lie from q (``oracle.tie_width``).  Here the
model's record part (the mean, the rows of T, the sums, qs/qw/qd and the
threshold: everything but the evaluation at a pixel, which the CPU pins
check against a float32 restatement) is checked against the records the
projection kernel actually writes: at pixel centres next to every visible
Gaussian's q = 9 ellipse, q from the GPU record, evaluated exactly, must lie
within that part of the window of the exact q.
"""
import numpy as np
import pytest

import oracle
import wsr_scenes as ws
from tests.gpu_util import gpu_render

pytestmark = pytest.mark.gpu

Q_MAX = np.float32(9.0) * np.float32(0.5 / np.log(2.0))      # the FP32 threshold 9 k


def _ellipse_pixels(P, idx_all, nang):
    a, b, c = (P["cov2d"][idx_all, k] for k in range(3))
    l00 = np.sqrt(a)
    l10 = b / l00
    l11 = np.sqrt(c - l10 * l10)
    th = np.linspace(0.0, 2.0 * np.pi, nang, endpoint=False)
    ct, st = np.cos(th)[None, :], np.sin(th)[None, :]
    x = np.floor(P["mean2d"][idx_all, 0][:, None] + 3.0 * l00[:, None] * ct) + 0.5
    y = np.floor(P["mean2d"][idx_all, 1][:, None] + 3.0 * (l10[:, None] * ct + l11[:, None] * st)) + 0.5
    return np.repeat(idx_all, nang), np.stack([x.reshape(-1), y.reshape(-1)], axis=1)


def _record_ratio(scene, cam, w, reduced=False, nang=8):
    views, (r, g, wpar, st) = gpu_render(scene, [cam], w, reduced=reduced, want_state=True)
    rec = st.records.cpu().numpy().reshape(-1, 12).astype(np.float64)
    P = oracle.project(scene, cam, w)
    vis = np.nonzero(P["visible"])[0]
    # the kernel culls exactly where the oracle does (behind the near plane), or at a zero depth factor
    assert np.all(rec[vis, 9] >= 0.0) or w.kind == ws.LC
    vis = vis[rec[vis, 9] >= 0.0]
    idx, xy = _ellipse_pixels(P, vis, nang)
    t = oracle.tie_width(scene, cam, w, idx, xy)
    part = t["terms"][:, :5].sum(1)              # mean, rows, sums, record, threshold
    mx, my, qs, qw, qd = (rec[idx, k] for k in range(5))
    dx, dy = xy[:, 0] - mx, xy[:, 1] - my
    q_gpu = 9.0 * ((qs * dy + qw * dx) ** 2 + qd * dx * dx) / float(Q_MAX)
    return np.abs(q_gpu - t["q"]) / part, len(vis)


@pytest.mark.parametrize("k", [2, 3])
def test_tie_model_covers_the_gpu_records(k):
    """Every visible Gaussian of the 200k-Gaussian 720p and the 1M-Gaussian
    1080p workloads, eight points each."""
    scene, cams, w, _ = ws.workload(k)
    ratio, nvis = _record_ratio(scene, cams[0].rounded(), w)
    assert nvis > 0.5 * scene.n
    assert ratio.max() <= 1.0, (ratio.max(), np.percentile(ratio, 99.9))


def test_tie_model_covers_the_gpu_records_of_needles_and_reduced_storage():
    """Needles (some conics formed in FP64) and bf16/f16 storage (the model
    runs on the stored values, as the oracle does)."""
    nd = ws.random_scene(20_000, 5, sh_degree=1, vd_opacity=True, clusters=0, box=1.0, log_scale_mu=-3.0,
                         log_scale_sd=0.3)
    nd.log_scales[:, 0] = -0.5
    cam = ws.look_at((0.3, 0.2, -3.0), width=320, height=240).rounded()
    ratio, _ = _record_ratio(nd, cam, ws.default_weight(ws.DIR))
    assert ratio.max() <= 1.0, ratio.max()
    q = ws.quantize_reduced(ws.random_scene(50_000, 12, sh_degree=3, vd_opacity=True, clusters=16, box=1.5,
                                            log_scale_mu=-3.5))
    ratio, _ = _record_ratio(q, ws.look_at((0.0, 0.0, -4.0), width=320, height=240).rounded(),
                             ws.default_weight(ws.LC), reduced=True)
    assert ratio.max() <= 1.0, ratio.max()
