"""Seeded synthetic scenes and cameras shared by the oracle and the CUDA path.

This module only draws random numbers and builds camera poses.  It holds none
of the rendering arithmetic (no projection, no spherical-harmonic evaluation,
no weighting): both the FP64 oracle and the GPU path receive the arrays made
here and compute everything else on their own.

Scene record (all float32 numpy arrays, C-contiguous):

* ``means``      [N, 3]   Gaussian centres p_i (world space)
* ``log_scales`` [N, 3]   log of the per-axis scale s_i
* ``quats``      [N, 4]   orientation q_i, (w, x, y, z), unit length on creation
* ``sh``         [N, K, 3] colour SH coefficients H_i, K = (deg + 1)^2
* ``opacity``    [N] logit o_i (view-independent, t_i = sigmoid(o_i)) or
                 [N, K] opacity SH coefficients (view-dependent, Eq. 11)
* ``lc_v``       [N]      per-Gaussian LC weight v_i (Eq. 10)

The paper evaluates on trained Mip-NeRF360 / Tanks&Temples / Deep Blending
scenes, which are not available here.  These generators stand in for them with
Gaussian counts and image sizes of the paper's scale (about 1-6 M Gaussians,
1920x1080 and up, Sec. 5.2).

Camera convention: world-to-camera rotation ``R`` (row-major 3x3) and
translation ``T``; camera axes x right, y down, z forward; pixel (j, i) has
its centre at (j + 0.5, i + 0.5); cx = W / 2, cy = H / 2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Weight-function kinds (Eqs. 8-10).
DIR, EXP, LC = 0, 1, 2
WEIGHT_NAMES = {DIR: "dir", EXP: "exp", LC: "lc"}

# Initial weight-function parameters stated in Sec. 4.4.
EXP_SIGMA0, EXP_BETA0 = 0.1, 0.8
LC_SIGMA0, LC_V0 = 10.0, 0.1

# 2*sqrt(pi): scaling that makes a degree-0 SH coefficient contribute the drawn
# value itself (the inverse of the l=0 basis constant).
_DC_SCALE = 2.0 * math.sqrt(math.pi)


@dataclass
class Camera:
    R: np.ndarray          # [3, 3] float64, world -> camera rotation
    T: np.ndarray          # [3] float64
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.2

    def rounded(self) -> "Camera":
        """The same camera with every real field rounded to float32.

        The GPU consumes float32 cameras; rounding once here means the oracle
        (which upcasts to float64) sees exactly the numbers the GPU sees.
        """
        f = lambda v: float(np.float32(v))
        return Camera(self.R.astype(np.float32).astype(np.float64),
                      self.T.astype(np.float32).astype(np.float64),
                      f(self.fx), f(self.fy), f(self.cx), f(self.cy),
                      int(self.width), int(self.height), f(self.znear))

    @property
    def n_pix(self) -> int:
        return self.width * self.height


@dataclass
class WeightParams:
    kind: int
    sigma: float = 0.0
    beta: float = 0.0
    w_bg: float = 1.0
    c_bg: tuple = (0.0, 0.0, 0.0)

    def as_array(self) -> np.ndarray:
        """[sigma, beta, w_bg, c_bg_r, c_bg_g, c_bg_b] as float32."""
        return np.array([self.sigma, self.beta, self.w_bg, *self.c_bg],
                        dtype=np.float32)

    def rounded(self) -> "WeightParams":
        """The same parameters rounded to float32, the values the GPU reads
        from ``as_array()``; the oracle then sees exactly those numbers (which
        matters where a result depends on an exact tie, e.g. the L1 gradient
        of a background pixel equal to its target)."""
        a = [float(x) for x in self.as_array()]
        return WeightParams(self.kind, a[0], a[1], a[2], tuple(a[3:6]))


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    sh: np.ndarray
    opacity: np.ndarray
    lc_v: np.ndarray
    sh_degree: int
    view_dependent_opacity: bool
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self) -> dict:
        return dict(means=self.means, log_scales=self.log_scales, quats=self.quats,
                    sh=self.sh, opacity=self.opacity, lc_v=self.lc_v)

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.sh[idx].copy(),
                     self.opacity[idx].copy(), self.lc_v[idx].copy(),
                     self.sh_degree, self.view_dependent_opacity, dict(self.meta))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def look_at(pos, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), width=128, height=128,
            fov_y_deg=60.0, znear=0.2) -> Camera:
    """Pinhole camera at ``pos`` looking at ``target``; vertical FOV ``fov_y_deg``."""
    pos = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    T = -R @ pos
    f = 0.5 * height / math.tan(math.radians(fov_y_deg) * 0.5)
    return Camera(R, T, f, f, 0.5 * width, 0.5 * height, int(width), int(height), znear)


def ring_cameras(k: int, radius: float, width: int, height: int) -> list:
    """``k`` cameras on a ring in the y = 0 plane, camera 0 at (0, 0, -radius)."""
    cams = []
    for j in range(k):
        a = 2.0 * math.pi * j / k
        cams.append(look_at((radius * math.sin(a), 0.0, -radius * math.cos(a)),
                            width=width, height=height))
    return cams


def sphere_cameras(k: int, radius: float, sizes) -> list:
    """``k`` cameras on a Fibonacci sphere; ``sizes`` gives (W, H) per camera."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for j in range(k):
        y = 1.0 - 2.0 * (j + 0.5) / k
        r = math.sqrt(max(0.0, 1.0 - y * y))
        ph = golden * j
        pos = (radius * r * math.cos(ph), radius * y, radius * r * math.sin(ph))
        up = (0.0, 0.0, 1.0) if abs(y) > 0.95 else (0.0, 1.0, 0.0)
        w, h = sizes[j]
        cams.append(look_at(pos, up=up, width=w, height=h))
    return cams


def random_scene(n: int, seed: int, *, sh_degree: int, vd_opacity: bool,
                 clusters: int = 0, cluster_sigma: float = 0.3, box: float = 3.0,
                 log_scale_mu: float = -4.0, log_scale_sd: float = 0.7,
                 sh_rest_sd: float = 0.2, opa_rest_sd: float = 0.05,
                 lc_v_range=(0.05, 0.15)) -> Scene:
    """Seeded Gaussian scene.

    ``clusters == 0``: centres uniform in [-box, box]^3.  Otherwise centres are
    drawn from an equal-weight mixture of ``clusters`` isotropic normals
    (std ``cluster_sigma``) whose centres are uniform in [-box, box]^3.
    Colour SH: DC so that its contribution is U[0,1] - 0.5, higher bands
    N(0, sh_rest_sd).  Opacity: logit N(0, 1) (view-independent) or opacity SH
    with DC contribution sigmoid(N(0, 1)) and higher bands N(0, opa_rest_sd)
    (view-dependent).
    """
    rng = np.random.default_rng(seed)
    K = (sh_degree + 1) ** 2
    if clusters > 0:
        centres = rng.uniform(-box, box, size=(clusters, 3))
        which = rng.integers(0, clusters, size=n)
        means = centres[which] + rng.normal(0.0, cluster_sigma, size=(n, 3))
    else:
        means = rng.uniform(-box, box, size=(n, 3))
    log_scales = rng.normal(log_scale_mu, log_scale_sd, size=(n, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sh = np.empty((n, K, 3))
    sh[:, 0, :] = (rng.uniform(0.0, 1.0, size=(n, 3)) - 0.5) * _DC_SCALE
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, sh_rest_sd, size=(n, K - 1, 3))
    logit = rng.normal(0.0, 1.0, size=n)
    if vd_opacity:
        opa = np.empty((n, K))
        opa[:, 0] = (1.0 / (1.0 + np.exp(-logit))) * _DC_SCALE
        if K > 1:
            opa[:, 1:] = rng.normal(0.0, opa_rest_sd, size=(n, K - 1))
    else:
        opa = logit
    lc_v = rng.uniform(lc_v_range[0], lc_v_range[1], size=n)
    return Scene(_f32(means), _f32(log_scales), _f32(q), _f32(sh), _f32(opa), _f32(lc_v),
                 sh_degree, vd_opacity, dict(seed=seed, clusters=clusters))


def default_weight(kind: int, w_bg: float = 1.0, c_bg=(0.0, 0.0, 0.0)) -> WeightParams:
    """Weight parameters at the initial values of Sec. 4.4."""
    if kind == EXP:
        return WeightParams(EXP, EXP_SIGMA0, EXP_BETA0, w_bg, tuple(c_bg))
    if kind == LC:
        return WeightParams(LC, LC_SIGMA0, 0.0, w_bg, tuple(c_bg))
    return WeightParams(DIR, 0.0, 0.0, w_bg, tuple(c_bg))


# --------------------------------------------------------------------------
# The five workloads: (1) small plain forward, (2) 200k 720p forward,
# (3) 1M 1080p forward+backward, (4) 3M batched 16 uneven views,
# (5) 6M reduced-precision 8 x 4K views.
# --------------------------------------------------------------------------

def workload(idx: int, *, n_override: int | None = None, weight_kind: int | None = None):
    """Return (scene, cameras, weight, extra) for workload ``idx`` in 1..5."""
    if idx == 1:
        n = n_override or 1000
        rng_seed = 0
        sc = random_scene(n, rng_seed, sh_degree=0, vd_opacity=False, clusters=0,
                          box=1.0, log_scale_mu=-3.0, log_scale_sd=0.5,
                          lc_v_range=(LC_V0, LC_V0))
        cams = [look_at((0.0, 0.0, -4.0), width=128, height=128)]
        w = default_weight(EXP if weight_kind is None else weight_kind)
        return sc, cams, w, dict(tile=(16, 16), name="1k-128x128")
    if idx == 2:
        n = n_override or 200_000
        sc = random_scene(n, 2, sh_degree=3, vd_opacity=True, clusters=32)
        cams = ring_cameras(1, 5.0, 1280, 720)
        w = default_weight(LC if weight_kind is None else weight_kind)
        return sc, cams, w, dict(tile=(16, 16), name="200k-1280x720")
    if idx == 3:
        n = n_override or 1_000_000
        sc = random_scene(n, 3, sh_degree=3, vd_opacity=True, clusters=64)
        cams = ring_cameras(1, 5.0, 1920, 1080)
        w = default_weight(LC if weight_kind is None else weight_kind)
        return sc, cams, w, dict(tile=(16, 16), name="1M-1920x1080", target_seed=3)
    if idx == 4:
        n = n_override or 3_000_000
        sc = random_scene(n, 4, sh_degree=3, vd_opacity=True, clusters=128)
        sizes = [(640, 360)] * 4 + [(1280, 720)] * 4 + [(1920, 1080)] * 4 + [(2560, 1440)] * 4
        # interleave resolutions around the sphere
        order = [0, 4, 8, 12, 1, 5, 9, 13, 2, 6, 10, 14, 3, 7, 11, 15]
        cams = sphere_cameras(16, 6.0, [sizes[o] for o in order])
        w = default_weight(LC if weight_kind is None else weight_kind)
        return sc, cams, w, dict(tile=None, name="3M-16views-uneven", target_seed=4)
    if idx == 5:
        n = n_override or 6_000_000
        sc = random_scene(n, 5, sh_degree=3, vd_opacity=True, clusters=256)
        cams = sphere_cameras(8, 6.0, [(3840, 2160)] * 8)
        w = default_weight(LC if weight_kind is None else weight_kind)
        return sc, cams, w, dict(tile=None, name="6M-8x3840x2160-reduced")
    raise ValueError(f"unknown workload {idx}")


def target_image(seed: int, height: int, width: int) -> np.ndarray:
    """Seeded random target image U[0,1]^3, [H, W, 3] float32 (for the L1 loss)."""
    rng = np.random.default_rng(seed)
    return _f32(rng.uniform(0.0, 1.0, size=(height, width, 3)))


def quantize_reduced(scene: Scene) -> Scene:
    """Reduced-precision storage of workload 5: SH and opacity rounded to
    float16, log-scales and quaternions rounded to bfloat16 (round to nearest
    even), means and the LC weights v_i kept in float32.  Returned as float32 arrays holding the
    rounded values, so any consumer sees exactly the stored numbers."""
    def bf16_round(a):
        u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
        rounding = ((u >> 16) & 1) + 0x7FFF
        u = ((u + rounding) & 0xFFFF0000).astype(np.uint32)
        return u.view(np.float32)
    return Scene(scene.means.copy(), bf16_round(scene.log_scales), bf16_round(scene.quats),
                 _f32(scene.sh.astype(np.float16)), _f32(scene.opacity.astype(np.float16)),
                 scene.lc_v.copy(), scene.sh_degree,
                 scene.view_dependent_opacity, dict(scene.meta, reduced=True))


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """Upper 16 bits of already bf16-rounded float32 values (uint16 array)."""
    return (np.ascontiguousarray(a, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)
