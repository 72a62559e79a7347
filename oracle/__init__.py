"""Python front end of the FP64 WSR oracle (``wsr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The CUDA library never imports this
package and this package never imports the CUDA library; the two share only
the seeded generators of ``wsr_scenes``.

Every array handed to the C code is float64; scenes made by ``wsr_scenes``
hold float32 values, which are upcast exactly, so the oracle sees the same
numbers as the GPU.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wsr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libwsr_oracle.so")
PROJ_STRIDE = 22
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            common = [ctypes.c_long, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp,
                      dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp]
            lib.wsro_project.argtypes = common + [dp]
            lib.wsro_render.argtypes = common + [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                                 ctypes.c_double, ctypes.POINTER(ctypes.c_longlong),
                                                 ctypes.c_double, dp]
            lib.wsro_render_pixels.argtypes = common + [ctypes.c_int, ctypes.c_long,
                                                        ctypes.POINTER(ctypes.c_int), dp, dp, dp,
                                                        ctypes.c_double]
            lib.wsro_grad.argtypes = (common + [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp] + [dp] * 8
                                      + [ctypes.c_double, ctypes.c_double] + [dp] * 8)
            lib.wsro_tie_width.argtypes = common + [ctypes.c_long, ctypes.POINTER(ctypes.c_long), dp, dp, dp, dp]
            lib.wsro_sh_basis.argtypes = [ctypes.c_long, ctypes.c_int, dp, dp, dp]
            lib.wsro_set_tie_flips.argtypes = [ctypes.c_uint, ctypes.c_uint, ctypes.c_double]
            lib.wsro_set_tie_flips.restype = None
            for f in (lib.wsro_project, lib.wsro_render, lib.wsro_render_pixels, lib.wsro_grad,
                      lib.wsro_tie_width, lib.wsro_sh_basis):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class _Args:
    """Marshalled (scene, camera, weight) argument block."""

    def __init__(self, scene, cam, weight):
        self.keep = [_d(scene.means), _d(scene.log_scales), _d(scene.quats), _d(scene.sh),
                     _d(scene.opacity), _d(scene.lc_v)]
        cam16 = np.concatenate([np.asarray(cam.R, np.float64).reshape(9),
                                np.asarray(cam.T, np.float64).reshape(3),
                                [cam.fx, cam.fy, cam.cx, cam.cy]]).astype(np.float64)
        wpar = np.array([weight.sigma, weight.beta, weight.w_bg, *weight.c_bg], np.float64)
        self.keep += [cam16, wpar]
        self.n = scene.n
        self.K = (scene.sh_degree + 1) ** 2
        self.vd = bool(scene.view_dependent_opacity)
        self.args = ([ctypes.c_long(scene.n), ctypes.c_int(scene.sh_degree), ctypes.c_int(int(self.vd))]
                     + [_ptr(a) for a in self.keep[:6]]
                     + [_ptr(cam16), ctypes.c_int(cam.width), ctypes.c_int(cam.height),
                        ctypes.c_double(cam.znear), ctypes.c_int(weight.kind), _ptr(wpar)])


def project(scene, cam, weight) -> dict:
    """Per-Gaussian projection table (Eqs. 3-5, 4, 11, 8-10)."""
    lib = _load()
    a = _Args(scene, cam, weight)
    out = np.zeros((scene.n, PROJ_STRIDE), np.float64)
    rc = lib.wsro_project(*a.args, _ptr(out))
    if rc:
        raise RuntimeError(f"wsro_project failed ({rc})")
    return dict(visible=out[:, 0] > 0.5, t=out[:, 1:4], mean2d=out[:, 4:6], cov2d=out[:, 6:9],
                conic=out[:, 9:12], color=out[:, 12:15], u=out[:, 15], w=out[:, 16],
                depth=out[:, 17], rx=out[:, 18], ry=out[:, 19])


def _tie_arg(tie) -> float:
    """Window argument of the C functions: "fp32" (each pair's window from
    the FP32 rounding model, ``tie_width``) is passed as -1."""
    if tie is None:
        return 0.0
    if isinstance(tie, str):
        if tie != "fp32":
            raise ValueError(f"unknown tie window {tie!r}")
        return -1.0
    if not tie > 0:
        raise ValueError("a fixed tie window must be positive")
    return float(tie)


def render(scene, cam, weight, *, threads: int | None = None, amb_tau=None, rows=None,
           cutoff: float = 9.0):
    """WSR forward (Eq. 7) over the whole image, or over image rows
    ``rows = (y_lo, y_hi)`` of the same camera.

    Returns dict(rgb [h, W, 3], den [h, W] = w_B + sum a_i, pairs, amb [h, W]
    or None, tie_mass [h, W] or None).  ``amb`` bounds how far a pixel can
    move if the pairs within the tie window of the q <= 9 cutoff were decided
    the other way, and ``tie_mass`` is the sum of |a_i| over those pairs.
    The window is ``amb_tau``: a number (|q - 9| <= amb_tau for every pair)
    or "fp32" (each pair's bound on an FP32 renderer's rounding of q).
    """
    lib = _load()
    a = _Args(scene, cam, weight)
    y_lo, y_hi = rows if rows is not None else (0, cam.height)
    H, W = y_hi - y_lo, cam.width
    rgb = np.zeros((H, W, 3), np.float64)
    den = np.zeros((H, W), np.float64)
    amb = np.zeros((H, W), np.float64) if amb_tau is not None else None
    mass = np.zeros((H, W), np.float64) if amb_tau is not None else None
    pairs = ctypes.c_longlong(0)
    rc = lib.wsro_render(*a.args, ctypes.c_int(threads or default_threads()), ctypes.c_int(y_lo),
                         ctypes.c_int(y_hi), _ptr(rgb), _ptr(den), _ptr(amb), ctypes.c_double(_tie_arg(amb_tau)),
                         ctypes.byref(pairs), ctypes.c_double(cutoff), _ptr(mass))
    if rc:
        raise RuntimeError(f"wsro_render failed ({rc})")
    return dict(rgb=rgb, den=den, pairs=int(pairs.value), amb=amb, tie_mass=mass)


def render_pixels(scene, cam, weight, xy, *, threads: int | None = None, amb_tau: float = 0.0):
    """WSR at the listed pixels (``xy`` [M, 2] int: column, row), each summed
    over every Gaussian.  Returns dict(rgb [M, 3], den [M], amb [M])."""
    lib = _load()
    a = _Args(scene, cam, weight)
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.int32))
    m = xy.shape[0]
    rgb = np.zeros((m, 3), np.float64)
    den = np.zeros(m, np.float64)
    amb = np.zeros(m, np.float64)
    rc = lib.wsro_render_pixels(*a.args, ctypes.c_int(threads or default_threads()), ctypes.c_long(m),
                                xy.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(rgb), _ptr(den),
                                _ptr(amb), ctypes.c_double(amb_tau))
    if rc:
        raise RuntimeError(f"wsro_render_pixels failed ({rc})")
    return dict(rgb=rgb, den=den, amb=amb)


def grad(scene, cam, weight, grad_rgb, *, threads: int | None = None, rows=None, cutoff: float = 9.0,
         tie=None) -> dict:
    """Analytic gradient of <grad_rgb, C> with respect to every parameter;
    with ``rows = (y_lo, y_hi)``, grad_rgb covers only those image rows.
    ``cutoff`` is the footprint bound on q (9 for Eq. 7 as read here).

    With ``tie`` (a fixed window, or "fp32" as in ``render``), the result
    also holds ``tie``: per entry of every output, a first-order bound on how
    far it moves if the pairs within the window are decided the other way,
    by the backward's own sum or through the forward's C and D."""
    lib = _load()
    a = _Args(scene, cam, weight)
    n, K = scene.n, a.K
    y_lo, y_hi = rows if rows is not None else (0, cam.height)
    G = _d(grad_rgb).reshape(y_hi - y_lo, cam.width, 3)

    def shapes():
        return dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                    sh=np.zeros((n, K, 3)), opacity=np.zeros((n, K)) if a.vd else np.zeros(n),
                    lc_v=np.zeros(n), wpar=np.zeros(6), g2d=np.zeros((n, 9)))

    keys = ("means", "log_scales", "quats", "sh", "opacity", "lc_v", "wpar", "g2d")
    out = shapes()
    t = _tie_arg(tie)
    bnd = shapes() if t else None
    rc = lib.wsro_grad(*a.args, ctypes.c_int(threads or default_threads()), ctypes.c_int(y_lo),
                       ctypes.c_int(y_hi), _ptr(G), *[_ptr(out[k]) for k in keys], ctypes.c_double(cutoff),
                       ctypes.c_double(t), *[_ptr(bnd[k]) if bnd else None for k in keys])
    if rc:
        raise RuntimeError(f"wsro_grad failed ({rc})")
    if bnd is not None:
        out["tie"] = bnd
    return out


TIE_TERMS = ("mean", "rows", "sums", "record", "threshold", "evaluation")


def tie_width(scene, cam, weight, idx, xy) -> dict:
    """The FP32 rounding model's tie window at listed points: Gaussian
    ``idx[k]`` at the image position ``xy[k]`` (pixel units, any point).
    Returns dict(q [M] exact, tau [M] the window, terms [M, 6] its parts in
    the order of ``TIE_TERMS``); -1 for culled Gaussians."""
    lib = _load()
    a = _Args(scene, cam, weight)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    pts = _d(xy).reshape(-1, 2)
    m = idx.shape[0]
    q, tau, terms = np.zeros(m), np.zeros(m), np.zeros((m, 6))
    rc = lib.wsro_tie_width(*a.args, ctypes.c_long(m), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                            _ptr(pts), _ptr(q), _ptr(tau), _ptr(terms))
    if rc:
        raise RuntimeError(f"wsro_tie_width failed ({rc})")
    return dict(q=q, tau=tau, terms=terms)


def sh_basis(dirs, deg: int, with_grad: bool = False):
    """Real SH basis Y[M, K] (and polynomial gradient [M, K, 3]) at unit dirs."""
    lib = _load()
    d = _d(dirs).reshape(-1, 3)
    K = (deg + 1) ** 2
    Y = np.zeros((d.shape[0], K))
    dY = np.zeros((d.shape[0], K, 3)) if with_grad else None
    rc = lib.wsro_sh_basis(ctypes.c_long(d.shape[0]), ctypes.c_int(deg), _ptr(d), _ptr(Y), _ptr(dY))
    if rc:
        raise RuntimeError("wsro_sh_basis failed")
    return (Y, dY) if with_grad else Y


@contextlib.contextmanager
def tie_flips(fwd_seed: int, grad_seed: int, tau: float):
    """Within the block, pairs with |q - 9| <= tau are counted or not by a
    seeded hash of (seed, Gaussian, pixel), in the forward sums (``fwd_seed``)
    and in the gradient's sums (``grad_seed``); 0 keeps q <= 9.  It stands in
    for a renderer that decides cutoff ties either way (tests of the tie
    bounds only)."""
    lib = _load()
    with _lock:
        lib.wsro_set_tie_flips(int(fwd_seed), int(grad_seed), float(tau))
    try:
        yield
    finally:
        with _lock:
            lib.wsro_set_tie_flips(0, 0, 0.0)
