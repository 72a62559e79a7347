"""Helpers shared by the GPU parity tests: run the CUDA path, run the oracle,
compare with the cutoff-tie allowance.

Ties.  Eq. 7 sums the pairs with q <= 9 (Sec. 3's 3-sigma footprint); the
FP32 renderer decides that test from an FP32 record, so a pair whose q lies
within rounding of 9 may be decided the other way there.  ``TIE = "fp32"``
asks the oracle for each pair's window from its FP32 rounding model
(``oracle.tie_width``: the FP32 mean, the rows of T = J W R S, the sums, the
record's qs/qw/qd, the threshold and the evaluation at the pixel, to first
order, doubled), and for bounds of what deciding those pairs either way can
change: per pixel (``amb``) and per gradient entry (``tie``).  Nothing else
is forgiven: every pixel must lie within FWD_TOL of the oracle plus its
allowance, at most RAW_FRACTION of the pixels may need the allowance at all,
and every gradient entry must lie within GRAD_TOL of the tensor's largest
magnitude plus its tie bound.
"""
from __future__ import annotations

import numpy as np

import oracle

FWD_TOL = 1e-4        # max abs pixel error in FP32 (against the FP64 oracle)
GRAD_TOL = 1e-3       # per-tensor max error / max magnitude
TIE = "fp32"          # tie windows from the oracle's FP32 rounding model, per pair
RAW_FRACTION = 1e-3   # pixels allowed to exceed FWD_TOL before the tie allowance


def gpu_render(scene, cams, weight, tile=(16, 16), reduced=False, want_state=False):
    import torch

    from paper_2410_18931_gb300 import Gaussians, Renderer
    g = Gaussians.from_scene(scene, reduced=reduced)
    wpar = torch.tensor(weight.as_array(), device="cuda")
    r = Renderer(cams, tile=tile)
    st = r.forward(g, weight.kind, wpar)
    torch.cuda.synchronize()
    rgb = st.rgb.cpu().numpy()
    den = st.den.cpu().numpy()
    views, o = [], 0
    for c in cams:
        m = c.width * c.height
        views.append((rgb[o:o + m].reshape(c.height, c.width, 3), den[o:o + m].reshape(c.height, c.width)))
        o += m
    if want_state:
        return views, (r, g, wpar, st)
    return views


def compare_image(gpu_rgb, ref, tol=FWD_TOL):
    """Max error after the tie allowance, max raw error, pixels holding ties."""
    err = np.abs(gpu_rgb.astype(np.float64) - ref["rgb"])
    allow = ref["amb"][..., None] if ref.get("amb") is not None else 0.0
    excess = err - allow
    n_amb = int((ref["amb"] > 0).sum()) if ref.get("amb") is not None else 0
    return float(excess.max()), float(err.max()), n_amb


def image_stats(gpu_rgb, ref, tol=FWD_TOL) -> dict:
    """The comparison of one image in numbers: max error, max error beyond
    the allowance, pixels over ``tol`` before the allowance, pixels that
    need the allowance to pass, pixels holding a tie pair."""
    err = np.abs(gpu_rgb.astype(np.float64) - ref["rgb"]).max(axis=-1)
    amb = ref["amb"] if ref.get("amb") is not None else np.zeros_like(err)
    over = err > tol
    return dict(max_abs_err=float(err.max()), max_abs_err_beyond_tie_bound=float(max((err - amb).max(), 0.0)),
                pixels=int(err.size), pixels_over_tol_raw=int(over.sum()),
                pixels_using_allowance=int((over & (err <= tol + amb)).sum()),
                pixels_with_tie_pairs=int((amb > 0).sum()))


def assert_image_parity(gpu_rgb, ref, tol=FWD_TOL, what=""):
    """Every pixel within tol plus its allowance; in images of 10,000 pixels
    or more (where RAW_FRACTION of them is at least 10 pixels), at most
    RAW_FRACTION of the pixels over tol before it."""
    st = image_stats(gpu_rgb, ref, tol)
    assert st["max_abs_err_beyond_tie_bound"] <= tol, (what, st)
    if st["pixels"] >= 10_000:
        assert st["pixels_over_tol_raw"] <= RAW_FRACTION * st["pixels"], (what, st)
    return st


def rel_err(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-12))


def grad_envelope(scene, cam, weight, G, rows=None):
    """(lo, mid, hi): the oracle's gradient ``mid`` and mid -/+ its tie bound
    (per entry: what deciding the pairs within each pair's FP32 rounding
    window of q = 9 either way, in the forward and in the backward, can
    change), for every parameter tensor, ``wpar`` and the 2D records."""
    ref = oracle.grad(scene, cam, weight, G, rows=rows, tie=TIE)
    b = ref.pop("tie")
    lo = {k: ref[k] - b[k] for k in b}
    hi = {k: ref[k] + b[k] for k in b}
    return lo, ref, hi


def add_envelopes(a, b):
    return tuple({k: x[k] + y[k] for k in x} for x, y in zip(a, b))


def grad_excess(gpu, env, key):
    """max distance of the GPU tensor outside [lo, hi], relative to the
    tensor's largest magnitude (the per-tensor relative error)."""
    lo, mid, hi = (np.asarray(e[key], np.float64) for e in env)
    g = np.asarray(gpu, np.float64).reshape(mid.shape)
    d = np.maximum(0.0, np.maximum(lo - g, g - hi))
    return float(d.max() / max(np.abs(mid).max(), 1e-12))
