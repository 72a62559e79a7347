"""Helpers shared by the GPU parity tests: run the CUDA path, run the oracle,
compare with the cutoff-ambiguity allowance."""
from __future__ import annotations

import numpy as np

import oracle

FWD_TOL = 1e-4        # max abs pixel error in FP32 (against the FP64 oracle)
GRAD_TOL = 1e-3       # per-tensor max error / max magnitude
AMB_TAU = 0.02        # |q - 9| window treated as a cutoff tie (forward)
GRAD_TIE_TAU = 1e-3   # the same for gradients: FP32 and FP64 may decide q = 9 +- 1e-3 differently


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
    """Max error after the ambiguity allowance, and diagnostics."""
    err = np.abs(gpu_rgb.astype(np.float64) - ref["rgb"])
    allow = ref["amb"][..., None] if ref.get("amb") is not None else 0.0
    excess = err - allow
    n_amb = int((ref["amb"] > 0).sum()) if ref.get("amb") is not None else 0
    return float(excess.max()), float(err.max()), n_amb


def rel_err(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-12))


def grad_envelope(scene, cam, weight, G, rows=None):
    """Oracle gradients at the cutoffs 9 - tau, 9 and 9 + tau.  A pair whose
    q lies within tau of 9 may be counted by FP32 and not by FP64 (or the
    reverse); the GPU gradient must lie in the envelope these bracket."""
    lo = oracle.grad(scene, cam, weight, G, rows=rows, cutoff=9.0 - GRAD_TIE_TAU)
    mid = oracle.grad(scene, cam, weight, G, rows=rows)
    hi = oracle.grad(scene, cam, weight, G, rows=rows, cutoff=9.0 + GRAD_TIE_TAU)
    return lo, mid, hi


def add_envelopes(a, b):
    return tuple({k: x[k] + y[k] for k in x} for x, y in zip(a, b))


def grad_excess(gpu, env, key):
    """max distance of the GPU tensor outside the tie envelope, relative to
    the tensor's largest magnitude (the per-tensor relative error)."""
    lo, mid, hi = (np.asarray(e[key], np.float64) for e in env)
    g = np.asarray(gpu, np.float64).reshape(mid.shape)
    a, b = np.minimum(lo, hi), np.maximum(lo, hi)
    slack = b - a            # several ties of one Gaussian may be decided either way
    d = np.maximum(0.0, np.maximum((a - slack) - g, g - (b + slack)))
    return float(d.max() / max(np.abs(mid).max(), 1e-12))
