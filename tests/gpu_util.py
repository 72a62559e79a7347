"""Helpers shared by the GPU parity tests: run the CUDA path, run the oracle,
compare with the cutoff-ambiguity allowance."""
from __future__ import annotations

import numpy as np

import oracle

FWD_TOL = 1e-4        # max abs pixel error in FP32 (against the FP64 oracle)
GRAD_TOL = 1e-3       # per-tensor max error / max magnitude
AMB_TAU = 0.02        # |q - 9| window treated as a cutoff tie


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
