"""Deterministic mode (wsr_tiles.deterministic = 1): every output bit for bit
the same from run to run, the tile lists sorted by record index and holding
the same pairs as the default binning, the images and gradients within the
usual tolerances of the FP64 oracle and within rounding of the default mode,
and a tile beyond the sort's bound reported."""
import numpy as np
import pytest

import oracle
import wsr_scenes as ws
from tests.gpu_util import TIE, GRAD_TOL, add_envelopes, assert_image_parity, grad_envelope, grad_excess

pytestmark = pytest.mark.gpu

KEYS = ("means", "log_scales", "quats", "sh", "opacity", "lc_v", "weight_params")


def _run(sc, cams, w, G, tile, persistent, chunk, deterministic, reduced=False):
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer
    g = Gaussians.from_scene(sc, reduced=reduced)
    wpar = torch.tensor(w.as_array(), device="cuda")
    r = Renderer(cams, tile=tile, persistent=persistent, chunk=chunk, deterministic=deterministic)
    st = r.forward(g, w.kind, wpar)
    out = r.backward(g, w.kind, wpar, st, G)
    torch.cuda.synchronize()
    res = {k: out[k].clone() for k in KEYS}
    res["rgb"], res["den"] = st.rgb.clone(), st.den.clone()
    total = int(st.tile_offsets[-1])
    res["offsets"], res["list"] = st.tile_offsets.clone(), st.tile_list[:total].clone()
    return res


@pytest.mark.parametrize("tile,persistent,chunk", [((16, 16), True, 64), ((8, 8), False, 128), ((32, 8), True, 128)])
def test_deterministic_mode_is_bitwise_reproducible_and_matches_the_oracle(tile, persistent, chunk):
    import torch
    sc = ws.random_scene(6000, 81, sh_degree=3, vd_opacity=True, clusters=8, box=1.2, log_scale_mu=-3.2)
    cams = [ws.look_at((0.2, 0.1, -3.5), width=120, height=90).rounded(),
            ws.look_at((-1.4, 0.5, -3.0), width=77, height=61).rounded()]
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 0.7, (0.2, 0.1, 0.3)).rounded()
    rng = np.random.default_rng(82)
    Gs = [rng.normal(size=(c.height, c.width, 3)).astype(np.float32) for c in cams]
    G = torch.tensor(np.concatenate([x.reshape(-1, 3) for x in Gs]), device="cuda")
    a = _run(sc, cams, w, G, tile, persistent, chunk, True)
    b = _run(sc, cams, w, G, tile, persistent, chunk, True)
    for k in a:
        assert torch.equal(a[k], b[k]), k                       # bit for bit, every output
    # the lists: the default binning's pairs, each tile's segment in increasing record index
    d = _run(sc, cams, w, G, tile, persistent, chunk, False)
    off = a["offsets"].cpu().numpy().astype(np.int64)
    lst, lst_d = a["list"].cpu().numpy().astype(np.int64), d["list"].cpu().numpy().astype(np.int64)
    assert np.array_equal(off, d["offsets"].cpu().numpy().astype(np.int64))
    for t in range(len(off) - 1):
        seg = lst[off[t]:off[t + 1]]
        assert np.all(np.diff(seg) > 0), t
        assert np.array_equal(seg, np.sort(lst_d[off[t]:off[t + 1]])), t
    # the same results as the default mode up to rounding order
    for k in ("rgb", "den") + KEYS:
        x, y = a[k].double(), d[k].double()
        assert float((x - y).abs().max()) <= 1e-4 * max(float(y.abs().max()), 1e-12), k
    # and the method itself: images and gradients against the oracle
    rgb = a["rgb"].cpu().numpy()
    o, env = 0, None
    for c, Gv in zip(cams, Gs):
        m = c.width * c.height
        ref = oracle.render(sc, c, w, amb_tau=TIE)
        assert_image_parity(rgb[o:o + m].reshape(c.height, c.width, 3), ref, what=(c.width, c.height))
        o += m
        e = grad_envelope(sc, c, w, Gv.astype(np.float64))
        env = e if env is None else add_envelopes(env, e)
    for k in ("means", "log_scales", "quats", "sh", "opacity"):
        assert grad_excess(a[k].cpu().numpy(), env, k) <= GRAD_TOL, k


@pytest.mark.parametrize("kind,deg,vd,reduced", [(ws.LC, 3, True, True), (ws.DIR, 1, False, False),
                                                  (ws.LC, 2, False, True), (ws.EXP, 0, True, False)])
def test_deterministic_mode_across_weights_storage_and_opacity(kind, deg, vd, reduced):
    """Each weight function, SH degrees 0-3, both opacity modes, FP32 and
    bf16/f16 storage: two deterministic runs equal bit for bit, and within
    rounding of the default mode."""
    import torch
    sc = ws.random_scene(8000, 90 + deg, sh_degree=deg, vd_opacity=vd, clusters=8, box=1.3, log_scale_mu=-3.3)
    cams = [ws.look_at((0.3, -0.1, -3.4), width=100, height=70).rounded(),
            ws.look_at((1.1, 0.6, -3.1), width=64, height=48).rounded()]
    if kind == ws.DIR:
        w = ws.WeightParams(kind, 0.0, 0.0, 0.7, (0.2, 0.1, 0.3))
    elif kind == ws.LC:
        w = ws.WeightParams(kind, 4.5, 0.0, 0.7, (0.2, 0.1, 0.3)).rounded()
    else:
        w = ws.WeightParams(kind, 0.1, 0.8, 0.7, (0.2, 0.1, 0.3)).rounded()
    rng = np.random.default_rng(91 + deg)
    G = torch.tensor(rng.normal(size=(sum(c.width * c.height for c in cams), 3)).astype(np.float32), device="cuda")
    a = _run(sc, cams, w, G, (16, 16), True, 64, True, reduced)
    b = _run(sc, cams, w, G, (16, 16), True, 64, True, reduced)
    for k in a:
        assert torch.equal(a[k], b[k]), k
    d = _run(sc, cams, w, G, (16, 16), True, 64, False, reduced)
    for k in ("rgb", "den") + KEYS:
        x, y = a[k].double(), d[k].double()
        assert float((x - y).abs().max()) <= 1e-4 * max(float(y.abs().max()), 1e-12), k


def test_deterministic_mode_reports_a_tile_beyond_its_sort_bound():
    """20,000 Gaussians stacked where two tiles meet: more instances in a tile
    than the sort holds, reported as unsupported (nothing is rendered)."""
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer
    from paper_2410_18931_gb300 import _abi as A
    stack = ws.random_scene(20_000, 42, sh_degree=0, vd_opacity=False, box=0.01, log_scale_mu=-5.5,
                            log_scale_sd=0.2)
    stack.means[:] += np.array([0.05, 0.05, 0.0], np.float32)
    cam = ws.look_at((0.0, 0.0, -3.0), width=96, height=80).rounded()
    w = ws.WeightParams(ws.EXP, 0.1, 0.8, 1.0, (0.0, 0.0, 0.0))
    g = Gaussians.from_scene(stack)
    wpar = torch.tensor(w.as_array(), device="cuda")
    r = Renderer([cam], deterministic=True)
    with pytest.raises(A.WSRError) as err:
        r.forward(g, w.kind, wpar)
    assert err.value.status == A.WSR_ERR_UNSUPPORTED


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_deterministic_fixed_point_sums_stay_inside_their_bounds(tile):
    """The deterministic backward adds each record term as 64-bit fixed point
    in units of 2^(e - 60), 2^e above a per-Gaussian bound on the sum of the
    term's absolute pixel terms over the whole footprint (stored beside the
    sums).  Every integer sum stays below 2^60 in magnitude (three bits of
    headroom in an int64), and every decoded sum lies within its bound, on a
    scene of small, large and needle-shaped footprints under a random pixel
    gradient."""
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer
    from paper_2410_18931_gb300 import _abi as A
    rng = np.random.default_rng(91)
    base = ws.random_scene(8000, 92, sh_degree=2, vd_opacity=True, clusters=8, box=1.2, log_scale_mu=-3.3)
    base.log_scales[:200, 0] = rng.uniform(np.log(0.2), np.log(0.8), 200).astype(np.float32)    # needles
    base.log_scales[:200, 1:] = np.float32(np.log(3e-3))
    base.log_scales[200:220] = np.float32(np.log(0.4))                                          # large
    cam = ws.look_at((0.3, -0.2, -3.4), width=160, height=120).rounded()
    w = ws.default_weight(ws.LC)
    g = Gaussians.from_scene(base)
    wpar = torch.tensor(w.as_array(), device="cuda")
    r = Renderer([cam], tile=tile, persistent=True, deterministic=True)
    st = r.forward(g, w.kind, wpar)
    G = torch.tensor(rng.normal(size=(cam.height * cam.width, 3)).astype(np.float32), device="cuda")
    grec = torch.empty(g.n * A.WSR_GRAD_RECORD_FLOATS_DET, dtype=torch.float32, device="cuda")
    r.wsr_render_bwd_tiles(st.records, g.n, st.tile_offsets, st.tile_list, w.kind, wpar, st.rgb, st.den, G, grec)
    torch.cuda.synchronize()
    recs = grec.cpu().numpy().reshape(g.n, A.WSR_GRAD_RECORD_FLOATS_DET)
    sums = recs[:, :18].copy().view(np.int64)                 # [n, 9]
    bounds = recs[:, 18:27]
    assert np.all(bounds >= 0.0) and np.all(np.isfinite(bounds))
    assert int(np.abs(sums).max()) < 2 ** 60
    touched = bounds > 0
    assert touched.sum() > 1000
    e = np.frexp(bounds[touched])[1].astype(np.int64)         # bound < 2^e
    val = np.ldexp(sums[touched].astype(np.float64), e - 60)
    assert np.all(np.abs(val) <= bounds[touched].astype(np.float64) * (1 + 1e-6))
    assert np.all(sums[~touched] == 0)
