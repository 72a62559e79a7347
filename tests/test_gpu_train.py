"""Training step on the GPU against the FP64 oracle: the 3DGS loss of Sec. 4.4
(L1 + 0.2 D-SSIM) and its gradient, Adam, one whole step's gradients, the
overflow guard, and a short optimisation that must lower the loss."""
import numpy as np
import pytest

import oracle
import wsr_scenes as ws
from oracle import train as OT
from tests.gpu_util import GRAD_TOL, grad_envelope, grad_excess, rel_err

pytestmark = pytest.mark.gpu

LOSS_SIZES = [(37, 23), (70, 45), (128, 64), (1, 1), (33, 1)]


def _cams(sizes):
    return [ws.look_at((0.0, 0.0, -4.0), width=w, height=h).rounded() for w, h in sizes]


def _images(sizes, seed, smooth=False):
    r = np.random.default_rng(seed)
    out = []
    for w, h in sizes:
        if smooth:
            yy, xx = np.mgrid[0:h, 0:w]
            base = 0.5 + 0.3 * np.sin(xx[..., None] * 0.11 + np.arange(3) + yy[..., None] * 0.07)
            out.append((base + r.normal(0, 0.01, (h, w, 3))).astype(np.float32))
        else:
            out.append(r.random((h, w, 3), dtype=np.float32))
    return out


def _gpu_loss(sizes, xs, ys, lam):
    import torch
    from paper_2410_18931_gb300 import Renderer
    r = Renderer(_cams(sizes))
    rgb = torch.from_numpy(np.concatenate([a.reshape(-1, 3) for a in xs])).cuda()
    tgt = torch.from_numpy(np.concatenate([a.reshape(-1, 3) for a in ys])).cuda()
    loss = torch.full((3,), 7.0, device="cuda")
    grad = torch.full_like(rgb, 7.0)
    r.wsr_loss_3dgs(rgb, tgt, lam, loss, grad)
    torch.cuda.synchronize()
    g = grad.cpu().numpy()
    views, o = [], 0
    for w, h in sizes:
        views.append(g[o:o + w * h].reshape(h, w, 3))
        o += w * h
    return loss.cpu().numpy(), views


@pytest.mark.parametrize("lam,smooth", [(0.2, False), (0.2, True), (0.0, False), (1.0, True)])
def test_loss_3dgs_matches_oracle(lam, smooth):
    xs = _images(LOSS_SIZES, 1, smooth)
    ys = _images(LOSS_SIZES, 2, smooth)
    ref = OT.loss_3dgs(xs, ys, lam=lam)
    loss, grad = _gpu_loss(LOSS_SIZES, xs, ys, lam)
    assert abs(loss[0] - ref["loss"]) <= 1e-5 * max(abs(ref["loss"]), 1e-3)
    assert abs(loss[1] - ref["l1"]) <= 1e-5 * ref["l1"]
    assert abs(loss[2] - ref["ssim"]) <= 1e-5
    g = np.concatenate([a.reshape(-1) for a in grad])
    gr = np.concatenate([a.reshape(-1) for a in ref["grad"]])
    assert rel_err(g, gr) <= 1e-4, rel_err(g, gr)


def test_loss_3dgs_rejects_bad_arguments():
    import torch
    from paper_2410_18931_gb300 import Renderer, WSRError
    r = Renderer(_cams([(16, 16)]))
    x = torch.zeros(256, 3, device="cuda")
    loss = torch.zeros(3, device="cuda")
    for lam in (-0.1, 1.5, float("nan")):
        with pytest.raises(WSRError):
            r.wsr_loss_3dgs(x, x, lam, loss, x.clone())


def _adam_setup(seed):
    import torch
    from paper_2410_18931_gb300 import _abi as A
    r = np.random.default_rng(seed)
    n = 4099
    groups = [A.wsr_adam_group(0, 1001, 1e-2, 1e-2, 0, 0),          # plain
              A.wsr_adam_group(1004, 2030, 3e-3, 1.5e-4, 48, 3),    # SH-like: period 3K, head 3
              A.wsr_adam_group(3036, 1062, 5e-2, 2.5e-3, 16, 1)]    # opacity SH-like; 4098.. untouched
    lr = np.zeros(n)
    for g in groups:
        e = np.arange(g.count)
        lr[g.offset:g.offset + g.count] = np.where((g.period > 0) & (e % max(g.period, 1) >= g.head),
                                                   g.lr_tail, g.lr) if g.period else g.lr
    p0 = r.standard_normal(n).astype(np.float32)
    grads = [(r.standard_normal(n) * 10.0 ** r.uniform(-6, 1, n)).astype(np.float32) for _ in range(5)]
    dev = dict(p=torch.from_numpy(p0.copy()).cuda(), m=torch.zeros(n, device="cuda"),
               v=torch.zeros(n, device="cuda"), state=torch.zeros(4, dtype=torch.int32, device="cuda"))
    return groups, lr, p0, grads, dev


def _adam_call(groups, dev, grad, guard=None, eps=1e-15):
    import ctypes
    import torch
    from paper_2410_18931_gb300 import _abi as A
    lib = A.load()
    arr = (A.wsr_adam_group * len(groups))(*groups)
    hp = A.wsr_adam_hparams(0.9, 0.999, eps)
    g = torch.from_numpy(grad).cuda()
    st = lib.wsr_adam_step(ctypes.c_void_p(dev["p"].data_ptr()), ctypes.c_void_p(g.data_ptr()),
                           ctypes.c_void_p(dev["m"].data_ptr()), ctypes.c_void_p(dev["v"].data_ptr()), arr,
                           len(groups), ctypes.byref(hp), ctypes.c_void_p(dev["state"].data_ptr()),
                           None if guard is None else ctypes.c_void_p(guard.data_ptr()),
                           0 if guard is None else guard.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    A.check("wsr_adam_step", st)


def test_adam_matches_oracle_with_group_tails():
    import torch
    groups, lr, p0, grads, dev = _adam_setup(3)
    p, m, v = p0.astype(np.float64), np.zeros(len(p0)), np.zeros(len(p0))
    inside = lr > 0
    for t, g in enumerate(grads, start=1):
        _adam_call(groups, dev, g)
        p_new, m_new, v_new = OT.adam_step(p, g, m, v, t, lr, eps=1e-15)
        p = np.where(inside, p_new, p)
        m, v = np.where(inside, m_new, 0.0), np.where(inside, v_new, 0.0)
    torch.cuda.synchronize()
    pg = dev["p"].cpu().numpy().astype(np.float64)
    assert np.array_equal(pg[~inside], p0[~inside])            # gaps between groups untouched
    assert np.abs(pg - p).max() <= 2e-6 * max(1.0, np.abs(p).max())
    # the update itself, relative to the learning rate that scales it
    du_g, du_o = (pg - p0)[inside], (p - p0)[inside]
    assert np.abs(du_g - du_o).max() <= 1e-4 * lr.max() + 1e-6
    assert rel_err(dev["m"].cpu().numpy()[inside], m[inside]) <= 1e-5
    assert rel_err(dev["v"].cpu().numpy()[inside], v[inside]) <= 1e-5
    s = dev["state"].cpu().numpy()
    assert s[0] == len(grads) and s[3] == 0


def test_adam_guard_skips_update_after_tile_list_overflow():
    import torch
    from paper_2410_18931_gb300 import Gaussians, Renderer
    from paper_2410_18931_gb300 import _abi as A
    sc, cams, w, _ = ws.workload(1)
    r = Renderer([c.rounded() for c in cams])
    g = Gaussians.from_scene(sc)
    wpar = torch.tensor(w.as_array(), device="cuda")
    st = r.alloc_state(g.n)
    r.wsr_project(g, w.kind, wpar, st.records)
    tiny = torch.empty(4, dtype=torch.int32, device="cuda")
    r.wsr_bin(st.records, g.n, st.tile_offsets, tiny)          # overflows: error recorded in the workspace
    groups, lr, p0, grads, dev = _adam_setup(4)
    _adam_call(groups, dev, grads[0], guard=r.workspace)
    torch.cuda.synchronize()
    assert np.array_equal(dev["p"].cpu().numpy(), p0)
    assert dev["m"].abs().max().item() == 0.0
    s = dev["state"].cpu().numpy()
    assert s[0] == 0 and s[3] == 1
    assert r.wsr_check() == A.WSR_ERR_CAPACITY                 # clears the error
    _adam_call(groups, dev, grads[0], guard=r.workspace)
    torch.cuda.synchronize()
    s = dev["state"].cpu().numpy()
    assert s[0] == 1 and s[3] == 1
    assert not np.array_equal(dev["p"].cpu().numpy(), p0)


def _train_problem(n=3000, size=(96, 80), views=2, seed=11, kind=ws.EXP, deg=1, vd=False):
    truth = ws.random_scene(n, seed, sh_degree=deg, vd_opacity=vd, clusters=0, box=1.0, log_scale_mu=-3.2,
                            log_scale_sd=0.4)
    cams = [c.rounded() for c in ws.ring_cameras(views, 4.0, *size)]
    w = ws.default_weight(kind, c_bg=(0.1, 0.1, 0.1)).rounded()
    r = np.random.default_rng(seed + 1)
    opacity = truth.opacity.copy()
    if vd:      # only the DC band: the unclamped higher bands stay small so the denominator stays positive
        opacity[:, 0] += r.normal(0, 0.5, truth.n).astype(np.float32)
    else:
        opacity += r.normal(0, 0.5, truth.n).astype(np.float32)
    init = ws.Scene(truth.means + r.normal(0, 0.03, truth.means.shape).astype(np.float32),
                    truth.log_scales + r.normal(0, 0.2, truth.log_scales.shape).astype(np.float32),
                    truth.quats, truth.sh + r.normal(0, 0.3, truth.sh.shape).astype(np.float32),
                    opacity, truth.lc_v, deg, vd)
    targets = [oracle.render(truth, c, w)["rgb"].astype(np.float32) for c in cams]
    return truth, init, cams, w, targets


def test_train_step_gradients_and_update_match_oracle():
    import torch
    from paper_2410_18931_gb300 import FlatParams, TrainStep
    _, init, cams, w, targets = _train_problem(n=1500, views=1, kind=ws.LC, deg=2, vd=True)
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1, 3) for t in targets])).cuda()
    flat = FlatParams.from_scene(init, w.as_array())
    p0 = flat.data.clone()
    step = TrainStep(flat, init.sh_degree, init.view_dependent_opacity, cams, w.kind, tgt, capture=False)
    step.run()
    torch.cuda.synchronize()
    cam = cams[0]
    img = oracle.render(init, cam, w)["rgb"]
    ref = OT.loss_3dgs([img], targets)
    assert abs(step.loss[0].item() - ref["loss"]) <= 1e-4 * ref["loss"]
    env = grad_envelope(init, cam, w, ref["grad"][0])
    for key, gk in (("means", "means"), ("log_scales", "log_scales"), ("quats", "quats"), ("sh", "sh"),
                    ("opacity", "opacity"), ("lc_v", "lc_v"), ("wpar", "weight_params")):
        ex = grad_excess(flat.grad[gk].cpu().numpy(), env, key)
        assert ex <= GRAD_TOL, (key, ex)
    # Adam's first step from the GPU gradient: lr * g / (|g| + eps) per element
    lr = np.zeros(flat.numel)
    K = (init.sh_degree + 1) ** 2
    for name in ("means", "log_scales", "quats", "sh", "opacity", "lc_v", "weight_params"):
        o, c = flat.offsets[name], flat.count(name)
        rate = step.opt.lr[name]
        e = np.arange(c)
        if name == "sh":
            lr[o:o + c] = np.where(e % (3 * K) >= 3, rate / 20.0, rate)
        elif name == "opacity":
            lr[o:o + c] = np.where(e % K >= 1, rate / 20.0, rate)
        else:
            lr[o:o + c] = rate
    g = flat.grad_data.cpu().numpy()
    exp_p, _, _ = OT.adam_step(p0.cpu().numpy(), g, 0.0, 0.0, 1, lr, eps=1e-15)
    got = flat.data.cpu().numpy()
    assert np.abs(got - exp_p).max() <= 1e-6 * max(1.0, np.abs(exp_p).max()) + 1e-4 * lr.max()
    assert step.opt.read_state() == dict(step=1, skipped=0)


def test_graph_replay_matches_eager_steps():
    import torch
    from paper_2410_18931_gb300 import FlatParams, TrainStep
    _, init, cams, w, targets = _train_problem(n=2000)
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1, 3) for t in targets])).cuda()
    fa = FlatParams.from_scene(init, w.as_array())
    fb = FlatParams.from_scene(init, w.as_array())
    a = TrainStep(fa, init.sh_degree, False, cams, w.kind, tgt, capture=False)
    b = TrainStep(fb, init.sh_degree, False, cams, w.kind, tgt, capture=True)
    la, lb = [], []
    for _ in range(4):
        a.replay()
        la.append(a.loss.clone())
        b.replay()
        lb.append(b.loss.clone())
    torch.cuda.synchronize()
    for x, y in zip(la, lb):
        assert abs(x[0].item() - y[0].item()) <= 1e-4 * abs(x[0].item())
    assert a.opt.read_state()["step"] == b.opt.read_state()["step"] == 4


def test_deterministic_training_is_bitwise_reproducible():
    """Six graph-replayed Adam steps over two views in the deterministic mode,
    twice from the same scene: the parameters and both Adam moments end equal
    bit for bit (the loss kernel forms each pixel's gradient from its own
    halo; only the reported loss value is summed with atomics)."""
    import torch
    from paper_2410_18931_gb300 import FlatParams, TrainStep
    _, init, cams, w, targets = _train_problem(n=2000, views=2, kind=ws.LC, deg=2, vd=True)
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1, 3) for t in targets])).cuda()
    runs = []
    for _ in range(2):
        flat = FlatParams.from_scene(init, w.as_array())
        step = TrainStep(flat, init.sh_degree, True, cams, w.kind, tgt, persistent=True, chunk=64, capture=True,
                         deterministic=True)
        step.train(6, check_every=3)
        torch.cuda.synchronize()
        assert step.opt.read_state() == dict(step=6, skipped=0)
        runs.append((flat.data.clone(), step.opt.exp_avg.clone(), step.opt.exp_avg_sq.clone()))
    for a, b in zip(*runs):
        assert torch.equal(a, b)
    assert not torch.equal(runs[0][0], FlatParams.from_scene(init, w.as_array()).data)


def test_overflowed_step_is_skipped_then_redone():
    import torch
    from paper_2410_18931_gb300 import FlatParams, TrainStep
    _, init, cams, w, targets = _train_problem(n=1000, views=1)
    tgt = torch.from_numpy(targets[0].reshape(-1, 3)).cuda()
    flat = FlatParams.from_scene(init, w.as_array())
    step = TrainStep(flat, init.sh_degree, False, cams, w.kind, tgt, capture=False)
    p0 = flat.data.clone()
    step.st.tile_list = torch.empty(8, dtype=torch.int32, device="cuda")    # far too small
    step.run()
    torch.cuda.synchronize()
    assert torch.equal(flat.data, p0)
    assert step.opt.read_state() == dict(step=0, skipped=1)
    hist = step.train(3, check_every=1)
    assert hist.shape == (3, 3)
    assert step.opt.read_state()["step"] == 3
    assert not torch.equal(flat.data, p0)


@pytest.mark.parametrize("kind,vd", [(ws.EXP, False), (ws.LC, True)])
def test_training_lowers_the_loss_and_moves_the_weight_parameters(kind, vd):
    import torch
    from paper_2410_18931_gb300 import FlatParams, TrainStep
    _, init, cams, w, targets = _train_problem(kind=kind, vd=vd, views=3)
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1, 3) for t in targets])).cuda()
    flat = FlatParams.from_scene(init, w.as_array())
    w0 = flat.param["weight_params"].clone()
    step = TrainStep(flat, init.sh_degree, vd, cams, w.kind, tgt, capture=True)
    hist = step.train(150, check_every=50).cpu().numpy()
    assert np.isfinite(hist).all()
    first, last = hist[:3, 0].mean(), hist[-10:, 0].mean()
    assert last < 0.6 * first, (first, last)
    assert hist[-10:, 2].mean() > hist[:3, 2].mean()                 # SSIM rises
    wp = flat.param["weight_params"].cpu().numpy()
    moved = np.abs(wp - w0.cpu().numpy())
    assert moved[2] > 0 and moved[3:].max() > 0                     # w_B and c_B are learnt
    assert moved[0] > 0                                             # sigma (EXP and LC)
