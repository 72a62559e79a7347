"""Training-step driver: optimise a Gaussian scene against target views with
the paper's loss (Sec. 4.4: L1 + 0.2 D-SSIM) and Adam, every kernel a C-ABI
call of ``libwsr.so``, the whole step captured as one CUDA graph.

The topology is fixed (no densification or pruning): the step exercises the
renderer's gradients and the learnable weight parameters sigma, beta, w_B,
c_B and v_i (Eqs. 8-10, Table 5 of the paper) without a dataset.

Learning rates.  The paper trains as 3DGS does and states none of its own;
the defaults below are 3DGS's for the shared parameters (positions, log
scales, rotations, SH with the higher bands at 1/20 of the DC rate, opacity)
and a chosen 1e-3 for the WSR weight parameters and v_i, which the paper
leaves open.  The position rate is constant (3DGS decays it over 30k
iterations; a fixed-length driver has no schedule).
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi as A
from .render import Gaussians, Renderer, _ptr, _stream

PARAM_ORDER = ("means", "log_scales", "quats", "sh", "opacity", "lc_v", "weight_params")
DEFAULT_LR = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, sh=2.5e-3, opacity=5e-2, lc_v=1e-3,
                  weight_params=1e-3)
TAIL_RATIO = 1.0 / 20.0           # higher SH bands (colour and view-dependent opacity)
DSSIM_LAMBDA = 0.2


class FlatParams:
    """Every trainable tensor of a scene in one flat float32 buffer (each
    tensor starting on a 16-byte boundary), with a gradient buffer of the same
    layout; ``param[name]`` and ``grad[name]`` are shaped views into them."""

    def __init__(self, shapes: dict, device="cuda"):
        self.device = torch.device(device)
        self.shapes = {k: tuple(shapes[k]) for k in PARAM_ORDER}
        self.offsets, o = {}, 0
        for k in PARAM_ORDER:
            self.offsets[k] = o
            n = 1
            for d in self.shapes[k]:
                n *= d
            o += (n + 3) // 4 * 4
        self.numel = o
        self.data = torch.zeros(o, device=self.device)
        self.grad_data = torch.zeros(o, device=self.device)
        self.param = {k: self._view(self.data, k) for k in PARAM_ORDER}
        self.grad = {k: self._view(self.grad_data, k) for k in PARAM_ORDER}

    def _view(self, buf, k):
        n = 1
        for d in self.shapes[k]:
            n *= d
        return buf[self.offsets[k]:self.offsets[k] + n].view(self.shapes[k])

    def count(self, k) -> int:
        return self.param[k].numel()

    @staticmethod
    def from_scene(scene, wparams, device="cuda") -> "FlatParams":
        """Copy a ``wsr_scenes.Scene``-like object (numpy arrays) and the six
        weight parameters [sigma, beta, w_B, c_B] into a new flat buffer."""
        arrays = dict(means=scene.means, log_scales=scene.log_scales, quats=scene.quats, sh=scene.sh,
                      opacity=scene.opacity, lc_v=scene.lc_v, weight_params=wparams)
        f = FlatParams({k: tuple(torch.as_tensor(arrays[k]).shape) for k in PARAM_ORDER}, device)
        for k in PARAM_ORDER:
            f.param[k].copy_(torch.as_tensor(arrays[k], dtype=torch.float32))
        return f

    def gaussians(self, sh_degree: int, view_dependent: bool) -> Gaussians:
        p = self.param
        return Gaussians(p["means"], p["log_scales"], p["quats"], p["sh"], p["opacity"], p["lc_v"],
                         int(sh_degree), bool(view_dependent))

    def grads_c(self) -> A.wsr_grads:
        return A.wsr_grads(*[self.grad[k].data_ptr() for k in PARAM_ORDER])


class Adam:
    """Adam over a ``FlatParams`` buffer through ``wsr_adam_step``: one group
    per parameter tensor, the higher SH bands at ``tail_ratio`` of their
    tensor's rate.  The moments and the step count live on the device."""

    def __init__(self, flat: FlatParams, sh_degree: int, view_dependent: bool, lr: dict | None = None,
                 betas=(0.9, 0.999), eps: float = 1e-15, tail_ratio: float = TAIL_RATIO):
        self.lib = A.load()
        self.flat = flat
        self.lr = dict(DEFAULT_LR, **(lr or {}))
        K = (sh_degree + 1) ** 2
        groups = []
        for k in PARAM_ORDER:
            rate = float(self.lr.get(k, 0.0))
            if rate == 0.0 or flat.count(k) == 0:
                continue
            period = head = 0
            if k == "sh" and K > 1:
                period, head = 3 * K, 3
            elif k == "opacity" and view_dependent and K > 1:
                period, head = K, 1
            groups.append(A.wsr_adam_group(flat.offsets[k], flat.count(k), rate, rate * tail_ratio, period, head))
        if len(groups) > A.WSR_ADAM_MAX_GROUPS:
            raise ValueError("too many parameter groups")
        self.groups = (A.wsr_adam_group * max(1, len(groups)))(*groups)
        self.n_groups = len(groups)
        self.hp = A.wsr_adam_hparams(float(betas[0]), float(betas[1]), float(eps))
        self.exp_avg = torch.zeros_like(flat.data)
        self.exp_avg_sq = torch.zeros_like(flat.data)
        self.state = torch.zeros(4, dtype=torch.int32, device=flat.device)     # wsr_adam_state

    def wsr_adam_step(self, guard: torch.Tensor | None = None, stream=None):
        A.check("wsr_adam_step", self.lib.wsr_adam_step(
            _ptr(self.flat.data), _ptr(self.flat.grad_data), _ptr(self.exp_avg), _ptr(self.exp_avg_sq),
            self.groups, self.n_groups, ctypes.byref(self.hp), _ptr(self.state), _ptr(guard),
            0 if guard is None else guard.numel(), _stream(stream)))

    def read_state(self) -> dict:
        s = self.state.cpu()
        return dict(step=int(s[0]), skipped=int(s[3]))

    def snapshot(self):
        return (self.flat.data.clone(), self.exp_avg.clone(), self.exp_avg_sq.clone(), self.state.clone())

    def restore(self, snap):
        for dst, src in zip((self.flat.data, self.exp_avg, self.exp_avg_sq, self.state), snap):
            dst.copy_(src)


class TrainStep:
    """One optimisation step over a fixed set of views:

        project -> bin -> render -> loss (L1 + lam D-SSIM) -> render backward
        -> projection backward -> Adam

    captured as one CUDA graph.  The tile list is sized from an exact count
    at construction plus ``headroom``; a step whose binning overflows it
    updates nothing (Adam reads the workspace error on the device), and
    ``train`` rebuilds the step with a fresh count when that happens.
    """

    def __init__(self, flat: FlatParams, sh_degree: int, view_dependent: bool, cams, kind: int,
                 target: torch.Tensor, lr: dict | None = None, lam: float = DSSIM_LAMBDA, tile=(16, 16),
                 persistent: bool = False, headroom: float = 1.5, capture: bool = True, chunk: int = 0,
                 deterministic: bool = False):
        self.flat, self.kind, self.lam = flat, kind, float(lam)
        self.cams, self.tile, self.persistent, self.headroom = list(cams), tile, persistent, headroom
        self.chunk, self.deterministic = int(chunk), bool(deterministic)
        self.g = flat.gaussians(sh_degree, view_dependent)
        self.wparams = flat.param["weight_params"]
        self.target = target.reshape(-1, 3).contiguous().float()
        self.opt = Adam(flat, sh_degree, view_dependent, lr)
        if self.target.numel() != 3 * sum(int(c.width) * int(c.height) for c in self.cams):
            raise ValueError("target must hold num_pixels * 3 values")
        dev = flat.device
        self.loss = torch.zeros(3, device=dev)
        self.grads = flat.grads_c()
        self._build(capture)

    def _build(self, capture: bool):
        dev = self.flat.device
        self.r = Renderer(self.cams, tile=self.tile, persistent=self.persistent, headroom=self.headroom,
                          chunk=self.chunk, deterministic=self.deterministic)
        self.st = self.r.forward(self.g, self.kind, self.wparams)
        self.grad_rgb = torch.empty_like(self.st.rgb)
        self.grad_records = torch.empty(self.r.n_cams * self.g.n * self.r.record_floats, device=dev)
        self.graph = None
        if capture:
            snap = self.opt.snapshot()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                self.run()                  # first launches outside the capture
            torch.cuda.current_stream().wait_stream(side)
            self.opt.restore(snap)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self.run()

    def run(self):
        """The step as eager C-ABI calls on the current stream."""
        r, st, g, k, w = self.r, self.st, self.g, self.kind, self.wparams
        r.wsr_project(g, k, w, st.records)
        r.wsr_bin(st.records, g.n, st.tile_offsets, st.tile_list)
        r.wsr_render_fwd(st.records, g.n, st.tile_offsets, st.tile_list, k, w, st.rgb, st.den)
        r.wsr_loss_3dgs(st.rgb, self.target, self.lam, self.loss, self.grad_rgb)
        r.wsr_render_bwd_tiles(st.records, g.n, st.tile_offsets, st.tile_list, k, w, st.rgb, st.den,
                               self.grad_rgb, self.grad_records)
        r.wsr_project_bwd(g, k, w, self.grad_records, self.grads)
        self.opt.wsr_adam_step(guard=r.workspace)

    def replay(self):
        if self.graph is None:
            self.run()
        else:
            self.graph.replay()

    @property
    def kernels_per_step(self) -> int:
        # project 1, bin (Renderer.bin_kernels), fwd 1, loss 1, bwd 1, project bwd 1, Adam 2;
        # deterministic: + the largest-pixel-term kernel and two ordered reductions
        return 7 + self.r.bin_kernels + (3 if self.deterministic else 0)

    def train(self, steps: int, check_every: int = 10) -> torch.Tensor:
        """Make ``steps`` Adam updates; returns the loss triples {L, L1, SSIM}
        of the steps that made them, [steps, 3] on the device.  Every
        ``check_every`` replays the Adam state is read (one synchronisation);
        when a replay was skipped (tile-list overflow), the step is rebuilt
        with a fresh count and the missing updates are made."""
        st = self.opt.read_state()
        start, seen_skips = st["step"], st["skipped"]
        goal, done = start + steps, start
        losses, stepno = [], []
        while done < goal:
            n = min(check_every, goal - done)
            buf = torch.empty(n, 3, device=self.flat.device)
            sb = torch.empty(n, dtype=torch.int32, device=self.flat.device)
            for i in range(n):
                self.replay()
                buf[i].copy_(self.loss)
                sb[i].copy_(self.opt.state[0])
            losses.append(buf)
            stepno.append(sb)
            st = self.opt.read_state()
            done = st["step"]
            if st["skipped"] != seen_skips:
                seen_skips = st["skipped"]
                self._build(self.graph is not None)     # recount, regrow and recapture
        loss = torch.cat(losses)
        sn = torch.cat(stepno)
        prev = torch.cat([torch.tensor([start], dtype=torch.int32, device=sn.device), sn[:-1]])
        return loss[sn != prev]
