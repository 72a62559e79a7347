"""Torch-facing wrapper of the WSR C ABI: buffers, streams and autograd.

Everything computed here is computed by ``libwsr.so``; this module only owns
device buffers (torch tensors), passes pointers and the current stream, and
sizes the tile list.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import torch

from . import _abi as A

_DT = {torch.float32: A.WSR_F32, torch.float16: A.WSR_F16, torch.bfloat16: A.WSR_BF16}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Gaussians:
    """A Gaussian scene on the device (shapes as in ``include/wsr.h``)."""
    means: torch.Tensor          # [n, 3] float32
    log_scales: torch.Tensor     # [n, 3] float32 | bfloat16
    quats: torch.Tensor          # [n, 4] float32 | bfloat16, (w, x, y, z)
    sh: torch.Tensor             # [n, K, 3] float32 | float16
    opacity: torch.Tensor        # [n] logit or [n, K] SH, float32 | float16
    lc_v: torch.Tensor | None    # [n] float32
    sh_degree: int
    view_dependent: bool

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def c_struct(self) -> A.wsr_gaussians:
        return A.wsr_gaussians(
            self.n, self.sh_degree, A.WSR_OPACITY_SH if self.view_dependent else A.WSR_OPACITY_LOGIT,
            _DT[self.log_scales.dtype], _DT[self.sh.dtype],
            self.means.data_ptr(), self.log_scales.data_ptr(), self.quats.data_ptr(), self.sh.data_ptr(),
            self.opacity.data_ptr(), self.lc_v.data_ptr() if self.lc_v is not None else None)

    @staticmethod
    def from_scene(scene, device="cuda", reduced: bool = False) -> "Gaussians":
        """Upload a ``wsr_scenes.Scene``-like object (numpy arrays)."""
        def t(a, dt=torch.float32):
            return torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
        sq = torch.bfloat16 if reduced else torch.float32
        sh = torch.float16 if reduced else torch.float32
        return Gaussians(t(scene.means), t(scene.log_scales, sq), t(scene.quats, sq), t(scene.sh, sh),
                         t(scene.opacity, sh), t(scene.lc_v), int(scene.sh_degree),
                         bool(scene.view_dependent_opacity))


@dataclass
class FrameState:
    """Buffers produced by one forward pass and consumed by its backward."""
    records: torch.Tensor        # [V * n * 12] float32
    tile_offsets: torch.Tensor   # [T + 1] int32 (uint32 on the device)
    tile_list: torch.Tensor      # [capacity] int32 (uint32 on the device)
    rgb: torch.Tensor            # [P, 3]
    den: torch.Tensor            # [P]
    n: int


class Renderer:
    """Renders a fixed set of views at a fixed tile shape."""

    def __init__(self, cams, tile=(16, 16), device="cuda", headroom: float = 1.25, persistent: bool = False,
                 chunk: int = 0, deterministic: bool = False):
        self.lib = A.load()
        self.device = torch.device(device)
        self.cams = list(cams)
        self.cams_c, self.n_cams = A.make_cameras(self.cams)
        self.persistent = bool(persistent)
        self.deterministic = bool(deterministic)
        self.tiles_c = A.tiles(*tile, A.WSR_SCHEDULE_PERSISTENT if persistent else A.WSR_SCHEDULE_TILE_BLOCKS,
                               chunk, int(self.deterministic))
        # floats per gradient record of the render backward (wider in the deterministic mode)
        self.record_floats = A.WSR_GRAD_RECORD_FLOATS_DET if self.deterministic else A.WSR_GRAD_RECORD_FLOATS
        self.chunk = int(chunk)
        self.tile = tuple(tile)
        self.num_tiles = int(self.lib.wsr_num_tiles(self.cams_c, self.n_cams, ctypes.byref(self.tiles_c)))
        # kernels one wsr_bin launches: the count; the scan, in one kernel (with the persistent schedule's
        # tile order) up to WSR_SCAN_ONE_BLOCK_TILES tiles, else three (and three for the order); the
        # scatter; in the deterministic mode the sort of each tile's list
        if self.num_tiles <= A.WSR_SCAN_ONE_BLOCK_TILES:
            self.bin_kernels = 3
        else:
            self.bin_kernels = 5 + (3 if persistent else 0)
        self.bin_kernels += 1 if self.deterministic else 0
        self.num_pix = int(self.lib.wsr_num_pixels(self.cams_c, self.n_cams))
        ws = int(self.lib.wsr_workspace_size(self.cams_c, self.n_cams, ctypes.byref(self.tiles_c)))
        if self.num_tiles <= 0 or ws == 0:
            raise ValueError("invalid cameras or tile shape")
        self.workspace = torch.zeros(ws, dtype=torch.uint8, device=self.device)
        self.headroom = headroom
        self.capacity = 0
        self.last_total = 0

    # -- raw C-ABI calls (same names as include/wsr.h) --------------------
    def wsr_project(self, g: Gaussians, kind: int, wparams: torch.Tensor, records: torch.Tensor, stream=None):
        w = A.wsr_weight(kind, wparams.data_ptr())
        A.check("wsr_project", self.lib.wsr_project(ctypes.byref(g.c_struct()), self.cams_c, self.n_cams,
                                                    ctypes.byref(w), _ptr(records), _stream(stream)))

    def wsr_bin(self, records, n, offsets, tile_list, stream=None, total_dev=None):
        """``total_dev``: optional [1] int64 device tensor that receives the true instance count."""
        A.check("wsr_bin", self.lib.wsr_bin(_ptr(records), n, self.cams_c, self.n_cams, ctypes.byref(self.tiles_c),
                                            _ptr(offsets), _ptr(tile_list), tile_list.numel(),
                                            _ptr(total_dev) if total_dev is not None else None,
                                            _ptr(self.workspace), self.workspace.numel(), _stream(stream)))

    def wsr_bin_count(self, records, n, offsets, stream=None):
        A.check("wsr_bin_count", self.lib.wsr_bin_count(_ptr(records), n, self.cams_c, self.n_cams,
                                                        ctypes.byref(self.tiles_c), _ptr(offsets),
                                                        _ptr(self.workspace), self.workspace.numel(),
                                                        _stream(stream)))

    def wsr_bin_total(self, stream=None) -> int:
        t = ctypes.c_uint64(0)
        A.check("wsr_bin_total", self.lib.wsr_bin_total(_ptr(self.workspace), self.workspace.numel(),
                                                        ctypes.byref(t), _stream(stream)))
        return int(t.value)

    def wsr_render_fwd(self, records, n, offsets, tile_list, kind, wparams, rgb, den, stream=None):
        w = A.wsr_weight(kind, wparams.data_ptr())
        A.check("wsr_render_fwd", self.lib.wsr_render_fwd(
            _ptr(records), n, _ptr(offsets), _ptr(tile_list), self.cams_c, self.n_cams,
            ctypes.byref(self.tiles_c), ctypes.byref(w), _ptr(rgb), _ptr(den), _ptr(self.workspace),
            self.workspace.numel(), _stream(stream)))

    def wsr_render_bwd(self, g, records, offsets, tile_list, kind, wparams, rgb, den, grad_rgb, grad_records,
                       grads: A.wsr_grads, stream=None):
        w = A.wsr_weight(kind, wparams.data_ptr())
        A.check("wsr_render_bwd", self.lib.wsr_render_bwd(
            ctypes.byref(g.c_struct()), _ptr(records), _ptr(offsets), _ptr(tile_list), self.cams_c, self.n_cams,
            ctypes.byref(self.tiles_c), ctypes.byref(w), _ptr(rgb), _ptr(den), _ptr(grad_rgb), _ptr(grad_records),
            ctypes.byref(grads), _ptr(self.workspace), self.workspace.numel(), _stream(stream)))

    def wsr_render_bwd_tiles(self, records, n, offsets, tile_list, kind, wparams, rgb, den, grad_rgb, grad_records,
                             stream=None):
        w = A.wsr_weight(kind, wparams.data_ptr())
        A.check("wsr_render_bwd_tiles", self.lib.wsr_render_bwd_tiles(
            _ptr(records), n, _ptr(offsets), _ptr(tile_list), self.cams_c, self.n_cams, ctypes.byref(self.tiles_c),
            ctypes.byref(w), _ptr(rgb), _ptr(den), _ptr(grad_rgb), _ptr(grad_records), _ptr(self.workspace),
            self.workspace.numel(), _stream(stream)))

    def wsr_project_bwd(self, g, kind, wparams, grad_records, grads: A.wsr_grads, stream=None):
        w = A.wsr_weight(kind, wparams.data_ptr())
        A.check("wsr_project_bwd", self.lib.wsr_project_bwd(
            ctypes.byref(g.c_struct()), self.cams_c, self.n_cams, ctypes.byref(self.tiles_c), ctypes.byref(w),
            _ptr(grad_records), ctypes.byref(grads), _ptr(self.workspace), self.workspace.numel(), _stream(stream)))

    def wsr_count_pairs(self, st: FrameState, stream=None) -> tuple:
        """(pairs with q <= 9, slots the forward evaluates, slots the backward evaluates)."""
        cnt = torch.zeros(3, dtype=torch.int64, device=self.device)
        A.check("wsr_count_pairs", self.lib.wsr_count_pairs(
            _ptr(st.records), st.n, _ptr(st.tile_offsets), _ptr(st.tile_list), self.cams_c, self.n_cams,
            ctypes.byref(self.tiles_c), _ptr(cnt), _stream(stream)))
        return tuple(int(v) for v in cnt.cpu().tolist())

    def wsr_check(self, stream=None) -> int:
        return int(self.lib.wsr_check(_ptr(self.workspace), self.workspace.numel(), _stream(stream)))

    # -- convenience -------------------------------------------------------
    def alloc_state(self, n: int) -> FrameState:
        dev = self.device
        return FrameState(
            records=torch.empty(self.n_cams * n * A.WSR_RECORD_FLOATS, dtype=torch.float32, device=dev),
            tile_offsets=torch.empty(self.num_tiles + 1, dtype=torch.int32, device=dev),
            tile_list=torch.empty(max(self.capacity, 1), dtype=torch.int32, device=dev),
            rgb=torch.empty(self.num_pix, 3, dtype=torch.float32, device=dev),
            den=torch.empty(self.num_pix, dtype=torch.float32, device=dev), n=n)

    def _grow(self, total: int):
        self.capacity = max(int(math.ceil(total * self.headroom)) + 1024, self.capacity)

    def forward(self, g: Gaussians, kind: int, wparams: torch.Tensor, state: FrameState | None = None,
                stream=None, check: bool = True) -> FrameState:
        """Project, bin and render.  With ``check`` the tile list is sized
        exactly on first use and the capacity flag is verified (one host
        synchronisation); without it the caller checks ``wsr_check`` later."""
        n = g.n
        st = state or self.alloc_state(n)
        self.wsr_project(g, kind, wparams, st.records, stream)
        if self.capacity == 0:
            self.wsr_bin_count(st.records, n, st.tile_offsets, stream)
            self._grow(self.wsr_bin_total(stream))
        if st.tile_list.numel() < self.capacity:
            st.tile_list = torch.empty(self.capacity, dtype=torch.int32, device=self.device)
        self.wsr_bin(st.records, n, st.tile_offsets, st.tile_list, stream)
        if check:
            status = self.wsr_check(stream)
            if status == A.WSR_ERR_CAPACITY:
                self._grow(self.wsr_bin_total(stream))
                st.tile_list = torch.empty(self.capacity, dtype=torch.int32, device=self.device)
                self.wsr_bin(st.records, n, st.tile_offsets, st.tile_list, stream)
                A.check("wsr_bin", self.wsr_check(stream))
            else:
                A.check("wsr_bin", status)
        self.wsr_render_fwd(st.records, n, st.tile_offsets, st.tile_list, kind, wparams, st.rgb, st.den, stream)
        return st

    def backward(self, g: Gaussians, kind: int, wparams: torch.Tensor, st: FrameState, grad_rgb: torch.Tensor,
                 out: dict | None = None, grad_records: torch.Tensor | None = None, stream=None) -> dict:
        """Gradients of <grad_rgb, C> for every parameter (float32 tensors)."""
        dev = self.device
        n = g.n
        K = (g.sh_degree + 1) ** 2
        if out is None:
            out = dict(means=torch.empty(n, 3, device=dev), log_scales=torch.empty(n, 3, device=dev),
                       quats=torch.empty(n, 4, device=dev), sh=torch.empty(n, K, 3, device=dev),
                       opacity=torch.empty((n, K) if g.view_dependent else (n,), device=dev),
                       lc_v=torch.empty(n, device=dev), weight_params=torch.empty(6, device=dev))
        if grad_records is None:
            grad_records = torch.empty(self.n_cams * n * self.record_floats, device=dev)
        grads = A.wsr_grads(*[out[k].data_ptr() if out.get(k) is not None else None
                              for k in ("means", "log_scales", "quats", "sh", "opacity", "lc_v", "weight_params")])
        self.wsr_render_bwd(g, st.records, st.tile_offsets, st.tile_list, kind, wparams, st.rgb, st.den,
                            grad_rgb.contiguous(), grad_records, grads, stream)
        out["grad_records"] = grad_records
        return out

    def loss_l1(self, rgb, target, loss, grad, stream=None):
        A.check("wsr_loss_l1", self.lib.wsr_loss_l1(_ptr(rgb), _ptr(target), rgb.numel(), _ptr(loss), _ptr(grad),
                                                    _stream(stream)))

    def wsr_loss_3dgs(self, rgb, target, lam, loss, grad, stream=None):
        """L1 + lam * D-SSIM over this renderer's views; loss [3] = {L, L1, SSIM}."""
        A.check("wsr_loss_3dgs", self.lib.wsr_loss_3dgs(_ptr(rgb), _ptr(target), self.cams_c, self.n_cams,
                                                        float(lam), _ptr(loss), _ptr(grad), _stream(stream)))


class WSRRender(torch.autograd.Function):
    """Differentiable WSR image (Eq. 7) of ``renderer``'s views.

    Inputs: the Gaussian parameter tensors and the weight parameters
    [sigma, beta, w_B, c_B]; output: colours [P, 3] (views concatenated)."""

    @staticmethod
    def forward(ctx, renderer, kind, sh_degree, view_dependent, means, log_scales, quats, sh, opacity, lc_v,
                wparams):
        g = Gaussians(means.contiguous(), log_scales.contiguous(), quats.contiguous(), sh.contiguous(),
                      opacity.contiguous(), lc_v.contiguous() if lc_v is not None else None, sh_degree,
                      view_dependent)
        st = renderer.forward(g, kind, wparams.contiguous())
        ctx.renderer, ctx.kind, ctx.g, ctx.st, ctx.wparams = renderer, kind, g, st, wparams.contiguous()
        ctx.has_lcv = lc_v is not None
        return st.rgb.clone()

    @staticmethod
    def backward(ctx, grad_rgb):
        out = ctx.renderer.backward(ctx.g, ctx.kind, ctx.wparams, ctx.st, grad_rgb.float())
        return (None, None, None, None, out["means"], out["log_scales"], out["quats"], out["sh"],
                out["opacity"], out["lc_v"] if ctx.has_lcv else None, out["weight_params"])


def render(renderer: Renderer, kind: int, g: Gaussians, wparams: torch.Tensor) -> torch.Tensor:
    """Autograd entry point: returns colours [P, 3] for the renderer's views."""
    return WSRRender.apply(renderer, kind, g.sh_degree, g.view_dependent, g.means, g.log_scales, g.quats, g.sh,
                           g.opacity, g.lc_v, wparams)
