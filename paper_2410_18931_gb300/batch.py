"""Batched multi-view steps: one set of launches for many views, captured in
a CUDA graph, with the tile shape and schedule picked by measurement.

A step over V views is: project (parameters read once for all views), bin
all views' tiles in one index space, render every tile of every view, the L1
loss, the backward over every tile, and the projection backward summing the
views' gradients.  Every kernel is a C-ABI call of ``libwsr.so``; this module
only allocates buffers, captures the graph and times candidates.
"""
from __future__ import annotations

import torch

from . import _abi as A
from .render import Gaussians, Renderer

DEFAULT_SHAPES = ((8, 8), (16, 8), (16, 16), (32, 8))
DEFAULT_CHUNKS = (128, 64, 256, 512)   # Gaussians per block of the backward


class GraphStep:
    """Forward + L1 loss + backward over a fixed set of views, captured once.

    The tile list is sized from an exact count of the first frame plus
    ``headroom``; ``check()`` (one host synchronisation) reports whether a
    later replay overflowed it, in which case the caller rebuilds the step.
    """

    def __init__(self, g: Gaussians, cams, kind: int, wparams: torch.Tensor, target: torch.Tensor,
                 tile=(16, 16), persistent: bool = True, headroom: float = 1.3, capture: bool = True,
                 chunk: int = 0, deterministic: bool = False):
        self.g, self.kind, self.wparams = g, kind, wparams
        self.r = Renderer(cams, tile=tile, persistent=persistent, headroom=headroom, chunk=chunk,
                          deterministic=deterministic)
        self.st = self.r.forward(g, kind, wparams)           # sizes the tile list exactly (+ headroom)
        self.target = target.reshape(-1, 3).contiguous()
        dev = self.r.device
        n, K = g.n, (g.sh_degree + 1) ** 2
        self.loss = torch.zeros(1, device=dev)
        self.grad_rgb = torch.empty_like(self.st.rgb)
        self.grad_records = torch.empty(self.r.n_cams * n * self.r.record_floats, device=dev)
        self.out = dict(means=torch.empty(n, 3, device=dev), log_scales=torch.empty(n, 3, device=dev),
                        quats=torch.empty(n, 4, device=dev), sh=torch.empty(n, K, 3, device=dev),
                        opacity=torch.empty((n, K) if g.view_dependent else (n,), device=dev),
                        lc_v=torch.empty(n, device=dev), weight_params=torch.empty(6, device=dev))
        self.grads = A.wsr_grads(*[self.out[k].data_ptr() for k in
                                   ("means", "log_scales", "quats", "sh", "opacity", "lc_v", "weight_params")])
        self.graph = None
        if capture:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(2):
                    self.run()
            torch.cuda.current_stream().wait_stream(side)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self.run()

    def run(self):
        """The step as eager C-ABI calls on the current stream."""
        r, st, g, k, w = self.r, self.st, self.g, self.kind, self.wparams
        r.wsr_project(g, k, w, st.records)
        r.wsr_bin(st.records, g.n, st.tile_offsets, st.tile_list)
        r.wsr_render_fwd(st.records, g.n, st.tile_offsets, st.tile_list, k, w, st.rgb, st.den)
        r.loss_l1(st.rgb, self.target, self.loss, self.grad_rgb)
        r.wsr_render_bwd_tiles(st.records, g.n, st.tile_offsets, st.tile_list, k, w, st.rgb, st.den,
                               self.grad_rgb, self.grad_records)
        r.wsr_project_bwd(g, k, w, self.grad_records, self.grads)

    def replay(self):
        if self.graph is None:
            self.run()
        else:
            self.graph.replay()

    def check(self) -> int:
        """wsr_check of the workspace: WSR_OK, or WSR_ERR_CAPACITY after an overflow."""
        return self.r.wsr_check()

    @property
    def kernels_per_step(self) -> int:
        # project 1, bin (Renderer.bin_kernels), fwd 1, loss 1, bwd 1, project bwd 1;
        # deterministic: + the largest-pixel-term kernel and two ordered reductions
        return 5 + self.r.bin_kernels + (3 if self.r.deterministic else 0)


def time_step(step: GraphStep, reps: int = 5, warmup: int = 2, flush: torch.Tensor | None = None) -> float:
    """Mean milliseconds per replay (CUDA events on the current stream).  With
    ``flush`` (a buffer larger than L2), the buffer is overwritten before each
    replay, outside the events, so every replay starts from a cold L2."""
    for _ in range(warmup):
        step.replay()
    torch.cuda.synchronize()
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            step.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record()
        step.replay()
        e1.record()
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in ev) / reps


_cache: dict = {}


def autotune(g: Gaussians, cams, kind: int, wparams: torch.Tensor, target: torch.Tensor,
             shapes=DEFAULT_SHAPES, schedules=(False, True), chunks=DEFAULT_CHUNKS, reps: int = 3,
             flush: torch.Tensor | None = None) -> dict:
    """Time every (tile shape, schedule, Gaussians per backward block) on this
    workload and return the fastest as dict(tile=, persistent=, chunk=, ms=,
    table=[...]); ``reps`` and ``flush`` as in ``time_step``.  Results are
    cached per (Gaussian count, view sizes, storage types, weight kind)."""
    key = (g.n, tuple((c.width, c.height) for c in cams), str(g.sh.dtype), str(g.log_scales.dtype), kind,
           tuple(shapes), tuple(schedules), tuple(chunks))
    if key in _cache:
        return _cache[key]
    table = []
    for shape in shapes:
        for persistent in schedules:
            for chunk in chunks:
                step = GraphStep(g, cams, kind, wparams, target, tile=shape, persistent=persistent, chunk=chunk)
                ms = time_step(step, reps=reps, flush=flush)
                ok = step.check() == A.WSR_OK
                table.append(dict(tile=shape, persistent=persistent, chunk=chunk, ms=ms, ok=ok))
                del step
                torch.cuda.empty_cache()
    ran = [t for t in table if t["ok"]]
    if not ran:
        raise RuntimeError("autotune: every configuration overflowed its tile list")
    best = min(ran, key=lambda t: t["ms"])
    res = dict(tile=best["tile"], persistent=best["persistent"], chunk=best["chunk"], ms=best["ms"], table=table)
    _cache[key] = res
    return res
