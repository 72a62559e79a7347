"""GB300 (sm_103a) Weighted Sum Rendering: sort-free Gaussian splatting.

The compute lives in ``libwsr.so`` (C ABI in ``include/wsr.h``); this package
is its binding.  Importing it loads the library and fails if it is not built.
"""
from . import _abi
from ._abi import (WSR_BF16, WSR_F16, WSR_F32, WSR_WEIGHT_DIR, WSR_WEIGHT_EXP, WSR_WEIGHT_LC, WSRError,
                   exported_symbols, load)

load()

from .render import FrameState, Gaussians, Renderer, WSRRender, render  # noqa: E402
from .batch import GraphStep, autotune, time_step  # noqa: E402
from .train import Adam, FlatParams, TrainStep  # noqa: E402

__all__ = ["Gaussians", "Renderer", "FrameState", "WSRRender", "render", "GraphStep", "autotune", "time_step",
           "FlatParams", "Adam", "TrainStep",
           "WSRError", "load",
           "exported_symbols", "WSR_F32", "WSR_F16", "WSR_BF16", "WSR_WEIGHT_DIR", "WSR_WEIGHT_EXP",
           "WSR_WEIGHT_LC"]
