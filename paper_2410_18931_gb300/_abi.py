"""ctypes binding of ``libwsr.so`` (declarations in ``include/wsr.h``).

Argument marshalling only: every function here forwards to the C ABI of the
same name, turning torch tensors into device pointers and a torch stream into
a ``cudaStream_t``.  A missing library is an error (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwsr.so")

WSR_OK, WSR_ERR_INVALID_ARG, WSR_ERR_CAPACITY, WSR_ERR_CUDA, WSR_ERR_TIMEOUT, WSR_ERR_UNSUPPORTED = range(6)
WSR_F32, WSR_F16, WSR_BF16 = 0, 1, 2
WSR_WEIGHT_DIR, WSR_WEIGHT_EXP, WSR_WEIGHT_LC = 0, 1, 2
WSR_OPACITY_LOGIT, WSR_OPACITY_SH = 0, 1
WSR_MAX_VIEWS = 32
WSR_RECORD_FLOATS = 12
WSR_GRAD_RECORD_FLOATS = 12
WSR_GRAD_RECORD_FLOATS_DET = 32      # deterministic mode: 9 int64 sums and their 9 bounds per record
WSR_DET_MAX_SEGMENT = 8192
WSR_SCAN_ONE_BLOCK_TILES = 32768     # wsr_bin scans (and orders) up to this many tiles in one kernel
WSR_BIN_STATIC_MAX_TILES = 65536     # tiles over all views that wsr_bin_static handles
WSR_BIN_STATIC_BYTES = 270848        # its fixed scratch array, held by every GPU that loads the library

_c_void_p = ctypes.c_void_p


class wsr_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("T", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("znear", ctypes.c_float)]


class wsr_gaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("opacity_mode", ctypes.c_int32),
                ("dtype_scales_quats", ctypes.c_int32), ("dtype_sh", ctypes.c_int32),
                ("means", _c_void_p), ("log_scales", _c_void_p), ("quats", _c_void_p),
                ("sh", _c_void_p), ("opacity", _c_void_p), ("lc_v", _c_void_p)]


class wsr_weight(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("params", _c_void_p)]


class wsr_tiles(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("deterministic", ctypes.c_int32)]


class wsr_grads(ctypes.Structure):
    _fields_ = [("means", _c_void_p), ("log_scales", _c_void_p), ("quats", _c_void_p), ("sh", _c_void_p),
                ("opacity", _c_void_p), ("lc_v", _c_void_p), ("weight_params", _c_void_p)]


WSR_ADAM_MAX_GROUPS = 16


class wsr_adam_group(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int64), ("count", ctypes.c_int64), ("lr", ctypes.c_float),
                ("lr_tail", ctypes.c_float), ("period", ctypes.c_int32), ("head", ctypes.c_int32)]


class wsr_adam_hparams(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double)]


class wsr_adam_state(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int32), ("c1", ctypes.c_float), ("c2", ctypes.c_float),
                ("skipped", ctypes.c_int32)]


# name -> (restype, argtypes)
_P = ctypes.POINTER
_SIGS = {
    "wsr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "wsr_version": (ctypes.c_int32, []),
    "wsr_num_tiles": (ctypes.c_int64, [_P(wsr_camera), ctypes.c_int32, _P(wsr_tiles)]),
    "wsr_num_pixels": (ctypes.c_int64, [_P(wsr_camera), ctypes.c_int32]),
    "wsr_workspace_size": (ctypes.c_size_t, [_P(wsr_camera), ctypes.c_int32, _P(wsr_tiles)]),
    "wsr_project": (ctypes.c_int, [_P(wsr_gaussians), _P(wsr_camera), ctypes.c_int32, _P(wsr_weight),
                                   _c_void_p, _c_void_p]),
    "wsr_bin": (ctypes.c_int, [_c_void_p, ctypes.c_int64, _P(wsr_camera), ctypes.c_int32, _P(wsr_tiles),
                               _c_void_p, _c_void_p, ctypes.c_uint64, _c_void_p, _c_void_p, ctypes.c_size_t,
                               _c_void_p]),
    "wsr_bin_count": (ctypes.c_int, [_c_void_p, ctypes.c_int64, _P(wsr_camera), ctypes.c_int32,
                                     _P(wsr_tiles), _c_void_p, _c_void_p, ctypes.c_size_t, _c_void_p]),
    "wsr_bin_total": (ctypes.c_int, [_c_void_p, ctypes.c_size_t, _P(ctypes.c_uint64), _c_void_p]),
    "wsr_render_fwd": (ctypes.c_int, [_c_void_p, ctypes.c_int64, _c_void_p, _c_void_p, _P(wsr_camera),
                                      ctypes.c_int32, _P(wsr_tiles), _P(wsr_weight), _c_void_p, _c_void_p,
                                      _c_void_p, ctypes.c_size_t, _c_void_p]),
    "wsr_render_bwd": (ctypes.c_int, [_P(wsr_gaussians), _c_void_p, _c_void_p, _c_void_p, _P(wsr_camera),
                                      ctypes.c_int32, _P(wsr_tiles), _P(wsr_weight), _c_void_p, _c_void_p,
                                      _c_void_p, _c_void_p, _P(wsr_grads), _c_void_p, ctypes.c_size_t,
                                      _c_void_p]),
    "wsr_render_bwd_tiles": (ctypes.c_int, [_c_void_p, ctypes.c_int64, _c_void_p, _c_void_p, _P(wsr_camera),
                                            ctypes.c_int32, _P(wsr_tiles), _P(wsr_weight), _c_void_p, _c_void_p,
                                            _c_void_p, _c_void_p, _c_void_p, ctypes.c_size_t, _c_void_p]),
    "wsr_project_bwd": (ctypes.c_int, [_P(wsr_gaussians), _P(wsr_camera), ctypes.c_int32, _P(wsr_tiles),
                                       _P(wsr_weight), _c_void_p, _P(wsr_grads), _c_void_p, ctypes.c_size_t,
                                       _c_void_p]),
    "wsr_bin_static": (ctypes.c_int, [_c_void_p, ctypes.c_int64, _P(wsr_camera), ctypes.c_int32, _P(wsr_tiles),
                                      _c_void_p, _c_void_p, ctypes.c_uint64, _c_void_p, _c_void_p, _c_void_p]),
    "wsr_count_pairs": (ctypes.c_int, [_c_void_p, ctypes.c_int64, _c_void_p, _c_void_p, _P(wsr_camera),
                                       ctypes.c_int32, _P(wsr_tiles), _c_void_p, _c_void_p]),
    "wsr_loss_l1": (ctypes.c_int, [_c_void_p, _c_void_p, ctypes.c_int64, _c_void_p, _c_void_p, _c_void_p]),
    "wsr_loss_3dgs": (ctypes.c_int, [_c_void_p, _c_void_p, _P(wsr_camera), ctypes.c_int32, ctypes.c_float,
                                     _c_void_p, _c_void_p, _c_void_p]),
    "wsr_adam_step": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _P(wsr_adam_group), ctypes.c_int32,
                                     _P(wsr_adam_hparams), _c_void_p, _c_void_p, ctypes.c_size_t, _c_void_p]),
    "wsr_check": (ctypes.c_int, [_c_void_p, ctypes.c_size_t, _c_void_p]),
}

_lib = None


def load(path: str | None = None):
    """Load libwsr.so (built by ``paper_2410_18931_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libwsr.so is not built ({p}); run paper_2410_18931_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list:
    return sorted(_SIGS)


class WSRError(RuntimeError):
    def __init__(self, fn: str, status: int):
        lib = load()
        msg = lib.wsr_status_string(status).decode()
        super().__init__(f"{fn} failed: {msg} ({status})")
        self.status = status


def check(fn: str, status: int) -> None:
    if status != WSR_OK:
        raise WSRError(fn, status)


def make_cameras(cams) -> tuple:
    """(ctypes array of wsr_camera, count) from objects with R, T, fx, fy,
    cx, cy, width, height and znear attributes."""
    arr = (wsr_camera * len(cams))()
    for k, c in enumerate(cams):
        R = [float(v) for v in np.asarray(c.R, dtype=np.float64).reshape(9)]
        T = [float(v) for v in np.asarray(c.T, dtype=np.float64).reshape(3)]
        arr[k].R[:] = R
        arr[k].T[:] = T
        arr[k].fx, arr[k].fy, arr[k].cx, arr[k].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        arr[k].width, arr[k].height = int(c.width), int(c.height)
        arr[k].znear = float(c.znear)
    return arr, len(cams)


WSR_SCHEDULE_TILE_BLOCKS, WSR_SCHEDULE_PERSISTENT = 0, 1


def tiles(tw: int, th: int, schedule: int = WSR_SCHEDULE_TILE_BLOCKS, chunk: int = 0,
          deterministic: int = 0) -> wsr_tiles:
    """Tile shape, schedule, the backward's Gaussians per block (0: the default) and
    the deterministic mode (1: bitwise-reproducible results)."""
    return wsr_tiles(int(tw), int(th), int(schedule), int(chunk), int(deterministic))
