"""The C-ABI library on a machine without a GPU: it builds, loads, exports
every function that ``include/wsr.h`` declares, and rejects bad arguments on
the host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wsr.h")


def _cuda_present() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


# The argument-error tests pass made-up device addresses that validation must
# reject before any launch.  They run where no GPU is present, so that a
# check that goes missing can never hand such an address to a kernel.
host_validation_only = pytest.mark.skipif(_cuda_present(), reason="fake device pointers: run without a GPU")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__._build_module().build()
    from paper_2410_18931_gb300 import _abi
    return _abi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(wsr_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("wsr_project", "wsr_bin", "wsr_render_fwd", "wsr_render_bwd"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2410_18931_gb300 import _abi
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _abi.exported_symbols(), f"binding lacks {name}"


def test_status_strings(lib):
    assert lib.wsr_status_string(0) == b"ok"
    assert b"capacity" in lib.wsr_status_string(2)
    assert lib.wsr_version() >= 10000


def _cam(w=1920, h=1080):
    from paper_2410_18931_gb300 import _abi
    import wsr_scenes as ws
    arr, n = _abi.make_cameras([ws.look_at((0, 0, -5), width=w, height=h)])
    return arr, n


def test_tile_and_pixel_counts(lib):
    from paper_2410_18931_gb300 import _abi
    cams, n = _cam()
    t16 = _abi.tiles(16, 16)
    assert lib.wsr_num_tiles(cams, n, ctypes.byref(t16)) == 120 * 68
    assert lib.wsr_num_tiles(cams, n, ctypes.byref(_abi.tiles(32, 8))) == 60 * 135
    assert lib.wsr_num_pixels(cams, n) == 1920 * 1080
    assert lib.wsr_workspace_size(cams, n, ctypes.byref(t16)) >= 256 + 4 * (8160 + 1)
    # unsupported tile shape
    assert lib.wsr_workspace_size(cams, n, ctypes.byref(_abi.tiles(12, 12))) == 0
    assert lib.wsr_num_tiles(cams, 0, ctypes.byref(t16)) == 0


@host_validation_only
def test_argument_errors_are_returned(lib):
    from paper_2410_18931_gb300 import _abi as A
    cams, n = _cam(64, 48)
    t16 = A.tiles(16, 16)
    fake = 1 << 20   # never dereferenced: validation fails first
    w = A.wsr_weight(A.WSR_WEIGHT_EXP, fake)
    g = A.wsr_gaussians(10, 3, A.WSR_OPACITY_SH, A.WSR_F32, A.WSR_F32, fake, fake, fake, fake, fake, None)
    # null scene / weight
    assert lib.wsr_project(None, cams, n, ctypes.byref(w), fake, None) == A.WSR_ERR_INVALID_ARG
    assert lib.wsr_project(ctypes.byref(g), cams, n, None, fake, None) == A.WSR_ERR_INVALID_ARG
    # SH degree out of range
    bad = A.wsr_gaussians(10, 4, 1, 0, 0, fake, fake, fake, fake, fake, None)
    assert lib.wsr_project(ctypes.byref(bad), cams, n, ctypes.byref(w), fake, None) == A.WSR_ERR_INVALID_ARG
    # LC needs the per-Gaussian v_i
    wlc = A.wsr_weight(A.WSR_WEIGHT_LC, fake)
    assert lib.wsr_project(ctypes.byref(g), cams, n, ctypes.byref(wlc), fake, None) == A.WSR_ERR_INVALID_ARG
    # unknown weight kind
    wbad = A.wsr_weight(7, fake)
    assert lib.wsr_project(ctypes.byref(g), cams, n, ctypes.byref(wbad), fake, None) == A.WSR_ERR_INVALID_ARG
    # mixed storage types are valid enums but unsupported
    mix = A.wsr_gaussians(10, 3, 1, A.WSR_BF16, A.WSR_F32, fake, fake, fake, fake, fake, None)
    assert lib.wsr_project(ctypes.byref(mix), cams, n, ctypes.byref(w), fake, None) == A.WSR_ERR_UNSUPPORTED
    # misaligned record buffer
    assert lib.wsr_project(ctypes.byref(g), cams, n, ctypes.byref(w), fake + 4, None) == A.WSR_ERR_INVALID_ARG
    # too many views
    many = (A.wsr_camera * 40)(*([cams[0]] * 40))
    assert lib.wsr_project(ctypes.byref(g), many, 40, ctypes.byref(w), fake, None) == A.WSR_ERR_INVALID_ARG
    # a zero-size camera
    zc = (A.wsr_camera * 1)(cams[0])
    zc[0].width = 0
    assert lib.wsr_workspace_size(zc, 1, ctypes.byref(t16)) == 0
    # workspace too small
    ws = lib.wsr_workspace_size(cams, n, ctypes.byref(t16))
    assert lib.wsr_bin(fake, 10, cams, n, ctypes.byref(t16), fake, fake, 100, None, fake, ws - 16,
                       None) == A.WSR_ERR_INVALID_ARG
    # unsupported tile shape
    assert lib.wsr_bin(fake, 10, cams, n, ctypes.byref(A.tiles(24, 24)), fake, fake, 100, None, fake, ws,
                       None) == A.WSR_ERR_UNSUPPORTED
    # a misaligned device total (uint64), and the static entry's misaligned total and status (int32)
    assert lib.wsr_bin(fake, 10, cams, n, ctypes.byref(t16), fake, fake, 100, fake + 4, fake, ws,
                       None) == A.WSR_ERR_INVALID_ARG
    assert lib.wsr_bin_static(fake, 10, cams, n, ctypes.byref(t16), fake, fake, 100, fake + 4, None,
                              None) == A.WSR_ERR_INVALID_ARG
    assert lib.wsr_bin_static(fake, 10, cams, n, ctypes.byref(t16), fake, fake, 100, None, fake + 2,
                              None) == A.WSR_ERR_INVALID_ARG
    # null outputs of the renderer
    assert lib.wsr_render_fwd(fake, 10, fake, fake, cams, n, ctypes.byref(t16), ctypes.byref(w), None, fake,
                              fake, ws, None) == A.WSR_ERR_INVALID_ARG
    # backward without gradient outputs
    assert lib.wsr_render_bwd(ctypes.byref(g), fake, fake, fake, cams, n, ctypes.byref(t16), ctypes.byref(w),
                              fake, fake, fake, fake, None, fake, ws, None) == A.WSR_ERR_INVALID_ARG
    # negative counts
    assert lib.wsr_loss_l1(fake, fake, -1, fake, fake, None) == A.WSR_ERR_INVALID_ARG
    # the L1 loss reads and writes float4: every array 16-byte aligned
    assert lib.wsr_loss_l1(fake + 4, fake, 12, fake, fake, None) == A.WSR_ERR_INVALID_ARG
    assert lib.wsr_loss_l1(fake, fake, 12, fake, fake + 8, None) == A.WSR_ERR_INVALID_ARG
    assert lib.wsr_check(None, 0, None) == A.WSR_ERR_INVALID_ARG


@host_validation_only
def test_training_entry_points_reject_bad_arguments(lib):
    from paper_2410_18931_gb300 import _abi as A
    cams, n = _cam(64, 48)
    fake = 1 << 20   # never dereferenced: validation fails first
    # 3DGS loss: lambda outside [0, 1], null outputs, zero-size view
    for lam in (-0.5, 1.01, float("nan")):
        assert lib.wsr_loss_3dgs(fake, fake, cams, n, lam, fake, fake, None) == A.WSR_ERR_INVALID_ARG
    assert lib.wsr_loss_3dgs(fake, fake, cams, n, 0.2, None, fake, None) == A.WSR_ERR_INVALID_ARG
    assert lib.wsr_loss_3dgs(fake, fake, cams, 0, 0.2, fake, fake, None) == A.WSR_ERR_INVALID_ARG
    zc = (A.wsr_camera * 1)(cams[0])
    zc[0].height = 0
    assert lib.wsr_loss_3dgs(fake, fake, zc, 1, 0.2, fake, fake, None) == A.WSR_ERR_INVALID_ARG
    hp = A.wsr_adam_hparams(0.9, 0.999, 1e-15)

    def adam(groups, hp=hp, p=fake, state=fake, guard=None, guard_bytes=0):
        arr = (A.wsr_adam_group * max(1, len(groups)))(*groups)
        return lib.wsr_adam_step(p, fake, fake, fake, arr, len(groups), ctypes.byref(hp), state, guard,
                                 guard_bytes, None)

    ok = A.wsr_adam_group(0, 100, 1e-3, 1e-3, 0, 0)
    assert adam([ok], p=fake + 4) == A.WSR_ERR_INVALID_ARG                       # misaligned buffer
    assert adam([ok], state=fake + 2) == A.WSR_ERR_INVALID_ARG                   # misaligned state
    assert adam([A.wsr_adam_group(2, 100, 1e-3, 1e-3, 0, 0)]) == A.WSR_ERR_INVALID_ARG      # offset % 4
    assert adam([A.wsr_adam_group(0, 1 << 32, 1e-3, 1e-3, 0, 0)]) == A.WSR_ERR_INVALID_ARG  # count
    assert adam([A.wsr_adam_group(0, 100, 1e-3, 1e-3, 8, 9)]) == A.WSR_ERR_INVALID_ARG     # head > period
    assert adam([ok, A.wsr_adam_group(96, 10, 1e-3, 1e-3, 0, 0)]) == A.WSR_ERR_INVALID_ARG  # overlap
    assert adam([ok] * (A.WSR_ADAM_MAX_GROUPS + 1)) == A.WSR_ERR_INVALID_ARG
    assert adam([A.wsr_adam_group(0, 100, float("inf"), 1e-3, 0, 0)]) == A.WSR_ERR_INVALID_ARG
    assert adam([ok], hp=A.wsr_adam_hparams(1.0, 0.999, 1e-8)) == A.WSR_ERR_INVALID_ARG
    assert adam([ok], hp=A.wsr_adam_hparams(0.9, 0.999, -1.0)) == A.WSR_ERR_INVALID_ARG
    assert adam([ok], guard=fake, guard_bytes=16) == A.WSR_ERR_INVALID_ARG        # guard smaller than a header
    assert lib.wsr_adam_step(fake, fake, fake, fake, None, 0, ctypes.byref(hp), None, None, 0,
                             None) == A.WSR_ERR_INVALID_ARG                       # no state


def test_weight_params_rounded_are_float32_exact():
    import numpy as np
    import wsr_scenes as ws
    w = ws.default_weight(ws.EXP, c_bg=(0.1, 0.2, 0.3))
    r = w.rounded()
    assert r.kind == w.kind
    vals = [r.sigma, r.beta, r.w_bg, *r.c_bg]
    assert all(float(np.float32(v)) == v for v in vals)
    assert np.array_equal(r.as_array(), w.as_array())


@host_validation_only
def test_tiles_chunk_is_validated(lib):
    from paper_2410_18931_gb300 import _abi as A
    cams, n = _cam(64, 48)
    for chunk, expect in ((0, True), (64, True), (128, True), (256, True), (512, True)):
        assert (lib.wsr_workspace_size(cams, n, ctypes.byref(A.tiles(16, 16, 0, chunk))) > 0) == expect
    fake = 1 << 20
    ws = lib.wsr_workspace_size(cams, n, ctypes.byref(A.tiles(16, 16)))
    w = A.wsr_weight(A.WSR_WEIGHT_EXP, fake)
    for chunk, status in ((32, A.WSR_ERR_UNSUPPORTED), (1024, A.WSR_ERR_UNSUPPORTED), (-1, A.WSR_ERR_INVALID_ARG)):
        t = A.tiles(16, 16, 0, chunk)
        assert lib.wsr_render_fwd(fake, 10, fake, fake, cams, n, ctypes.byref(t), ctypes.byref(w), fake, fake,
                                  fake, ws, None) == status


def test_bench_uses_a_fixed_launch_configuration_as_given():
    """With tile shape, schedule and backward block size all given, the bench
    runs them without tuning (nothing is launched)."""
    import argparse

    import bench
    args = argparse.Namespace(tile="16x8", schedule="persistent", chunk="64")
    assert bench.launch_config(args, None, None, None, None) == ((16, 8), True, 64, None)
    args = argparse.Namespace(tile="32x8", schedule="per-tile", chunk="128")
    assert bench.launch_config(args, None, None, None, None) == ((32, 8), False, 128, None)


@host_validation_only
def test_deterministic_flag_is_validated(lib):
    """wsr_tiles.deterministic: 0 or 1; the deterministic workspace holds the
    per-tile background terms as well; wsr_project_bwd checks the flag too."""
    from paper_2410_18931_gb300 import _abi as A
    cams, n = _cam(64, 48)
    base = lib.wsr_workspace_size(cams, n, ctypes.byref(A.tiles(16, 16)))
    det = lib.wsr_workspace_size(cams, n, ctypes.byref(A.tiles(16, 16, 0, 0, 1)))
    assert det > base > 0
    assert lib.wsr_workspace_size(cams, n, ctypes.byref(A.tiles(16, 16, 0, 0, 2))) == 0
    assert lib.wsr_workspace_size(cams, n, ctypes.byref(A.tiles(16, 16, 0, 0, -1))) == 0
    fake = 1 << 20   # never dereferenced: validation fails first
    g = A.wsr_gaussians()
    w = A.wsr_weight(0, fake)
    grads = A.wsr_grads()
    assert lib.wsr_project_bwd(ctypes.byref(g), cams, n, ctypes.byref(A.tiles(16, 16, 0, 0, 3)), ctypes.byref(w),
                               fake, ctypes.byref(grads), fake, 1 << 16, None) == A.WSR_ERR_INVALID_ARG


@host_validation_only
def test_misaligned_record_buffers_are_rejected(lib):
    """Render records are read, and gradient records updated, as 16-byte
    vectors; tile offsets and lists are 32-bit words."""
    from paper_2410_18931_gb300 import _abi as A
    cams, n = _cam(64, 48)
    fake = 1 << 20   # never dereferenced: validation fails first
    for det in (0, 1):
        t = A.tiles(16, 16, 0, 0, det)
        ws = lib.wsr_workspace_size(cams, n, ctypes.byref(t))
        w = A.wsr_weight(A.WSR_WEIGHT_EXP, fake)
        fwd = lambda rec, lst: lib.wsr_render_fwd(rec, 10, fake, lst, cams, n, ctypes.byref(t), ctypes.byref(w),
                                                  fake, fake, fake, ws, None)
        assert fwd(fake + 8, fake) == A.WSR_ERR_INVALID_ARG
        assert fwd(fake, fake + 2) == A.WSR_ERR_INVALID_ARG
        bwd = lambda rec, grec: lib.wsr_render_bwd_tiles(rec, 10, fake, fake, cams, n, ctypes.byref(t),
                                                         ctypes.byref(w), fake, fake, fake, grec, fake, ws, None)
        assert bwd(fake + 4, fake) == A.WSR_ERR_INVALID_ARG
        assert bwd(fake, fake + 8) == A.WSR_ERR_INVALID_ARG
        g = A.wsr_gaussians(10, 0, A.WSR_OPACITY_LOGIT, A.WSR_F32, A.WSR_F32, fake, fake, fake, fake, fake, None)
        grads = A.wsr_grads()
        assert lib.wsr_project_bwd(ctypes.byref(g), cams, n, ctypes.byref(t), ctypes.byref(w), fake + 4,
                                   ctypes.byref(grads), fake, ws, None) == A.WSR_ERR_INVALID_ARG
        assert lib.wsr_bin(fake, 10, cams, n, ctypes.byref(t), fake + 1, fake, 100, None, fake, ws,
                           None) == A.WSR_ERR_INVALID_ARG
        assert lib.wsr_count_pairs(fake + 4, 10, fake, fake, cams, n, ctypes.byref(t), fake,
                                   None) == A.WSR_ERR_INVALID_ARG


def test_binding_constants_match_the_header():
    """Every numeric #define and enum constant of include/wsr.h has the same
    value in the Python binding."""
    from paper_2410_18931_gb300 import _abi as A
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"^#define\s+(WSR_\w+)\s+(\d+)\s*$", text, flags=re.M)}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        consts.update({k: int(v) for k, v in re.findall(r"(WSR_\w+)\s*=\s*(\d+)", body)})
    assert len(consts) >= 20
    for k, v in consts.items():
        assert getattr(A, k) == v, k


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct crossing the ABI has the same size and field offsets in
    C (compiled with the host compiler from include/wsr.h) and in ctypes."""
    import shutil
    import subprocess
    from paper_2410_18931_gb300 import _abi as A
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = ["wsr_camera", "wsr_gaussians", "wsr_weight", "wsr_tiles", "wsr_grads", "wsr_adam_group",
               "wsr_adam_hparams", "wsr_adam_state"]
    lines = ['#include <stdio.h>', '#include "wsr.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for name, _ in getattr(A, s)._fields_:
            lines.append(f'printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln.strip())}
    for s in structs:
        cls = getattr(A, s)
        assert c_layout[(s, "size")] == ctypes.sizeof(cls), s
        for name, _ in cls._fields_:
            assert c_layout[(s, name)] == getattr(cls, name).offset, (s, name)


def test_binding_signatures_match_the_header_prototypes():
    """Each prototype of include/wsr.h and its ctypes signature agree on the
    return type and, argument by argument, on the C type."""
    from paper_2410_18931_gb300 import _abi as A
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = re.findall(r"^\s*(const\s+)?(\w+)\s*(\*?)\s*(wsr_\w+)\s*\(([^)]*)\)\s*;", text, flags=re.M)
    assert len(protos) == len(A._SIGS)
    scalars = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
               "size_t": ctypes.c_size_t, "float": ctypes.c_float, "wsr_status": ctypes.c_int}
    device_structs = {"wsr_adam_state"}      # lives in device memory: a plain device pointer in the binding

    def ctype_of(decl):
        decl = decl.replace("const ", "").strip()
        if "*" in decl:
            base = decl.split("*")[0].strip()
            if base.startswith("wsr_") and base not in device_structs:
                return ctypes.POINTER(getattr(A, base))
            return ("ptr", base)
        return scalars[decl]

    for const, ret, star, name, params in protos:
        res, args = A._SIGS[name]
        want_ret = ctypes.c_char_p if star else scalars[ret]
        assert res is want_ret, name
        plist = [] if params.strip() in ("", "void") else [p.strip() for p in params.split(",")]
        assert len(plist) == len(args), name
        for p, a in zip(plist, args):
            decl = re.sub(r"\s*\w+$", "", p)            # drop the parameter name
            t = ctype_of(decl)
            if isinstance(t, tuple):                    # a plain data pointer: void* in the binding
                assert a in (ctypes.c_void_p, A._c_void_p) or t[1] == "uint64_t", (name, p)
            else:
                assert a is t, (name, p)
