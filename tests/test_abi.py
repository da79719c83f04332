"""C-ABI library checks that need no GPU: it loads, exports every entry point
declared in include/turbogs.h, and rejects bad arguments before any launch."""
import ctypes
import os
import re

import pytest

from paper_2412_13547_b300 import build_native, raster as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "turbogs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    build_native.build()
    lib = R.load()
    names = declared_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(R.SYMBOLS)


def test_python_constants_match_the_header():
    """Buffer sizes the binding allocates follow the header's #defines."""
    src = open(os.path.join(ROOT, "include", "turbogs.h")).read()
    defs = {m.group(1): m.group(2) for m in re.finditer(r"#define\s+(GS_[A-Z0-9_]+)\s+\(?([0-9]+)u?(?:\s*<<\s*([0-9]+))?",
                                                          src)}
    shifts = {m.group(1): int(m.group(2)) << int(m.group(3)) for m in
              re.finditer(r"#define\s+(GS_[A-Z0-9_]+)\s+\(([0-9]+)u\s*<<\s*([0-9]+)\)", src)}
    assert int(defs["GS_SPLAT_FLOATS"]) == R.SPLAT_FLOATS
    assert int(defs["GS_GRAD2D_FLOATS"]) == R.GRAD2D_FLOATS
    assert int(defs["GS_ADAM_MAX_TENSORS"]) == R.ADAM_MAX_TENSORS
    assert int(defs["GS_MAX_VIEWS"]) == R.MAX_VIEWS
    assert int(defs["GS_TARGET_F32"]) == R.TARGET_F32 and int(defs["GS_TARGET_U8"]) == R.TARGET_U8
    assert int(defs["GS_MAX_ROW_TENSORS"]) == R.GS_MAX_ROW_TENSORS
    assert shifts["GS_BIN_SORT_STATIC_SCRATCH_BYTES"] == R.BIN_SORT_STATIC_SCRATCH_BYTES
    for role in ("COPY", "MEANS", "LOG_SCALES", "QUATS", "STATE", "ZERO"):
        assert int(defs["GS_ROW_" + role]) == getattr(R, "GS_ROW_" + role)
    assert ctypes.sizeof(R.GsDilation) == 6 * 4


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the C layout of the header:
    a C program built with gcc against include/turbogs.h prints every field's
    offset and each struct's size."""
    structs = {"GsCamera": R.GsCamera, "GsDilation": R.GsDilation, "GsAdamTensor": R.GsAdamTensor,
               "GsAdamParams": R.GsAdamParams, "GsRowTensor": R.GsRowTensor, "GsView": R.GsView}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "turbogs.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], check=True, capture_output=True,
                                                    text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert int(got[f"{name}.{f[0]}"]) == getattr(cls, f[0]).offset, (name, f[0])


def test_host_only_calls():
    assert R.gs_version() >= 100
    cam = type("C", (), dict(R=[[1, 0, 0], [0, 1, 0], [0, 0, 1]], T=[0, 0, 0], fx=100.0, fy=100.0, cx=63.5,
                             cy=47.5, width=130, height=97))()
    assert R.gs_grid(cam, R.Dilation(1, 0, 0)) == (130, 97, 9, 7)
    assert R.gs_grid(cam, R.Dilation(2, 1, 0)) == (65, 49, 5, 4)
    assert R.gs_grid(cam, R.Dilation(3, 2, 2, tile=8)) == (43, 32, 6, 4)
    assert R.gs_bin_sort_workspace_size(1000, 5000, 8, 8) > 0
    # a grid larger than the counting path's limit needs the pair-sized sort buffers
    assert R.gs_bin_sort_workspace_size(1000, 10**6, 480, 270) > R.gs_bin_sort_workspace_size(1000, 10**6, 240, 135)
    with pytest.raises(R.GsError):
        R.gs_grid(cam, R.Dilation(2, 2, 0))       # offset >= d
    with pytest.raises(R.GsError):
        R.gs_grid(cam, R.Dilation(2, 0, 0, tile=12))


def test_bad_arguments_are_rejected_before_launch():
    lib = R.load()
    cam = R.GsCamera()
    cam.width, cam.height, cam.fx, cam.fy = 64, 64, 50.0, 50.0
    dil = R.GsDilation(1, 0, 0, 0, 16)
    P = ctypes.c_void_p
    # n < 0
    assert lib.gs_project(-1, 0, 0, *[None] * 5, ctypes.byref(cam), ctypes.byref(dil), *[None] * 5, None) == R.GS_ERR_ARG
    # sh degree 4
    assert lib.gs_project(0, 4, 0, *[None] * 5, ctypes.byref(cam), ctypes.byref(dil), *[None] * 5, None) == R.GS_ERR_ARG
    # null pointers with n > 0
    assert lib.gs_project(5, 0, 0, *[None] * 5, ctypes.byref(cam), ctypes.byref(dil), *[None] * 5, None) == R.GS_ERR_ARG
    assert "null" in lib.gs_last_error().decode()
    # bad dilation
    bad = R.GsDilation(0, 0, 0, 0, 16)
    assert lib.gs_render_fwd(0, None, None, P(16), ctypes.byref(cam), ctypes.byref(bad), None, None, None, None,
                             None, 0, None, None) == R.GS_ERR_ARG
    # bad launch shape: 3 pixels per thread
    bg = (ctypes.c_float * 3)()
    assert lib.gs_render_fwd(0, P(16), P(16), P(16), ctypes.byref(cam), ctypes.byref(dil), bg, P(16), P(16), P(16),
                             None, 3, None, None) == R.GS_ERR_ARG
    tile8 = R.GsDilation(1, 0, 0, 0, 8)  # 4 pixels per thread would leave a 16-thread CTA
    assert lib.gs_render_fwd(0, P(16), P(16), P(16), ctypes.byref(cam), ctypes.byref(tile8), bg, P(16), P(16),
                             P(16), None, 4, None, None) == R.GS_ERR_ARG
    assert lib.gs_tile_order(None, -1, None, None) == R.GS_ERR_ARG
    # capacity >= 2^31
    assert lib.gs_bin_sort(0, None, None, None, None, 1, 1, None, 0, 1 << 31, None, P(16), P(16), None, None) == R.GS_ERR_ARG
    # adam: too many tensors, bad step
    arr = (R.GsAdamTensor * 9)()
    assert lib.gs_adam(arr, 9, 0.9, 0.999, 1e-8, 1, None, None) == R.GS_ERR_ARG
    assert lib.gs_adam(arr, 1, 0.9, 0.999, 1e-8, 0, None, None) == R.GS_ERR_ARG
    # unknown forward flags, and the fused loss without its buffers
    assert lib.gs_render_fwd_batch(0, None, 0, bg, None, None, 0, 0, None) == R.GS_ERR_ARG
    v = (R.GsView * 1)()
    v[0].cam, v[0].dil = cam, dil
    v[0].ranges, v[0].img, v[0].t_final, v[0].last = 16, 16, 16, 16
    assert lib.gs_render_fwd_batch(0, v, 1, bg, None, None, 0, 4, None) == R.GS_ERR_ARG
    assert "flags" in lib.gs_last_error().decode()
    assert lib.gs_render_fwd_batch(0, v, 1, bg, None, None, 0, R.FWD_L1, None) == R.GS_ERR_ARG
    assert "fused loss" in lib.gs_last_error().decode()
    # a target type the kernels do not know
    assert lib.gs_loss_l1(ctypes.byref(cam), ctypes.byref(dil), P(16), P(16), 7, P(16), P(16), None) == R.GS_ERR_ARG
    assert "target_dtype" in lib.gs_last_error().decode()
    ws = P(256)
    assert lib.gs_ssim(ctypes.byref(cam), ctypes.byref(dil), P(16), P(16), 2, 0, P(16), None, ws, 1 << 30,
                       None) == R.GS_ERR_ARG
    # the optimizer pass with the next view's projection: the next view is required, the Adam
    # dense, and its output buffers present and 16-byte aligned
    adam = R.GsAdamParams()
    for t in range(5):
        adam.param[t], adam.m[t], adam.v[t] = 256 * (t + 1), 256 * (t + 6), 256 * (t + 11)
    adam.beta1, adam.beta2, adam.step = 0.9, 0.999, 1
    nxt = (R.GsView * 1)()
    nxt[0].cam, nxt[0].dil = cam, dil
    nxt[0].splats, nxt[0].radii, nxt[0].rects, nxt[0].tiles_touched = 4096, 4096, 4096, 4096

    def bwd_next(next_view):
        return lib.gs_project_bwd_adam_next(8, 0, 0, P(4096), ctypes.byref(cam), ctypes.byref(dil), P(4096),
                                            P(4096), ctypes.byref(adam), None, None, None, None, next_view, None)
    assert bwd_next(None) == R.GS_ERR_ARG
    assert "next view is null" in lib.gs_last_error().decode()
    adam.sparse = 1
    assert bwd_next(nxt) == R.GS_ERR_ARG
    assert "dense Adam" in lib.gs_last_error().decode()
    adam.sparse = 0
    nxt[0].splats = 4104  # 8-byte aligned only
    assert bwd_next(nxt) == R.GS_ERR_ARG
    assert "16-byte aligned" in lib.gs_last_error().decode()
    nxt[0].splats, nxt[0].radii = 4096, None
    assert bwd_next(nxt) == R.GS_ERR_ARG
    # empty inputs are a no-op success
    assert lib.gs_project(0, 0, 0, *[None] * 5, ctypes.byref(cam), ctypes.byref(dil), *[None] * 5, None) == R.GS_OK


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(R, "_lib", None)
    monkeypatch.setattr(R, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        R.load()
