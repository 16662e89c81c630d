"""The C-ABI library without a GPU: it loads, exports every function that
include/gray.h declares, and its host-side logic (layout sizes, defaults,
argument validation that returns before any CUDA call) behaves."""
import ctypes as C
import os
import re

import pytest

from paper_1303_5057_gb300 import build, gray


@pytest.fixture(scope="module")
def L():
    build.build()
    return gray.lib()


def test_exports_every_declared_function(L):
    names = gray.header_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name


def test_header_constants_match_binding():
    text = open(gray.HEADER).read()
    consts = dict(re.findall(r"#define (GRAY_[A-Z0-9_]+) \(?(-?\d+)\)?", text))
    for name, val in consts.items():
        py = name[len("GRAY_"):]
        if hasattr(gray, py):
            assert getattr(gray, py) == int(val), name


def test_state_bytes(L):
    for prec in (gray.FP64, gray.FP32, gray.FP32_KAHAN, gray.FP32_KAHAN_SEL64):
        assert gray.gray_state_bytes(0, prec) == 0
        b1 = gray.gray_state_bytes(1, prec)
        assert b1 > 0 and b1 % 256 == 0
        n = 1 << 20
        per = (32 * 3 if prec == gray.FP64 else 16 * 5 + 32) + 32 + 16 + 16 + 4
        if prec == gray.FP32_KAHAN_SEL64:
            per += 4  # the zone's return list
        assert gray.gray_state_bytes(n, prec) == per * n
    assert gray.gray_state_bytes(-1, gray.FP64) == 0
    assert gray.gray_state_bytes(10, 7) == 0


def test_defaults_and_strerror(L):
    o = gray.gray_default_options()
    assert o == gray.Options()
    assert gray.gray_strerror(0) == "success"
    assert "invalid" in gray.gray_strerror(gray.EINVAL)
    assert gray.gray_strerror(-99) == "unknown error code"
    assert "cancel" in gray.gray_strerror(gray.ECANCEL)
    assert gray.gray_launch_count() >= 0


@pytest.mark.parametrize("bad", [dict(precision=9), dict(step_rule=5), dict(max_steps=0), dict(block=48),
                                 dict(h_frac=0.0), dict(h_frac=float("nan")), dict(cap_frac=0.5),
                                 dict(eps_xi=-1.0), dict(r_sw=-0.1), dict(blocks_per_sm=-1)])
def test_create_rejects_bad_options_before_touching_the_device(L, bad):
    opt = gray.Options(**bad)
    h = C.c_void_p()
    o = opt._c()
    assert L.gray_create(C.byref(h), C.byref(o)) == gray.EINVAL
    assert not h.value


def test_calls_reject_null_context(L):
    assert L.gray_setup(None, None, 1, None, 0, 1, 0, None) == gray.EINVAL
    assert L.gray_trace(None, None, 0, 0, None, 0, 0, None, None, None) == gray.EINVAL
    assert L.gray_plan(None, None, 0, 0, None, 0, 0, 4, 100, None, 0, None) == gray.EINVAL
    assert L.gray_setup_plan(None, None, 1, None, 0, 1, 0, 4, 100, None, 0, None) == gray.EINVAL
    assert L.gray_render(None, None, 0, 0, 0, 0, 0, None, 0, None) == gray.EINVAL
    assert L.gray_shadow(None, None, 0, 0, 0, None, 0, None, 0, None) == gray.EINVAL
    assert L.gray_ring(None, None, 0, 0, 0, None, 0, None, 0, None, 0, None) == gray.EINVAL
    assert L.gray_splat(None, None, 0, 0, 0, 0, None, None, None, 0, None) == gray.EINVAL
    assert L.gray_clear(None, None, 0, 0, 0, 0, None) == gray.EINVAL
    assert L.gray_cancel(None, 1) == gray.EINVAL
    assert L.gray_range_stats(None, None, 0, 0, None, 0, None, None) == gray.EINVAL


def test_structures_match_the_header(tmp_path):
    """The binding's structures against the header as a C compiler lays it
    out (sizes and the offsets of the fields added last)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "gray.h"
int main(void) {
    printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gray_image), offsetof(gray_image, grid),
           sizeof(gray_options), sizeof(gray_camera), offsetof(gray_camera, status_mask),
           sizeof(gray_ring_info), sizeof(gray_shadow_info), sizeof(gray_pixel32));
    return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(gray.HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(gray._Image), gray._Image.grid.offset, ctypes.sizeof(gray._Options),
            ctypes.sizeof(gray._Camera), gray._Camera.status_mask.offset, gray.RING_DTYPE.itemsize,
            gray.SHADOW_DTYPE.itemsize, gray.PIXEL32_DTYPE.itemsize]
    assert got == want


def test_eval_rejects_bad_arguments(L):
    assert L.gray_eval(99, gray.FP64, None, 1, None, None) == gray.EINVAL
    assert L.gray_eval(gray.EVAL_RHS, gray.FP32_KAHAN, None, 1, None, None) == gray.EINVAL
    assert L.gray_eval(gray.EVAL_RHS, gray.FP64, None, -1, None, None) == gray.EINVAL
    assert L.gray_eval(gray.EVAL_RHS, gray.FP64, None, 0, None, None) == gray.OK


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libgray.so the binding raises: there is no fallback path."""
    monkeypatch.setattr(gray, "_lib", None)
    monkeypatch.setattr(gray, "LIB_PATH", str(tmp_path / "libgray.so"))
    with pytest.raises(RuntimeError, match="libgray.so not found"):
        gray.lib()
    with pytest.raises(RuntimeError):
        gray.Tracer(gray.Options(), 16)


def test_noalloc_rejects_a_state_beyond_32_bit_ray_indices(L):
    """gray_setup_noalloc takes the same state bound as gray_setup (ray
    indices are 32-bit in the work queues): 2^31 rays are refused before any
    CUDA call, even with a buffer size that would hold them."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("host-side validation test: runs where no GPU is visible")
    except ImportError:
        pass
    im = (gray._Image * 1)(gray._Image(0.5, 1.0, 1000.0, 1.0, 1, 1, -1.0, 1.0, -1.0, 1.0, 0, 0))
    n = 1 << 31
    big = gray.gray_state_bytes(n, gray.FP64)
    assert big > 0
    assert L.gray_setup_noalloc(gray.FP64, im, 1, C.c_void_p(4096), big, n, 0, None) == gray.EINVAL
    # one ray fewer passes validation and only then needs the device (absent here)
    assert L.gray_setup_noalloc(gray.FP64, im, 1, C.c_void_p(4096), big, n - 1, 0, None) == gray.ECUDA
