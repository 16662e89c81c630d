"""gray_setup_noalloc: the image-plane set-up for callers that cannot
allocate device memory (a host code that hands the tracer a slice of its own
memory pool, or a loop where allocator calls are not allowed).  It must write
exactly the state gray_setup writes, call after call, through the C ABI.

This file is collected last on purpose (tests/test_zz_*): if it fails, a run
that stops at the first failure has already run every other test.
"""
import ctypes as C
import math

import pytest
import torch

from paper_1303_5057_gb300 import build, gray
from paper_1303_5057_gb300.inputs import Image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    gray.lib()
    torch.cuda.init()


def _states(prec, images, first_ray, n_state):
    """The same images set up by gray_setup (with a context) and by
    gray_setup_noalloc (without), into zero-filled buffers."""
    nbytes = gray.gray_state_bytes(n_state, prec)
    ref = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    got = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    ctx = gray.gray_create(gray.Options(precision=prec))
    try:
        gray.gray_setup(ctx, images, ref, n_state, first_ray)
    finally:
        torch.cuda.synchronize()
        gray.gray_destroy(ctx)
    gray.gray_setup_noalloc(prec, images, got, n_state, first_ray)
    torch.cuda.synchronize()
    return ref, got


@pytest.mark.parametrize("prec", [gray.FP64, gray.FP32_KAHAN_SEL64])
def test_noalloc_setup_equals_setup_on_two_calls_in_a_row(prec):
    first = [Image(a=0.99, incl=math.radians(90.0), nx=37, ny=29),
             Image(a=0.3, incl=math.radians(12.0), nx=8, ny=64, alpha0=-3.0, alpha1=5.0)]
    second = [Image(a=0.0, incl=math.radians(60.0), nx=64, ny=64),
              Image(a=0.7, incl=math.radians(45.0), nx=5, ny=3, M=1.0, r_obs=5000.0),
              Image(a=-0.5, incl=math.radians(170.0), nx=100, ny=1)]
    n1 = sum(im.n for im in first)
    ref, got = _states(prec, first, 0, n1)
    assert torch.equal(ref, got)
    # the second call reuses the same device table with a different, longer
    # image list and a ray offset: nothing of the first call may leak through
    n2 = 7 + sum(im.n for im in second)
    ref, got = _states(prec, second, 7, n2)
    assert torch.equal(ref, got)


def test_noalloc_rejects_too_many_images_and_bad_arguments():
    L = gray.lib()
    n = gray.NOALLOC_MAX_IMAGES + 1
    arr = (gray._Image * n)()
    for k in range(n):
        arr[k] = gray._Image(0.5, 1.0, 1000.0, 1.0, 1, 1, -1.0, 1.0, -1.0, 1.0)
    state = torch.zeros(gray.gray_state_bytes(n, gray.FP64), dtype=torch.uint8, device="cuda")
    sb = state.numel()
    p = C.c_void_p(state.data_ptr())
    assert L.gray_setup_noalloc(gray.FP64, arr, n, p, sb, n, 0, None) == gray.EINVAL
    assert L.gray_setup_noalloc(gray.FP64, arr, n - 1, p, sb, n, 0, None) == gray.OK
    assert L.gray_setup_noalloc(7, arr, 1, p, sb, n, 0, None) == gray.EINVAL
    assert L.gray_setup_noalloc(gray.FP64, arr, 1, p, 16, n, 0, None) == gray.EINVAL
    assert L.gray_setup_noalloc(gray.FP64, arr, 1, p, sb, n, n, None) == gray.EINVAL
    torch.cuda.synchronize()
