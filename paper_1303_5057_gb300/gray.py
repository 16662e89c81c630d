"""Thin ctypes binding of libgray (C ABI in include/gray.h).

Argument marshalling only: every step of the tracer runs in the library's
CUDA kernels.  PyTorch supplies device memory (uint8 / float64 tensors) and
streams.  Function names are those of the C ABI; negative return codes raise
``GrayError``.  If libgray.so is missing the first call raises: there is no
other implementation to fall back to.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from dataclasses import dataclass, fields

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgray.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "gray.h")

# constants mirrored from include/gray.h (checked against it by the tests)
OK, EINVAL, ECUDA, ENOMEM, ECANCEL = 0, -1, -2, -3, -4
ACTIVE, CAPTURED, ESCAPED, STEP_CAP, NONFINITE, EMPTY, EQUATOR = 0, 1, 2, 3, 4, 5, 6
FP64, FP32, FP32_KAHAN, FP32_KAHAN_SEL64 = 0, 1, 2, 3
STEP_BENCH, STEP_EQ2 = 0, 1
RENDER_PIXELS64, RENDER_PIXELS32, RENDER_RECORD, RENDER_INVARIANTS = 0, 1, 3, 4
EVAL_CHRISTOFFEL, EVAL_RHS, EVAL_INITIAL, EVAL_XI, EVAL_SINCOS, EVAL_RECIP = 0, 1, 2, 3, 4, 5
EVAL_SINCOS_DS, EVAL_NORM = 6, 7
LAUNCH_PERSISTENT, LAUNCH_ONE_PER_THREAD = 0, 1
ZONE_DS, ZONE_FP64 = 0, 1
GRID_CARTESIAN, GRID_POLAR = 0, 1
RECORD = 17
NOALLOC_MAX_IMAGES = 4096

PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp32_kahan": FP32_KAHAN, "fp32_kahan_sel64": FP32_KAHAN_SEL64}


class GrayError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s failed: %s (%d)" % (where, gray_strerror(code), code))
        self.code = code


class _Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("step_rule", C.c_int32), ("max_steps", C.c_int32),
                ("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("refill", C.c_int32),
                ("launch", C.c_int32), ("stop_equator", C.c_int32),
                ("zone_arith", C.c_int32), ("reserved", C.c_int32),
                ("h_frac", C.c_double), ("h_min", C.c_double), ("cap_frac", C.c_double),
                ("eps_xi", C.c_double), ("r_esc_frac", C.c_double), ("r_sw", C.c_double)]


class _Image(C.Structure):
    _fields_ = [("a", C.c_double), ("M", C.c_double), ("r_obs", C.c_double), ("incl", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32), ("alpha0", C.c_double), ("alpha1", C.c_double),
                ("beta0", C.c_double), ("beta1", C.c_double), ("grid", C.c_int32), ("reserved", C.c_int32)]


class _Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("look", C.c_double * 3), ("up", C.c_double * 3), ("fov", C.c_double),
                ("half_height", C.c_double), ("sprite", C.c_double), ("width", C.c_int32), ("height", C.c_int32),
                ("status_mask", C.c_int32), ("clear", C.c_int32)]


@dataclass
class Camera:
    """Camera of gray_splat (see include/gray.h): eye, look-at point and up
    vector in Cartesian units of M; vertical field of view in radians (0 =
    orthographic with the given half height); sprite radius in pixels;
    status_mask selects the rays drawn by status (bit 1 << status)."""
    eye: tuple = (60.0, 0.0, 20.0)
    look: tuple = (0.0, 0.0, 0.0)
    up: tuple = (0.0, 0.0, 1.0)
    fov: float = 0.7
    half_height: float = 10.0
    sprite: float = 0.0
    width: int = 640
    height: int = 480
    status_mask: int = 1
    clear: int = 1

    def _c(self):
        d3 = C.c_double * 3
        return _Camera(d3(*self.eye), d3(*self.look), d3(*self.up), float(self.fov), float(self.half_height),
                       float(self.sprite), int(self.width), int(self.height), int(self.status_mask), int(self.clear))


SHADOW_DTYPE = np.dtype([("n_captured", "<i8"), ("n_escaped", "<i8"), ("n_other", "<i8"),
                         ("area", "<f8"), ("radius", "<f8"), ("alpha_c", "<f8"), ("beta_c", "<f8")])
PIXEL64_DTYPE = np.dtype([("r", "<f8"), ("theta", "<f8"), ("phi", "<f8"), ("status", "<i4"), ("steps", "<i4")])
PIXEL32_DTYPE = np.dtype([("r", "<f4"), ("theta", "<f4"), ("phi", "<f4"), ("status", "<i4")])
RING_DTYPE = np.dtype([("D", "<f8"), ("R_mean", "<f8"), ("A", "<f8"), ("alpha_min", "<f8"), ("alpha_max", "<f8"),
                       ("n_captured", "<i8"), ("n_wrong", "<i8"), ("n_open", "<i4"), ("n_rows", "<i4")])


@dataclass
class Options:
    """gray_options; defaults are gray_default_options()."""
    precision: int = FP64
    step_rule: int = STEP_BENCH
    max_steps: int = 100000
    block: int = 0
    blocks_per_sm: int = 0
    refill: int = 0
    launch: int = LAUNCH_PERSISTENT
    stop_equator: int = 0
    zone_arith: int = 0  # ZONE_DS
    reserved: int = 0
    h_frac: float = 1.0 / 32.0
    h_min: float = 1e-3
    cap_frac: float = 1.01
    eps_xi: float = 1e-3
    r_esc_frac: float = 1.0
    r_sw: float = 0.0

    def _c(self):
        return _Options(*[getattr(self, f.name) for f in fields(self)])


_lib = None


def lib():
    """Load libgray.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libgray.so not found at %s: build it with "
                           "`python -m paper_1303_5057_gb300.build`" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, sz, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.POINTER(C.c_double)
    L.gray_default_options.argtypes = [C.POINTER(_Options)]
    L.gray_default_options.restype = None
    L.gray_state_bytes.argtypes = [i64, i32]
    L.gray_state_bytes.restype = sz
    L.gray_create.argtypes = [C.POINTER(vp), C.POINTER(_Options)]
    L.gray_create.restype = C.c_int
    L.gray_destroy.argtypes = [vp]
    L.gray_destroy.restype = None
    L.gray_setup.argtypes = [vp, C.POINTER(_Image), i32, vp, sz, i64, i64, vp]
    L.gray_setup.restype = C.c_int
    L.gray_setup_noalloc.argtypes = [i32, C.POINTER(_Image), i32, vp, sz, i64, i64, vp]
    L.gray_setup_noalloc.restype = C.c_int
    L.gray_setup_rays.argtypes = [vp, vp, i64, C.c_double, vp, sz, i64, i64, vp]
    L.gray_setup_rays.restype = C.c_int
    L.gray_trace.argtypes = [vp, vp, sz, i64, vp, i64, i64, C.POINTER(i64), C.POINTER(i64), vp]
    L.gray_trace.restype = C.c_int
    L.gray_plan.argtypes = [vp, vp, sz, i64, C.POINTER(_Image), i32, i64, i32, i32, vp, sz, vp]
    L.gray_plan.restype = C.c_int
    L.gray_setup_plan.argtypes = [vp, C.POINTER(_Image), i32, vp, sz, i64, i64, i32, i32, vp, sz, vp]
    L.gray_setup_plan.restype = C.c_int
    L.gray_trace.restype = C.c_int
    L.gray_clear.argtypes = [vp, vp, sz, i64, i64, i64, vp]
    L.gray_clear.restype = C.c_int
    L.gray_count_active.argtypes = [vp, vp, sz, i64, C.POINTER(i64), i32, C.POINTER(i64), vp]
    L.gray_count_active.restype = C.c_int
    L.gray_range_stats.argtypes = [vp, vp, sz, i64, vp, i32, vp, vp]
    L.gray_range_stats.restype = C.c_int
    L.gray_render.argtypes = [vp, vp, sz, i64, i64, i64, i32, vp, sz, vp]
    L.gray_render.restype = C.c_int
    L.gray_shadow.argtypes = [vp, vp, sz, i64, i64, C.POINTER(_Image), i32, vp, sz, vp]
    L.gray_shadow.restype = C.c_int
    L.gray_ring.argtypes = [vp, vp, sz, i64, i64, C.POINTER(_Image), i32, vp, sz, vp, sz, vp]
    L.gray_ring.restype = C.c_int
    L.gray_splat.argtypes = [vp, vp, sz, i64, i64, i64, C.POINTER(_Camera), vp, vp, sz, vp]
    L.gray_splat.restype = C.c_int
    L.gray_eval.argtypes = [i32, i32, vp, i64, vp, vp]
    L.gray_eval.restype = C.c_int
    L.gray_cancel.argtypes = [vp, i32]
    L.gray_cancel.restype = C.c_int
    L.gray_set_timing.argtypes = [vp, i32]
    L.gray_set_timing.restype = C.c_int
    L.gray_timings.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i64)]
    L.gray_timings.restype = C.c_int
    L.gray_strerror.argtypes = [C.c_int]
    L.gray_strerror.restype = C.c_char_p
    L.gray_fma_peak.argtypes = [i32, i32, i32, i64, vp, sz, vp]
    L.gray_fma_peak.restype = C.c_int
    L.gray_launch_count.argtypes = []
    L.gray_launch_count.restype = i64
    _lib = L
    return L


def header_functions():
    """Names of the functions declared in include/gray.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(gray_[a-z_0-9]+)\s*\(", text)))


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _check(rc, where):
    if rc < 0:
        raise GrayError(rc, where)
    return rc


def _images(images):
    arr = (_Image * len(images))()
    for k, im in enumerate(images):
        arr[k] = _Image(float(im.a), float(getattr(im, "M", 1.0)), float(im.r_obs), float(im.incl),
                        int(im.nx), int(im.ny), float(im.alpha0), float(im.alpha1),
                        float(im.beta0), float(im.beta1), int(getattr(im, "grid", GRID_CARTESIAN)), 0)
    return arr


# ---------------------------------------------------------------- C ABI ---

def gray_strerror(code: int) -> str:
    return lib().gray_strerror(int(code)).decode()


def gray_default_options() -> Options:
    o = _Options()
    lib().gray_default_options(C.byref(o))
    return Options(*[getattr(o, f.name) for f in fields(Options)])


def gray_state_bytes(n: int, precision: int) -> int:
    return int(lib().gray_state_bytes(int(n), int(precision)))


def gray_launch_count() -> int:
    return int(lib().gray_launch_count())


def gray_create(opt: Options):
    h = C.c_void_p()
    o = opt._c()
    _check(lib().gray_create(C.byref(h), C.byref(o)), "gray_create")
    return h


def gray_destroy(ctx) -> None:
    lib().gray_destroy(ctx)


def gray_setup(ctx, images, state, n_state, first_ray=0, stream=None):
    arr = _images(images)
    return _check(lib().gray_setup(ctx, arr, len(images), _ptr(state), state.numel() * state.element_size(),
                                   int(n_state), int(first_ray), _stream(stream)), "gray_setup")


def gray_setup_noalloc(precision, images, state, n_state, first_ray=0, stream=None):
    """gray_setup without a context and without any device allocation: the
    image table goes through a fixed device array of GRAY_NOALLOC_MAX_IMAGES
    entries inside the library (for callers that cannot allocate)."""
    arr = _images(images)
    return _check(lib().gray_setup_noalloc(int(precision), arr, len(images), _ptr(state),
                                           state.numel() * state.element_size(), int(n_state), int(first_ray),
                                           _stream(stream)), "gray_setup_noalloc")


def gray_setup_rays(ctx, rays, M, state, n_state, first_ray=0, stream=None):
    assert rays.is_cuda and rays.dtype.itemsize == 8 and rays.is_contiguous()
    n = rays.numel() // 5
    return _check(lib().gray_setup_rays(ctx, _ptr(rays), int(n), float(M), _ptr(state),
                                        state.numel() * state.element_size(), int(n_state), int(first_ray),
                                        _stream(stream)), "gray_setup_rays")


def gray_trace(ctx, state, n_state, step_budget=0, wait=True, stream=None, order=None):
    """Returns (rc, n_active, stats) with stats = (steps, euler, fp64 steps,
    active) of this call; n_active and stats are None when wait=False.  rc is
    ECANCEL when the context's cancel flag stopped the call (gray_cancel).
    ``order``: optional int32 CUDA tensor, the work queue of ray indices."""
    op = _ptr(order) if order is not None else None
    no = order.numel() if order is not None else 0
    if wait:
        na = C.c_int64()
        st = (C.c_int64 * 4)()
        rc = lib().gray_trace(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state), op, no,
                              int(step_budget), C.byref(na), st, _stream(stream))
        if rc != ECANCEL:  # a cancelled trace is not a failure: its counts are valid
            _check(rc, "gray_trace")
        return rc, int(na.value), tuple(int(x) for x in st)
    rc = _check(lib().gray_trace(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state), op, no,
                                 int(step_budget), None, None, _stream(stream)), "gray_trace")
    return rc, None, None


def gray_plan(ctx, state, n_state, images, first_ray=0, probe_stride=6, probe_budget=400, order=None, stream=None):
    """Longest-first work queue (int32 CUDA tensor) for the rays of ``images``
    set up at ``first_ray``; the probe rays advance by up to probe_budget."""
    import torch
    arr = _images(images)
    total = sum(int(im.nx) * int(im.ny) for im in images)
    if order is None:
        order = torch.empty(max(1, total), dtype=torch.int32, device=state.device)
    _check(lib().gray_plan(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state), arr, len(images),
                           int(first_ray), int(probe_stride), int(probe_budget), _ptr(order),
                           order.numel() * order.element_size(), _stream(stream)), "gray_plan")
    return order[:total]


def gray_setup_plan(ctx, images, state, n_state, first_ray=0, probe_stride=6, probe_budget=400, order=None,
                    stream=None):
    """gray_setup then gray_plan in one call, the set-up of the non-probe rays
    overlapping the probe pass; returns the queue as gray_plan does."""
    import torch
    arr = _images(images)
    total = sum(int(im.nx) * int(im.ny) for im in images)
    if order is None:
        order = torch.empty(max(1, total), dtype=torch.int32, device=state.device)
    _check(lib().gray_setup_plan(ctx, arr, len(images), _ptr(state), state.numel() * state.element_size(),
                                 int(n_state), int(first_ray), int(probe_stride), int(probe_budget), _ptr(order),
                                 order.numel() * order.element_size(), _stream(stream)), "gray_setup_plan")
    return order[:total]


def gray_fma_peak(precision, blocks, threads, iters, sink, stream=None):
    """Launch the FMA-chain microbenchmark (asynchronous); returns the
    floating-point operations of the launch.  ``sink``: CUDA tensor of at
    least blocks x threads elements of the precision's type."""
    _check(lib().gray_fma_peak(int(precision), int(blocks), int(threads), int(iters), _ptr(sink),
                               sink.numel() * sink.element_size(), _stream(stream)), "gray_fma_peak")
    return 2 * 8 * int(iters) * int(blocks) * int(threads)


def gray_cancel(ctx, on=True):
    """Set (or clear) the context's cancel flag; safe to call from another
    thread while gray_trace runs."""
    return _check(lib().gray_cancel(ctx, 1 if on else 0), "gray_cancel")


def gray_set_timing(ctx, on=True):
    return _check(lib().gray_set_timing(ctx, 1 if on else 0), "gray_set_timing")


def gray_timings(ctx):
    """(single pass ms, zone pass ms, probe pass ms, zone steps) of the last calls."""
    ms = (C.c_double * 3)()
    zs = C.c_int64()
    _check(lib().gray_timings(ctx, ms, C.byref(zs)), "gray_timings")
    return float(ms[0]), float(ms[1]), float(ms[2]), int(zs.value)


def gray_clear(ctx, state, n_state, first_ray, n, stream=None):
    return _check(lib().gray_clear(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state),
                                   int(first_ray), int(n), _stream(stream)), "gray_clear")


def gray_count_active(ctx, state, n_state, ranges, stream=None):
    """ranges: list of (first_ray, count).  Returns a list of active counts."""
    k = len(ranges)
    arr = (C.c_int64 * max(1, 2 * k))()
    for j, (f, c) in enumerate(ranges):
        arr[2 * j], arr[2 * j + 1] = int(f), int(c)
    out = (C.c_int64 * max(1, k))()
    _check(lib().gray_count_active(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state), arr, k, out,
                                   _stream(stream)), "gray_count_active")
    return [int(out[j]) for j in range(k)]


def gray_range_stats(ctx, state, n_state, ranges_dev, out_dev, n_ranges=None, stream=None):
    """Asynchronous (active rays, steps) per range: ranges_dev an int64 CUDA
    tensor of (first_ray, count) pairs, out_dev an int64 CUDA tensor of at
    least 2 x n_ranges entries."""
    if n_ranges is None:
        n_ranges = ranges_dev.numel() // 2
    assert ranges_dev.is_cuda and out_dev.is_cuda and out_dev.numel() >= 2 * n_ranges
    return _check(lib().gray_range_stats(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state),
                                         _ptr(ranges_dev), int(n_ranges), _ptr(out_dev), _stream(stream)),
                  "gray_range_stats")


_PER = {RENDER_PIXELS64: 32, RENDER_PIXELS32: 16, RENDER_RECORD: 17 * 8, RENDER_INVARIANTS: 4 * 8}


def gray_render(ctx, state, n_state, kind, first_ray=0, n=None, out=None, stream=None):
    """Render rays [first_ray, first_ray + n) into ``out`` (a uint8 CUDA tensor
    of at least n * record bytes; allocated if None).  Returns ``out``."""
    import torch
    if n is None:
        n = n_state - first_ray
    per = _PER[kind]
    if out is None:
        out = torch.empty(max(1, per * n), dtype=torch.uint8, device=state.device)
    _check(lib().gray_render(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state),
                             int(first_ray), int(n), int(kind), _ptr(out), out.numel() * out.element_size(),
                             _stream(stream)), "gray_render")
    return out


def gray_shadow(ctx, state, n_state, images, first_ray=0, out=None, stream=None):
    import torch
    arr = _images(images)
    if out is None:
        out = torch.empty(SHADOW_DTYPE.itemsize * len(images), dtype=torch.uint8, device=state.device)
    _check(lib().gray_shadow(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state),
                             int(first_ray), arr, len(images), _ptr(out), out.numel() * out.element_size(),
                             _stream(stream)), "gray_shadow")
    return out


def gray_ring(ctx, state, n_state, images, first_ray=0, out=None, boundary=None, stream=None):
    """Ring metrics (Sec. 4) of traced polar images: a uint8 CUDA tensor of
    len(images) RING_DTYPE records.  ``boundary``: optional float64 CUDA
    tensor that receives every image's boundary radius per angle row."""
    import torch
    arr = _images(images)
    if out is None:
        out = torch.empty(RING_DTYPE.itemsize * len(images), dtype=torch.uint8, device=state.device)
    bp = _ptr(boundary) if boundary is not None else None
    bb = boundary.numel() * boundary.element_size() if boundary is not None else 0
    _check(lib().gray_ring(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state),
                           int(first_ray), arr, len(images), _ptr(out), out.numel() * out.element_size(),
                           bp, bb, _stream(stream)), "gray_ring")
    return out


def gray_splat(ctx, state, n_state, camera, count=None, depth=None, first_ray=0, n=None, stream=None):
    """Draw rays first_ray .. first_ray + n - 1 into count (uint32 as int32
    CUDA tensor of height x width) and optionally depth (float32, same
    shape).  Returns (count, depth)."""
    import torch
    if n is None:
        n = n_state - first_ray
    if count is None:
        count = torch.empty((camera.height, camera.width), dtype=torch.int32, device=state.device)
    nbytes = count.numel() * count.element_size()
    if depth is not None:
        assert depth.numel() * depth.element_size() == nbytes
    cam = camera._c()
    _check(lib().gray_splat(ctx, _ptr(state), state.numel() * state.element_size(), int(n_state), int(first_ray),
                            int(n), C.byref(cam), _ptr(count), _ptr(depth) if depth is not None else None, nbytes,
                            _stream(stream)), "gray_splat")
    return count, depth


def gray_eval(what, precision, inp, stream=None):
    """inp: float64 CUDA tensor of n rows (4, 10, 6 or 10 doubles by ``what``).
    Returns a float64 CUDA tensor of n rows (64, 8, 8 or 1 doubles)."""
    import torch
    width_in = {EVAL_CHRISTOFFEL: 4, EVAL_RHS: 10, EVAL_INITIAL: 6, EVAL_XI: 10, EVAL_SINCOS: 1, EVAL_RECIP: 1,
                EVAL_SINCOS_DS: 1, EVAL_NORM: 10}[what]
    width_out = {EVAL_CHRISTOFFEL: 64, EVAL_RHS: 8, EVAL_INITIAL: 8, EVAL_XI: 1, EVAL_SINCOS: 2, EVAL_RECIP: 2,
                 EVAL_SINCOS_DS: 2, EVAL_NORM: 6}[what]
    inp = inp.contiguous()
    n = inp.numel() // width_in
    out = torch.empty((n, width_out), dtype=torch.float64, device=inp.device)
    _check(lib().gray_eval(int(what), int(precision), _ptr(inp), int(n), _ptr(out), _stream(stream)),
           "gray_eval")
    return out


# ------------------------------------------------------------ helpers ---

def as_numpy(out_tensor, dtype):
    """Copy a rendered uint8 tensor to the host as a numpy array of ``dtype``."""
    return out_tensor.cpu().numpy().view(dtype)


class Tracer:
    """Convenience owner of a context and one state buffer."""

    def __init__(self, opt: Options, n_state: int, device="cuda"):
        import torch
        self.opt = opt
        self.n = int(n_state)
        self.ctx = gray_create(opt)
        nbytes = gray_state_bytes(self.n, opt.precision)
        self.state = torch.zeros(max(256, nbytes), dtype=torch.uint8, device=device)

    def close(self):
        if self.ctx is not None:
            gray_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setup(self, images, first_ray=0, stream=None):
        return gray_setup(self.ctx, images, self.state, self.n, first_ray, stream)

    def setup_rays(self, rays, M=1.0, first_ray=0, stream=None):
        return gray_setup_rays(self.ctx, rays, M, self.state, self.n, first_ray, stream)

    def trace(self, step_budget=0, wait=True, stream=None, order=None):
        return gray_trace(self.ctx, self.state, self.n, step_budget, wait, stream, order)

    def plan(self, images, first_ray=0, probe_stride=6, probe_budget=400, order=None, stream=None):
        return gray_plan(self.ctx, self.state, self.n, images, first_ray, probe_stride, probe_budget, order, stream)

    def setup_plan(self, images, first_ray=0, probe_stride=6, probe_budget=400, order=None, stream=None):
        return gray_setup_plan(self.ctx, images, self.state, self.n, first_ray, probe_stride, probe_budget, order,
                               stream)

    def render(self, kind, first_ray=0, n=None, out=None, stream=None):
        return gray_render(self.ctx, self.state, self.n, kind, first_ray, n, out, stream)

    def records(self, first_ray=0, n=None):
        """Per-ray records as an (n, 17) float64 numpy array."""
        t = self.render(RENDER_RECORD, first_ray, n)
        import torch
        torch.cuda.synchronize()
        return t.cpu().numpy().view(np.float64).reshape(-1, RECORD)[: (self.n - first_ray if n is None else n)]

    def invariants(self, first_ray=0, n=None):
        t = self.render(RENDER_INVARIANTS, first_ray, n)
        import torch
        torch.cuda.synchronize()
        return t.cpu().numpy().view(np.float64).reshape(-1, 4)[: (self.n - first_ray if n is None else n)]

    def shadow(self, images, first_ray=0):
        t = gray_shadow(self.ctx, self.state, self.n, images, first_ray)
        import torch
        torch.cuda.synchronize()
        return as_numpy(t, SHADOW_DTYPE)

    def ring(self, images, first_ray=0):
        """(RING_DTYPE records, boundary radii per image as a list of arrays)."""
        import torch
        rows = sum(int(im.ny) for im in images)
        b = torch.empty(max(1, rows), dtype=torch.float64, device=self.state.device)
        t = gray_ring(self.ctx, self.state, self.n, images, first_ray, boundary=b)
        torch.cuda.synchronize()
        bh = b.cpu().numpy()
        out, k = [], 0
        for im in images:
            out.append(bh[k:k + int(im.ny)])
            k += int(im.ny)
        return as_numpy(t, RING_DTYPE), out
