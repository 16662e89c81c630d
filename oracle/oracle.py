"""ctypes binding of the FP64 C oracle (``kerr_oracle.c``).

Test infrastructure only: the parity reference for the CUDA tracer.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
use it.  Nothing here imports the CUDA library.

Every function follows the paper (Chan, Psaltis & Ozel 2013, Sec. 2) or the
textbook Kerr relations it defers to; see the C source for the statement of
each step.  Argument order follows the C functions.
"""
import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

ACTIVE, CAPTURED, ESCAPED, STEP_CAP, NONFINITE, EQUATOR = 0, 1, 2, 3, 4, 6
STEP_BENCH, STEP_EQ2 = 0, 1
REC = 17  # doubles per ray record, see ``orc_trace``

_dp = C.POINTER(C.c_double)


class _Options(C.Structure):
    _fields_ = [("M", C.c_double), ("h_frac", C.c_double), ("h_min", C.c_double),
                ("cap_frac", C.c_double), ("eps_xi", C.c_double),
                ("r_esc_frac", C.c_double), ("max_steps", C.c_int32),
                ("step_rule", C.c_int32), ("stop_equator", C.c_int32)]


@dataclass
class Options:
    """Integration options.  Defaults are the benchmark's: |h| = r/32 with the
    horizon guard of Eq. 2, floor 1e-3, capture at 1.01 r_h, xi threshold 1e-3
    (Sec. 2), escape at r_obs, cap 1e5 steps."""
    M: float = 1.0
    h_frac: float = 1.0 / 32.0
    h_min: float = 1e-3
    cap_frac: float = 1.01
    eps_xi: float = 1e-3
    r_esc_frac: float = 1.0
    max_steps: int = 100000
    step_rule: int = STEP_BENCH
    stop_equator: int = 0

    def _c(self):
        return _Options(self.M, self.h_frac, self.h_min, self.cap_frac, self.eps_xi,
                        self.r_esc_frac, int(self.max_steps), int(self.step_rule),
                        int(self.stop_equator))


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, i32, i64 = C.c_double, C.c_int32, C.c_int64
        L.orc_horizon.restype = d
        L.orc_horizon.argtypes = [d, d]
        for name in ("orc_metric", "orc_inverse_metric", "orc_metric_derivs", "orc_christoffel"):
            f = getattr(L, name)
            f.restype = None
            f.argtypes = [d, d, d, d, _dp]
        L.orc_rhs.restype = None
        L.orc_rhs.argtypes = [d, d, _dp, _dp]
        L.orc_null_norm.restype = d
        L.orc_null_norm.argtypes = [d, d, _dp]
        L.orc_xi.restype = d
        L.orc_xi.argtypes = [d, d, _dp]
        L.orc_invariants.restype = None
        L.orc_invariants.argtypes = [d, d, _dp, _dp]
        L.orc_initial.restype = None
        L.orc_initial.argtypes = [d, d, d, d, d, d, _dp]
        L.orc_step_size.restype = d
        L.orc_step_size.argtypes = [C.POINTER(_Options), d, _dp]
        L.orc_rk4.restype = None
        L.orc_rk4.argtypes = [d, d, _dp, d, _dp, _dp]
        L.orc_remap.restype = C.c_int
        L.orc_remap.argtypes = [_dp]
        L.orc_hermite.restype = d
        L.orc_hermite.argtypes = [d, d, d, d, d, d]
        L.orc_stop_surface.restype = None
        L.orc_stop_surface.argtypes = [_dp, _dp, d, d, _dp]
        L.orc_trace.restype = C.c_int
        L.orc_trace.argtypes = [d, d, d, C.POINTER(_Options), _dp, _dp]
        L.orc_trace_many.restype = C.c_int
        L.orc_trace_many.argtypes = [i64, _dp, C.POINTER(_Options), _dp, C.c_int]
        L.orc_trace_states.restype = C.c_int
        L.orc_trace_states.argtypes = [i64, _dp, _dp, C.POINTER(_Options), _dp, C.c_int]
        L.orc_initial_many.restype = None
        L.orc_initial_many.argtypes = [i64, _dp, d, _dp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _vec(y, n):
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(n))
    return y


def horizon(M, a):
    """r_h = M + sqrt(M^2 - a^2) (Sec. 2)."""
    return lib().orc_horizon(M, a)


def metric(M, a, r, th):
    g = np.zeros((4, 4))
    lib().orc_metric(M, a, r, th, _ptr(g))
    return g


def inverse_metric(M, a, r, th):
    g = np.zeros((4, 4))
    lib().orc_inverse_metric(M, a, r, th, _ptr(g))
    return g


def metric_derivs(M, a, r, th):
    """dg[k, mu, nu] = d g_{mu nu} / d x^k."""
    g = np.zeros((4, 4, 4))
    lib().orc_metric_derivs(M, a, r, th, _ptr(g))
    return g


def christoffel(M, a, r, th):
    """G[mu, a, b] = Gamma^mu_ab from the general formula."""
    g = np.zeros((4, 4, 4))
    lib().orc_christoffel(M, a, r, th, _ptr(g))
    return g


def rhs(M, a, y):
    y = _vec(y, 8)
    dy = np.zeros(8)
    lib().orc_rhs(M, a, _ptr(y), _ptr(dy))
    return dy


def null_norm(M, a, y):
    y = _vec(y, 8)
    return lib().orc_null_norm(M, a, _ptr(y))


def xi(M, a, y):
    """Eq. 4."""
    y = _vec(y, 8)
    return lib().orc_xi(M, a, _ptr(y))


def invariants(M, a, y):
    """(E, L_z, Q, N) of the state y."""
    y = _vec(y, 8)
    out = np.zeros(4)
    lib().orc_invariants(M, a, _ptr(y), _ptr(out))
    return out


def initial(M, a, r_obs, incl, alpha, beta):
    """State (x^mu, k^mu) of the pixel (alpha, beta), normalised to E = 1."""
    y = np.zeros(8)
    lib().orc_initial(M, a, r_obs, incl, alpha, beta, _ptr(y))
    return y


def step_size(opts, r_h, y):
    y = _vec(y, 8)
    o = opts._c()
    return lib().orc_step_size(C.byref(o), r_h, _ptr(y))


def rk4(M, a, y, h):
    y = _vec(y, 8)
    out = np.zeros(8)
    k1 = np.zeros(8)
    lib().orc_rk4(M, a, _ptr(y), h, _ptr(out), _ptr(k1))
    return out, k1


def remap(y):
    """Eq. 3; returns (new state, whether it applied)."""
    y = _vec(y, 8).copy()
    n = lib().orc_remap(_ptr(y))
    return y, bool(n)


def hermite(x0, v0, x1, v1, h, s):
    return lib().orc_hermite(x0, v0, x1, v1, h, s)


def stop_surface(y0, y1, h, r_stop):
    y0 = _vec(y0, 8)
    y1 = _vec(y1, 8)
    fin = np.zeros(4)
    lib().orc_stop_surface(_ptr(y0), _ptr(y1), h, r_stop, _ptr(fin))
    return fin


def trace(a, r_obs, y, opts=None):
    """Trace one ray from state y.  Returns the 17-double record:
    [status, steps, euler redos, pole remaps, t_f, r_f, th_f, ph_f,
     y_end[8], affine length]."""
    opts = opts or Options()
    y = _vec(y, 8).copy()
    rec = np.zeros(REC)
    o = opts._c()
    lib().orc_trace(opts.M, a, r_obs, C.byref(o), _ptr(y), _ptr(rec))
    return rec


def trace_many(rays, opts=None, nthreads=None):
    """rays: (n, 5) array of (alpha, beta, a, incl, r_obs).  Returns (n, 17)."""
    opts = opts or Options()
    rays = np.ascontiguousarray(np.asarray(rays, dtype=np.float64).reshape(-1, 5))
    n = rays.shape[0]
    out = np.zeros((n, REC))
    if n == 0:
        return out
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    o = opts._c()
    lib().orc_trace_many(n, _ptr(rays), C.byref(o), _ptr(out), int(nthreads))
    return out


def initial_many(rays, M=1.0):
    """Start states (n, 8) of the rays (alpha, beta, a, incl, r_obs)."""
    rays = np.ascontiguousarray(np.asarray(rays, dtype=np.float64).reshape(-1, 5))
    out = np.zeros((rays.shape[0], 8))
    if rays.shape[0]:
        lib().orc_initial_many(rays.shape[0], _ptr(rays), float(M), _ptr(out))
    return out


def trace_states(states, a, r_obs, opts=None, nthreads=None):
    """Trace from given start states: states (n, 8); a and r_obs per ray
    (arrays of n, or scalars).  Returns (n, 17) records as trace_many."""
    opts = opts or Options()
    states = np.ascontiguousarray(np.asarray(states, dtype=np.float64).reshape(-1, 8))
    n = states.shape[0]
    params = np.empty((n, 2))
    params[:, 0] = a
    params[:, 1] = r_obs
    out = np.zeros((n, REC))
    if n == 0:
        return out
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    o = opts._c()
    lib().orc_trace_states(n, _ptr(states), _ptr(params), C.byref(o), _ptr(out), int(nthreads))
    return out


def pixel_centres(nx, ny, a0, a1, b0, b1):
    """Pixel-centre grid of one image (reading: alpha_j = a0 + (j + 1/2)
    (a1 - a0)/nx, likewise beta; ray index = row * nx + column, row along
    beta).  Returns (alpha, beta) flat arrays of length nx * ny."""
    j = np.arange(nx, dtype=np.float64)
    i = np.arange(ny, dtype=np.float64)
    al = a0 + (j + 0.5) * ((a1 - a0) / nx)
    be = b0 + (i + 0.5) * ((b1 - b0) / ny)
    A, B = np.meshgrid(al, be)
    return A.ravel(), B.ravel()


def image_rays(a, incl, r_obs, nx, ny, a0, a1, b0, b1):
    """(n, 5) ray table of one image for ``trace_many``."""
    al, be = pixel_centres(nx, ny, a0, a1, b0, b1)
    n = al.size
    rays = np.empty((n, 5))
    rays[:, 0] = al
    rays[:, 1] = be
    rays[:, 2] = a
    rays[:, 3] = incl
    rays[:, 4] = r_obs
    return rays


__all__ = [
    "ACTIVE", "CAPTURED", "ESCAPED", "STEP_CAP", "NONFINITE", "EQUATOR", "STEP_BENCH", "STEP_EQ2",
    "REC", "Options", "horizon", "metric", "inverse_metric", "metric_derivs",
    "christoffel", "rhs", "null_norm", "xi", "invariants", "initial", "step_size",
    "rk4", "remap", "hermite", "stop_surface", "trace", "trace_many", "trace_states", "initial_many",
    "pixel_centres", "image_rays", "lib",
]
