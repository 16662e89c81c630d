"""Seeded synthetic workloads for the Kerr photon tracer.

This module only draws numbers: image-plane windows, spins, inclinations,
image sizes, Poisson arrival times and, for the mixed workload, per-ray impact
parameters.  It holds none of the tracer's arithmetic (no metric, no geodesic,
no step rule, no pixel-centre rule) and is shared, unchanged, by the CUDA path's
tests and benchmark and by the CPU oracle's tests.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014), mapped to
doubles in [0, 1) by the top 53 bits, seeded with ``1303057 + workload index``.

The workloads mirror the paper's: image-plane grids at r_obs = 1000 M
(Sec. 3 grid projection, Sec. 4 photon-ring study), a 1024 x 1024 image
(Sec. 5 discussion of image cost), and sweeps over spin and inclination
(Sec. 4).  The paper uses no dataset.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1303057
_MASK = (1 << 64) - 1


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of the splitmix64 sequence from ``seed``
    (the generator is counter based, so any slice can be drawn directly)."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = (np.uint64(seed & _MASK) + idx * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from splitmix64 (slice ``offset``)."""
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return lo + (hi - lo) * u


@dataclass
class Image:
    """One image request: a black hole of spin ``a`` seen by an observer at
    ``r_obs`` and inclination ``incl`` (radians), through an nx x ny pixel grid
    over [alpha0, alpha1] x [beta0, beta1] (units of M).  grid = 1 makes it
    the polar grid of the ring study instead: nx radii cell-centred on
    (alpha0, alpha1), ny angles from beta0 to beta1 inclusive."""
    a: float
    incl: float
    nx: int
    ny: int
    r_obs: float = 1000.0
    M: float = 1.0
    alpha0: float = -10.0
    alpha1: float = 10.0
    beta0: float = -10.0
    beta1: float = 10.0
    grid: int = 0

    @property
    def n(self) -> int:
        return self.nx * self.ny


@dataclass
class Workload:
    name: str
    images: list = field(default_factory=list)
    precision: str = "fp64"
    max_steps: int = 100000

    @property
    def n_rays(self) -> int:
        return sum(im.n for im in self.images)


def schwarzschild_64():
    """a = 0, i = 60 deg, 64 x 64 over [-10, 10]^2, FP64, cap 1e5 steps."""
    return Workload("schwarzschild_a0_i60_64x64_fp64",
                    [Image(a=0.0, incl=math.radians(60.0), nx=64, ny=64)],
                    precision="fp64", max_steps=100000)


def kerr_1024(side: int = 1024):
    """a = 0.99, i = 90 deg, side x side over [-10, 10]^2, FP32 bulk with
    selective FP64, cap 1e4 steps.  ``side`` < 1024 gives the same image at a
    coarser resolution (same window) for CPU-sized parity runs."""
    return Workload("kerr_a0.99_i90_%dx%d" % (side, side),
                    [Image(a=0.99, incl=math.radians(90.0), nx=side, ny=side)],
                    precision="fp32_kahan_sel64", max_steps=10000)


def shadow_sweep(n_images: int = 256, side_lo: int = 64, side_hi: int = 1024,
                 seed_index: int = 3):
    """Batched sweep: n_images (a, i) pairs, a ~ U[0, 0.999], i ~ U[0, 90] deg,
    square images of side ~ U{side_lo..side_hi} over [-10, 10]^2."""
    s = SEED_BASE + seed_index
    a = uniform(s, n_images, 0.0, 0.999)
    inc = uniform(s + 101, n_images, 0.0, 90.0)
    side = np.floor(uniform(s + 202, n_images, side_lo, side_hi + 1)).astype(int)
    ims = [Image(a=float(a[k]), incl=math.radians(float(inc[k])), nx=int(side[k]),
                 ny=int(side[k])) for k in range(n_images)]
    return Workload("shadow_sweep_%d" % n_images, ims, precision="fp32_kahan_sel64",
                    max_steps=10000)


def polar_image(a: float, incl_deg: float, n_R: int = 6000, n_th: int = 181, R0: float = 1.5,
                R1: float = 7.5, th0: float = 0.0, th1: float = math.pi, r_obs: float = 1000.0) -> Image:
    """One image of the Sec. 4 ring study: the polar grid of n_R radii over
    (R0, R1) by n_th angles over [th0, th1] (the paper's 6000 x 181 over
    (1.5, 7.5) M x [0, pi]), observer at r_obs and inclination incl_deg."""
    return Image(a=float(a), incl=math.radians(float(incl_deg)), nx=int(n_R), ny=int(n_th), r_obs=r_obs,
                 alpha0=R0, alpha1=R1, beta0=th0, beta1=th1, grid=1)


def ring_spins():
    """The 16 spins of the ring study, a_j = 1 - 10^(-j/5), j = 0..15."""
    return [1.0 - 10.0 ** (-j / 5.0) for j in range(16)]


def ring_sweep(n_R: int = 6000, n_th: int = 181, spins=None, incls_deg=None):
    """Sec. 4 parameter study: 16 spins x 19 inclinations (0, 5, .., 90 deg),
    each a polar image of n_R x n_th rays (3.3e8 rays at the paper's size).
    Deterministic; no random draws."""
    spins = ring_spins() if spins is None else list(spins)
    incls = list(range(0, 91, 5)) if incls_deg is None else list(incls_deg)
    ims = [polar_image(a, i, n_R, n_th) for a in spins for i in incls]
    return Workload("ring_sweep_%dx%dx%dx%d" % (len(spins), len(incls), n_R, n_th), ims,
                    precision="fp32_kahan_sel64", max_steps=100000)


def _bardeen_point(a, incl, u):
    """Point of the Kerr shadow boundary (Bardeen 1973, M = 1) at fraction u
    between the prograde and retrograde circular photon orbits, per element.
    Returns (alpha, beta >= 0, valid).  Used only to place near-critical rays."""
    a = np.maximum(np.abs(a), 1e-6)
    r_pro = 2.0 * (1.0 + np.cos(2.0 / 3.0 * np.arccos(-a)))
    r_ret = 2.0 * (1.0 + np.cos(2.0 / 3.0 * np.arccos(a)))
    rp = r_pro + u * (r_ret - r_pro)
    xi = (rp * rp * (3.0 - rp) - a * a * (rp + 1.0)) / (a * (rp - 1.0))
    eta = rp ** 3 * (4.0 * a * a - rp * (rp - 3.0) ** 2) / (a * a * (rp - 1.0) ** 2)
    si = np.maximum(np.sin(incl), 1e-9)
    ci = np.cos(incl)
    al = -xi / si
    b2 = eta + a * a * ci * ci - xi * xi * (ci / si) ** 2
    ok = b2 >= 0.0
    return al, np.sqrt(np.where(ok, b2, 0.0)), ok


def mixed_rays(n: int = 1 << 26, seed_index: int = 2, offset: int = 0):
    """Per-ray workload: rows (alpha, beta, a, incl, r_obs) for rays
    offset .. offset+n-1 of the stream.  Even rays are uniform in |alpha|,
    |beta| <= 20; odd rays lie within +-0.1 M (along the normal) of the
    analytic shadow boundary for their own (a, i), where that boundary exists
    at the drawn point (up to 8 redraws, else the ray stays uniform).
    a ~ U[0, 0.999], i ~ U[0, 90] deg, r_obs = 1000."""
    s = SEED_BASE + seed_index
    a = uniform(s, n, 0.0, 0.999, offset)
    inc = np.radians(uniform(s + 11, n, 0.0, 90.0, offset))
    al = uniform(s + 22, n, -20.0, 20.0, offset)
    be = uniform(s + 33, n, -20.0, 20.0, offset)
    near = (np.arange(offset, offset + n) % 2) == 1
    sgn = np.where(uniform(s + 55, n, offset=offset) < 0.5, -1.0, 1.0)
    off = uniform(s + 66, n, -0.1, 0.1, offset)
    todo = np.nonzero(near)[0]
    for attempt in range(8):
        if todo.size == 0:
            break
        u = uniform(s + 44 + 1000 * attempt, n, 0.02, 0.98, offset)[todo]
        at, it = a[todo], inc[todo]
        pa, pb, ok = _bardeen_point(at, it, u)
        qa, qb, ok2 = _bardeen_point(at, it, np.minimum(u + 1e-4, 1.0))
        take = ok & ok2
        sg = sgn[todo]
        ta, tb = qa - pa, sg * (qb - pb)
        nrm = np.hypot(ta, tb)
        nrm = np.where(nrm > 0, nrm, 1.0)
        idx = todo[take]
        al[idx] = (pa + off[todo] * (tb / nrm))[take]
        be[idx] = (sg * pb - off[todo] * (ta / nrm))[take]
        todo = todo[~take]
    rays = np.empty((n, 5))
    rays[:, 0] = al
    rays[:, 1] = be
    rays[:, 2] = a
    rays[:, 3] = inc
    rays[:, 4] = 1000.0
    return rays


@dataclass
class Request:
    rid: int
    t_arrive: float
    image: Image


def request_stream(rate: float, n_requests: int, seed_index: int = 4,
                   sides=(32, 64, 128, 256, 512, 1024, 2048)):
    """Poisson arrivals at ``rate`` per second of render requests with side
    uniform over ``sides``, a ~ U[0, 0.999], i ~ U[0, 90] deg, r_obs = 1000."""
    s = SEED_BASE + seed_index + int(rate * 1000)
    gaps = -np.log1p(-uniform(s, n_requests)) / rate
    t = np.cumsum(gaps)
    a = uniform(s + 1, n_requests, 0.0, 0.999)
    inc = uniform(s + 2, n_requests, 0.0, 90.0)
    pick = np.floor(uniform(s + 3, n_requests, 0, len(sides))).astype(int)
    out = []
    for k in range(n_requests):
        side = int(sides[min(pick[k], len(sides) - 1)])
        out.append(Request(k, float(t[k]), Image(a=float(a[k]), incl=math.radians(float(inc[k])),
                                                  nx=side, ny=side)))
    return out
