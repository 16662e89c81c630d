"""Closed forms from textbook general relativity, used to pin the oracle.

Nothing here calls the oracle or the CUDA library; each function is an
independent statement of a known result:

* Schwarzschild Christoffel symbols (any GR text, e.g. Carroll Eq. 5.13 ff.);
* the boundary of the Kerr shadow (Bardeen 1973), the critical curve the
  paper's photon rings trace (Sec. 4);
* the exact deflection of an equatorial Kerr photon as a one-dimensional
  quadrature of the radial and azimuthal first integrals;
* straight lines of flat space in (oblate) spheroidal coordinates, which is
  what the Kerr metric becomes at M = 0.
"""
import math

import numpy as np
from scipy import integrate


# ---------------------------------------------------------------------------
# Schwarzschild
# ---------------------------------------------------------------------------

def schwarzschild_gamma(M, r, th):
    """Nonzero Gamma^mu_ab (a <= b) of the Schwarzschild metric, keyed by
    (mu, a, b) with indices t=0, r=1, theta=2, phi=3."""
    f = 1.0 - 2.0 * M / r
    s, c = math.sin(th), math.cos(th)
    return {
        (0, 0, 1): M / (r * r * f),
        (1, 0, 0): M * f / (r * r),
        (1, 1, 1): -M / (r * r * f),
        (1, 2, 2): -r * f,
        (1, 3, 3): -r * f * s * s,
        (2, 1, 2): 1.0 / r,
        (2, 3, 3): -s * c,
        (3, 1, 3): 1.0 / r,
        (3, 2, 3): c / s,
    }


def schwarzschild_deflection_series(M, b):
    """Weak-field bending angle of light, to second order in M/b:
    4M/b + 15 pi M^2 / (4 b^2)."""
    return 4.0 * M / b + 15.0 * math.pi * M * M / (4.0 * b * b)


# ---------------------------------------------------------------------------
# Kerr shadow boundary (Bardeen 1973), M = 1
# ---------------------------------------------------------------------------

def photon_orbit_radii(a):
    """Prograde and retrograde circular equatorial photon orbits."""
    a = abs(a)
    return (2.0 * (1.0 + math.cos(2.0 / 3.0 * math.acos(-a))),
            2.0 * (1.0 + math.cos(2.0 / 3.0 * math.acos(a))))


def bardeen_curve(a, incl, n=100000):
    """Closed polygon (alpha, beta) of the shadow boundary seen at inclination
    ``incl`` for spin ``a`` (M = 1), with the convention L_z / E = -alpha sin i.
    a = 0 gives the circle of radius 3 sqrt 3."""
    if abs(a) < 1e-12:
        t = np.linspace(0.0, 2.0 * math.pi, n, endpoint=False)
        R = 3.0 * math.sqrt(3.0)
        return R * np.cos(t), R * np.sin(t)
    r_pro, r_ret = photon_orbit_radii(a)
    # cluster samples near both ends, where the curve meets beta = 0
    u = 0.5 - 0.5 * np.cos(np.linspace(0.0, math.pi, n))
    rp = r_pro + u * (r_ret - r_pro)
    aa = abs(a)
    xi = (rp * rp * (3.0 - rp) - aa * aa * (rp + 1.0)) / (aa * (rp - 1.0))
    eta = rp ** 3 * (4.0 * aa * aa - rp * (rp - 3.0) ** 2) / (aa * aa * (rp - 1.0) ** 2)
    si, ci = math.sin(incl), math.cos(incl)
    al = -xi / si
    b2 = eta + aa * aa * ci * ci - xi * xi * (ci / si) ** 2
    ok = b2 >= 0.0
    al, be = al[ok], np.sqrt(b2[ok])
    if a < 0:  # (a, alpha) -> (-a, -alpha) symmetry
        al = -al
    # upper half then lower half reversed: a closed curve
    A = np.concatenate([al, al[::-1]])
    B = np.concatenate([be, -be[::-1]])
    return A, B


def polar_shadow_radius(a):
    """Radius of the (circular) shadow seen from the spin axis, i = 0: the
    spherical photon orbit with xi = L/E = 0 has sqrt(eta + a^2) as its
    image radius (M = 1)."""
    aa = abs(a)
    if aa < 1e-12:
        return 3.0 * math.sqrt(3.0)
    lo, hi = photon_orbit_radii(aa)

    def xi(r):
        return (r * r * (3.0 - r) - aa * aa * (r + 1.0)) / (aa * (r - 1.0))

    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (xi(mid) > 0.0) == (xi(lo) > 0.0):
            lo = mid
        else:
            hi = mid
    r = 0.5 * (lo + hi)
    eta = r ** 3 * (4.0 * aa * aa - r * (r - 3.0) ** 2) / (aa * aa * (r - 1.0) ** 2)
    return math.sqrt(eta + aa * aa)


def inside_polygon(px, py, cx, cy):
    """Even-odd rule point-in-polygon test, vectorised over points."""
    px = np.asarray(px, dtype=np.float64)
    py = np.asarray(py, dtype=np.float64)
    inside = np.zeros(px.shape, dtype=bool)
    x0, y0 = cx, cy
    x1, y1 = np.roll(cx, -1), np.roll(cy, -1)
    for k in range(cx.size):
        ya, yb = y0[k], y1[k]
        if ya == yb:
            continue
        cond = (py >= min(ya, yb)) & (py < max(ya, yb))
        xin = x0[k] + (py - ya) * (x1[k] - x0[k]) / (yb - ya)
        inside ^= cond & (px < xin)
    return inside


def curve_distance(px, py, cx, cy):
    """Distance from each point to the nearest sample of a dense curve."""
    px = np.asarray(px, dtype=np.float64).ravel()
    py = np.asarray(py, dtype=np.float64).ravel()
    out = np.empty(px.size)
    for i in range(0, px.size, 256):
        dx = px[i:i + 256, None] - cx[None, :]
        dy = py[i:i + 256, None] - cy[None, :]
        out[i:i + 256] = np.sqrt((dx * dx + dy * dy).min(axis=1))
    return out


def shadow_truth(alpha, beta, a, incl, band=0.05, n_curve=100000):
    """(inside, far) for each pixel: inside the analytic shadow, and farther
    than ``band`` from its boundary.  For speed the polygon test uses a
    decimated copy of the curve, which is safe away from the band."""
    cx, cy = bardeen_curve(a, incl, n_curve)
    d = curve_distance(alpha, beta, cx, cy)
    step = max(1, cx.size // 4000)
    inside = inside_polygon(alpha, beta, cx[::step], cy[::step])
    return inside.reshape(np.shape(alpha)), (d > band).reshape(np.shape(alpha))


# ---------------------------------------------------------------------------
# Exact equatorial Kerr deflection (M = 1, E = 1, L_z = b)
# ---------------------------------------------------------------------------

def _radial_cubic(a, b):
    """R(r) = (r^2 + a^2 - a b)^2 - Delta (b - a)^2 = r * C(r) with the cubic
    C(r) = r^3 + (2a^2 - 2ab - (b - a)^2) r + 2 (b - a)^2."""
    return np.array([1.0, 0.0, 2 * a * a - 2 * a * b - (b - a) ** 2, 2 * (b - a) ** 2])


def turning_point(a, b):
    roots = np.roots(_radial_cubic(a, b))
    real = roots[np.abs(roots.imag) < 1e-9].real
    return float(real.max())


def equatorial_phi_integral(a, b, R):
    """Signed azimuth swept from the turning point r_min out to radius R along
    an equatorial photon of E = 1, L_z = b:
        phi(R) - phi(r_min) = int_{r_min}^{R} [a (r^2 + a^2 - a b)/Delta + b - a] / sqrt(R(r)) dr
    for the outgoing branch.  Substitution r = r_min + u^2 removes the
    inverse square-root singularity at the turning point."""
    c3 = _radial_cubic(a, b)
    rm = turning_point(a, b)
    # deflate the cubic: C(r) = (r - rm)(r^2 + p r + q)
    p = c3[1] + rm
    q = c3[2] + rm * p

    def f(u):
        r = rm + u * u
        delta = r * r - 2.0 * r + a * a
        num = a * (r * r + a * a - a * b) / delta + (b - a)
        return 2.0 * num / math.sqrt(r * (r * r + p * r + q))

    val, err = integrate.quad(f, 0.0, math.sqrt(R - rm), epsabs=1e-13, epsrel=1e-13, limit=400)
    return val


def equatorial_sweep(a, b, R_start, R_end):
    """Total azimuth swept by an equatorial photon (E = 1, L_z = b) that comes
    in from radius R_end, passes its turning point and leaves to R_start, in
    the photon's forward direction."""
    return equatorial_phi_integral(a, b, R_start) + equatorial_phi_integral(a, b, R_end)


# ---------------------------------------------------------------------------
# Flat space in Boyer-Lindquist (oblate spheroidal) coordinates, M = 0
# ---------------------------------------------------------------------------

def oblate_to_cart(a, r, th, ph):
    rho = math.sqrt(r * r + a * a)
    return np.array([rho * math.sin(th) * math.cos(ph),
                     rho * math.sin(th) * math.sin(ph),
                     r * math.cos(th)])


def oblate_velocity(a, r, th, ph, kr, kth, kph):
    """Cartesian velocity of (dr, dtheta, dphi) at (r, theta, phi)."""
    rho = math.sqrt(r * r + a * a)
    s, c = math.sin(th), math.cos(th)
    cp, sp = math.cos(ph), math.sin(ph)
    drho = r / rho
    return np.array([
        drho * kr * s * cp + rho * c * cp * kth - rho * s * sp * kph,
        drho * kr * s * sp + rho * c * sp * kth + rho * s * cp * kph,
        kr * c - r * s * kth,
    ])


def cart_to_oblate(a, X):
    x, y, z = X
    R2 = x * x + y * y + z * z
    w = R2 - a * a
    r2 = 0.5 * (w + math.sqrt(w * w + 4.0 * a * a * z * z))
    r = math.sqrt(r2)
    th = math.acos(max(-1.0, min(1.0, z / r)))
    ph = math.atan2(y, x)
    return r, th, ph


def straight_line_exit(a, y0, r_exit):
    """Follow the straight line through the state y0 (t, r, th, ph, k^t,
    k^r, k^th, k^ph) backwards in the affine parameter and return (theta, phi)
    where it leaves through the spheroid r = r_exit on the far side."""
    X0 = oblate_to_cart(a, y0[1], y0[2], y0[3])
    V = oblate_velocity(a, y0[1], y0[2], y0[3], y0[5], y0[6], y0[7])

    def r_of(lam):
        return cart_to_oblate(a, X0 + lam * V)[0]

    # the closest approach is at lam_c = -(X0.V)/(V.V) < 0; the exit lies beyond
    lam_c = -float(X0 @ V) / float(V @ V)
    lo, hi = lam_c, lam_c
    step = abs(lam_c) + 10.0
    while r_of(hi) < r_exit:
        hi -= step
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if r_of(mid) < r_exit:
            lo = mid
        else:
            hi = mid
    _, th, ph = cart_to_oblate(a, X0 + 0.5 * (lo + hi) * V)
    return th, ph


def angle_diff(x, y):
    """x - y wrapped into (-pi, pi]."""
    d = (np.asarray(x) - np.asarray(y) + math.pi) % (2.0 * math.pi) - math.pi
    return d


# ---------------------------------------------------------------------------
# Schwarzschild orbit: radius at a given swept angle (M = 1)
# ---------------------------------------------------------------------------

def schwarzschild_radius_at_angle(b, r0, psi):
    """Radius where a photon of impact parameter b, followed inward from r0,
    has swept the orbital angle psi (on the inward leg, or past its turning
    point on the outward leg).  d psi / d r = 1 / (r^2 sqrt(1/b^2 - (1 - 2/r)/r^2))."""
    from scipy import optimize

    def g(r):
        return 1.0 / (r * r * math.sqrt(max(1.0 / (b * b) - (1.0 - 2.0 / r) / (r * r), 1e-300)))

    bc = 3.0 * math.sqrt(3.0)
    if b > bc:
        # turning point: largest root of r^3 - b^2 r + 2 b^2 = 0
        roots = np.roots([1.0, 0.0, -b * b, 2.0 * b * b])
        rmin = float(roots[np.abs(roots.imag) < 1e-9].real.max())

        def swept_in(r):  # from r0 down to r >= rmin; u-substitution near rmin
            def f(u):
                rr = rmin + u * u
                return 2.0 * u * g(rr)
            return integrate.quad(f, math.sqrt(r - rmin), math.sqrt(r0 - rmin), epsabs=1e-13, epsrel=1e-13,
                                  limit=400)[0]
        total_in = swept_in(rmin)
        if psi <= total_in:
            return optimize.brentq(lambda r: swept_in(r) - psi, rmin, r0, xtol=1e-13, rtol=1e-14)
        return optimize.brentq(lambda r: total_in + (total_in - swept_in(r)) - psi, rmin, r0, xtol=1e-13,
                               rtol=1e-14)

    def swept(r):
        return integrate.quad(g, r, r0, epsabs=1e-13, epsrel=1e-13, limit=400)[0]
    return optimize.brentq(lambda r: swept(r) - psi, 2.0 + 1e-9, r0, xtol=1e-13, rtol=1e-14)


def schwarzschild_swept_to(b, r0, r1):
    """Orbital angle a plunging photon (b < 3 sqrt 3) sweeps from r0 in to r1."""
    def g(r):
        return 1.0 / (r * r * math.sqrt(1.0 / (b * b) - (1.0 - 2.0 / r) / (r * r)))
    return integrate.quad(g, r1, r0, epsabs=1e-13, epsrel=1e-13, limit=400)[0]


# ---------------------------------------------------------------------------
# Photon ring along polar rays from the image-plane origin (Sec. 4)
# ---------------------------------------------------------------------------

def shadow_radius_at_angle(a, incl, th):
    """Exact distance from the image-plane origin to Bardeen's critical curve
    along the polar angle th (array, in [0, pi]; M = 1, a >= 0).  The curve
    is star-shaped about the origin; each angle is solved by Brent's method
    on the polar angle of the curve's upper branch as a function of the
    photon-orbit radius."""
    from scipy import optimize
    th = np.asarray(th, dtype=np.float64)
    aa = abs(a)
    if aa < 1e-12:
        return np.full(th.shape, 3.0 * math.sqrt(3.0))
    si, ci = math.sin(incl), math.cos(incl)
    if si < 1e-12:
        return np.full(th.shape, polar_shadow_radius(aa))
    r_pro, r_ret = photon_orbit_radii(aa)

    def xi(r):
        return (r * r * (3.0 - r) - aa * aa * (r + 1.0)) / (aa * (r - 1.0))

    def b2(r):
        eta = r ** 3 * (4.0 * aa * aa - r * (r - 3.0) ** 2) / (aa * aa * (r - 1.0) ** 2)
        return eta + aa * aa * ci * ci - xi(r) ** 2 * (ci / si) ** 2

    rs = np.linspace(r_pro, r_ret, 200001)
    ok = np.nonzero(b2(rs) >= 0.0)[0]
    i0, i1 = int(ok[0]), int(ok[-1])
    r1 = optimize.brentq(b2, rs[i0 - 1], rs[i0], xtol=1e-15) if i0 > 0 else r_pro
    r2 = optimize.brentq(b2, rs[i1], rs[i1 + 1], xtol=1e-15) if i1 < rs.size - 1 else r_ret

    def point(r):
        return -xi(r) / si, math.sqrt(max(b2(r), 0.0))

    def angle(r):
        al, be = point(r)
        return math.atan2(be, al)

    out = np.empty(th.shape)
    for k, t in enumerate(th.ravel()):
        fa, fb = angle(r1) - t, angle(r2) - t
        if fa * fb >= 0.0:  # at an end of the curve (beta = 0)
            r = r1 if abs(fa) < abs(fb) else r2
        else:
            r = optimize.brentq(lambda x: angle(x) - t, r1, r2, xtol=1e-15, rtol=1e-15)
        out.flat[k] = math.hypot(*point(r))
    return out


def paper_ring_fits(a, incl_deg):
    """The paper's empirical fits (Eqs. 11-14, M = 1; angles in degrees):
    returns (<R>, A)."""
    R0 = 5.2 - 0.209 * a + 0.445 * a * a - 0.567 * a ** 3
    R1 = (0.24 - 3.3 / ((a - 0.9017) ** 2 + 0.059)) * 1e-3
    R_mean = R0 + R1 * math.cos(math.radians(2.14 * incl_deg - 22.9))
    A0 = 0.332 * a ** 3 + 0.176 * a ** 21.7 + 0.0756 * a ** 195
    n = 1.55 * (1.0 - a) ** (-0.022) + 1.3 * (1.0 - a) ** 0.98
    return R_mean, A0 * math.sin(math.radians(incl_deg)) ** n


def captured_from_invariants(a, lam, eta):
    """Exact fate of photons with lam = L_z / E and eta = Q / E^2 coming in
    from far away (M = 1): captured iff the radial potential
    R(r) = (r^2 + a^2 - a lam)^2 - Delta ((lam - a)^2 + eta) has no real root
    outside the horizon.  Returns (captured, margin) arrays; margin is the
    distance of the nearest real root above r_h (or of the smallest |Im| of a
    complex pair) -- near zero for rays on the critical curve."""
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    eta = np.atleast_1d(np.asarray(eta, dtype=np.float64))
    r_h = 1.0 + math.sqrt(1.0 - a * a)
    cap = np.empty(lam.shape, dtype=bool)
    margin = np.empty(lam.shape)
    for k in range(lam.size):
        K = (lam[k] - a) ** 2 + eta[k]
        u = a * a - a * lam[k]
        roots = np.roots([1.0, 0.0, 2.0 * u - K, 2.0 * K, u * u - a * a * K])
        real = np.abs(roots.imag) <= 1e-7 * np.maximum(1.0, np.abs(roots))
        outside = roots.real[real & (roots.real > r_h)]
        cap[k] = outside.size == 0
        im = np.abs(roots.imag[~real & (roots.real > r_h)])
        margin[k] = float(np.min(np.concatenate([im, [np.inf]]))) if cap[k] else 0.0
    return cap, margin
