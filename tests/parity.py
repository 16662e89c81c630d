"""Shared comparison helpers for the GPU-vs-oracle parity tests.

Records are the 17-double rows written by both sides: status, steps, Euler
redos, pole remaps, final (t, r, theta, phi) on the stop surface, state y[8]
at the end of the last step, and one side-specific diagnostic.

Which rays a tolerance applies to is decided by the oracle alone, from
perturbed re-traces of each ray (``Reference``):

* band: pixels within 0.05 M of the analytic critical curve (the acceptance's
  own exclusion; rays there are chaotic);
* chaotic: a relative change of 1e-12 in alpha moves the oracle's final
  angles by more than 1e-6 rad (or changes the status);
* diverged: the oracle's own trajectory does not keep Carter's constant even
  to order one (relative drift >= 1).  These are rays that graze a pole under
  the benchmark step rule; their state leaves the null geodesic of their start
  (theta runs to thousands of radians, the drift reaches 1e30), and their
  digits are set by rounding (a different but equally exact formula for the
  Christoffel symbols gives different ones);
* conditioned at a precision: the oracle's final angles stay within that
  precision's tolerance when the start state is perturbed at the size of that
  precision's accumulated rounding: k rescaled by 1 + u (the same null
  geodesic with a rescaled affine parameter, which changes only the step
  sequence) and k^r changed by -+u (a null-norm offset of ~2u).  For the
  single-precision paths u = 1e-6 (16 units of 2^-24; the compensated state's
  null norm drifts by up to 3e-7 of (k^t)^2 over a trace, measured, and its
  spin and constants are rounded to 2^-24) against the 1e-4 rad tolerance;
  for the double path u = 1e-13 (the GPU's closed-form Christoffel symbols
  and the oracle's general formula round differently by ~1e-16 per
  evaluation, over thousands of steps) against 1e-9.  A ray that fails this
  is decided by the method's discrete choices (an Eq. 4 test within that
  rounding of its threshold, hundreds of first-order Euler steps) below that
  precision's resolution: its final angles move by more than the tolerance
  for an amplification above 100 (single) or 1e4 (double) of the start
  perturbation.

Every excluded set is counted and reported by the tests; classification is
compared on every ray outside the band.
"""
import math

import numpy as np

import oracle
import theory as T

TWO_PI = 2.0 * math.pi

CHAOS_ALPHA, CHAOS_MOVE = 1e-12, 1e-6
DIVERGED_Q = 1.0
SINGLE_U, SINGLE_TOL = 1e-6, 1e-4
DOUBLE_U, DOUBLE_TOL = 1e-13, 1e-9


def wrap(d):
    """Angle difference wrapped into (-pi, pi]."""
    return (np.asarray(d) + math.pi) % TWO_PI - math.pi


def band_mask(images_alpha_beta, a, incl, band=0.05):
    """True for pixels farther than ``band`` from the analytic shadow boundary."""
    al, be = images_alpha_beta
    _, far = T.shadow_truth(al, be, a, incl, band=band)
    return far


def per_ray_far(rays, band=0.05):
    """Band mask of per-ray (alpha, beta, a, incl) rays against each ray's own
    analytic critical curve (nearly polar observers: the boundary is nearly a
    circle, and a wider margin covers its small departure from one)."""
    far = np.ones(len(rays), dtype=bool)
    for k in range(len(rays)):
        cx, cy = T.bardeen_curve(rays[k, 2], rays[k, 3], 4000)
        if cx.size < 200:
            far[k] = abs(math.hypot(rays[k, 0], rays[k, 1]) - T.polar_shadow_radius(rays[k, 2])) > 0.6
        else:
            far[k] = T.curve_distance([rays[k, 0]], [rays[k, 1]], cx, cy)[0] > band
    return far


def angle_move(a, b):
    """max(|d theta|, |d phi| mod 2 pi) between two record arrays; inf where
    the statuses differ."""
    d = np.maximum(np.abs(a[:, 6] - b[:, 6]), np.abs(wrap(a[:, 7] - b[:, 7])))
    return np.where(a[:, 0] == b[:, 0], d, np.inf)


def rel_move(a, b):
    """The FP64 comparison's relative difference of the final angles."""
    dth = np.abs(a[:, 6] - b[:, 6])
    dph = np.abs(wrap(a[:, 7] - b[:, 7]))
    d = np.maximum(dth / np.maximum(1.0, np.abs(b[:, 6])), dph / np.maximum(1.0, np.abs(b[:, 7])))
    return np.where(a[:, 0] == b[:, 0], d, np.inf)


def q_drift(inv0, inv1, a):
    """Relative drift of Carter's constant: |Q1 - Q0| / (Q0 + (L - a E)^2)."""
    E0, L0, Q0 = inv0[:, 0], inv0[:, 1], inv0[:, 2]
    K = Q0 + (L0 - a * E0) ** 2
    return np.abs(inv1[:, 2] - Q0) / np.maximum(K, 1e-300)


class Reference:
    """Oracle records of a set of rays with the per-ray conditioning flags
    described in the module docstring.

    rays: (n, 5) (alpha, beta, a, incl, r_obs); far: band mask (n,).
    single / double: compute the conditioning at that precision."""

    def __init__(self, rays, opts, far, single=True, double=False, M=1.0):
        self.rays = np.ascontiguousarray(rays, dtype=np.float64)
        self.opts = opts
        self.far = np.asarray(far, dtype=bool)
        self.M = M
        a, ro = self.rays[:, 2], self.rays[:, 4]
        self.y0 = oracle.initial_many(self.rays, M)
        self.ref = oracle.trace_states(self.y0, a, ro, opts)
        pr = self.rays.copy()
        pr[:, 0] *= 1.0 + CHAOS_ALPHA
        self.chaotic = ~(angle_move(oracle.trace_many(pr, opts), self.ref) <= CHAOS_MOVE)
        self.inv0 = self._invariants(self.y0)
        self.inv1 = self._invariants(self.ref[:, 8:16])
        self.qd = q_drift(self.inv0, self.inv1, a)
        self.diverged = ~(self.qd < DIVERGED_Q)
        self.single_ill = self._ill(SINGLE_U, SINGLE_TOL, angle_move) if single else None
        self.double_ill = self._ill(DOUBLE_U, DOUBLE_TOL, rel_move) if double else None

    def _invariants(self, ys):
        out = np.empty((len(ys), 4))
        for i in range(len(ys)):
            out[i] = oracle.invariants(self.M, self.rays[i, 2], ys[i])
        return out

    def _ill(self, u, tol, move):
        a, ro = self.rays[:, 2], self.rays[:, 4]
        ill = np.zeros(len(self.rays), dtype=bool)
        for kind, sgn in (("scale", 1.0), ("kr", 1.0), ("kr", -1.0)):
            y = self.y0.copy()
            if kind == "scale":
                y[:, 4:] *= 1.0 + u
            else:
                y[:, 5] *= 1.0 + sgn * u
            ill |= ~(move(oracle.trace_states(y, a, ro, self.opts), self.ref) <= tol)
        return ill

    @property
    def n(self):
        return len(self.rays)

    def done(self):
        """Rays the oracle traces to a stop surface: capture, escape, or the
        equatorial plane of the Sec. 3 projection."""
        st = self.ref[:, 0]
        return (st == oracle.CAPTURED) | (st == oracle.ESCAPED) | (st == oracle.EQUATOR)

    def faithful(self):
        """Rays outside the band that are neither chaotic nor diverged, and
        that the oracle traces to a stop surface."""
        return self.far & ~self.chaotic & ~self.diverged & self.done()

    def compared(self, precision="single"):
        """Rays whose final angles are compared at the precision's tolerance:
        the faithful rays that are conditioned at that precision."""
        ill = self.single_ill if precision == "single" else self.double_ill
        m = self.faithful()
        return m & ~ill if ill is not None else m

    def census(self, precision="single"):
        cap = self.ref[:, 0] == oracle.CAPTURED
        far = self.far & self.done()
        cmp_ = self.compared(precision)
        ill = self.single_ill if precision == "single" else self.double_ill
        out = {"n": self.n, "far": int(self.far.sum()), "far_captured": int((far & cap).sum()),
               "chaotic": int((far & self.chaotic).sum()), "diverged": int((far & self.diverged).sum()),
               "compared": int(cmp_.sum()), "compared_captured": int((cmp_ & cap).sum())}
        if ill is not None:
            out["ill_conditioned"] = int((far & ~self.chaotic & ~self.diverged & ill).sum())
        return out


def compare(gpu, ref, sel):
    """Differences between GPU and oracle records on the selected rays (both
    sides with the same status there, else counted as disagreements)."""
    same = gpu[:, 0] == ref[:, 0]
    s = sel & same
    dang = angle_move(gpu, ref)[s]
    rel = rel_move(gpu, ref)[s]
    return {
        "n_selected": int(sel.sum()),
        "status_disagree": int((sel & ~same).sum()),
        "n_compared": int(s.sum()),
        "max_dang": float(dang.max()) if dang.size else 0.0,
        "max_rel": float(rel.max()) if rel.size else 0.0,
        "n_ang_gt_1e-4": int((dang > 1e-4).sum()),
        "steps_equal_frac": float((gpu[s, 1] == ref[s, 1]).mean()) if s.any() else 1.0,
        "redos_equal_frac": float((gpu[s, 2] == ref[s, 2]).mean()) if s.any() else 1.0,
    }


def class_agreement(gpu, ref, far):
    """Capture/escape classification agreement outside the band."""
    same = gpu[:, 0] == ref[:, 0]
    return float(same[far].mean()) if far.any() else 1.0, int((~same & far).sum())
