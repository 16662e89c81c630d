"""Shared comparison helpers for the GPU-vs-oracle parity tests.

Records are the 17-double rows written by both sides: status, steps, Euler
redos, pole remaps, final (t, r, theta, phi) on the stop surface, state y[8]
at the end of the last step, and one side-specific diagnostic.
"""
import math

import numpy as np

import theory as T

TWO_PI = 2.0 * math.pi


def wrap(d):
    """Angle difference wrapped into (-pi, pi]."""
    return (np.asarray(d) + math.pi) % TWO_PI - math.pi


def band_mask(images_alpha_beta, a, incl, band=0.05):
    """True for pixels farther than ``band`` from the analytic shadow boundary."""
    al, be = images_alpha_beta
    _, far = T.shadow_truth(al, be, a, incl, band=band)
    return far


def compare(gpu, ref, far=None):
    """Summary of the differences between two record arrays."""
    n = len(ref)
    if far is None:
        far = np.ones(n, dtype=bool)
    st_g, st_r = gpu[:, 0], ref[:, 0]
    agree = st_g == st_r
    both_done = agree & ((st_r == 1) | (st_r == 2))
    sel = both_done & far
    dth = np.abs(gpu[sel, 6] - ref[sel, 6])
    dph = np.abs(wrap(gpu[sel, 7] - ref[sel, 7]))
    rel = np.maximum(dth / np.maximum(1.0, np.abs(ref[sel, 6])), dph / np.maximum(1.0, np.abs(ref[sel, 7])))
    out = {
        "n": n,
        "n_far": int(far.sum()),
        "class_agree_far": float(agree[far].mean()) if far.any() else 1.0,
        "class_disagree_far": int((~agree & far).sum()),
        "n_compared": int(sel.sum()),
        "max_dtheta": float(dth.max()) if dth.size else 0.0,
        "max_dphi": float(dph.max()) if dph.size else 0.0,
        "p9999_dang": float(np.percentile(np.maximum(dth, dph), 99.99)) if dth.size else 0.0,
        "max_rel": float(rel.max()) if rel.size else 0.0,
        "n_ang_gt_1e-4": int((np.maximum(dth, dph) > 1e-4).sum()),
        "steps_equal_frac": float((gpu[sel, 1] == ref[sel, 1]).mean()) if sel.any() else 1.0,
    }
    return out


def q_drift(inv0, inv1, a):
    """Relative drift of Carter's constant: |Q1 - Q0| / (Q0 + (L - a E)^2)."""
    E0, L0, Q0 = inv0[:, 0], inv0[:, 1], inv0[:, 2]
    K = Q0 + (L0 - a * E0) ** 2
    return np.abs(inv1[:, 2] - Q0) / np.maximum(K, 1e-300)


def oracle_q_drift(orc, rays, ref, M=1.0):
    """Relative Carter drift of the oracle's own trajectories, from its
    initial state to the state at the end of its last step.  Rays whose
    oracle trajectory does not conserve Q (drift above ~1e-4) were not
    integrated faithfully by the method itself (for instance rays grazing a
    pole under a step rule that ignores d phi / d lambda); their final angles
    are numerical noise on both sides and are not compared."""
    n = len(rays)
    inv0 = np.empty((n, 4))
    inv1 = np.empty((n, 4))
    for i in range(n):
        a = rays[i, 2]
        inv0[i] = orc.invariants(M, a, orc.initial(M, a, rays[i, 4], rays[i, 3], rays[i, 0], rays[i, 1]))
        inv1[i] = orc.invariants(M, a, ref[i, 8:16])
    E0, L0, Q0 = inv0[:, 0], inv0[:, 1], inv0[:, 2]
    K = Q0 + (L0 - rays[:, 2] * E0) ** 2
    return np.abs(inv1[:, 2] - Q0) / np.maximum(K, 1e-300)


SANE_Q = 1e-4
