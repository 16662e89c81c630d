"""Photon-ring metrics of Sec. 4 (Eqs. 6-10), in plain numpy.

Test infrastructure only: the parity reference for the CUDA ring reduction.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  Nothing here imports the CUDA library.

The polar image-plane grid of Sec. 4: n_R radii R cell-centred on (R0, R1)
and n_th angles vartheta from th0 to th1 with both ends included (the paper's
6000 x 181 rays over (1.5, 7.5) x [0, pi]: an open radial interval, a closed
angular one, one degree apart).  Ray index = angle row * n_R + radius column.
A ray's Cartesian image-plane position is alpha = R cos(vartheta),
beta = R sin(vartheta) (Eqs. 9-10).

Readings (the paper leaves these to the reader):
* boundary of a row: the cell edge that leaves the fewest of the row's rays
  on the wrong side (captured outside, or not captured inside); for a row
  whose captured rays are exactly its innermost ones, the midpoint between
  the last captured and the first uncaptured ray centre.  A ray that the
  integrator got wrong away from the boundary (a pole crossing gone bad, for
  instance) does not move it; such rays are counted.
* the integrals over [0, 2 pi] of Eqs. 7-8 are the trapezoidal mean over the
  sampled angles; the sampled half-plane beta >= 0 gives the full-circle mean
  because the image is symmetric under beta -> -beta.
* R is measured from the midpoint c = (alpha_min + alpha_max) / 2 of the
  ring's horizontal extent, D = |c| (Eq. 6).  The paper writes alpha_0 - D,
  which is alpha_0 - c whenever c >= 0, as it is for a >= 0 with the image
  orientation L_z = -alpha E sin i used here.
"""
import math

import numpy as np

CAPTURED = 1  # status code of a captured ray in the oracle's records


def polar_grid(n_R, n_th, R0=1.5, R1=7.5, th0=0.0, th1=math.pi):
    """Radii (cell centres) and angles (ends included) of the polar grid."""
    R = R0 + (np.arange(n_R, dtype=np.float64) + 0.5) * ((R1 - R0) / n_R)
    if n_th > 1:
        th = th0 + np.arange(n_th, dtype=np.float64) * ((th1 - th0) / (n_th - 1))
    else:
        th = np.array([float(th0)])
    return R, th


def polar_rays(a, incl, r_obs, n_R, n_th, R0=1.5, R1=7.5, th0=0.0, th1=math.pi):
    """(n, 5) ray table (alpha, beta, a, incl, r_obs) of one polar image for
    ``oracle.trace_many``; rows of the grid are angles (Eqs. 9-10)."""
    R, th = polar_grid(n_R, n_th, R0, R1, th0, th1)
    Rg, Tg = np.meshgrid(R, th)
    n = Rg.size
    rays = np.empty((n, 5))
    rays[:, 0] = (Rg * np.cos(Tg)).ravel()
    rays[:, 1] = (Rg * np.sin(Tg)).ravel()
    rays[:, 2] = a
    rays[:, 3] = incl
    rays[:, 4] = r_obs
    return rays


def ring_boundary(status, R0=1.5, R1=7.5):
    """Boundary radius of each angle row of an (n_th, n_R) status array.

    The boundary of a row is the radius R0 + k dR (a cell edge, k = 0..n_R)
    that leaves the fewest of the row's rays on the wrong side: captured
    outside it or not captured inside it.  With C(k) the number of captured
    rays among the k innermost, k maximises 2 C(k) - k; ties go to the
    smallest k.  When the captured rays of the row are exactly its innermost
    ones, k is their count and the boundary is the midpoint between the last
    captured and the first uncaptured ray centre.

    Returns (R_b, wrong, open): wrong[j] = rays of row j on the wrong side
    of its boundary (0 for a clean row); open[j] when the boundary is an end
    of the radial range (k = 0 or n_R, the ring lies off the grid)."""
    st = np.asarray(status)
    n_th, n_R = st.shape
    cap = (st == CAPTURED).astype(np.int64)
    C = np.concatenate([np.zeros((n_th, 1), np.int64), np.cumsum(cap, axis=1)], axis=1)
    k = np.argmax(2 * C - np.arange(n_R + 1)[None, :], axis=1)  # first maximum
    Ck = C[np.arange(n_th), k]
    wrong = (k - Ck) + (C[:, -1] - Ck)
    dR = (R1 - R0) / n_R
    R_b = R0 + dR * k
    open_ = (k == 0) | (k == n_R)
    return R_b, wrong, open_


def ring_metrics(R_b, th):
    """D, <R>, A (Eqs. 6-8) of the ring whose boundary radius along the angle
    th[j] from the image-plane origin is R_b[j].  Returns a dict with D,
    R_mean, A, alpha_min, alpha_max."""
    R_b = np.asarray(R_b, dtype=np.float64)
    th = np.asarray(th, dtype=np.float64)
    alpha0 = R_b * np.cos(th)  # Eq. 9
    beta0 = R_b * np.sin(th)  # Eq. 10
    a_min, a_max = float(alpha0.min()), float(alpha0.max())
    c = 0.5 * (a_min + a_max)
    D = abs(c)  # Eq. 6
    R = np.sqrt((alpha0 - c) ** 2 + beta0 ** 2)

    def mean(f):
        if f.size == 1:
            return float(f[0])
        w = np.ones_like(f)
        w[0] = w[-1] = 0.5
        return float((w * f).sum() / w.sum())

    R_mean = mean(R)  # Eq. 7
    A = 2.0 * math.sqrt(mean((R - R_mean) ** 2))  # Eq. 8
    return {"D": D, "R_mean": R_mean, "A": A, "alpha_min": a_min, "alpha_max": a_max}


def ring_from_records(rec, n_R, n_th, R0=1.5, R1=7.5, th0=0.0, th1=math.pi):
    """Ring metrics of one traced polar image from its (n, 17) oracle records
    (status in column 0).  Adds R_b, wrong and open to the dict."""
    st = np.asarray(rec)[:, 0].astype(np.int64).reshape(n_th, n_R)
    R_b, wrong, open_ = ring_boundary(st, R0, R1)
    _, th = polar_grid(n_R, n_th, R0, R1, th0, th1)
    out = ring_metrics(R_b, th)
    out.update({"R_b": R_b, "wrong": wrong, "open": open_})
    return out


__all__ = ["polar_grid", "polar_rays", "ring_boundary", "ring_metrics", "ring_from_records"]
