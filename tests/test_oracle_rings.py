"""Pins of the ring-study oracle (Sec. 4, Eqs. 5-14) against what geometry and
the theory fix: the polar grid's layout, the boundary estimator by brute force,
closed-form rings (an off-centre circle, an ellipse), Bardeen's critical curve
against the paper's fitted formulae (Eqs. 11-14), and the traced capture of
every ray against its exact fate from the conserved quantities."""
import itertools
import math

import numpy as np
import pytest
from scipy.special import ellipk

import oracle
from oracle import rings
from paper_1303_5057_gb300 import inputs

import theory as T

# The ring study integrates with Eq. 2 (Delta = 1/32) and no floor under the
# step (the 1e-3 floor belongs to the benchmark rule, and near a pole it would
# force the Euler fallback on every step).
RING_OPTS = oracle.Options(step_rule=oracle.STEP_EQ2, h_min=1e-9)


def test_polar_grid_layout():
    R, th = rings.polar_grid(6000, 181)
    assert R[0] == pytest.approx(1.5005, abs=1e-12) and R[-1] == pytest.approx(7.4995, abs=1e-12)
    assert np.allclose(np.diff(R), 0.001, atol=1e-12)
    assert th[0] == 0.0 and th[-1] == pytest.approx(math.pi, abs=1e-15)
    assert np.allclose(np.degrees(np.diff(th)), 1.0, atol=1e-12)
    rays = rings.polar_rays(0.5, 0.3, 1000.0, 7, 5)
    Rg, Tg = np.meshgrid(*rings.polar_grid(7, 5))
    # row-major: angle rows of 7 radii each (Eqs. 9-10)
    assert np.allclose(np.hypot(rays[:, 0], rays[:, 1]), Rg.ravel(), atol=1e-14)
    assert np.allclose(np.arctan2(rays[:, 1], rays[:, 0])[7:35], Tg.ravel()[7:35], atol=1e-14)
    assert np.allclose(rays[:7, 1], 0.0) and np.all(rays[:7, 0] > 0)
    assert np.all(rays[:, 2] == 0.5) and np.all(rays[:, 3] == 0.3) and np.all(rays[:, 4] == 1000.0)
    assert rings.polar_grid(4, 1)[1].tolist() == [0.0]


def _brute_boundary(row):
    """k in 0..n minimising the rays on the wrong side, smallest k on ties."""
    n = len(row)
    costs = [sum(1 for j in range(k) if row[j] != 1) + sum(1 for j in range(k, n) if row[j] == 1)
             for k in range(n + 1)]
    k = int(np.argmin(costs))
    return k, costs[k]


def test_boundary_estimator_matches_brute_force():
    rng = np.random.default_rng(1303)
    rows = [list(p) for n in range(1, 7) for p in itertools.product((1, 2), repeat=n)]
    rows += [list(rng.choice([1, 2, 0, 3], size=int(rng.integers(1, 15)))) for _ in range(300)]
    for row in rows:
        st = np.array([row])
        R_b, wrong, open_ = rings.ring_boundary(st, 0.0, float(len(row)))
        k, cost = _brute_boundary(row)
        assert R_b[0] == pytest.approx(k, abs=1e-12), row
        assert wrong[0] == cost, row
        assert open_[0] == (k == 0 or k == len(row)), row


def test_boundary_of_clean_rows_is_the_cell_edge():
    n_R = 50
    counts = np.array([0, 1, 17, 49, 50])
    st = np.where(np.arange(n_R)[None, :] < counts[:, None], 1, 2)
    R_b, wrong, open_ = rings.ring_boundary(st, 1.5, 7.5)
    assert np.allclose(R_b, 1.5 + counts * 0.12, atol=1e-14)
    assert wrong.tolist() == [0] * 5
    assert open_.tolist() == [True, False, False, False, True]
    # an isolated wrong ray on either side leaves the boundary in place
    st2 = st.copy()
    st2[2, 3] = 2   # escaped deep inside
    st2[2, 40] = 1  # captured far outside
    R_b2, wrong2, _ = rings.ring_boundary(st2, 1.5, 7.5)
    assert R_b2[2] == R_b[2] and wrong2[2] == 2


def test_metrics_of_an_off_centre_circle():
    # circle of radius rho about (c, 0), seen along rays from the origin
    for c, rho in ((0.0, 5.196), (0.7, 5.0), (-1.2, 4.5), (2.4, 4.9)):
        _, th = rings.polar_grid(10, 181)
        R_b = c * np.cos(th) + np.sqrt(rho ** 2 - (c * np.sin(th)) ** 2)
        m = rings.ring_metrics(R_b, th)
        assert m["D"] == pytest.approx(abs(c), abs=1e-12)
        assert m["alpha_min"] == pytest.approx(c - rho, abs=1e-12)
        assert m["alpha_max"] == pytest.approx(c + rho, abs=1e-12)
        assert m["R_mean"] == pytest.approx(rho, abs=1e-12)
        assert m["A"] < 1e-6


@pytest.mark.parametrize("p,q", [(5.2, 4.8), (4.0, 5.5), (7.0, 2.0)])
def test_metrics_of_an_ellipse_closed_form(p, q):
    """Centred ellipse with semi-axes p (along alpha) and q: over the polar
    angle, <R> = (2 q / pi) K(1 - q^2/p^2) (complete elliptic integral of the
    first kind, parameter m) and <R^2> = p q, so A = 2 sqrt(p q - <R>^2)."""
    _, th = rings.polar_grid(10, 181)
    R_b = p * q / np.sqrt((q * np.cos(th)) ** 2 + (p * np.sin(th)) ** 2)
    m = rings.ring_metrics(R_b, th)
    if p >= q:
        R_mean = 2.0 * q / math.pi * ellipk(1.0 - q * q / (p * p))
    else:
        R_mean = 2.0 * p / math.pi * ellipk(1.0 - p * p / (q * q))
    assert m["D"] == pytest.approx(0.0, abs=1e-12)
    assert m["R_mean"] == pytest.approx(R_mean, rel=1e-9)
    assert m["A"] == pytest.approx(2.0 * math.sqrt(p * q - R_mean ** 2), rel=1e-6)


def test_bardeen_ring_against_the_paper_fits():
    """Eqs. 6-8 on the exact critical curve (r_obs -> infinity, the paper's
    181 angles) reproduce the paper's fits (Eqs. 11-14) over its whole
    16 x 19 parameter grid: the fits are good to ~0.5% in <R> and ~0.05 M in
    A, which also rules out the other readings of Eqs. 6-8 (R about the
    origin instead of the centre misses A by up to 3 M)."""
    _, th = rings.polar_grid(10, 181)
    worst_R = worst_A = 0.0
    for a in inputs.ring_spins():
        for i_deg in range(0, 91, 5):
            R_b = T.shadow_radius_at_angle(a, math.radians(i_deg), th)
            m = rings.ring_metrics(R_b, th)
            fit_R, fit_A = T.paper_ring_fits(a, i_deg)
            worst_R = max(worst_R, abs(m["R_mean"] - fit_R))
            worst_A = max(worst_A, abs(m["A"] - fit_A))
            if a == 0.0:
                assert m["R_mean"] == pytest.approx(3.0 * math.sqrt(3.0), abs=1e-12)
                assert m["D"] < 1e-12 and m["A"] < 1e-12
            if i_deg == 0:
                assert m["D"] < 1e-12 and m["A"] < 1e-12
    assert worst_R < 0.03
    assert worst_A < 0.05


def test_spins_of_the_study():
    a = inputs.ring_spins()
    assert len(a) == 16 and a[0] == 0.0 and a[-1] == pytest.approx(0.999, abs=1e-12)
    assert np.allclose(np.diff(np.log10(1.0 - np.array(a))), -0.2)


def _exact_fate(a, incl, rays):
    """Capture of each ray from the invariants of its initial state."""
    lam, eta = np.empty(len(rays)), np.empty(len(rays))
    for k, q in enumerate(rays):
        y = oracle.initial(1.0, a, q[4], incl, q[0], q[1])
        E, L, Q, _ = oracle.invariants(1.0, a, y)
        lam[k], eta[k] = L / E, Q / (E * E)
    return T.captured_from_invariants(a, lam, eta)


def test_exact_fate_reproduces_bardeen_far_away():
    """The invariants of the image-plane set-up at r_obs = 1000 put the
    boundary within a grid cell plus O(1/r_obs) of Bardeen's curve."""
    n_R, n_th = 300, 7
    for a, i_deg in ((0.9, 90), (0.6, 35), (0.999, 0)):
        incl = math.radians(i_deg)
        rays = rings.polar_rays(a, incl, 1000.0, n_R, n_th)
        cap, _ = _exact_fate(a, incl, rays)
        R_b, wrong, _ = rings.ring_boundary(np.where(cap, 1, 2).reshape(n_th, n_R))
        assert wrong.sum() == 0
        _, th = rings.polar_grid(n_R, n_th)
        exact = T.shadow_radius_at_angle(a, incl, th)
        assert np.max(np.abs(R_b - exact)) <= 0.5 * 0.02 + 2e-3


@pytest.mark.parametrize("a,i_deg", [(0.9, 90), (0.99, 45), (0.3, 30)])
def test_traced_rings_match_the_exact_fate(a, i_deg):
    """Every traced ray (Eq. 2 rule, Sec. 2 pole treatment) has the fate its
    invariants fix, the ray through the pole (the row vartheta = 90 deg at
    i = 90 deg) included, so the traced ring is the exact one on this grid."""
    n_R, n_th = 400, 10
    incl = math.radians(i_deg)
    rays = rings.polar_rays(a, incl, 1000.0, n_R, n_th)
    cap, _ = _exact_fate(a, incl, rays)
    rec = oracle.trace_many(rays, RING_OPTS)
    st = rec[:, 0].astype(int)
    assert np.all((st == oracle.CAPTURED) | (st == oracle.ESCAPED))
    assert np.array_equal(st == oracle.CAPTURED, cap)
    m = rings.ring_from_records(rec, n_R, n_th)
    R_b, _, _ = rings.ring_boundary(np.where(cap, 1, 2).reshape(n_th, n_R))
    assert np.array_equal(m["R_b"], R_b) and m["wrong"].sum() == 0


def test_face_on_rings_lose_a_few_pole_crossings():
    """Seen face-on (i = 0) every ray crosses a pole.  With the Sec. 2
    treatment as read here a few of them are mis-integrated (a full step lands
    within ~1e-4 rad of the pole, the Euler redo from there breaks the null
    condition and the Eq. 4 test then rejects every later RK4 step); the
    boundary estimator keeps the ring within a few cells regardless."""
    a, n_R, n_th = 0.999, 400, 4
    rays = rings.polar_rays(a, 0.0, 1000.0, n_R, n_th)
    cap, _ = _exact_fate(a, 0.0, rays)
    rec = oracle.trace_many(rays, RING_OPTS)
    st = rec[:, 0].astype(int)
    bad = (st == oracle.CAPTURED) != cap
    assert bad.mean() < 0.01
    m = rings.ring_from_records(rec, n_R, n_th)
    R_b, _, _ = rings.ring_boundary(np.where(cap, 1, 2).reshape(n_th, n_R))
    dR = 6.0 / n_R
    assert np.max(np.abs(m["R_b"] - R_b)) <= 3 * dR + 1e-12
