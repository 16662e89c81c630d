"""Pins of the FP64 CPU oracle against what theory fixes (no GPU).

Each test checks the oracle against something other than itself: a textbook
closed form, an exact quadrature, an identity, a symmetry, or the paper's own
worked example.  A plausible mistake anywhere in the oracle -- a dropped
Christoffel term, a wrong sign, a transposed index, a wrong RK4 weight, a
wrong initial direction, a wrong remap -- fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import theory as T

M = 1.0
HERE = os.path.dirname(os.path.abspath(__file__))
RNG = np.random.default_rng(1303057)
POINTS = [(M, a, r, th) for a in (0.0, 0.5, 0.99, -0.7)
          for r, th in ((2.5, 0.3), (3.7, 1.2), (12.0, 2.6), (150.0, 1.5707))]


# ---------------------------------------------------------------- metric ---

@pytest.mark.parametrize("M_,a,r,th", POINTS)
def test_metric_determinant_and_inverse(orc, M_, a, r, th):
    """det g = -Sigma^2 sin^2 th for Kerr; g^{-1} g = 1."""
    g = orc.metric(M_, a, r, th)
    gi = orc.inverse_metric(M_, a, r, th)
    Sigma = r * r + a * a * math.cos(th) ** 2
    assert np.linalg.det(g) == pytest.approx(-Sigma ** 2 * math.sin(th) ** 2, rel=1e-12)
    assert np.allclose(gi @ g, np.eye(4), atol=1e-12)
    # the (t, phi) block determinant is -Delta sin^2 th
    Delta = r * r - 2 * M_ * r + a * a
    det2 = g[0, 0] * g[3, 3] - g[0, 3] ** 2
    assert det2 == pytest.approx(-Delta * math.sin(th) ** 2, rel=1e-12)


@pytest.mark.parametrize("M_,a,r,th", POINTS)
def test_metric_derivatives_match_finite_differences(orc, M_, a, r, th):
    dg = orc.metric_derivs(M_, a, r, th)
    for k, (dr, dth) in ((1, (1e-5 * r, 0.0)), (2, (0.0, 1e-5))):
        hi = orc.metric(M_, a, r + dr, th + dth)
        lo = orc.metric(M_, a, r - dr, th - dth)
        fd = (hi - lo) / (2 * (dr + dth))
        scale = np.abs(fd).max() + 1e-30
        assert np.abs(dg[k] - fd).max() <= 1e-7 * scale
    assert np.all(dg[0] == 0) and np.all(dg[3] == 0)


def test_horizon(orc):
    assert orc.horizon(1.0, 0.0) == 2.0
    a = 0.99
    rh = orc.horizon(1.0, a)
    assert rh * rh - 2 * rh + a * a == pytest.approx(0.0, abs=1e-14)


# ----------------------------------------------------------- christoffel ---

@pytest.mark.parametrize("r,th", [(2.5, 0.4), (3.0, 1.1), (40.0, 2.9)])
def test_christoffel_reduces_to_schwarzschild(orc, r, th):
    G = orc.christoffel(M, 0.0, r, th)
    ref = T.schwarzschild_gamma(M, r, th)
    for mu in range(4):
        for a in range(4):
            for b in range(4):
                key = (mu, min(a, b), max(a, b))
                want = ref.get(key, 0.0)
                assert G[mu, a, b] == pytest.approx(want, rel=1e-12, abs=1e-15), (mu, a, b)


@pytest.mark.parametrize("M_,a,r,th", POINTS)
def test_christoffel_symmetric_and_metric_compatible(orc, M_, a, r, th):
    """Gamma^mu_ab = Gamma^mu_ba and nabla g = 0:
    d_c g_ab = Gamma^l_ca g_lb + Gamma^l_cb g_al (a transposed index in the
    general formula breaks this)."""
    G = orc.christoffel(M_, a, r, th)
    g = orc.metric(M_, a, r, th)
    dg = orc.metric_derivs(M_, a, r, th)
    assert np.allclose(G, np.transpose(G, (0, 2, 1)), rtol=0, atol=1e-14 * np.abs(G).max())
    rhs = np.einsum("lca,lb->cab", G, g) + np.einsum("lcb,al->cab", G, g)
    assert np.allclose(dg, rhs, rtol=1e-11, atol=1e-12 * np.abs(dg).max())


def test_christoffel_general_formula_against_fd_metric(orc):
    """Gamma from finite differences of the metric (no analytic derivative at
    all) agrees with the oracle's analytic-derivative Gamma."""
    for (M_, a, r, th) in POINTS:
        gi = orc.inverse_metric(M_, a, r, th)
        dg = np.zeros((4, 4, 4))
        for k, (dr, dth) in ((1, (1e-5 * r, 0.0)), (2, (0.0, 1e-5))):
            dg[k] = (orc.metric(M_, a, r + dr, th + dth) - orc.metric(M_, a, r - dr, th - dth)) / (2 * (dr + dth))
        Gfd = 0.5 * (np.einsum("mn,anb->mab", gi, dg) + np.einsum("mn,bna->mab", gi, dg)
                     - np.einsum("mn,nab->mab", gi, dg))
        G = orc.christoffel(M_, a, r, th)
        assert np.abs(G - Gfd).max() <= 1e-7 * (np.abs(G).max() + 1e-30)


# ---------------------------------------------------------- set-up (C2) ---

@pytest.mark.parametrize("a", [0.0, 0.6, 0.99])
@pytest.mark.parametrize("incl_deg", [17.0, 60.0, 90.0])
def test_initial_conditions_far_field_invariants(orc, a, incl_deg):
    """Far from the hole the image-plane coordinates are Bardeen's: L_z/E ->
    -alpha sin i and Q/E^2 -> beta^2 + (alpha^2 - a^2) cos^2 i, with errors of
    order M/r_obs; the initial momentum is null and E = 1."""
    incl = math.radians(incl_deg)
    for alpha, beta in ((3.0, -4.0), (-7.5, 2.25), (0.3, 9.0)):
        for r_obs, tol in ((1e3, 3e-3), (1e6, 3e-6)):
            y = orc.initial(M, a, r_obs, incl, alpha, beta)
            E, L, Q, N = orc.invariants(M, a, y)
            assert E == pytest.approx(1.0, rel=1e-14)
            assert abs(N) <= 1e-12 * y[4] ** 2
            scale = alpha * alpha + beta * beta + 1.0
            assert abs(L / E + alpha * math.sin(incl)) <= tol * math.sqrt(scale)
            q_ref = beta ** 2 + (alpha ** 2 - a * a) * math.cos(incl) ** 2
            assert abs(Q / E ** 2 - q_ref) <= tol * scale
            assert y[5] > 0  # moving towards the observer


def test_xi_is_minus_one_on_null_vectors(orc):
    """Eq. 4 equals -1 exactly when g k k = 0, and xi + 1 = N/(g_tt k^t^2)."""
    for a in (0.0, 0.9):
        y = orc.initial(M, a, 1000.0, 1.0, 4.0, 3.0)
        assert orc.xi(M, a, y) == pytest.approx(-1.0, abs=1e-12)
        y2 = y.copy()
        y2[5] *= 1.01
        N = orc.null_norm(M, a, y2)
        gtt = orc.metric(M, a, y2[1], y2[2])[0, 0]
        assert orc.xi(M, a, y2) + 1.0 == pytest.approx(N / (gtt * y2[4] ** 2), rel=1e-10)


# ----------------------------------------------------- steps of Sec. 2 ---

def test_remap_eq3(orc):
    y = np.array([0.0, 5.0, math.pi + 0.1, 0.2, 1.0, 0.1, 0.3, 0.05])
    z, did = orc.remap(y)
    assert did and z[2] == pytest.approx(math.pi - 0.1) and z[3] == pytest.approx(0.2 + math.pi)
    assert z[6] == -0.3 and np.all(z[[0, 1, 4, 5, 7]] == y[[0, 1, 4, 5, 7]])
    y[2] = -0.1
    z, did = orc.remap(y)
    assert did and z[2] == pytest.approx(0.1) and z[3] == pytest.approx(0.2 - math.pi) and z[6] == -0.3
    for th in (0.0, 1.0, math.pi):
        y[2] = th
        z, did = orc.remap(y)
        assert not did and np.all(z == y)


def test_rk4_is_fourth_order(orc):
    """One RK4 step vs two half steps: the difference scales as h^5."""
    a = 0.7
    y = orc.initial(M, a, 1000.0, 1.0, 5.5, 2.0)
    # move in close to the hole first
    for _ in range(120):
        y, _ = orc.rk4(M, a, y, orc.step_size(orc.Options(), orc.horizon(M, a), y))
    diffs = []
    for h in (-0.2, -0.1, -0.05):
        one, _ = orc.rk4(M, a, y, h)
        half, _ = orc.rk4(M, a, y, h / 2)
        two, _ = orc.rk4(M, a, half, h / 2)
        diffs.append(np.abs(one - two)[1:4].max())
    ratios = [diffs[0] / diffs[1], diffs[1] / diffs[2]]
    assert all(25 < q < 40 for q in ratios), ratios


def test_step_rule(orc):
    o = orc.Options()
    rh = orc.horizon(M, 0.5)
    y = orc.initial(M, 0.5, 1000.0, 1.0, 4.0, 3.0)
    h = orc.step_size(o, rh, y)
    assert h < 0 and -h == pytest.approx(y[1] / 32.0)
    # close to the horizon the guard halves the distance to it (linearly)
    y2 = y.copy()
    y2[1] = rh + 0.02
    y2[5] = -1.5
    assert -orc.step_size(o, rh, y2) == pytest.approx(max(0.02 / 3.0, 1e-3))
    y2[1] = rh + 1e-4
    assert -orc.step_size(o, rh, y2) == pytest.approx(1e-3)
    # Eq. 2: the angular rates shrink the step
    o2 = orc.Options(step_rule=orc.STEP_EQ2)
    y3 = y.copy()
    y3[6], y3[7] = 0.5, 0.25
    assert -orc.step_size(o2, rh, y3) == pytest.approx((1 / 32) / (abs(y3[5] / y3[1]) + 0.75))


def test_hermite_is_exact_on_cubics_and_lands_on_surface(orc):
    p = np.poly1d([0.3, -1.1, 0.7, 2.0])
    dp = p.deriv()
    h = 0.7
    for s in (0.0, 0.25, 0.5, 0.9, 1.0):
        assert orc.hermite(p(0), dp(0), p(h), dp(h), h, s) == pytest.approx(p(s * h), abs=1e-13)
    a = 0.9
    y0 = orc.initial(M, a, 1000.0, 1.2, 2.0, 1.0)
    y1, _ = orc.rk4(M, a, y0, -20.0)
    r_stop = 0.5 * (y0[1] + y1[1])
    fin = orc.stop_surface(y0, y1, -20.0, r_stop)
    assert fin[1] == pytest.approx(r_stop, abs=1e-12)


# ------------------------------------------------------ whole rays (M=0) ---

@pytest.mark.parametrize("a", [0.0, 0.8])
def test_flat_space_rays_are_straight_lines(orc, a):
    """M = 0: Kerr reduces to flat space in oblate spheroidal coordinates, no
    capture, and every ray leaves along the straight line it came in on."""
    o = orc.Options(M=0.0)
    # (rays with impact parameter below |a| would thread the r = 0 disk of the
    # oblate chart, where Boyer-Lindquist coordinates end; none is used here)
    for alpha, beta, incl in ((3.0, 4.0, 0.7), (9.0, -2.0, 1.57), (1.6, 1.5, 0.2), (-5.0, -6.0, 2.0)):
        y0 = orc.initial(0.0, a, 1000.0, incl, alpha, beta)
        rec = orc.trace(a, 1000.0, y0, o)
        assert rec[0] == orc.ESCAPED and rec[2] == 0
        th, ph = T.straight_line_exit(a, y0, rec[5])
        assert rec[5] == pytest.approx(1000.0, abs=1e-9)
        assert abs(rec[6] - th) < 1e-6
        assert abs(T.angle_diff(rec[7], ph)) < 1e-6


@pytest.mark.parametrize("a", [0.0, 0.8])
def test_near_axis_rays_need_eq2(orc, a):
    """Rays that graze the polar axis: the benchmark rule |h| = r/32 ignores
    d phi / d lambda, so RK4 fails the xi test (Eq. 4) step after step and the
    ray crawls past the pole on Euler redos, losing accuracy; the paper's own
    Eq. 2 shrinks the step with the angular rates and stays on the line."""
    for alpha, beta, incl in ((-0.4, 7.0, 1.3), (0.05, 3.0, 0.9)):
        y0 = orc.initial(0.0, a, 1000.0, incl, alpha, beta)
        bench = orc.trace(a, 1000.0, y0, orc.Options(M=0.0))
        eq2 = orc.trace(a, 1000.0, y0, orc.Options(M=0.0, step_rule=orc.STEP_EQ2))
        th, ph = T.straight_line_exit(a, y0, eq2[5])
        assert eq2[0] == orc.ESCAPED and eq2[2] == 0
        assert abs(eq2[6] - th) < 1e-6 and abs(T.angle_diff(eq2[7], ph)) < 5e-6
        assert bench[0] == orc.ESCAPED and bench[2] > 1000


# ------------------------------------------------- whole rays (Kerr) -------

@pytest.mark.parametrize("a", [0.0, 0.5, 0.9, -0.9])
@pytest.mark.parametrize("alpha", [7.0, -7.0, 12.0])
def test_equatorial_deflection_matches_exact_quadrature(orc, a, alpha):
    """Equatorial photons (i = 90 deg, beta = 0): the azimuth swept between the
    start and the escape radius equals the exact quadrature of the Kerr first
    integrals, to RK4 truncation error, and the error falls 16x when the step
    halves."""
    errs = []
    for hf in (1 / 32, 1 / 64):
        y0 = orc.initial(M, a, 1000.0, math.pi / 2, alpha, 0.0)
        E, L, _, _ = orc.invariants(M, a, y0)
        rec = orc.trace(a, 1000.0, y0, orc.Options(h_frac=hf))
        assert rec[0] == orc.ESCAPED
        assert abs(rec[6] - math.pi / 2) < 1e-12
        exact = -T.equatorial_sweep(a, L / E, y0[1], rec[5])
        errs.append(abs((rec[7] - y0[3]) - exact))
    assert errs[0] < 5e-5
    assert 12.0 < errs[0] / errs[1] < 20.0, errs


def test_polar_shadow_radius_limits():
    """a = 0 gives 3 sqrt 3; the i -> 0 limit of the sampled Bardeen curve
    approaches the same circle."""
    assert T.polar_shadow_radius(0.0) == pytest.approx(3.0 * math.sqrt(3.0))
    cx, cy = T.bardeen_curve(0.99, 0.01, 200000)
    assert np.hypot(cx, cy).max() == pytest.approx(T.polar_shadow_radius(0.99), abs=0.03)


def test_quadrature_reproduces_weak_field_series():
    """The exact quadrature itself against the textbook 4M/b + 15 pi M^2/(4b^2)."""
    for b in (300.0, 1000.0):
        defl = T.equatorial_sweep(0.0, b, 1e12, 1e12) - math.pi
        assert defl == pytest.approx(T.schwarzschild_deflection_series(M, b), rel=5e-4)


def test_schwarzschild_capture_radius(orc):
    """a = 0: captured iff b < 3 sqrt 3 (b^2 = alpha^2 + beta^2 on the plane)."""
    bc = 3.0 * math.sqrt(3.0)
    bs = np.concatenate([np.linspace(0.3, bc - 0.05, 9), np.linspace(bc + 0.05, 9.5, 9)])
    phis = np.linspace(0.1, 2 * math.pi, len(bs), endpoint=False)
    rays = np.array([[b * math.cos(p), b * math.sin(p), 0.0, 1.0, 1000.0] for b, p in zip(bs, phis)])
    out = orc.trace_many(rays)
    captured = out[:, 0] == orc.CAPTURED
    assert np.all(captured == (bs < bc))
    assert np.all((out[:, 0] == orc.CAPTURED) | (out[:, 0] == orc.ESCAPED))


@pytest.mark.parametrize("a,incl_deg", [(0.99, 90.0), (0.6, 45.0)])
@pytest.mark.parametrize("rule", ["bench", "eq2"])
def test_kerr_capture_map_matches_bardeen_shadow(orc, a, incl_deg, rule):
    """Outside a 0.05 M band around Bardeen's critical curve the capture map
    equals the analytic shadow exactly.  Under the benchmark step rule the
    near-axis column (|alpha| < 0.5, i.e. L_z ~ 0, rays that graze the poles)
    is left out: that rule ignores d phi / d lambda and can misclassify there
    (see test_near_axis_rays_need_eq2); the paper's Eq. 2 needs no exclusion."""
    incl = math.radians(incl_deg)
    rays = orc.image_rays(a, incl, 1000.0, 40, 40, -8.0, 8.0, -8.0, 8.0)
    step_rule = orc.STEP_EQ2 if rule == "eq2" else orc.STEP_BENCH
    out = orc.trace_many(rays, orc.Options(max_steps=20000, step_rule=step_rule))
    inside, far = T.shadow_truth(rays[:, 0], rays[:, 1], a, incl, band=0.05)
    if rule == "bench":
        far &= np.abs(rays[:, 0]) >= 0.5
    got = out[:, 0] == orc.CAPTURED
    assert far.sum() > 1400
    assert np.all(got[far] == inside[far])


def test_constants_of_motion_conserved_with_fourth_order_drift(orc):
    """E and L_z are conserved by the continuous equations and Q is Carter's
    constant; along whole rays their drift is truncation error that falls ~16x
    when the step halves."""
    a = 0.9
    drift = {}
    for hf in (1 / 32, 1 / 64):
        rows = []
        for alpha, beta in ((6.0, 5.0), (-9.0, 3.0), (2.0, -8.0)):
            y0 = orc.initial(M, a, 1000.0, 1.1, alpha, beta)
            E0, L0, Q0, _ = orc.invariants(M, a, y0)
            rec = orc.trace(a, 1000.0, y0, orc.Options(h_frac=hf))
            assert rec[0] == orc.ESCAPED and rec[2] == 0
            E1, L1, Q1, N1 = orc.invariants(M, a, rec[8:16])
            K = Q0 + (L0 - a * E0) ** 2
            rows.append([abs(E1 - E0), abs(L1 - L0), abs(Q1 - Q0) / K, abs(N1)])
        drift[hf] = np.array(rows)
    d32, d64 = drift[1 / 32], drift[1 / 64]
    assert d32.max() < 1e-5
    assert np.all(d32[:, 2] / d64[:, 2] > 8.0)


def test_symmetries(orc):
    """beta -> -beta mirrors theta about the equator; (a, alpha) -> (-a, -alpha)
    flips phi.  Status and step counts are unchanged."""
    a = 0.8
    for alpha, beta, incl in ((4.0, 3.0, 1.57079632679), (-6.0, 5.5, 1.57079632679)):
        r1 = orc.trace(a, 1000.0, orc.initial(M, a, 1000.0, incl, alpha, beta))
        r2 = orc.trace(a, 1000.0, orc.initial(M, a, 1000.0, incl, alpha, -beta))
        assert r1[0] == r2[0] and abs(r1[1] - r2[1]) <= 1
        if r1[0] == orc.ESCAPED:
            assert r1[6] == pytest.approx(math.pi - r2[6], abs=1e-6)
    for alpha, beta, incl in ((4.0, 3.0, 1.0), (-7.0, -2.0, 0.5)):
        r1 = orc.trace(a, 1000.0, orc.initial(M, a, 1000.0, incl, alpha, beta))
        r2 = orc.trace(-a, 1000.0, orc.initial(M, -a, 1000.0, incl, -alpha, beta))
        assert r1[0] == r2[0] and r1[1] == r2[1]
        assert r1[6] == pytest.approx(r2[6], abs=1e-10)
        assert abs(T.angle_diff(r1[7], -r2[7])) < 1e-10


def test_pole_crossing_ray_from_the_paper(orc):
    """Sec. 2 worked example (golden/pole_ray.json): the production scheme
    (Eq. 2 steps, RK4, Euler fallback of Eq. 4, remap of Eq. 3) carries the
    ray across both poles and into the horizon, and the analytic shadow agrees
    that it is captured."""
    with open(os.path.join(HERE, "golden", "pole_ray.json")) as f:
        g = json.load(f)
    a = g["a"]
    # observer on the spin axis, photon travelling along it (reading C10)
    y0 = orc.initial(M, a, g["r0_cos_theta0"], 0.0, g["r0_sin_theta0"], 0.0)
    assert y0[1] * math.cos(y0[2]) == pytest.approx(g["r0_cos_theta0"], rel=1e-12)
    assert y0[1] * math.sin(y0[2]) == pytest.approx(g["r0_sin_theta0"], rel=1e-12)
    assert g["step_rule"] == "eq2"
    rec = orc.trace(a, g["r0_cos_theta0"], y0, orc.Options(step_rule=orc.STEP_EQ2, h_frac=g["Delta"]))
    assert rec[0] == orc.CAPTURED
    assert rec[3] >= g["min_pole_crossings"]
    assert rec[2] >= 1  # the Euler fallback of Eq. 4 fired
    assert g["r0_sin_theta0"] < T.polar_shadow_radius(a)


@pytest.mark.parametrize("a,r,th", [(0.9, 6.0, 1.1), (0.5, 40.0, 0.3), (0.99, 2.5, 1.6)])
def test_euler_redo_is_one_ninth_step_from_the_old_state(orc, a, r, th):
    """Sec. 2, text after Eq. 4: when the null condition fails by more than
    eps after an RK4 step, the step is taken again as a forward-Euler step of
    one ninth of its length from the state it started from.  A one-step trace
    of a state whose k is pushed off the null cone must end exactly on
    y + (h/9) dy/dl(y), with one redo counted and an affine length of |h|/9;
    the same trace from the null state takes the RK4 step of full length."""
    y = np.array([0.0, r, th, 0.3, 0.0, -0.7, 0.05, 0.02])
    g = orc.metric(M, a, r, th)
    # k^t the future root of g(k, k) = 0, so y starts on the null cone
    A, B = g[0, 0], 2 * (g[0, 3] * y[7])
    C = g[1, 1] * y[5] ** 2 + g[2, 2] * y[6] ** 2 + g[3, 3] * y[7] ** 2
    assert A < 0  # outside the ergoregion: the larger root is the future one
    y[4] = (-B - math.sqrt(B * B - 4 * A * C)) / (2 * A)
    r_h = orc.horizon(M, a)
    # the benchmark step rule written out: |h| = max(min(r/32, (r - r_h)/(2|k^r|)), 1e-3), backward
    h = -max(min(r / 32.0, (r - r_h) / (2.0 * abs(y[5]))), 1e-3)
    one = orc.Options(max_steps=1)
    rec = orc.trace(a, 1000.0, y, one)
    y_rk4, _ = orc.rk4(M, a, y, h)
    assert rec[0] == orc.STEP_CAP and rec[1] == 1 and rec[2] == 0
    assert np.allclose(rec[8:16], orc.remap(y_rk4)[0], rtol=0, atol=1e-15 * np.abs(y_rk4).max())
    assert rec[16] == pytest.approx(abs(h), rel=1e-15)
    bad = y.copy()
    bad[5] *= 1.05  # off the null cone by ~10 %: |xi + 1| >> 1e-3
    assert abs(orc.xi(M, a, bad) + 1.0) > 1e-2
    h_bad = -max(min(r / 32.0, (r - r_h) / (2.0 * abs(bad[5]))), 1e-3)
    rec = orc.trace(a, 1000.0, bad, one)
    want = bad + (h_bad / 9.0) * orc.rhs(M, a, bad)
    assert rec[0] == orc.STEP_CAP and rec[1] == 1 and rec[2] == 1
    assert np.allclose(rec[8:16], orc.remap(want)[0], rtol=0, atol=1e-15 * np.abs(want).max())
    assert rec[16] == pytest.approx(abs(h_bad) / 9.0, rel=1e-15)
    # neither a third of the step nor a redo from the rejected RK4 end point
    y1_bad, _ = orc.rk4(M, a, bad, h_bad)
    for wrong in (bad + (h_bad / 3.0) * orc.rhs(M, a, bad), y1_bad + (h_bad / 9.0) * orc.rhs(M, a, y1_bad)):
        assert np.abs(rec[8:16] - orc.remap(wrong)[0]).max() > 1e-6


@pytest.mark.parametrize("b", [2.5, 4.0, 6.0, 9.0, 20.0])
def test_equator_crossing_matches_schwarzschild_quadrature(orc, b):
    """Grid projection (Sec. 3): seen face-on, a Schwarzschild photon's orbit
    contains the axis, so it meets the equatorial plane where its swept
    orbital angle reaches pi/2 - theta_0, or is captured first when it plunges
    before sweeping that much.  The oracle's interpolated crossing radius
    matches the exact quadrature (impact parameter from the ray's own
    invariants, b^2 = Q + L_z^2) to RK4 truncation, falling ~16x when the step
    halves."""
    errs = []
    for hf in (1 / 32, 1 / 64):
        y0 = orc.initial(M, 0.0, 1000.0, 0.0, b, 0.0)
        E, L, Q, _ = orc.invariants(M, 0.0, y0)
        b_true = math.sqrt(Q + L * L) / E
        rec = orc.trace(0.0, 1000.0, y0, orc.Options(h_frac=hf, stop_equator=1))
        target = math.pi / 2 - y0[2]
        r_cap = 1.01 * 2.0
        if b_true < 3 * math.sqrt(3) and T.schwarzschild_swept_to(b_true, y0[1], r_cap) < target:
            assert rec[0] == orc.CAPTURED
            return
        assert rec[0] == orc.EQUATOR
        assert rec[6] == pytest.approx(math.pi / 2)
        r_eq = T.schwarzschild_radius_at_angle(b_true, y0[1], target)
        errs.append(abs(rec[5] - r_eq) / r_eq)
    assert errs[0] < 2e-6, errs
    assert errs[1] < errs[0] / 6 or errs[1] < 1e-9, errs
