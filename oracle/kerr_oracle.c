/*
 * kerr_oracle.c -- plain FP64 CPU oracle for backward RK4 tracing of null
 * geodesics in the Kerr metric (Boyer-Lindquist coordinates).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity reference for the CUDA
 * tracer.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header, table or constant with the
 * CUDA library, and it imports nothing from it.
 *
 * What it computes, in the paper's order (Chan, Psaltis & Ozel 2013, "GRay",
 * Sec. 2):
 *   - one photon at a time (Sec. 2: one geodesic per thread);
 *   - the second-order geodesic equation d^2x/dl^2 = -Gamma k k, integrated
 *     with classic 4th-order Runge-Kutta (Sec. 2, the RK4 scheme the paper
 *     takes over from Psaltis & Johannsen 2012);
 *   - the step size rule (Eq. 2 horizon guard; the benchmark rule
 *     |h| = max(min(f r, (r - r_h)/(2|k^r|)), h_min) is the default, the full
 *     Eq. 2 is selectable);
 *   - the null-norm monitor xi (Eq. 4) with a forward-Euler redo of the step
 *     at one ninth of the step when |xi + 1| > eps (Sec. 2);
 *   - the pole remap theta, phi, k_theta (Eq. 3);
 *   - the stop at the horizon (Sec. 2, "stop integrating at r_bh + delta",
 *     here r <= cap_frac * r_h) or at escape.
 *
 * The Christoffel symbols are NOT taken in closed form here.  They come from
 * the general formula
 *     Gamma^mu_ab = 1/2 g^{mu nu} (d_a g_{nu b} + d_b g_{nu a} - d_nu g_{ab})
 * with hand-written analytic d_r g and d_theta g and the (t,phi) 2x2 block
 * inverse of the metric, so that the CUDA path's closed forms are checked
 * against an independent derivation.
 *
 * The paper defers the geodesic equations and the image-plane set-up to
 * Psaltis & Johannsen (2012); both are restated here from textbook general
 * relativity (units G = c = 1, mass M; M = 1 in the paper):
 *   Sigma = r^2 + a^2 cos^2 th,  Delta = r^2 - 2 M r + a^2,
 *   g_tt = -(1 - 2 M r / Sigma),  g_tph = -2 M a r sin^2 th / Sigma,
 *   g_rr = Sigma / Delta,  g_thth = Sigma,
 *   g_phph = (r^2 + a^2 + 2 M a^2 r sin^2 th / Sigma) sin^2 th,
 *   r_h = M + sqrt(M^2 - a^2)   (Sec. 2, r_bh with M = 1).
 *
 * Readings where the paper is silent are listed in the repository's design
 * notes; each is marked "reading" where it is applied below.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define T_ 0
#define R_ 1
#define TH_ 2
#define PH_ 3

/* Status codes written per ray. */
enum { ORC_ACTIVE = 0, ORC_CAPTURED = 1, ORC_ESCAPED = 2, ORC_STEP_CAP = 3, ORC_NONFINITE = 4, ORC_EQUATOR = 6 };

/* Step rules: the benchmark rule (default) and the paper's full Eq. 2. */
enum { ORC_STEP_BENCH = 0, ORC_STEP_EQ2 = 1 };

typedef struct {
    double M;          /* mass */
    double h_frac;     /* benchmark rule: |h| <= h_frac * r ; Eq. 2: Delta */
    double h_min;      /* floor on |h| */
    double cap_frac;   /* capture when r <= cap_frac * r_h */
    double eps_xi;     /* threshold on |xi + 1| (Eq. 4) */
    double r_esc_frac; /* escape radius as a multiple of r_obs (reading: 1) */
    int32_t max_steps; /* hard step cap per ray */
    int32_t step_rule; /* ORC_STEP_BENCH or ORC_STEP_EQ2 */
    int32_t stop_equator; /* 1: also stop at the first crossing of theta = pi/2 (Sec. 3 projection) */
} orc_options;

/* ------------------------------------------------------------------ */
/* Metric and its first derivatives (textbook Kerr, BL coordinates).  */
/* ------------------------------------------------------------------ */

double orc_horizon(double M, double a)
{
    /* Sec. 2: r_bh = 1 + sqrt(1 - a^2) for M = 1. */
    return M + sqrt(M * M - a * a);
}

void orc_metric(double M, double a, double r, double th, double g[4][4])
{
    double s = sin(th), c = cos(th);
    double Sigma = r * r + a * a * c * c;
    double Delta = r * r - 2.0 * M * r + a * a;
    memset(g, 0, 16 * sizeof(double));
    g[T_][T_] = -(1.0 - 2.0 * M * r / Sigma);
    g[T_][PH_] = g[PH_][T_] = -2.0 * M * a * r * s * s / Sigma;
    g[R_][R_] = Sigma / Delta;
    g[TH_][TH_] = Sigma;
    g[PH_][PH_] = (r * r + a * a + 2.0 * M * a * a * r * s * s / Sigma) * s * s;
}

/* dg[k][mu][nu] = d g_{mu nu} / d x^k ; only k = r and k = theta are nonzero
 * because the metric does not depend on t or phi. */
void orc_metric_derivs(double M, double a, double r, double th, double dg[4][4][4])
{
    double s = sin(th), c = cos(th);
    double s2 = s * s;
    double Sigma = r * r + a * a * c * c;
    double Delta = r * r - 2.0 * M * r + a * a;
    double Sigma_r = 2.0 * r;
    double Sigma_th = -2.0 * a * a * c * s;
    double Delta_r = 2.0 * r - 2.0 * M;
    double S2 = Sigma * Sigma;
    double F = r * r + a * a + 2.0 * M * a * a * r * s2 / Sigma;
    double F_r = 2.0 * r + 2.0 * M * a * a * s2 * (Sigma - r * Sigma_r) / S2;
    double F_th = 2.0 * M * a * a * r * (2.0 * s * c * Sigma - s2 * Sigma_th) / S2;

    memset(dg, 0, 64 * sizeof(double));
    /* d/dr */
    dg[R_][T_][T_] = 2.0 * M * (Sigma - r * Sigma_r) / S2;
    dg[R_][T_][PH_] = dg[R_][PH_][T_] = -2.0 * M * a * s2 * (Sigma - r * Sigma_r) / S2;
    dg[R_][R_][R_] = (Sigma_r * Delta - Sigma * Delta_r) / (Delta * Delta);
    dg[R_][TH_][TH_] = Sigma_r;
    dg[R_][PH_][PH_] = F_r * s2;
    /* d/dtheta */
    dg[TH_][T_][T_] = -2.0 * M * r * Sigma_th / S2;
    dg[TH_][T_][PH_] = dg[TH_][PH_][T_] = -2.0 * M * a * r * (2.0 * s * c * Sigma - s2 * Sigma_th) / S2;
    dg[TH_][R_][R_] = Sigma_th / Delta;
    dg[TH_][TH_][TH_] = Sigma_th;
    dg[TH_][PH_][PH_] = F_th * s2 + F * 2.0 * s * c;
}

/* Inverse metric: diagonal in r, theta; 2x2 block inverse in (t, phi). */
void orc_inverse_metric(double M, double a, double r, double th, double gi[4][4])
{
    double g[4][4];
    orc_metric(M, a, r, th, g);
    double det = g[T_][T_] * g[PH_][PH_] - g[T_][PH_] * g[T_][PH_];
    memset(gi, 0, 16 * sizeof(double));
    gi[T_][T_] = g[PH_][PH_] / det;
    gi[PH_][PH_] = g[T_][T_] / det;
    gi[T_][PH_] = gi[PH_][T_] = -g[T_][PH_] / det;
    gi[R_][R_] = 1.0 / g[R_][R_];
    gi[TH_][TH_] = 1.0 / g[TH_][TH_];
}

/* General formula for the Christoffel symbols of the second kind. */
void orc_christoffel(double M, double a, double r, double th, double G[4][4][4])
{
    double gi[4][4], dg[4][4][4];
    orc_inverse_metric(M, a, r, th, gi);
    orc_metric_derivs(M, a, r, th, dg);
    for (int mu = 0; mu < 4; ++mu)
        for (int al = 0; al < 4; ++al)
            for (int be = 0; be < 4; ++be) {
                double sum = 0.0;
                for (int nu = 0; nu < 4; ++nu)
                    sum += gi[mu][nu] * (dg[al][nu][be] + dg[be][nu][al] - dg[nu][al][be]);
                G[mu][al][be] = 0.5 * sum;
            }
}

/* Right-hand side of the first-order system: y = (x^mu, k^mu),
 * dx^mu/dl = k^mu, dk^mu/dl = -Gamma^mu_ab k^a k^b. */
void orc_rhs(double M, double a, const double y[8], double dy[8])
{
    double G[4][4][4];
    const double *k = y + 4;
    orc_christoffel(M, a, y[R_], y[TH_], G);
    for (int mu = 0; mu < 4; ++mu) {
        dy[mu] = k[mu];
        double acc = 0.0;
        for (int al = 0; al < 4; ++al)
            for (int be = 0; be < 4; ++be)
                acc += G[mu][al][be] * k[al] * k[be];
        dy[4 + mu] = -acc;
    }
}

/* ------------------------------------------------------------------ */
/* Diagnostics: null norm, xi (Eq. 4), constants of motion.           */
/* ------------------------------------------------------------------ */

double orc_null_norm(double M, double a, const double y[8])
{
    double g[4][4];
    orc_metric(M, a, y[R_], y[TH_], g);
    const double *k = y + 4;
    double N = 0.0;
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
            N += g[m][n] * k[m] * k[n];
    return N;
}

/* Eq. 4: xi = [g_rr k^r^2 + g_phph k^ph^2 + g_thth k^th^2 + 2 g_tph k^t k^ph]
 *             / [g_tt k^t^2], which is -1 on a null vector. */
double orc_xi(double M, double a, const double y[8])
{
    double g[4][4];
    orc_metric(M, a, y[R_], y[TH_], g);
    const double *k = y + 4;
    double num = g[R_][R_] * k[R_] * k[R_] + g[PH_][PH_] * k[PH_] * k[PH_]
               + g[TH_][TH_] * k[TH_] * k[TH_] + 2.0 * g[T_][PH_] * k[T_] * k[PH_];
    return num / (g[T_][T_] * k[T_] * k[T_]);
}

/* E = -k_t, L_z = k_phi, Carter constant Q = k_th^2 + cos^2 th (-a^2 E^2 +
 * L_z^2 / sin^2 th), and the null norm N = g k k. */
void orc_invariants(double M, double a, const double y[8], double out[4])
{
    double g[4][4];
    orc_metric(M, a, y[R_], y[TH_], g);
    const double *k = y + 4;
    double kl[4];
    for (int m = 0; m < 4; ++m) {
        kl[m] = 0.0;
        for (int n = 0; n < 4; ++n)
            kl[m] += g[m][n] * k[n];
    }
    double E = -kl[T_], L = kl[PH_];
    double s = sin(y[TH_]), c = cos(y[TH_]);
    double Q = kl[TH_] * kl[TH_] + c * c * (-a * a * E * E + L * L / (s * s));
    out[0] = E;
    out[1] = L;
    out[2] = Q;
    out[3] = orc_null_norm(M, a, y);
}

/* ------------------------------------------------------------------ */
/* Image-plane initial conditions (reading of the set-up the paper    */
/* takes from Psaltis & Johannsen 2012; plane at r_obs, Sec. 4).      */
/* ------------------------------------------------------------------ */

/* Flat-space construction: the observer direction is n = (sin i, 0, cos i);
 * the pixel (alpha, beta) sits at X = D n + alpha y_hat + beta (-cos i, 0,
 * sin i) with D = r_obs, and the photon moves along +n (towards the
 * observer).  Spherical components of position and direction follow from
 * that Cartesian picture; k^t is the future root of g k k = 0 in the full
 * Kerr metric; finally k is scaled so that E = -k_t = 1 (reading: the
 * affine parameter of the paper is normalised to unit energy). */
void orc_initial(double M, double a, double r_obs, double incl,
                 double alpha, double beta, double y[8])
{
    double D = r_obs, si = sin(incl), ci = cos(incl);
    double x = D * si - beta * ci;
    double yy = alpha;
    double z = D * ci + beta * si;
    double r = sqrt(D * D + alpha * alpha + beta * beta);
    double rho = sqrt(x * x + yy * yy);
    double th = atan2(rho, z);
    double ph = atan2(yy, x);
    /* direction n in spherical components (flat space) */
    double kr = D / r;
    double kth = (z * D - r * r * ci) / (rho * r * r);
    double kph = -alpha * si / (rho * rho);

    double g[4][4];
    orc_metric(M, a, r, th, g);
    double A = g[T_][T_];
    double B = 2.0 * g[T_][PH_] * kph;
    double C = g[R_][R_] * kr * kr + g[TH_][TH_] * kth * kth + g[PH_][PH_] * kph * kph;
    /* A < 0 outside the ergosphere: the future-directed root is the positive one. */
    double kt = (-B - sqrt(B * B - 4.0 * A * C)) / (2.0 * A);

    double E = -(g[T_][T_] * kt + g[T_][PH_] * kph);
    y[T_] = 0.0;
    y[R_] = r;
    y[TH_] = th;
    y[PH_] = ph;
    y[4 + T_] = kt / E;
    y[4 + R_] = kr / E;
    y[4 + TH_] = kth / E;
    y[4 + PH_] = kph / E;
}

/* ------------------------------------------------------------------ */
/* One integration step, in the order of Sec. 2.                      */
/* ------------------------------------------------------------------ */

/* Step size (negative: the photon is traced backward from the observer).
 * ORC_STEP_BENCH: |h| = max(min(h_frac r, (r - r_h)/(2|k^r|)), h_min),
 *   the benchmark rule; its second term is the horizon guard of Eq. 2.
 * ORC_STEP_EQ2:   |h| = min(h_frac / (|k^r / r| + |k^th| + |k^ph|),
 *                          (r - r_h)/(2|k^r|)),  floored at h_min (Eq. 2). */
double orc_step_size(const orc_options *o, double r_h, const double y[8])
{
    double r = y[R_], kr = y[4 + R_];
    double guard = (r - r_h) / (2.0 * fabs(kr));
    double h;
    if (o->step_rule == ORC_STEP_EQ2) {
        double first = o->h_frac / (fabs(kr / r) + fabs(y[4 + TH_]) + fabs(y[4 + PH_]));
        h = fmin(first, guard);
    } else {
        h = fmin(o->h_frac * r, guard);
    }
    h = fmax(h, o->h_min);
    return -h;
}

/* Classic RK4 on the 8-component state. */
void orc_rk4(double M, double a, const double y[8], double h, double out[8], double k1_out[8])
{
    double k1[8], k2[8], k3[8], k4[8], tmp[8];
    orc_rhs(M, a, y, k1);
    for (int i = 0; i < 8; ++i) tmp[i] = y[i] + 0.5 * h * k1[i];
    orc_rhs(M, a, tmp, k2);
    for (int i = 0; i < 8; ++i) tmp[i] = y[i] + 0.5 * h * k2[i];
    orc_rhs(M, a, tmp, k3);
    for (int i = 0; i < 8; ++i) tmp[i] = y[i] + h * k3[i];
    orc_rhs(M, a, tmp, k4);
    for (int i = 0; i < 8; ++i)
        out[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    if (k1_out)
        memcpy(k1_out, k1, sizeof k1);
}

/* Eq. 3: keep theta in [0, pi]. */
int orc_remap(double y[8])
{
    if (y[TH_] > ORC_PI) {
        y[TH_] = 2.0 * ORC_PI - y[TH_];
        y[PH_] = y[PH_] + ORC_PI;
        y[4 + TH_] = -y[4 + TH_];
        return 1;
    }
    if (y[TH_] < 0.0) {
        y[TH_] = -y[TH_];
        y[PH_] = y[PH_] - ORC_PI;
        y[4 + TH_] = -y[4 + TH_];
        return 1;
    }
    return 0;
}

/* Cubic Hermite interpolation of one coordinate over a step of length h,
 * from value/derivative (x0, v0) to (x1, v1), at fraction s in [0, 1]. */
double orc_hermite(double x0, double v0, double x1, double v1, double h, double s)
{
    double s2 = s * s, s3 = s2 * s;
    double h00 = 2.0 * s3 - 3.0 * s2 + 1.0;
    double h10 = s3 - 2.0 * s2 + s;
    double h01 = -2.0 * s3 + 3.0 * s2;
    double h11 = s3 - s2;
    return h00 * x0 + h10 * h * v0 + h01 * x1 + h11 * h * v1;
}

/* Reading: the final (t, r, theta, phi) are taken on the stop surface
 * r = r_stop itself, by cubic Hermite interpolation within the last step
 * (positions with their derivatives k).  The crossing fraction s is found by
 * 60 bisections of r(s) - r_stop on [0, 1]; the pole remap (Eq. 3) is applied
 * to the interpolated point. */
void orc_stop_surface(const double y0[8], const double y1[8], double h, double r_stop, double fin[4])
{
    double lo = 0.0, hi = 1.0;
    double f_lo = y0[R_] - r_stop;
    for (int it = 0; it < 60; ++it) {
        double mid = 0.5 * (lo + hi);
        double f_mid = orc_hermite(y0[R_], y0[4 + R_], y1[R_], y1[4 + R_], h, mid) - r_stop;
        if ((f_mid > 0.0) == (f_lo > 0.0)) {
            lo = mid;
            f_lo = f_mid;
        } else {
            hi = mid;
        }
    }
    double s = 0.5 * (lo + hi);
    double p[8];
    for (int m = 0; m < 4; ++m) {
        p[m] = orc_hermite(y0[m], y0[4 + m], y1[m], y1[4 + m], h, s);
        p[4 + m] = y1[4 + m];
    }
    orc_remap(p);
    for (int m = 0; m < 4; ++m)
        fin[m] = p[m];
}

/* Grid projection (Sec. 3): the point where the ray first crosses the
 * equatorial plane theta = pi/2 within the step (y0, y1): 60 bisections of
 * the Hermite theta(s) - pi/2 on [0, 1], then Hermite for the other
 * coordinates.  The pre-remap end state is used, so theta is continuous. */
void orc_equator_crossing(const double y0[8], const double y1[8], double h, double fin[4])
{
    double lo = 0.0, hi = 1.0;
    double f_lo = y0[TH_] - 0.5 * ORC_PI;
    for (int it = 0; it < 60; ++it) {
        double mid = 0.5 * (lo + hi);
        double f_mid = orc_hermite(y0[TH_], y0[4 + TH_], y1[TH_], y1[4 + TH_], h, mid) - 0.5 * ORC_PI;
        if ((f_mid > 0.0) == (f_lo > 0.0)) {
            lo = mid;
            f_lo = f_mid;
        } else {
            hi = mid;
        }
    }
    double s = 0.5 * (lo + hi);
    for (int m = 0; m < 4; ++m)
        fin[m] = orc_hermite(y0[m], y0[4 + m], y1[m], y1[4 + m], h, s);
    fin[TH_] = 0.5 * ORC_PI;
}

/* Per-ray result record (all doubles so that one flat array carries it):
 *  [0] status  [1] steps  [2] euler redos  [3] pole remaps
 *  [4..7] final (t, r, theta, phi) on the stop surface
 *  [8..15] state y at the end of the last step (after the remap)
 *  [16] sum of |h| over the accepted steps (affine length)              */
#define ORC_REC 17

int orc_trace(double M, double a, double r_obs, const orc_options *o, double y[8], double rec[ORC_REC])
{
    double r_h = orc_horizon(M, a);
    /* Reading: with M = 0 there is no horizon and no capture. */
    double r_cap = (M > 0.0) ? o->cap_frac * r_h : -1.0;
    double r_esc = o->r_esc_frac * r_obs;
    int status = ORC_ACTIVE, steps = 0, euler = 0, remaps = 0;
    double fin[4] = {y[T_], y[R_], y[TH_], y[PH_]};
    double lam = 0.0;

    while (status == ORC_ACTIVE) {
        if (steps >= o->max_steps) {
            status = ORC_STEP_CAP;
            memcpy(fin, y, 4 * sizeof(double));
            break;
        }
        double h = orc_step_size(o, r_h, y);
        double y1[8], k1[8];
        orc_rk4(M, a, y, h, y1, k1);
        /* Eq. 4 monitor: on failure redo the step as forward Euler at h/9. */
        double xi = orc_xi(M, a, y1);
        if (!(fabs(xi + 1.0) <= o->eps_xi)) {
            h = h / 9.0;
            for (int i = 0; i < 8; ++i)
                y1[i] = y[i] + h * k1[i];
            ++euler;
        }
        ++steps;
        lam += fabs(h);
        int finite = 1;
        for (int i = 0; i < 8; ++i)
            finite &= isfinite(y1[i]);
        if (!finite) {
            status = ORC_NONFINITE;
            memcpy(y, y1, sizeof y1);
            memcpy(fin, y1, 4 * sizeof(double));
            break;
        }
        if (o->stop_equator && (y[TH_] - 0.5 * ORC_PI) * (y1[TH_] - 0.5 * ORC_PI) < 0.0) {
            /* reading: the crossing is tested before the horizon and escape
             * stops, on the step's start state (theta in [0, pi]) and its
             * pre-remap end state */
            orc_equator_crossing(y, y1, h, fin);
            status = ORC_EQUATOR;
        } else if (y1[R_] <= r_cap) {
            orc_stop_surface(y, y1, h, r_cap, fin);
            status = ORC_CAPTURED;
        } else if (y1[R_] >= r_esc && h * y1[4 + R_] > 0.0) {
            /* Reading: escape needs r >= r_esc and the ray moving outward
             * along the backward trace (h k^r > 0); the start point itself
             * lies at r > r_obs. */
            orc_stop_surface(y, y1, h, r_esc, fin);
            status = ORC_ESCAPED;
        }
        remaps += orc_remap(y1);
        memcpy(y, y1, sizeof y1);
    }
    rec[0] = status;
    rec[1] = steps;
    rec[2] = euler;
    rec[3] = remaps;
    for (int m = 0; m < 4; ++m)
        rec[4 + m] = fin[m];
    for (int i = 0; i < 8; ++i)
        rec[8 + i] = y[i];
    rec[16] = lam;
    return status;
}

/* ------------------------------------------------------------------ */
/* Many rays, split over host threads (for timing the CPU baseline).  */
/* ------------------------------------------------------------------ */

/* rays: n x 5 doubles (alpha, beta, a, incl, r_obs). out: n x ORC_REC. */
typedef struct {
    const double *rays;
    const orc_options *o;
    double *out;
    int64_t begin, end;
} orc_job;

static void *orc_worker(void *arg)
{
    orc_job *j = (orc_job *)arg;
    for (int64_t i = j->begin; i < j->end; ++i) {
        const double *p = j->rays + 5 * i;
        double y[8];
        orc_initial(j->o->M, p[2], p[4], p[3], p[0], p[1], y);
        orc_trace(j->o->M, p[2], p[4], j->o, y, j->out + ORC_REC * i);
    }
    return NULL;
}

int orc_trace_many(int64_t n, const double *rays, const orc_options *o, double *out, int nthreads)
{
    if (n <= 0)
        return 0;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 1024)
        nthreads = 1024;
    if ((int64_t)nthreads > n)
        nthreads = (int)n;
    pthread_t th[1024];
    int created[1024];
    orc_job jobs[1024];
    int64_t chunk = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].rays = rays;
        jobs[t].o = o;
        jobs[t].out = out;
        jobs[t].begin = t * chunk < n ? t * chunk : n;
        jobs[t].end = (t + 1) * chunk < n ? (t + 1) * chunk : n;
        created[t] = 0;
        if (jobs[t].begin >= jobs[t].end)
            continue;
        if (pthread_create(&th[t], NULL, orc_worker, &jobs[t]) == 0)
            created[t] = 1;
        else
            orc_worker(&jobs[t]); /* no thread available: run it here */
    }
    for (int t = 0; t < nthreads; ++t)
        if (created[t])
            pthread_join(th[t], NULL);
    return 0;
}

/* Start states of n image-plane rays (alpha, beta, a, incl, r_obs) -> n x 8. */
void orc_initial_many(int64_t n, const double *rays, double M, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        const double *p = rays + 5 * i;
        orc_initial(M, p[2], p[4], p[3], p[0], p[1], out + 8 * i);
    }
}

/* The same over given start states instead of image-plane pixels (used by
 * the tests' conditioning checks, which trace perturbed start states):
 * states n x 8 doubles, params n x 2 doubles (a, r_obs). out: n x ORC_REC. */
typedef struct {
    const double *states, *params;
    const orc_options *o;
    double *out;
    int64_t begin, end;
} orc_state_job;

static void *orc_state_worker(void *arg)
{
    orc_state_job *j = (orc_state_job *)arg;
    for (int64_t i = j->begin; i < j->end; ++i) {
        double y[8];
        memcpy(y, j->states + 8 * i, sizeof y);
        orc_trace(j->o->M, j->params[2 * i], j->params[2 * i + 1], j->o, y, j->out + ORC_REC * i);
    }
    return NULL;
}

int orc_trace_states(int64_t n, const double *states, const double *params, const orc_options *o, double *out,
                     int nthreads)
{
    if (n <= 0)
        return 0;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 1024)
        nthreads = 1024;
    if ((int64_t)nthreads > n)
        nthreads = (int)n;
    pthread_t th[1024];
    int created[1024];
    orc_state_job jobs[1024];
    int64_t chunk = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].states = states;
        jobs[t].params = params;
        jobs[t].o = o;
        jobs[t].out = out;
        jobs[t].begin = t * chunk < n ? t * chunk : n;
        jobs[t].end = (t + 1) * chunk < n ? (t + 1) * chunk : n;
        created[t] = 0;
        if (jobs[t].begin >= jobs[t].end)
            continue;
        if (pthread_create(&th[t], NULL, orc_state_worker, &jobs[t]) == 0)
            created[t] = 1;
        else
            orc_state_worker(&jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t)
        if (created[t])
            pthread_join(th[t], NULL);
    return 0;
}
