// kerr.cuh -- device arithmetic of the Kerr photon tracer, templated on the
// floating-point type (float or double).
//
// Kerr metric in Boyer-Lindquist coordinates x = (t, r, theta, phi), units
// G = c = 1, mass M, spin a:
//   Sigma = r^2 + a^2 cos^2 th,   Delta = r^2 - 2 M r + a^2,
//   g_tt = -(1 - 2 M r/Sigma), g_tph = -2 M a r sin^2 th / Sigma,
//   g_rr = Sigma/Delta, g_thth = Sigma,
//   g_phph = (r^2 + a^2 + 2 M a^2 r sin^2 th / Sigma) sin^2 th.
// The geodesic equation d^2 x^mu/dl^2 = -Gamma^mu_ab k^a k^b (GRay, Sec. 2,
// which takes it from Psaltis & Johannsen 2012) is integrated with RK4.
//
// The Christoffel symbols are used in closed form.  With s = sin th,
// c = cos th, A = r^2 - a^2 c^2, P = r^2 + a^2, the twenty independent
// nonzero symbols are (christoffel_closed_form below):
//   G^t_tr  = M P A / (Sigma^2 Delta)       G^t_tth = -2 M a^2 r s c / Sigma^2
//   G^t_rph = -M a s^2 (a^2 c^2 (r^2 - a^2) + r^2 (a^2 + 3 r^2)) / (Sigma^2 Delta)
//   G^t_thph = 2 M a^3 r s^3 c / Sigma^2
//   G^r_tt  = M Delta A / Sigma^3           G^r_tph = -M a Delta s^2 A / Sigma^3
//   G^r_rr  = (a^2 r s^2 - M A) / (Sigma Delta)
//   G^r_rth = -a^2 s c / Sigma              G^r_thth = -r Delta / Sigma
//   G^r_phph = -Delta s^2 (r Sigma^2 - M a^2 s^2 A) / Sigma^3
//   G^th_tt = -2 M a^2 r s c / Sigma^3      G^th_tph = 2 M a r P s c / Sigma^3
//   G^th_rr = a^2 s c / (Sigma Delta)       G^th_rth = r / Sigma
//   G^th_thth = -a^2 s c / Sigma
//   G^th_phph = -s c (P Sigma^2 + 2 M a^2 r s^2 (Sigma + P)) / Sigma^3
//   G^ph_tr = M a A / (Sigma^2 Delta)       G^ph_tth = -2 M a r cot th / Sigma^2
//   G^ph_rph = (r Sigma^2 + M (a^4 s^2 c^2 - r^2 (Sigma + P))) / (Sigma^2 Delta)
//   G^ph_thph = cot th (Sigma^2 + 2 M a^2 r s^2) / Sigma^2
// The right-hand side contracts them with k k.  Grouping the terms with
// w = k^t - a s^2 k^ph (and using P - a^2 s^2 = Sigma) gives the exact,
// shorter form evaluated per RK4 stage in geodesic_accel.
//
// Delta is evaluated as (r - r_+)(r - r_-) + dc with the horizon roots r_+-
// taken once per ray in double precision (dc = max(a^2 - M^2, 0) covers M = 0):
// in single precision this keeps Delta's relative error at the rounding of r
// itself near the horizon, where r^2 - 2 M r + a^2 cancels.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace gray {

// Single-precision sin and cos of the angles the tracer meets (|x| < 2^22;
// theta stays within a few pi): x = k pi/2 + d with k rounded by the
// 1.5 * 2^23 addition (whose low bits give the quadrant) and pi/2 split in
// three floats (Cody and Waite's reduction), then the Taylor series of sin d
// and cos d to degrees 9 and 10 (truncation below 2^-28 for |d| <= pi/4).
// Within 1.5 ulp of the double values (a unit test bounds it by 4); unlike
// the library's sincosf it has no float-integer conversion, which on this
// part runs on the narrow double-precision pipe.
__device__ __forceinline__ void fsincos(float x, float *s, float *c)
{
    const float t = fmaf(x, 0.636619772367581343f, 12582912.0f);
    const float k = t - 12582912.0f;
    const int q = __float_as_int(t) & 3;
    float d = fmaf(-k, 1.57079637050628662109375f, x);
    d = fmaf(-k, -4.37113882867379317e-08f, d);
    d = fmaf(-k, -1.71512451e-15f, d);
    const float d2 = d * d;
    float ps = fmaf(d2, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = fmaf(ps, d2, 1.0f / 120.0f);
    ps = fmaf(ps, d2, -1.0f / 6.0f);
    const float sd = fmaf(ps * d2, d, d);
    float pc = fmaf(d2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = fmaf(pc, d2, -1.0f / 720.0f);
    pc = fmaf(pc, d2, 1.0f / 24.0f);
    pc = fmaf(pc, d2, -0.5f);
    const float cd = fmaf(pc, d2, 1.0f);
    const float sa = (q & 1) ? cd : sd, ca = (q & 1) ? sd : cd;
    *s = (q & 2) ? -sa : sa;
    *c = ((q + 1) & 2) ? -ca : ca;
}
__device__ __forceinline__ void fsincos(double x, double *s, double *c) { sincos(x, s, c); }
template <typename T> __device__ __forceinline__ T pi_v();
template <> __device__ __forceinline__ float pi_v<float>() { return 3.14159265358979323846f; }
template <> __device__ __forceinline__ double pi_v<double>() { return 3.14159265358979323846; }

// Per-ray constants of the spacetime and of the stop surfaces.
template <typename T> struct Hole {
    T a, M;
    T a2, Ma, m2M;     // a^2, M a, -2 M
    T t2a, t2a2, t2Ma; // 2 a, 2 a^2, 2 M a
    T rp, rm, dc; // Delta = (r - rp)(r - rm) + dc
    T rp_lo;      // single precision: rp - (float)rp, so rp is carried to ~48 bits
    T r_h;        // horizon used by the step guard; -inf when M = 0 (no guard)
    T r_cap;      // capture radius cap_frac * r_h; -1 when M = 0 (no capture)
    T r_esc;      // escape radius
    T r_promote;  // FP32_KAHAN_SEL64: steps with r below this run in double
};

// Integration options used inside a step.
template <typename T> struct StepOpt {
    T h_frac, h_min, eps_xi;
    int step_rule;    // 0: benchmark rule, 1: Eq. 2
    int stop_equator; // 1: stop at the first crossing of theta = pi/2 (Sec. 3 projection)
};

// Build the per-ray constants in double precision (one square root per ray).
__host__ __device__ inline Hole<double> make_hole(double a, double M, double r_obs, double cap_frac,
                                                  double r_esc_frac, double r_sw)
{
    Hole<double> H;
    H.a = a;
    H.M = M;
    H.a2 = a * a;
    H.Ma = M * a;
    H.m2M = -2.0 * M;
    H.t2a = 2.0 * a;
    H.t2a2 = 2.0 * H.a2;
    H.t2Ma = 2.0 * H.Ma;
    double disc = M * M - a * a;
    double root = disc > 0.0 ? sqrt(disc) : 0.0;
    H.rp = M + root;
    H.rm = M - root;
    H.dc = disc < 0.0 ? -disc : 0.0;
    H.rp_lo = 0.0;
    if (M > 0.0) {
        H.r_h = H.rp;
        H.r_cap = cap_frac * H.rp;
        H.r_promote = H.r_cap + r_sw;
    } else {
        H.r_h = -INFINITY;
        H.r_cap = -1.0;
        H.r_promote = -INFINITY;
    }
    H.r_esc = r_esc_frac * r_obs;
    return H;
}

template <typename T> __host__ __device__ inline Hole<T> cast_hole(const Hole<double> &h)
{
    Hole<T> o;
    o.a = (T)h.a;
    o.M = (T)h.M;
    o.a2 = o.a * o.a;
    o.Ma = o.M * o.a;
    o.m2M = T(-2) * o.M;
    o.t2a = T(2) * o.a;
    o.t2a2 = T(2) * o.a2;
    o.t2Ma = T(2) * o.Ma;
    o.rp = (T)h.rp;
    o.rp_lo = (T)(h.rp - (double)o.rp);
    o.rm = (T)h.rm;
    o.dc = (T)h.dc;
    o.r_h = (T)h.r_h;
    o.r_cap = (T)h.r_cap;
    o.r_esc = (T)h.r_esc;
    o.r_promote = (T)h.r_promote;
    return o;
}

// Single-precision per-ray constants, computed once in double at set-up and
// stored as two float4: (a, M, r_+ high, r_+ low) and (r_-, dc, r_h, r_obs).
__host__ __device__ inline void hole_constants_f(double a, double M, double r_obs, float *c8)
{
    const Hole<double> H = make_hole(a, M, r_obs, 1.0, 1.0, 0.0);
    const float rp_hi = (float)H.rp;
    c8[0] = (float)a;
    c8[1] = (float)M;
    c8[2] = rp_hi;
    c8[3] = (float)(H.rp - (double)rp_hi);
    c8[4] = (float)H.rm;
    c8[5] = (float)H.dc;
    c8[6] = (float)H.r_h;
    c8[7] = (float)r_obs;
}

__device__ __forceinline__ Hole<float> make_hole_f(float4 c0, float4 c1, float cap_frac, float r_esc_frac, float r_sw)
{
    Hole<float> H;
    H.a = c0.x;
    H.M = c0.y;
    H.a2 = H.a * H.a;
    H.Ma = H.M * H.a;
    H.m2M = -2.0f * H.M;
    H.t2a = 2.0f * H.a;
    H.t2a2 = 2.0f * H.a2;
    H.t2Ma = 2.0f * H.Ma;
    H.rp = c0.z;
    H.rp_lo = c0.w;
    H.rm = c1.x;
    H.dc = c1.y;
    H.r_h = c1.z;
    if (H.M > 0.0f) {
        H.r_cap = cap_frac * H.r_h;
        H.r_promote = H.r_cap + r_sw;
    } else {
        H.r_cap = -1.0f;
        H.r_promote = -INFINITY;
    }
    H.r_esc = r_esc_frac * c1.w;
    return H;
}

// Metric pieces at (r, theta) with sin/cos given.
template <typename T> struct MetricPieces {
    T s2, Sigma, Delta, gtt, gtp, grr, gthth, gpp;
};

template <typename T>
__device__ __forceinline__ MetricPieces<T> metric_pieces(const Hole<T> &H, T r, T s, T c)
{
    MetricPieces<T> m;
    T a2 = H.a * H.a;
    m.s2 = s * s;
    m.Sigma = fma(a2, c * c, r * r);
    m.Delta = fma(r - H.rp, r - H.rm, H.dc);
    T iS = T(1) / m.Sigma;
    T twoMr = T(2) * H.M * r;
    m.gtt = -(T(1) - twoMr * iS);
    m.gtp = -twoMr * H.a * m.s2 * iS;
    m.grr = m.Sigma / m.Delta;
    m.gthth = m.Sigma;
    m.gpp = (r * r + a2 + twoMr * a2 * m.s2 * iS) * m.s2;
    return m;
}

// Eq. 4: xi = [g_rr (k^r)^2 + g_phph (k^ph)^2 + g_thth (k^th)^2
//             + 2 g_tph k^t k^ph] / [g_tt (k^t)^2]; -1 on a null vector.
template <typename T> __device__ __forceinline__ T xi_eq4(const Hole<T> &H, const T *y)
{
    T s, c;
    fsincos(y[2], &s, &c);
    MetricPieces<T> m = metric_pieces(H, y[1], s, c);
    T kt = y[4], kr = y[5], kh = y[6], kp = y[7];
    T num = m.grr * kr * kr + m.gpp * kp * kp + m.gthth * kh * kh + T(2) * m.gtp * kt * kp;
    return num / (m.gtt * kt * kt);
}

// The twenty closed-form symbols, written into G[mu][a][b] (symmetric in a,b).
template <typename T>
__device__ inline void christoffel_closed_form(const Hole<T> &H, T r, T th, T *G)
{
    T s, c;
    fsincos(th, &s, &c);
    const T a = H.a, M = H.M;
    const T a2 = a * a, r2 = r * r, s2 = s * s, c2 = c * c, sc = s * c;
    const T Sigma = fma(a2, c2, r2);
    const T Delta = fma(r - H.rp, r - H.rm, H.dc);
    const T iS = T(1) / Sigma, iD = T(1) / Delta;
    const T iS2 = iS * iS, iS3 = iS2 * iS;
    const T A = fma(-a2, c2, r2), P = r2 + a2;
    const T cot = c / s;
    for (int i = 0; i < 64; ++i) G[i] = T(0);
#define GSET(m, i, j, v)                                                                                         \
    do {                                                                                                         \
        T v_ = (v);                                                                                              \
        G[(m) * 16 + (i) * 4 + (j)] = v_;                                                                        \
        G[(m) * 16 + (j) * 4 + (i)] = v_;                                                                        \
    } while (0)
    GSET(0, 0, 1, M * P * A * iS2 * iD);
    GSET(0, 0, 2, -T(2) * M * a2 * r * sc * iS2);
    GSET(0, 1, 3, -M * a * s2 * (a2 * c2 * (r2 - a2) + r2 * (a2 + T(3) * r2)) * iS2 * iD);
    GSET(0, 2, 3, T(2) * M * a2 * a * r * s2 * sc * iS2);
    GSET(1, 0, 0, M * Delta * A * iS3);
    GSET(1, 0, 3, -M * a * Delta * s2 * A * iS3);
    GSET(1, 1, 1, (a2 * r * s2 - M * A) * iS * iD);
    GSET(1, 1, 2, -a2 * sc * iS);
    GSET(1, 2, 2, -r * Delta * iS);
    GSET(1, 3, 3, -Delta * s2 * (r * Sigma * Sigma - M * a2 * s2 * A) * iS3);
    GSET(2, 0, 0, -T(2) * M * a2 * r * sc * iS3);
    GSET(2, 0, 3, T(2) * M * a * r * P * sc * iS3);
    GSET(2, 1, 1, a2 * sc * iS * iD);
    GSET(2, 1, 2, r * iS);
    GSET(2, 2, 2, -a2 * sc * iS);
    GSET(2, 3, 3, -sc * (P * Sigma * Sigma + T(2) * M * a2 * r * s2 * (Sigma + P)) * iS3);
    GSET(3, 0, 1, M * a * A * iS2 * iD);
    GSET(3, 0, 2, -T(2) * M * a * r * cot * iS2);
    GSET(3, 1, 3, (r * Sigma * Sigma + M * (a2 * a2 * s2 * c2 - r2 * (Sigma + P))) * iS2 * iD);
    GSET(3, 2, 3, cot * (Sigma * Sigma + T(2) * M * a2 * r * s2) * iS2);
#undef GSET
}

// Reciprocal: the hardware approximation refined by Newton-Raphson steps
// r <- r + r (1 - x r): one in single precision, two in double (each step
// squares the relative error; about 1 ulp at the end).  On GB300 a double
// divide is a long sequence on the narrow FP64 pipe.
__device__ __forceinline__ float recip(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    const float e = fmaf(-x, r, 1.0f);
    return fmaf(r, e, r);
}
__device__ __forceinline__ double recip(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// The hardware reciprocal alone (bounded by 2 ulp in a unit test): single
// precision takes it for the geometry of a point, whose other operations
// round as much; double keeps the refined one.
__device__ __forceinline__ float recip_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double recip_approx(double x) { return recip(x); }

// Geometry of one point (r, theta): the quantities every right-hand side and
// the Eq. 4 monitor need, with the reciprocals of Sigma, Delta and sin(theta).
template <typename T> struct Geo {
    T r, s, c, Sigma, Delta, iS, iD, is;
};

// 1/Sigma, 1/Delta and 1/sin.  Single precision: three hardware
// reciprocals, one issue slot each (they run on the SFU pipe, beside the
// FMA pipe), each within 2 ulp (unit test); forming the three from one
// reciprocal of Sigma Delta sin takes eight issue slots and rounds up to
// five times (single-precision pass 8.33 -> 8.00 ms on the 1024^2 image).
// Double and double-single keep the one reciprocal (there each reciprocal
// is a refined sequence).
template <typename T> __device__ __forceinline__ void geometry_reciprocals(Geo<T> &g)
{
    if constexpr (sizeof(T) == 4) {
        g.iS = recip_approx(g.Sigma);
        g.iD = recip_approx(g.Delta);
        g.is = recip_approx(g.s);
    } else {
        const T Ds = g.Delta * g.s, SD = g.Sigma * g.Delta;
        const T inv = recip_approx(SD * g.s);
        g.iS = inv * Ds;
        g.iD = inv * (g.Sigma * g.s);
        g.is = inv * SD;
    }
}

// dr and dth are the low words of a compensated single-precision point (the
// true point is (r + dr, th + dth)): sin and cos get their first-order
// correction and Delta is formed from the compensated r and the split r_+, so
// near theta = pi and near the horizon single precision keeps the bits that
// the high words alone lose.
template <typename T>
__device__ __forceinline__ Geo<T> geometry(const Hole<T> &H, T r, T th, T dr = T(0), T dth = T(0))
{
    Geo<T> g;
    g.r = r;
    T s0, c0;
    fsincos(th, &s0, &c0);
    if (sizeof(T) == 4) {
        g.s = fma(dth, c0, s0);
        g.c = fma(-dth, s0, c0);
        g.Delta = fma((r - H.rp) + (dr - H.rp_lo), (r - H.rm) + dr, H.dc);
    } else {
        g.s = s0;
        g.c = c0;
        g.Delta = fma(r - H.rp, r - H.rm, H.dc);
    }
    g.Sigma = fma(H.a * H.a, g.c * g.c, r * r);
    geometry_reciprocals(g);
    return g;
}

// sin and cos of a small angle d by their Taylor series: single precision
// for |d| <= 0.125 (degrees 5 and 6, truncation below 1e-10), double for
// |d| <= 0.25 (degrees 11 and 12, below 3e-18; degrees 7 and 8 for
// |d| <= 1/64).  Returns false for larger |d|.
__device__ __forceinline__ bool small_sincos(float d, float *s, float *c)
{
    if (!(fabsf(d) <= 0.125f))
        return false;
    const float d2 = d * d;
    const float ps = fmaf(d2, 8.33333333e-03f, -1.66666667e-01f);
    *s = fmaf(ps * d2, d, d);
    float pc = fmaf(d2, -1.38888889e-03f, 4.16666667e-02f);
    pc = fmaf(pc, d2, -0.5f);
    *c = fmaf(pc, d2, 1.0f);
    return true;
}
__device__ __forceinline__ bool small_sincos(double d, double *s, double *c)
{
    if (!(fabs(d) <= 0.25))
        return false;
    const double d2 = d * d;
    if (fabs(d) <= 0.015625) {
        // degrees 7 and 8 (truncation below 1e-22 for |d| <= 1/64), the
        // usual case of the short steps near the horizon
        double ps = fma(d2, -1.984126984126984e-04, 8.333333333333333e-03);
        ps = fma(ps, d2, -1.6666666666666666e-01);
        *s = fma(ps * d2, d, d);
        double pc = fma(d2, 2.48015873015873e-05, -1.388888888888889e-03);
        pc = fma(pc, d2, 4.1666666666666664e-02);
        pc = fma(pc, d2, -0.5);
        *c = fma(pc, d2, 1.0);
        return true;
    }
    double ps = fma(d2, -2.505210838544172e-08, 2.7557319223985893e-06);
    ps = fma(ps, d2, -1.984126984126984e-04);
    ps = fma(ps, d2, 8.333333333333333e-03);
    ps = fma(ps, d2, -1.6666666666666666e-01);
    *s = fma(ps * d2, d, d);
    double pc = fma(d2, 2.08767569878681e-09, -2.755731922398589e-07);
    pc = fma(pc, d2, 2.48015873015873e-05);
    pc = fma(pc, d2, -1.388888888888889e-03);
    pc = fma(pc, d2, 4.1666666666666664e-02);
    pc = fma(pc, d2, -0.5);
    *c = fma(pc, d2, 1.0);
    return true;
}

// Geometry of an RK4 stage point whose polar angle is the step's start angle
// plus d: sin and cos come from the start point's by the angle-addition
// formulas (the start point's values already carry the compensation), which
// costs two short series instead of a full sin/cos; far stages (|d| > 0.25)
// take the full evaluation at th with its low word dth.
template <typename T>
__device__ __forceinline__ Geo<T> geometry_rel(const Hole<T> &H, const Geo<T> &g0, T r, T d, T th, T dr, T dth)
{
    T sd, cd;
    if (!small_sincos(d, &sd, &cd))
        return geometry(H, r, th, dr, dth);
    Geo<T> g;
    g.r = r;
    g.s = fma(g0.s, cd, g0.c * sd);
    g.c = fma(g0.c, cd, -(g0.s * sd));
    if (sizeof(T) == 4)
        g.Delta = fma((r - H.rp) + (dr - H.rp_lo), (r - H.rm) + dr, H.dc);
    else
        g.Delta = fma(r - H.rp, r - H.rm, H.dc);
    g.Sigma = fma(H.a * H.a, g.c * g.c, r * r);
    geometry_reciprocals(g);
    return g;
}

// dk^mu/dl at a point whose geometry is known: the closed-form symbols
// contracted with k k, grouped with X = (k^t - a s^2 k^ph)/Sigma,
// V = -2 a s^2 k^ph (so X = (k^t + V/2)/Sigma), u = k^r/Delta, q = k^r u,
// Z = 2 M a r X, A = r^2 - a^2 c^2 = 2 r^2 - Sigma, P = r^2 + a^2:
//   a^t  = -2M/Sigma [ u (P A X + r^2 V) - 2 a^2 r s c k^th X ]
//   a^r  = [ M A (q - Delta X^2) + Delta r (s^2 k^ph^2 + k^th^2)
//            - a^2 r s^2 q + 2 a^2 s c k^r k^th ] / Sigma
//   a^th = [ s c (Z (a X - 2 k^ph) + P k^ph^2 + a^2 (k^th^2 - q))
//            - 2 r k^r k^th ] / Sigma
//   a^ph = -2 [ u ((M a A X - 2 M r^2 k^ph)/Sigma + r k^ph)
//               + cot(th) k^th (k^ph - Z/Sigma) ]
template <typename T>
__device__ __forceinline__ void accel_geo(const Hole<T> &H, const Geo<T> &g, T kt, T kr, T kh, T kp, T *acc)
{
    const T r = g.r, iS = g.iS;
    const T r2 = r * r, s2 = g.s * g.s, sc = g.s * g.c;
    const T A = fma(T(2), r2, -g.Sigma);
    const T P = r2 + H.a2;
    const T V = -(H.t2a * s2) * kp;
    const T X = fma(V, T(0.5), kt) * iS;
    const T u = kr * g.iD;
    const T q = kr * u;
    const T krkh = kr * kh, kh2 = kh * kh, kp2 = kp * kp;
    // t
    const T ut = fma(P * A, X, r2 * V);
    const T xt = -(H.t2a2 * (r * sc)) * (kh * X);
    acc[0] = (H.m2M * iS) * fma(u, ut, xt);
    // r
    const T DX = g.Delta * X;
    T sr = fma(H.M * A, fma(-DX, X, q), (g.Delta * r) * fma(s2, kp2, kh2));
    sr = fma(-((H.a2 * r) * s2), q, sr);
    sr = fma(H.t2a2 * sc, krkh, sr);
    acc[1] = iS * sr;
    // theta
    const T Z = (H.t2Ma * r) * X;
    const T hth = fma(Z, fma(H.a, X, T(-2) * kp), fma(P, kp2, H.a2 * (kh2 - q)));
    acc[2] = iS * fma(r * krkh, T(-2), sc * hth);
    // phi
    const T inner = fma(iS, fma(H.m2M * r2, kp, (H.Ma * A) * X), r * kp);
    const T up2 = fma(-Z, iS, kp);
    acc[3] = T(-2) * fma(u, inner, ((g.c * g.is) * kh) * up2);
}

// Eq. 4 test without its division: |xi + 1| > eps  <=>
// |g(k, k)| > eps |g_tt (k^t)^2| (NaN fails, as in the oracle).  The norm
// g(k, k) = num + g_tt (k^t)^2 is taken in the metric's Carter-frame form
//   g(k, k) = [s^2 v^2 - Delta w^2] / Sigma + Sigma ((k^r)^2/Delta + (k^th)^2),
//   w = k^t - a s^2 k^ph,  v = (r^2 + a^2) k^ph - a k^t,
// which is the same quadratic form in fewer operations.
template <typename T> __device__ __forceinline__ bool xi_fails(const Hole<T> &H, const Geo<T> &g, const T *y, T eps)
{
    const T r = g.r, s2 = g.s * g.s;
    const T kt = y[4], kr = y[5], kh = y[6], kp = y[7];
    const T w = fma(-(H.a * s2), kp, kt);
    const T v = fma(fma(r, r, H.a2), kp, -(H.a * kt));
    const T E = fma(s2 * v, v, -((g.Delta * w) * w));
    const T norm = fma(g.Sigma, fma(kr * g.iD, kr, kh * kh), E * g.iS);
    const T den = fma(H.m2M * r, g.iS, T(1)) * (kt * kt);
    return !(fabs(norm) <= eps * fabs(den));
}

// The null norm g(k, k) of the single-precision Eq. 4 test, in the metric's
// Carter-frame form, with the size of the terms that make it up (the sum of
// their magnitudes) and g_tt (k^t)^2.
struct NormF {
    float norm, size, den;
};
__device__ __forceinline__ NormF null_norm_f(const Hole<float> &H, const Geo<float> &g, const float *y)
{
    const float r = g.r, s2 = g.s * g.s;
    const float kt = y[4], kr = y[5], kh = y[6], kp = y[7];
    const float w = fmaf(-(H.a * s2), kp, kt);
    const float v = fmaf(fmaf(r, r, H.a2), kp, -(H.a * kt));
    const float sv2 = (s2 * v) * v, dw2 = (g.Delta * w) * w;
    const float q = fmaf(kr * g.iD, kr, kh * kh);
    NormF o;
    o.norm = fmaf(g.Sigma, q, (sv2 - dw2) * g.iS);
    o.size = fmaf(g.Sigma, fabsf(q), (sv2 + fabsf(dw2)) * g.iS);
    o.den = fmaf(H.m2M * r, g.iS, 1.0f) * (kt * kt);
    return o;
}

// The single-precision Eq. 4 test, with a flag set when its outcome lies
// within the rounding of its own evaluation: |g(k, k)| and the threshold
// eps |g_tt (k^t)^2| closer than 2^-20 of the size of the terms that make up
// g(k, k).  Single precision evaluates g(k, k) to a few units of 2^-24 of
// that size (the geometry's reciprocal and sin/cos to 2-4 ulp, the high words
// of k to 2^-24 relative); such a test is taken again in double-single
// arithmetic (xi_fails_ds).
__device__ __forceinline__ bool xi_fails_flag(const Hole<float> &H, const Geo<float> &g, const float *y, float eps,
                                              bool &ambiguous)
{
    const NormF n = null_norm_f(H, g, y);
    const float thr = eps * fabsf(n.den);
    ambiguous = fabsf(fabsf(n.norm) - thr) <= 9.5367431640625e-7f * n.size;
    return !(fabsf(n.norm) <= thr);
}

// ---- double-single arithmetic -------------------------------------------
// A value carried as an unevaluated sum hi + lo of two floats (about 48
// significant bits), with the error-free transformations of Knuth (TwoSum)
// and Dekker (TwoProduct by fused multiply-add).  The tracer uses it only on
// the rare path that re-takes an ambiguous Eq. 4 test, so that the test is
// decided to ~2^-40 of its terms without leaving the single-precision pipe
// (GB300's FP64 rate is 1/64 of FP32's).
struct ds {
    float hi, lo;
    ds() = default;
    __host__ __device__ constexpr ds(float h, float l) : hi(h), lo(l) {}
    // from a double constant (folded at compile time for literals)
    __host__ __device__ constexpr explicit ds(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};
__device__ __forceinline__ ds ds_two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return ds{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ds ds_fast(float a, float b) // |a| >= |b| or a == 0
{
    const float s = a + b;
    return ds{s, b - (s - a)};
}
__device__ __forceinline__ ds ds_add(ds x, ds y)
{
    const ds s = ds_two_sum(x.hi, y.hi);
    return ds_fast(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ds ds_neg(ds x) { return ds{-x.hi, -x.lo}; }
__device__ __forceinline__ ds ds_mul(ds x, ds y)
{
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return ds_fast(p, e);
}
__device__ __forceinline__ ds ds_mulf(ds x, float y)
{
    const float p = x.hi * y;
    float e = fmaf(x.hi, y, -p);
    e = fmaf(x.lo, y, e);
    return ds_fast(p, e);
}
// 1/x: the single-precision reciprocal refined by one Newton-Raphson step
// r + r (1 - x r) whose residual 1 - x r is formed exactly.
__device__ __forceinline__ ds ds_recip(ds x)
{
    const float r = recip(x.hi);
    const ds xr = ds_mulf(x, r);
    const float e = (1.0f - xr.hi) - xr.lo;
    return ds_fast(r, r * e);
}

// ---- double-single as a number type ---------------------------------------
// (the library's float and double overloads stay visible next to these)
using ::fabs;
using ::fma;
using ::fmax;
using ::fmin;
// The arithmetic the templated tracer functions need (step size, right-hand
// side, RK4, Eq. 4, Eq. 3, stop tests), so that the steps near the horizon
// can run in double-single on the single-precision pipe instead of in double
// (GB300's FP64 pipe runs at 1/64 of the FP32 rate).  Values are kept
// normalised (|lo| <= ulp(hi)/2); comparisons order by hi, then lo.
__device__ __forceinline__ ds operator+(ds a, ds b) { return ds_add(a, b); }
__device__ __forceinline__ ds operator-(ds a) { return ds_neg(a); }
__device__ __forceinline__ ds operator-(ds a, ds b) { return ds_add(a, ds_neg(b)); }
__device__ __forceinline__ ds operator*(ds a, ds b) { return ds_mul(a, b); }
__device__ __forceinline__ ds operator/(ds a, ds b) { return ds_mul(a, ds_recip(b)); }
__device__ __forceinline__ bool operator<(ds a, ds b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(ds a, ds b) { return b < a; }
__device__ __forceinline__ bool operator<=(ds a, ds b) { return !(b < a) && a.hi == a.hi && b.hi == b.hi; }
__device__ __forceinline__ bool operator>=(ds a, ds b) { return b <= a; }
__device__ __forceinline__ ds fma(ds a, ds b, ds c) { return ds_add(ds_mul(a, b), c); }
__device__ __forceinline__ ds fabs(ds a) { return a.hi < 0.0f ? ds_neg(a) : a; }
__device__ __forceinline__ ds fmin(ds a, ds b) { return b < a ? b : a; }
__device__ __forceinline__ ds fmax(ds a, ds b) { return a < b ? b : a; }
__device__ __forceinline__ ds recip(ds a) { return ds_recip(a); }
__device__ __forceinline__ ds recip_approx(ds a) { return ds_recip(a); }
template <> __device__ __forceinline__ ds pi_v<ds>() { return ds(3.14159265358979323846); }
__device__ __forceinline__ bool finite_v(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_v(double x) { return isfinite(x); }
__device__ __forceinline__ bool finite_v(ds x) { return isfinite(x.hi) && isfinite(x.lo); }

// sin and cos of a float angle x (|x| < 8) in double-single, from a table
// of sin and cos at the multiples x0 = j/32 (each as the two floats nearest to
// the double value and to its remainder, filled from the host once per
// device) and angle addition: d = x - x0 is exact, |d| <= 1/64, and
// sin d = d - d^3/6 + d^5/120, cos d = 1 - d^2/2 + d^4/24 (truncation below
// 2e-15) need double-single only for d and d^2.  j comes from the 1.5 * 2^23
// rounding addition: no float-integer conversion.
constexpr int SINCOS_TABLE_HALF = 256; // entries j/32 for j in [-256, 256)
__constant__ float4 c_sincos_table[2 * SINCOS_TABLE_HALF];
__device__ __forceinline__ void ds_sincos(float x, ds &s, ds &c)
{
    const float t = fmaf(x, 32.0f, 12582912.0f);
    const float jf = t - 12582912.0f;
    int j = __float_as_int(t) - 0x4B400000; // jf as an integer
    j = j < -SINCOS_TABLE_HALF ? -SINCOS_TABLE_HALF : (j > SINCOS_TABLE_HALF - 1 ? SINCOS_TABLE_HALF - 1 : j);
    const float4 e = c_sincos_table[j + SINCOS_TABLE_HALF];
    const ds S0{e.x, e.y}, C0{e.z, e.w};
    const float d = fmaf(-jf, 0.03125f, x); // exact
    const float p = d * d, pe = fmaf(d, d, -p); // d^2 = p + pe exactly
    const ds sd = ds_fast(d, d * p * fmaf(p, 1.0f / 120.0f, -1.0f / 6.0f));
    const ds cd = ds_add(ds{1.0f, 0.0f}, ds{-0.5f * p, fmaf(p * p, 1.0f / 24.0f, -0.5f * pe)});
    s = ds_add(ds_mul(S0, cd), ds_mul(C0, sd));
    c = ds_add(ds_mul(C0, cd), ds_neg(ds_mul(S0, sd)));
}

// sin and cos of a double-single angle (|x| < 8): ds_sincos of the high
// word, then the first-order term of the low one (|lo| <= 2^-24 |x|).
__device__ __forceinline__ void fsincos(ds x, ds *s, ds *c)
{
    ds s0, c0;
    ds_sincos(x.hi, s0, c0);
    *s = ds_add(s0, ds{c0.hi * x.lo, 0.0f});
    *c = ds_add(c0, ds{-s0.hi * x.lo, 0.0f});
}

// sin and cos of a small double-single angle d (|d| <= 1/64, the stage
// increments near the horizon) by their series: d and -d^2/2 in
// double-single, the smaller terms in single precision (truncation below
// 1e-17).  Returns false for larger |d|.
__device__ __forceinline__ bool small_sincos(ds d, ds *s, ds *c)
{
    if (!(fabsf(d.hi) <= 0.015625f))
        return false;
    const float p = d.hi * d.hi;
    *s = ds_add(d, ds{d.hi * p * fmaf(p, fmaf(p, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 0.0f});
    const ds d2 = ds_mul(d, d);
    *c = ds_add(ds{1.0f, 0.0f}, ds{-0.5f * d2.hi, fmaf(p * p, fmaf(p, -1.0f / 720.0f, 1.0f / 24.0f), -0.5f * d2.lo)});
    return true;
}

// The null norm g(k, k) in double-single arithmetic of a compensated
// single-precision state (the true state is hi - lo: y1 the high words, c1
// the low ones) with the spin and mass split into two floats each, aM =
// (a_hi, a_lo, M_hi, M_lo): accurate to ~2^-40 of its terms, where single
// precision resolves ~2^-21.  Also returns 1/Sigma (high word).
__device__ __forceinline__ ds null_norm_ds(const float *y1, const float *c1, float4 aM, float &iS_hi)
{
    const ds r = ds_fast(y1[1], -c1[1]);
    const ds kt = ds_fast(y1[4], -c1[4]), kr = ds_fast(y1[5], -c1[5]);
    const ds kh = ds_fast(y1[6], -c1[6]), kp = ds_fast(y1[7], -c1[7]);
    const ds a = ds_fast(aM.x, aM.y), M = ds_fast(aM.z, aM.w);
    ds s, c;
    ds_sincos(y1[2], s, c);
    // sin and cos of theta_hi - theta_lo to first order in the low word
    const float tl = c1[2];
    const ds sn = ds_add(s, ds{-c.hi * tl, 0.0f});
    const ds cs = ds_add(c, ds{s.hi * tl, 0.0f});
    const ds r2 = ds_mul(r, r), a2 = ds_mul(a, a), s2 = ds_mul(sn, sn);
    const ds Sigma = ds_add(r2, ds_mul(a2, ds_mul(cs, cs)));
    const ds Delta = ds_add(ds_add(r2, ds_neg(ds_mulf(ds_mul(M, r), 2.0f))), a2);
    const ds w = ds_add(kt, ds_neg(ds_mul(ds_mul(a, s2), kp)));
    const ds v = ds_add(ds_mul(ds_add(r2, a2), kp), ds_neg(ds_mul(a, kt)));
    const ds E = ds_add(ds_mul(s2, ds_mul(v, v)), ds_neg(ds_mul(Delta, ds_mul(w, w))));
    const ds iS = ds_recip(Sigma), iD = ds_recip(Delta);
    const ds q = ds_add(ds_mul(ds_mul(kr, kr), iD), ds_mul(kh, kh));
    iS_hi = iS.hi;
    return ds_add(ds_mul(Sigma, q), ds_mul(E, iS));
}

// The Eq. 4 test re-taken in double-single arithmetic: |g(k, k)| of
// null_norm_ds against eps |g_tt (k^t)^2|.  The threshold needs no such care:
// single precision forms it to ~2^-23 of itself.
__device__ __forceinline__ bool xi_fails_ds(const float *y1, const float *c1, float4 aM, float eps)
{
    float iS;
    const ds norm = null_norm_ds(y1, c1, aM, iS);
    const float r = y1[1] - c1[1], kt = y1[4] - c1[4];
    const float gtt = fmaf(-2.0f * aM.z * r, iS, 1.0f);
    return !(fabsf(norm.hi + norm.lo) <= eps * fabsf(gtt * (kt * kt)));
}

// dk^mu/dl = -Gamma^mu_ab k^a k^b, from the closed-form symbols grouped with
// w = k^t - a s^2 k^ph.  Inputs: r, theta and k = (kt, kr, kh, kp).
template <typename T>
__device__ __forceinline__ void geodesic_accel(const Hole<T> &H, T r, T th, T kt, T kr, T kh, T kp, T *acc)
{
    const Geo<T> g = geometry(H, r, th);
    accel_geo(H, g, kt, kr, kh, kp, acc);
}

// Step size (negative: backward trace).  Benchmark rule
// |h| = max(min(h_frac r, (r - r_h)/(2|k^r|)), h_min), or Eq. 2
// |h| = max(min(h_frac / (|k^r/r| + |k^th| + |k^ph|), (r - r_h)/(2|k^r|)), h_min).
template <typename T> __device__ __forceinline__ T step_size(const Hole<T> &H, const StepOpt<T> &O, const T *y)
{
    const T r = y[1], kr = y[5];
    const T guard = (r - H.r_h) * (T(0.5) * recip(fabs(kr)));
    T h;
    if (O.step_rule == 1)
        h = fmin(O.h_frac * recip(fabs(kr) * recip(r) + fabs(y[6]) + fabs(y[7])), guard);
    else
        h = fmin(O.h_frac * r, guard);
    h = fmax(h, O.h_min);
    return -h;
}

// Cubic Hermite interpolation within one step of length h.
template <typename T> __device__ __forceinline__ T hermite(T x0, T v0, T x1, T v1, T h, T s)
{
    const T s2 = s * s, s3 = s2 * s;
    const T h00 = T(2) * s3 - T(3) * s2 + T(1);
    const T h10 = s3 - T(2) * s2 + s;
    const T h01 = -T(2) * s3 + T(3) * s2;
    const T h11 = s3 - s2;
    return h00 * x0 + h10 * h * v0 + h01 * x1 + h11 * h * v1;
}

// Fraction s of the last step at which coordinate m (1: r, 2: theta) of the
// Hermite interpolant reaches `target`, starting from the secant estimate and
// kept inside the bracket (a step that leaves it is replaced by a bisection
// step).  Double: the chord iteration s <- s - f(s) / f'(s0) with the slope
// at the secant point (one reciprocal; GB300's double divide is costly),
// 10 iterations -- it converges linearly with the ratio |1 - f'/f'(s0)|,
// small over one step, onto the root the oracle's bisection finds (8 and 16
// iterations pass the same parity tests; each costs the zone pass ~1.5 %).
// Single:
// Newton's method, 6 iterations.
template <typename T>
__device__ __forceinline__ T crossing_fraction(const T *y0, const T *y1, T h, T target, int m = 1)
{
    T lo = T(0), hi = T(1);
    T f_lo = y0[m] - target;
    if (sizeof(T) == 8) {
        const T f_h = y1[m] - target;
        T s = f_lo / (f_lo - f_h);
        if (!(s > T(0) && s < T(1)))
            s = T(0.5);
        const T p0 = y0[m], m0 = h * y0[4 + m], p1 = y1[m], m1 = h * y1[4 + m];
        const T s2 = s * s;
        const T df = (T(6) * s2 - T(6) * s) * p0 + (T(3) * s2 - T(4) * s + T(1)) * m0 + (T(6) * s - T(6) * s2) * p1 +
                     (T(3) * s2 - T(2) * s) * m1;
        const T idf = recip(df);
        for (int it = 0; it < 10; ++it) {
            const T f = hermite(p0, y0[4 + m], p1, y1[4 + m], h, s) - target;
            if ((f > T(0)) == (f_lo > T(0)))
                lo = s;
            else
                hi = s;
            T sn = s - f * idf;
            if (!(sn >= lo && sn <= hi))
                sn = T(0.5) * (lo + hi);
            s = sn;
        }
        return s;
    }
    const T f_hi = y1[m] - target;
    T s = f_lo / (f_lo - f_hi);
    if (!(s > T(0) && s < T(1)))
        s = T(0.5);
    const T p0 = y0[m], m0 = h * y0[4 + m], p1 = y1[m], m1 = h * y1[4 + m];
    for (int it = 0; it < 6; ++it) {
        const T s2 = s * s;
        const T f = hermite(p0, y0[4 + m], p1, y1[4 + m], h, s) - target;
        const T df = (T(6) * s2 - T(6) * s) * p0 + (T(3) * s2 - T(4) * s + T(1)) * m0 + (T(6) * s - T(6) * s2) * p1 +
                     (T(3) * s2 - T(2) * s) * m1;
        if ((f > T(0)) == (f_lo > T(0)))
            lo = s;
        else
            hi = s;
        T sn = s - f / df;
        if (!(sn >= lo && sn <= hi)) // inclusive: f = 0 keeps s (the root)
            sn = T(0.5) * (lo + hi);
        s = sn;
    }
    return s;
}

// Grid projection (Sec. 3): the point where the step first crosses the
// equatorial plane theta = pi/2 (start state and pre-remap end state).
template <typename T> __device__ __noinline__ void equator_crossing(const T *y0, const T *y1, T h, T *fin)
{
    const T half_pi = T(0.5) * pi_v<T>();
    const T s = crossing_fraction(y0, y1, h, half_pi, 2);
    for (int m = 0; m < 4; ++m)
        fin[m] = hermite(y0[m], y0[4 + m], y1[m], y1[4 + m], h, s);
    fin[2] = half_pi;
}

// Final (t, r, theta, phi) on the stop surface r = r_stop: the crossing
// fraction, Hermite for the other coordinates, then the pole remap of Eq. 3
// applied to the interpolated point.
template <typename T>
__device__ __noinline__ void stop_surface(const T *y0, const T *y1, T h, T r_stop, T *fin)
{
    const T s = crossing_fraction(y0, y1, h, r_stop);
    for (int m = 0; m < 4; ++m)
        fin[m] = hermite(y0[m], y0[4 + m], y1[m], y1[4 + m], h, s);
    if (fin[2] > pi_v<T>()) {
        fin[2] = T(2) * pi_v<T>() - fin[2];
        fin[3] = fin[3] + pi_v<T>();
    } else if (fin[2] < T(0)) {
        fin[2] = -fin[2];
        fin[3] = fin[3] - pi_v<T>();
    }
}

// The stop surface of a double step taken in the single-precision zone
// tracer: the step's offsets y1 - y0 and the surface's offset r_stop - r0
// are formed in double, the crossing fraction and the Hermite increments in
// single precision, and the increments are added back in double.  The
// increments are small (one step), so the crossing point keeps a relative
// accuracy of ~1e-7 of one step's displacement while the double pipe does
// ~30 operations instead of the double chord iteration's ~300.
__device__ __noinline__ void stop_surface_mixed(const double *y0, const double *y1, double h, double r_stop,
                                                double *fin)
{
    float z0[8], z1[8];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        z0[m] = 0.0f;
        z1[m] = (float)(y1[m] - y0[m]);
        z0[4 + m] = (float)y0[4 + m];
        z1[4 + m] = (float)y1[4 + m];
    }
    const float hf = (float)h;
    const float s = crossing_fraction<float>(z0, z1, hf, (float)(r_stop - y0[1]));
#pragma unroll
    for (int m = 0; m < 4; ++m)
        fin[m] = y0[m] + (double)hermite<float>(0.0f, z0[4 + m], z1[m], z1[4 + m], hf, s);
    if (fin[2] > pi_v<double>()) {
        fin[2] = 2.0 * pi_v<double>() - fin[2];
        fin[3] = fin[3] + pi_v<double>();
    } else if (fin[2] < 0.0) {
        fin[2] = -fin[2];
        fin[3] = fin[3] - pi_v<double>();
    }
}

// The same for double-single steps (the zone tracer's default arithmetic):
// offsets in double-single, crossing and Hermite increments in single
// precision, added back in double-single.
__device__ __noinline__ void stop_surface_mixed(const ds *y0, const ds *y1, ds h, ds r_stop, ds *fin)
{
    float z0[8], z1[8];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        z0[m] = 0.0f;
        z1[m] = (y1[m] - y0[m]).hi;
        z0[4 + m] = y0[4 + m].hi;
        z1[4 + m] = y1[4 + m].hi;
    }
    const float hf = h.hi;
    const float sf = crossing_fraction<float>(z0, z1, hf, (r_stop - y0[1]).hi);
#pragma unroll
    for (int m = 0; m < 4; ++m)
        fin[m] = y0[m] + ds{hermite<float>(0.0f, z0[4 + m], z1[m], z1[4 + m], hf, sf), 0.0f};
    if (fin[2] > pi_v<ds>()) {
        fin[2] = ds(2.0) * pi_v<ds>() - fin[2];
        fin[3] = fin[3] + pi_v<ds>();
    } else if (fin[2] < ds(0.0)) {
        fin[2] = -fin[2];
        fin[3] = fin[3] - pi_v<ds>();
    }
}

// Per-ray constants in double-single from the single-precision planes
// (PF0: a, M, r_+ high, r_+ low; PF1: r_-, dc, r_h, r_obs) and the low
// words of a and M (the fourth slot of P): r_- = 2M - r_+ and dc = 0 below
// extremal spin, the surfaces from the double options.
__device__ __forceinline__ Hole<ds> make_hole_ds(float4 c0, float4 c1, float2 lows, ds cap_frac, ds r_esc_frac,
                                                 ds r_sw)
{
    Hole<ds> H;
    H.a = ds_fast(c0.x, lows.x);
    H.M = ds_fast(c0.y, lows.y);
    H.a2 = H.a * H.a;
    H.Ma = H.M * H.a;
    H.m2M = ds(-2.0) * H.M;
    H.t2a = ds(2.0) * H.a;
    H.t2a2 = ds(2.0) * H.a2;
    H.t2Ma = ds(2.0) * H.Ma;
    H.rp = ds_fast(c0.z, c0.w);
    H.rp_lo = ds(0.0);
    if (c1.y > 0.0f) { // |a| > M: no horizon roots (Delta = (r - M)^2 + a^2 - M^2)
        H.rp = H.M;
        H.rm = H.M;
        H.dc = H.a2 - H.M * H.M;
    } else {
        H.rm = ds(2.0) * H.M - H.rp;
        H.dc = ds(0.0);
    }
    if (c0.y > 0.0f) {
        H.r_h = H.rp;
        H.r_cap = cap_frac * H.rp;
        H.r_promote = H.r_cap + r_sw;
    } else {
        H.r_h = ds(-INFINITY, 0.0f);
        H.r_cap = ds(-1.0);
        H.r_promote = ds(-INFINITY, 0.0f);
    }
    H.r_esc = r_esc_frac * ds(c1.w, 0.0f);
    return H;
}

// Image-plane initial conditions in double precision: flat-space picture of
// the pixel (alpha, beta) at distance D = r_obs, observer direction
// n = (sin i, 0, cos i), photon moving along +n; k^t is the future root of the
// null condition in the Kerr metric; k is scaled to unit energy E = -k_t.
__device__ inline void initial_state_sc(double M, double a, double r_obs, double si, double ci, double alpha,
                                        double beta, double *y)
{
    const double D = r_obs;
    const double x = D * si - beta * ci;
    const double z = D * ci + beta * si;
    const double r = sqrt(D * D + alpha * alpha + beta * beta);
    const double rho = sqrt(x * x + alpha * alpha);
    const double ir = recip(r), irho = recip(rho);
    const double th = atan2(rho, z);
    const double ph = atan2(alpha, x);
    const double kr = D * ir;
    const double kth = (z * D - r * r * ci) * (irho * ir * ir);
    const double kph = -alpha * si * (irho * irho);
    // the metric at the start point; sin and cos of th = atan2(rho, z) with
    // rho^2 + z^2 = r^2 (reciprocals, no divides: far from the horizon
    // Delta = r (r - 2M) + a^2 does not cancel)
    const double s = rho * ir, c = z * ir, s2 = s * s, a2 = a * a;
    const double Sigma = fma(a2, c * c, r * r);
    const double iS = recip(Sigma);
    const double twoMr = 2.0 * M * r;
    const double gtt = twoMr * iS - 1.0;
    const double gtp = -(twoMr * a) * s2 * iS;
    const double grr = Sigma * recip(fma(r, r - 2.0 * M, a2));
    const double gpp = (r * r + a2 + (twoMr * a2) * s2 * iS) * s2;
    const double A = gtt;
    const double B = 2.0 * gtp * kph;
    const double C = grr * kr * kr + Sigma * kth * kth + gpp * kph * kph;
    const double kt = (-B - sqrt(B * B - 4.0 * A * C)) * (0.5 * recip(A));
    const double iE = -recip(gtt * kt + gtp * kph);
    y[0] = 0.0;
    y[1] = r;
    y[2] = th;
    y[3] = ph;
    y[4] = kt * iE;
    y[5] = kr * iE;
    y[6] = kth * iE;
    y[7] = kph * iE;
}

__device__ inline void initial_state(double M, double a, double r_obs, double incl, double alpha, double beta,
                                     double *y)
{
    double si, ci;
    sincos(incl, &si, &ci);
    initial_state_sc(M, a, r_obs, si, ci, alpha, beta, y);
}

} // namespace gray
