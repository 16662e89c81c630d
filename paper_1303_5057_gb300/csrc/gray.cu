// gray.cu -- kernels and C ABI of libgray (declared in include/gray.h).
//
// Kernels:
//   setup_images_kernel / setup_rays_kernel  image-plane initial conditions (double)
//   trace32_kernel<MODE>, trace64_kernel     persistent backward RK4 tracers
//                                            (single precision, double)
//   zone_kernel<RETURN, T>                   the near-horizon zone of the
//                                            selective mode (double-single or double)
//   probe_rays_kernel, plan_*_kernel         the longest-first planner
//   render_kernel, shadow_*, ring_*, splat   read-out of results
//   eval_kernel<T>                           unit evaluations for parity tests
//
// Trace kernel design (GRay Sec. 2 puts one photon in one thread; here a
// warp owns 32 photons at a time and keeps each photon's state in registers):
//   * a persistent grid (blocks_per_sm x SMs blocks) drains a global work
//     queue of ray indices with one atomicAdd per warp refill;
//   * every `refill` steps the warp ballots its idle lanes (rays that
//     finished) and hands them new rays, so warps do not idle while a few
//     long rays (near-critical orbits) run on;
//   * rays are loaded and stored with 16-byte vector accesses from a
//     structure-of-arrays state (one plane per 4-vector);
//   * per-call statistics are reduced in the warp and added once per warp.
// There is no spin-wait anywhere: a warp leaves when the queue is empty and
// its lanes are idle, so every launch ends.
#include "gray.h"
#include "kerr.cuh"

#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <type_traits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using namespace gray;

namespace {

std::atomic<int64_t> g_launches{0};

struct alignas(32) d4 {
    double x, y, z, w;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Structure-of-arrays layout of the state of n rays (all planes 256-byte aligned):
//   X  position (t, r, theta, phi)      float4 (FP32 modes) / d4 (FP64)
//   K  momentum (k^t, k^r, k^th, k^ph)  float4 / d4
//   CX, CK  Kahan compensations         float4 (FP32 modes only)
//   F  final position on the stop surface  float4 / d4
//   P  per-ray constants (a, M, r_obs, w)  d4; w holds the low words of a and M as
//      two floats (a = (float)a + a_lo, likewise M)
//   PF0, PF1 the same constants for single precision: (a, M, r_+ hi, r_+ lo),
//           (r_-, dc, r_h, r_obs)  float4 each (FP32 modes only)
//   S0 (status, steps, Euler redos, pole remaps)  int4
//   S1 (steps in double, call epoch, steps in that call, flags)  int4
//   L  hand-off list of ray indices (selective-double mode)  int
struct Layout {
    size_t X, K, CX, CK, F, P, PF0, PF1, S0, S1, L, R, total;
};

inline bool is_f64(int prec) { return prec == GRAY_FP64; }

Layout make_layout(int64_t n, int prec)
{
    Layout L{};
    size_t off = 0;
    const size_t un = (size_t)n;
    const size_t v = is_f64(prec) ? 32 : 16;
    L.X = off;
    off = align256(off + v * un);
    L.K = off;
    off = align256(off + v * un);
    if (!is_f64(prec)) {
        L.CX = off;
        off = align256(off + 16 * un);
        L.CK = off;
        off = align256(off + 16 * un);
    } else {
        L.CX = L.CK = 0;
    }
    L.F = off;
    off = align256(off + v * un);
    L.P = off;
    off = align256(off + 32 * un);
    if (!is_f64(prec)) {
        L.PF0 = off;
        off = align256(off + 16 * un);
        L.PF1 = off;
        off = align256(off + 16 * un);
    } else {
        L.PF0 = L.PF1 = 0;
    }
    L.S0 = off;
    off = align256(off + 16 * un);
    L.S1 = off;
    off = align256(off + 16 * un);
    L.L = off;
    off = align256(off + 4 * un);
    if (prec == GRAY_FP32_KAHAN_SEL64) {
        L.R = off; // rays the zone pass returns to single precision
        off = align256(off + 4 * un);
    } else {
        L.R = 0;
    }
    L.total = off;
    return L;
}

struct StateView {
    char *X, *K, *CX, *CK, *F;
    d4 *P;
    float4 *PF0, *PF1;
    int4 *S0;
    int4 *S1;
    int *L;
    int *R;
};

StateView make_view(void *base, int64_t n, int prec)
{
    Layout L = make_layout(n, prec);
    char *b = (char *)base;
    StateView v;
    v.X = b + L.X;
    v.K = b + L.K;
    v.CX = is_f64(prec) ? nullptr : b + L.CX;
    v.CK = is_f64(prec) ? nullptr : b + L.CK;
    v.F = b + L.F;
    v.P = (d4 *)(b + L.P);
    v.PF0 = is_f64(prec) ? nullptr : (float4 *)(b + L.PF0);
    v.PF1 = is_f64(prec) ? nullptr : (float4 *)(b + L.PF1);
    v.S0 = (int4 *)(b + L.S0);
    v.S1 = (int4 *)(b + L.S1);
    v.L = (int *)(b + L.L);
    v.R = prec == GRAY_FP32_KAHAN_SEL64 ? (int *)(b + L.R) : nullptr;
    return v;
}

__device__ __forceinline__ d4 ld_d4(const void *p, int64_t i)
{
    const double2 *q = (const double2 *)p + 2 * i;
    double2 a = q[0], b = q[1];
    return d4{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st_d4(void *p, int64_t i, double x, double y, double z, double w)
{
    double2 *q = (double2 *)p + 2 * i;
    q[0] = make_double2(x, y);
    q[1] = make_double2(z, w);
}
__device__ __forceinline__ float4 ld_f4(const void *p, int64_t i) { return ((const float4 *)p)[i]; }
__device__ __forceinline__ void st_f4(void *p, int64_t i, float x, float y, float z, float w)
{
    ((float4 *)p)[i] = make_float4(x, y, z, w);
}

// Workspace of one context (device memory, zeroed before each trace).
struct Workspace {
    unsigned long long head;    // next ray (or list slot) handed out by the queue of a pass
    unsigned long long steps;   // steps taken in this call
    unsigned long long euler;   // Euler redos in this call
    unsigned long long fp64;    // steps taken in double by the selective mode in this call
    unsigned long long active;  // rays left active by this call
    unsigned long long handoff; // rays appended to the hand-off list by the current pass
    unsigned long long demoted; // rays returned to single precision by the current zone pass
    unsigned long long zone_steps; // steps taken by the zone kernel in this call
    unsigned long long cancel;     // the cancel flag as the call ended (copied in by gray_trace)
};

} // namespace

struct gray_ctx {
    gray_options opt;
    Workspace *ws = nullptr;      // device
    Workspace *ws_host = nullptr; // pinned host mirror
    int device = 0;
    int num_sms = 0;
    unsigned long long *aux = nullptr; // device: planning counters, histograms, call epoch
    bool timing = false;               // record events around the passes of each call
    cudaEvent_t ev[6] = {};            // [0,1] single pass, [2,3] zone pass, [4,5] plan probe pass
    bool ev_used[3] = {false, false, false};
    cudaStream_t side = nullptr;       // gray_setup_plan: the planning passes (high priority)
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaStream_t cancel_stream = nullptr; // gray_cancel writes the flag through it (non-blocking)
};

namespace {

// --------------------------------------------------------------------------
// Set-up
// --------------------------------------------------------------------------

struct ImageDev {
    double a, M, r_obs, incl;
    double si, ci; // sin and cos of incl (host)
    double a0, da; // Cartesian: alpha of the first pixel edge, pixel width; polar: R0, dR
    double b0, db; // Cartesian: beta likewise; polar: first angle, angle step
    long long first; // first ray of the image relative to the call's first ray
    int nx, ny;
    int grid;
    int probe_first; // planning: the image's first probe among the call's probes (0 otherwise)
    float hc[8]; // single-precision per-ray constants (hole_constants_f), once per image
};
static_assert(sizeof(ImageDev) == 136, "gray_setup_noalloc's table size is documented in gray.h");

// Image-plane position of the ray in (row, col) of an image: a pixel centre
// of the Cartesian grid, or the polar grid point of Sec. 4 (Eqs. 9-10).
__device__ __forceinline__ void image_point(const ImageDev &im, int64_t row, int64_t col, double &alpha,
                                            double &beta)
{
    if (im.grid == GRAY_GRID_POLAR) {
        const double R = im.a0 + ((double)col + 0.5) * im.da;
        double s, c;
        sincos(im.b0 + (double)row * im.db, &s, &c);
        alpha = R * c;
        beta = R * s;
    } else {
        alpha = im.a0 + ((double)col + 0.5) * im.da;
        beta = im.b0 + ((double)row + 0.5) * im.db;
    }
}

// Store one initial state (double) into the layout of `prec`.  FP32 modes keep
// the rounding error of each component in the compensation plane, so a
// compensated trace starts from the double-precision initial condition.
// hc: the single-precision constants of (a, M, r_obs), or NULL to compute them.
__device__ void store_initial(const StateView &v, int prec, int64_t i, const double *y, double a, double M,
                              double r_obs, const float *hc)
{
    if (prec == GRAY_FP64) {
        st_d4(v.X, i, y[0], y[1], y[2], y[3]);
        st_d4(v.K, i, y[4], y[5], y[6], y[7]);
        st_d4(v.F, i, y[0], y[1], y[2], y[3]);
    } else {
        float hi[8], lo[8];
        for (int m = 0; m < 8; ++m) {
            hi[m] = (float)y[m];
            lo[m] = (prec == GRAY_FP32) ? 0.0f : (float)((double)hi[m] - y[m]);
        }
        st_f4(v.X, i, hi[0], hi[1], hi[2], hi[3]);
        st_f4(v.K, i, hi[4], hi[5], hi[6], hi[7]);
        st_f4(v.CX, i, lo[0], lo[1], lo[2], lo[3]);
        st_f4(v.CK, i, lo[4], lo[5], lo[6], lo[7]);
        st_f4(v.F, i, hi[0], hi[1], hi[2], hi[3]);
        float c8[8];
        if (hc) {
            for (int m = 0; m < 8; ++m)
                c8[m] = hc[m];
        } else {
            hole_constants_f(a, M, r_obs, c8);
        }
        v.PF0[i] = make_float4(c8[0], c8[1], c8[2], c8[3]);
        v.PF1[i] = make_float4(c8[4], c8[5], c8[6], c8[7]);
    }
    // the fourth slot of P holds the low words of a and M as two floats
    // (a = (float)a + a_lo): the double-single Eq. 4 test needs them
    const float a_hi = (float)a, M_hi = (float)M;
    const float2 low = make_float2((float)(a - (double)a_hi), (float)(M - (double)M_hi));
    double w;
    memcpy(&w, &low, sizeof w);
    st_d4(v.P, i, a, M, r_obs, w);
    v.S0[i] = make_int4(GRAY_RAY_ACTIVE, 0, 0, 0);
    v.S1[i] = make_int4(0, 0, 0, 0);
}

// Set-up of the rays of a call's images.  probe_stride > 0 selects part of
// them: probe rays (every probe_stride-th pixel of each row and column,
// which_probes = 1) or the others (which_probes = 0); probe_stride = 0 sets
// up every ray.
__global__ void setup_images_kernel(const ImageDev *imgs, int n_images, int64_t total, int64_t first_ray,
                                    StateView v, int prec, int probe_stride = 0, int which_probes = 0)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total)
        return;
    int lo = 0, hi = n_images - 1;
    while (lo < hi) { // last image with first <= i
        int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].first <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ImageDev im = imgs[lo];
    const int64_t p = i - im.first;
    const int64_t row = p / im.nx, col = p - row * im.nx;
    if (probe_stride > 0 && ((row % probe_stride == 0 && col % probe_stride == 0) ? 1 : 0) != which_probes)
        return;
    double alpha, beta;
    image_point(im, row, col, alpha, beta);
    double y[8];
    initial_state_sc(im.M, im.a, im.r_obs, im.si, im.ci, alpha, beta, y);
    store_initial(v, prec, first_ray + i, y, im.a, im.M, im.r_obs, im.hc);
}

__global__ void setup_rays_kernel(const double *rays, int64_t n, double M, int64_t first_ray, StateView v, int prec)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const double *q = rays + 5 * i;
    double y[8];
    initial_state(M, q[2], q[4], q[3], q[0], q[1], y);
    store_initial(v, prec, first_ray + i, y, q[2], M, q[4], nullptr);
}

// --------------------------------------------------------------------------
// One integration step (GRay Sec. 2 order): step size -> RK4 -> Eq. 4
// monitor, Euler redo at h/9 on failure -> finite check -> stop tests with
// the final point on the stop surface -> Eq. 3 remap.
// --------------------------------------------------------------------------

// State update y1 = y + inc, plain or compensated (Kahan: the true value is
// y - c).
template <typename T, bool KAHAN>
__device__ __forceinline__ void add_update(const T *y, const T *c, const T *inc, T *y1, T *c1)
{
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        if (KAHAN) {
            const T d = inc[m] - c[m];
            const T t = y[m] + d;
            c1[m] = (t - y[m]) - d;
            y1[m] = t;
        } else {
            y1[m] = y[m] + inc[m];
        }
    }
}

// Eq. 3 on the state; with compensation the new theta and phi are formed in
// double-single from the pair (hi, lo) so that the remap itself adds no
// rounding beyond the pair's own.
template <typename T, bool KAHAN> __device__ __forceinline__ int remap_eq3(T *y, T *c)
{
    const T pi = pi_v<T>();
    if (!(y[2] > pi) && !(y[2] < T(0)))
        return 0;
    const bool over = y[2] > pi;
    if constexpr (KAHAN) {
        const ds th = ds_fast(y[2], -c[2]), ph = ds_fast(y[3], -c[3]);
        const ds th2 = over ? ds(2.0 * 3.14159265358979323846) - th : -th;
        const ds ph2 = over ? ph + pi_v<ds>() : ph - pi_v<ds>();
        y[2] = th2.hi;
        c[2] = -th2.lo;
        y[3] = ph2.hi;
        c[3] = -ph2.lo;
        y[6] = -y[6];
        c[6] = -c[6];
    } else {
        if (over) {
            y[2] = T(2) * pi - y[2];
            y[3] = y[3] + pi;
        } else {
            y[2] = -y[2];
            y[3] = y[3] - pi;
        }
        y[6] = -y[6];
    }
    return 1;
}

__device__ __forceinline__ float sixth(float h) { return h * (1.0f / 6.0f); }
__device__ __forceinline__ double sixth(double h) { return h * (1.0 / 6.0); }
__device__ __forceinline__ float ninth(float h) { return h * (1.0f / 9.0f); }
__device__ __forceinline__ double ninth(double h) { return h * (1.0 / 9.0); }
__device__ __forceinline__ ds sixth(ds h) { return h * ds(1.0 / 6.0); }
__device__ __forceinline__ ds ninth(ds h) { return h * ds(1.0 / 9.0); }

// One step.  Returns the ray's new status; writes fin[4] when it stops.  g
// holds the geometry of the current point on entry and of the new point on
// exit, so the first RK4 stage reuses what the previous step's Eq. 4 test
// computed.  MIXED_STOP (double steps of the single-precision zone tracer):
// the stop surfaces are interpolated by stop_surface_mixed.
template <typename T, bool KAHAN, bool MIXED_STOP = false>
__device__ __forceinline__ int step_once(const Hole<T> &H, const StepOpt<T> &O, T *y, T *c, Geo<T> &g, T *fin,
                                         int &euler, int &remaps, const float2 *aM_lo = nullptr)
{
    T h = step_size(H, O, y);
    T a1[4];
    accel_geo(H, g, y[4], y[5], y[6], y[7], a1);
    const T hh = T(0.5) * h;
    const T dr = KAHAN ? -c[1] : T(0), dth = KAHAN ? -c[2] : T(0);
    const T h6 = sixth(h);
    T inc[8];
    if constexpr (std::is_same<T, ds>::value) {
        // double-single (the zone): the three later stages in one rolled loop,
        // one copy of the stage's ~8x longer code (the zone pass is 1.6x
        // faster rolled; the single-precision pass is 1-8 % slower rolled, so
        // float and double keep the stages written out below).  Stage s
        // starts from y + c_s h (k, a) of stage s - 1 (c = 1/2, 1/2, 1) and
        // enters the sums k1 + 2 k2 + 2 k3 + k4 with weight 2, 2, 1.
        T sk[4], sa[4], pk[4], pa[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            sk[m] = pk[m] = y[4 + m];
            sa[m] = pa[m] = a1[m];
        }
#pragma unroll 1
        for (int stage = 0; stage < 3; ++stage) {
            const T cs = stage < 2 ? hh : h;
            const T w = stage < 2 ? T(2) : T(1);
            const T rs = fma(cs, pk[1], y[1]), ths = fma(cs, pk[2], y[2]);
            T ks[4], as[4];
#pragma unroll
            for (int m = 0; m < 4; ++m)
                ks[m] = fma(cs, pa[m], y[4 + m]);
            accel_geo(H, geometry_rel(H, g, rs, cs * pk[2], ths, dr, dth), ks[0], ks[1], ks[2], ks[3], as);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                sk[m] = fma(w, ks[m], sk[m]);
                sa[m] = fma(w, as[m], sa[m]);
                pk[m] = ks[m];
                pa[m] = as[m];
            }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            inc[m] = h6 * sk[m];
            inc[4 + m] = h6 * sa[m];
        }
    } else {
        T a2[4], a3[4], a4[4];
        const T r2 = fma(hh, y[5], y[1]), th2 = fma(hh, y[6], y[2]);
        const T kt2 = fma(hh, a1[0], y[4]), kr2 = fma(hh, a1[1], y[5]), kh2 = fma(hh, a1[2], y[6]),
                kp2 = fma(hh, a1[3], y[7]);
        accel_geo(H, geometry_rel(H, g, r2, hh * y[6], th2, dr, dth), kt2, kr2, kh2, kp2, a2);
        const T r3 = fma(hh, kr2, y[1]), th3 = fma(hh, kh2, y[2]);
        const T kt3 = fma(hh, a2[0], y[4]), kr3 = fma(hh, a2[1], y[5]), kh3 = fma(hh, a2[2], y[6]),
                kp3 = fma(hh, a2[3], y[7]);
        accel_geo(H, geometry_rel(H, g, r3, hh * kh2, th3, dr, dth), kt3, kr3, kh3, kp3, a3);
        const T r4 = fma(h, kr3, y[1]), th4 = fma(h, kh3, y[2]);
        const T kt4 = fma(h, a3[0], y[4]), kr4 = fma(h, a3[1], y[5]), kh4 = fma(h, a3[2], y[6]),
                kp4 = fma(h, a3[3], y[7]);
        accel_geo(H, geometry_rel(H, g, r4, h * kh3, th4, dr, dth), kt4, kr4, kh4, kp4, a4);
        inc[0] = h6 * (y[4] + T(2) * (kt2 + kt3) + kt4);
        inc[1] = h6 * (y[5] + T(2) * (kr2 + kr3) + kr4);
        inc[2] = h6 * (y[6] + T(2) * (kh2 + kh3) + kh4);
        inc[3] = h6 * (y[7] + T(2) * (kp2 + kp3) + kp4);
#pragma unroll
        for (int m = 0; m < 4; ++m)
            inc[4 + m] = h6 * (a1[m] + T(2) * (a2[m] + a3[m]) + a4[m]);
    }
    T y1[8], c1[8];
    add_update<T, KAHAN>(y, c, inc, y1, c1);
    Geo<T> g1 = geometry(H, y1[1], y1[2], KAHAN ? -c1[1] : T(0), KAHAN ? -c1[2] : T(0));

    // Eq. 4 monitor: redo the step as forward Euler at h/9 when |xi + 1| > eps.
    // Compensated single precision: a test whose outcome lies within its own
    // rounding is taken again in double-single arithmetic on the compensated
    // state, with the ray's spin and mass split into two floats (aM), so the
    // decision follows the one the double method takes at that state.
    bool redo;
    if constexpr (sizeof(T) == 4 && KAHAN) {
        bool ambiguous;
        redo = xi_fails_flag(H, g1, y1, O.eps_xi, ambiguous);
        if (ambiguous && aM_lo) {
            const float2 lo = *aM_lo;
            redo = xi_fails_ds(y1, c1, make_float4(H.a, lo.x, H.M, lo.y), O.eps_xi);
        }
    } else {
        redo = xi_fails(H, g1, y1, O.eps_xi);
    }
    if (redo) {
        h = ninth(h);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            inc[m] = h * y[4 + m];
            inc[4 + m] = h * a1[m];
        }
        add_update<T, KAHAN>(y, c, inc, y1, c1);
        g1 = geometry(H, y1[1], y1[2], KAHAN ? -c1[1] : T(0), KAHAN ? -c1[2] : T(0));
        ++euler;
    }

    int status = GRAY_RAY_ACTIVE;
    bool finite = true;
#pragma unroll
    for (int m = 0; m < 8; ++m)
        finite &= finite_v(y1[m]);
    // The rare outcomes (a non-finite state, a stop, a pole crossing) sit
    // behind one test, so a plain step takes a single branch here.
    const T half_pi = T(0.5) * pi_v<T>();
    const bool equator = O.stop_equator && (y[2] - half_pi) * (y1[2] - half_pi) < T(0);
    if (!finite || equator || y1[1] <= H.r_cap || y1[1] >= H.r_esc || y1[2] > pi_v<T>() || y1[2] < T(0)) {
        // the out-of-line helpers get copies made here: only these copies
        // have their address taken, so the step's states stay in registers
        // (without them the pass stored ~6 words to local memory per warp
        // step; with them, 0.3 % faster)
        T s0[8], s1[8], sf[4];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            s0[m] = y[m];
            s1[m] = y1[m];
        }
        if (!finite) {
            status = GRAY_RAY_NONFINITE;
            for (int m = 0; m < 4; ++m)
                fin[m] = y1[m];
        } else if (equator) {
            equator_crossing(s0, s1, h, sf);
            status = GRAY_RAY_EQUATOR;
        } else if (y1[1] <= H.r_cap) {
            if constexpr (MIXED_STOP)
                stop_surface_mixed(s0, s1, h, H.r_cap, sf);
            else
                stop_surface(s0, s1, h, H.r_cap, sf);
            status = GRAY_RAY_CAPTURED;
        } else if (y1[1] >= H.r_esc && h * y1[5] > T(0)) {
            if constexpr (MIXED_STOP)
                stop_surface_mixed(s0, s1, h, H.r_esc, sf);
            else
                stop_surface(s0, s1, h, H.r_esc, sf);
            status = GRAY_RAY_ESCAPED;
        }
        if (status == GRAY_RAY_EQUATOR || status == GRAY_RAY_CAPTURED || status == GRAY_RAY_ESCAPED) {
#pragma unroll
            for (int m = 0; m < 4; ++m)
                fin[m] = sf[m];
        }
        if (status != GRAY_RAY_NONFINITE && remap_eq3<T, KAHAN>(y1, c1)) {
            ++remaps;
            g1 = geometry(H, y1[1], y1[2], KAHAN ? -c1[1] : T(0), KAHAN ? -c1[2] : T(0));
        }
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        y[m] = y1[m];
        if (KAHAN)
            c[m] = c1[m];
    }
    g = g1;
    return status;
}

// --------------------------------------------------------------------------
// Persistent trace kernels
// --------------------------------------------------------------------------
//
// Single-precision modes run trace32_kernel over every ray of the buffer.
// In GRAY_FP32_KAHAN_SEL64 a ray that reaches the zone (r below
// cap_frac r_h + r_sw at the start of a step) is handed off: its state is
// stored and its index appended to the hand-off list.  zone_kernel then
// runs the listed rays in extended precision (double-single by default,
// IEEE double as an option), 32 to a warp, until they stop or climb out of
// the zone (r above cap_frac r_h + 2 r_sw), when they return to single
// precision for the next pass.  The zone's arithmetic is ~8 times longer
// per step (and the FP64 pipe of this part runs at 1/64 of the FP32 rate),
// so a zone step must never hold a warp of single-precision lanes; the
// hand-off keeps the two populations apart and the single-precision kernel
// free of the zone's registers.  GRAY_FP64 runs trace64_kernel over every
// ray, with double planes.

enum : int { FLAG_DOUBLE_MODE = 1, FLAG_DOUBLE_REPR = 2 };

struct TraceArgs {
    StateView v;
    int64_t n;                                   // rays in the buffer
    const int *order;                            // queue of ray indices, or NULL: 0 .. n-1
    int64_t n_queue;                             // queue length (order != NULL)
    const unsigned long long *n_queue_dev;       // if not NULL: queue length read on the device
    int64_t budget; // per-call step budget per ray, <= 0: none
    int max_steps;
    int refill;
    int step_rule;
    const int *epoch_dev; // call counter on the device (bumped by every gray_trace / gray_plan):
                          // S1.y == epoch means S1.z counts this call's steps
    int one_per_thread; // the paper's launch: thread g takes queue slot g only
    int stop_equator;   // Sec. 3 grid projection: stop at the equatorial plane
    int zone_return;    // zone pass: a ray climbing out of the zone goes to the return list
    double h_frac, h_min, eps_xi, cap_frac, r_esc_frac, r_sw;
    Workspace *ws;
    const int *cancel;          // the context's cancel flag (gray_cancel), read at each refill
};

template <int MODE> struct ModeTraits {
    static constexpr bool kahan = (MODE == GRAY_FP32_KAHAN || MODE == GRAY_FP32_KAHAN_SEL64);
    static constexpr bool sel64 = (MODE == GRAY_FP32_KAHAN_SEL64);
};

// Length of the work queue of a pass, and the ray behind a queue slot (-1 for
// an index outside the buffer, which is skipped).
__device__ __forceinline__ int64_t queue_length(const TraceArgs &A)
{
    if (A.n_queue_dev)
        return (int64_t)*(volatile const unsigned long long *)A.n_queue_dev;
    return A.order ? A.n_queue : A.n;
}
__device__ __forceinline__ int64_t queue_ray(const TraceArgs &A, int64_t slot)
{
    if (!A.order)
        return slot;
    const int64_t my = (int64_t)A.order[slot];
    return (my >= 0 && my < A.n) ? my : -1;
}

// The context's cancel flag, read by lane 0 and shared with the warp
// (warp-uniform call).
__device__ __forceinline__ bool cancelled(const TraceArgs &A, int lane)
{
    int f = 0;
    if (lane == 0)
        f = *(volatile const int *)A.cancel;
    return __shfl_sync(0xffffffffu, f, 0) != 0;
}

// Warp-aggregated counter increment (warp-uniform call).
__device__ __forceinline__ unsigned long long warp_count(unsigned long long *ctr, bool pred, int lane,
                                                         int *rank_out)
{
    const unsigned FULL = 0xffffffffu;
    const unsigned m = __ballot_sync(FULL, pred);
    unsigned long long base = 0;
    if (m) {
        const int leader = __ffs(m) - 1;
        if (lane == leader)
            base = atomicAdd(ctr, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, leader);
    }
    *rank_out = __popc(m & ((1u << lane) - 1u));
    return base;
}

template <typename T>
__device__ __forceinline__ void warp_stats(const TraceArgs &A, int lane, unsigned long long steps,
                                           unsigned long long euler, unsigned long long fp64,
                                           bool zone = false)
{
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        steps += __shfl_xor_sync(FULL, steps, off);
        euler += __shfl_xor_sync(FULL, euler, off);
        fp64 += __shfl_xor_sync(FULL, fp64, off);
    }
    if (lane == 0) {
        if (steps)
            atomicAdd(&A.ws->steps, steps);
        if (steps && zone)
            atomicAdd(&A.ws->zone_steps, steps);
        if (euler)
            atomicAdd(&A.ws->euler, euler);
        if (fp64)
            atomicAdd(&A.ws->fp64, fp64);
    }
}

// Single-precision persistent tracer (modes FP32, FP32_KAHAN, FP32_KAHAN_SEL64).
// MAXREG: 128 registers keep four 128-thread blocks per SM for the main pass;
// the probe pass of the planner (~900 warps for a 1024^2 image, latency-bound
// over its 400 sequential steps) runs the same code uncapped (~140 registers:
// nothing re-formed under register pressure), 0.56 -> 0.52 ms.
template <int MODE, int MAXREG = 128> __global__ void __maxnreg__(MAXREG) trace32_kernel(TraceArgs A)
{
    constexpr bool KAHAN = ModeTraits<MODE>::kahan;
    constexpr bool SEL64 = ModeTraits<MODE>::sel64;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const StateView &v = A.v;
    StepOpt<float> O;
    O.h_frac = (float)A.h_frac;
    O.h_min = (float)A.h_min;
    O.eps_xi = (float)A.eps_xi;
    O.step_rule = A.step_rule;
    O.stop_equator = A.stop_equator;

    bool has = false, exhausted = false;
    int64_t id = 0;
    const int64_t nq = queue_length(A);
    const int epoch = *A.epoch_dev;
    float y[8], c[8], fin[4];
    Hole<float> H;
    Geo<float> geo;
    float r_promote = -INFINITY;
    int steps = 0, euler = 0, remaps = 0, n64 = 0;
    int steps0 = 0, euler0 = 0, used0 = 0; // at load: this call's counts follow from them
    int stop_at = 0;                        // step count at which the ray hits the cap or its budget
    unsigned long long tot_steps = 0, tot_euler = 0;
    bool pending = false; // this lane handed its ray off; its index is not yet on the list

    for (;;) {
        // gray_cancel: no more rays are picked up, and the rays in flight
        // are stored as they stand (still ACTIVE) at their next step
        const bool stop = cancelled(A, lane);
        if (stop)
            exhausted = true;
        if (SEL64) {
            int rank;
            const unsigned long long hb = warp_count(&A.ws->handoff, pending, lane, &rank);
            if (pending)
                v.L[hb + rank] = (int)id;
            pending = false;
        }
        // ---- refill idle lanes from the work queue (warp-uniform loop) ----
        while (!exhausted) {
            const unsigned idle = __ballot_sync(FULL, !has);
            if (idle == 0)
                break;
            const int cnt = __popc(idle);
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if (!A.one_per_thread) {
                if (lane == leader)
                    base = atomicAdd(&A.ws->head, (unsigned long long)cnt);
                base = __shfl_sync(FULL, base, leader);
            }
            bool handoff_now = false;
            if (!has) {
                const int64_t slot = A.one_per_thread
                                         ? (int64_t)blockIdx.x * blockDim.x + threadIdx.x
                                         : (int64_t)base + __popc(idle & ((1u << lane) - 1u));
                const int64_t my = slot < nq ? queue_ray(A, slot) : -1;
                if (my >= 0) {
                    const int4 s0 = v.S0[my];
                    if (s0.x == GRAY_RAY_ACTIVE) {
                        const int4 s1 = v.S1[my];
                        if (SEL64 && (s1.w & FLAG_DOUBLE_MODE)) {
                            handoff_now = true; // resumed inside the zone
                            id = my;
                        } else {
                            has = true;
                            id = my;
                            steps = s0.y;
                            euler = s0.z;
                            remaps = s0.w;
                            n64 = s1.x;
                            used0 = (s1.y == epoch) ? s1.z : 0;
                            steps0 = steps;
                            euler0 = euler;
                            stop_at = A.max_steps;
                            if (A.budget > 0) {
                                const int64_t b = (int64_t)steps0 + A.budget - used0;
                                if (b < stop_at)
                                    stop_at = (int)b;
                            }
                            H = make_hole_f(v.PF0[my], v.PF1[my], (float)A.cap_frac, (float)A.r_esc_frac,
                                            (float)A.r_sw);
                            r_promote = H.r_promote;
                            const float4 X = ld_f4(v.X, my), K = ld_f4(v.K, my);
                            y[0] = X.x; y[1] = X.y; y[2] = X.z; y[3] = X.w;
                            y[4] = K.x; y[5] = K.y; y[6] = K.z; y[7] = K.w;
                            if (KAHAN) {
                                const float4 CX = ld_f4(v.CX, my), CK = ld_f4(v.CK, my);
                                c[0] = CX.x; c[1] = CX.y; c[2] = CX.z; c[3] = CX.w;
                                c[4] = CK.x; c[5] = CK.y; c[6] = CK.z; c[7] = CK.w;
                            } else {
#pragma unroll
                                for (int m = 0; m < 8; ++m)
                                    c[m] = 0.0f;
                            }
                            geo = geometry(H, y[1], y[2], KAHAN ? -c[1] : 0.0f, KAHAN ? -c[2] : 0.0f);
                        }
                    }
                }
            }
            if (SEL64) {
                int rank;
                const unsigned long long hb = warp_count(&A.ws->handoff, handoff_now, lane, &rank);
                if (handoff_now)
                    v.L[hb + rank] = (int)id;
            }
            if (A.one_per_thread || (int64_t)base + cnt >= nq)
                exhausted = true;
        }
        if (!__any_sync(FULL, has))
            break;

        // ---- step block: `refill` steps, then look for idle lanes again ----
        for (int k = 0; k < A.refill; ++k) {
            bool handoff = false;
            if (has) {
                int status = GRAY_RAY_ACTIVE;
                bool yield = false;
                if (steps >= stop_at || (SEL64 && y[1] - c[1] < r_promote) || stop) {
                    if (steps >= A.max_steps) {
                        status = GRAY_RAY_STEP_CAP;
                        for (int m = 0; m < 4; ++m)
                            fin[m] = y[m];
                    } else if (stop || (A.budget > 0 && used0 + (steps - steps0) >= A.budget)) {
                        yield = true;
                    } else {
                        handoff = true;
                    }
                } else {
                    status = step_once<float, KAHAN>(H, O, y, c, geo, fin, euler, remaps, (const float2 *)&v.P[id].w);
                    ++steps;
                }
                if (status != GRAY_RAY_ACTIVE || yield || handoff) {
                    st_f4(v.X, id, y[0], y[1], y[2], y[3]);
                    st_f4(v.K, id, y[4], y[5], y[6], y[7]);
                    if (KAHAN) {
                        st_f4(v.CX, id, c[0], c[1], c[2], c[3]);
                        st_f4(v.CK, id, c[4], c[5], c[6], c[7]);
                    }
                    if (status != GRAY_RAY_ACTIVE)
                        st_f4(v.F, id, fin[0], fin[1], fin[2], fin[3]);
                    v.S0[id] = make_int4(status, steps, euler, remaps);
                    v.S1[id] = make_int4(n64, epoch, used0 + (steps - steps0), handoff ? FLAG_DOUBLE_MODE : 0);
                    tot_steps += (unsigned long long)(steps - steps0);
                    tot_euler += (unsigned long long)(euler - euler0);
                    has = false;
                    pending = handoff;
                }
            }
        }
    }
    warp_stats<float>(A, lane, tot_steps, tot_euler, 0ull);
}

// Double-precision persistent tracer over every ray of a GRAY_FP64 buffer.
__global__ void __launch_bounds__(128) trace64_kernel(TraceArgs A)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const StateView &v = A.v;
    StepOpt<double> O;
    O.h_frac = A.h_frac;
    O.h_min = A.h_min;
    O.eps_xi = A.eps_xi;
    O.step_rule = A.step_rule;
    O.stop_equator = A.stop_equator;

    bool has = false, exhausted = false;
    int64_t id = 0;
    double y[8], cz[8], fin[4];
    Hole<double> H;
    Geo<double> geo;
    int steps = 0, euler = 0, remaps = 0, n64 = 0, used = 0;
    unsigned long long tot_steps = 0, tot_euler = 0;
    const int64_t nq = queue_length(A);
    const int epoch = *A.epoch_dev;
#pragma unroll
    for (int m = 0; m < 8; ++m)
        cz[m] = 0.0;

    for (;;) {
        const bool stop = cancelled(A, lane); // gray_cancel, as in trace32_kernel
        if (stop)
            exhausted = true;
        while (!exhausted) {
            const unsigned idle = __ballot_sync(FULL, !has);
            if (idle == 0)
                break;
            const int cnt = __popc(idle);
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if (lane == leader)
                base = atomicAdd(&A.ws->head, (unsigned long long)cnt);
            base = __shfl_sync(FULL, base, leader);
            if (!has) {
                const int64_t slot = (int64_t)base + __popc(idle & ((1u << lane) - 1u));
                const int64_t my = slot < nq ? queue_ray(A, slot) : -1;
                if (my >= 0) {
                    const int4 s0 = v.S0[my];
                    if (s0.x == GRAY_RAY_ACTIVE) {
                        const int4 s1 = v.S1[my];
                        has = true;
                        id = my;
                        steps = s0.y;
                        euler = s0.z;
                        remaps = s0.w;
                        n64 = s1.x;
                        used = (s1.y == epoch) ? s1.z : 0;
                        const d4 p = ld_d4(v.P, my);
                        H = make_hole(p.x, p.y, p.z, A.cap_frac, A.r_esc_frac, A.r_sw);
                        const d4 X = ld_d4(v.X, my), K = ld_d4(v.K, my);
                        y[0] = X.x; y[1] = X.y; y[2] = X.z; y[3] = X.w;
                        y[4] = K.x; y[5] = K.y; y[6] = K.z; y[7] = K.w;
                        geo = geometry(H, y[1], y[2]);
                    }
                }
            }
            if ((int64_t)base + cnt >= nq)
                exhausted = true;
        }
        if (!__any_sync(FULL, has))
            break;

        for (int k = 0; k < A.refill; ++k) {
            if (has) {
                int status = GRAY_RAY_ACTIVE;
                bool yield = false;
                if (steps >= A.max_steps) {
                    status = GRAY_RAY_STEP_CAP;
                    for (int m = 0; m < 4; ++m)
                        fin[m] = y[m];
                } else if (stop || (A.budget > 0 && used >= A.budget)) {
                    yield = true;
                } else {
                    const int e0 = euler;
                    status = step_once<double, false>(H, O, y, cz, geo, fin, euler, remaps);
                    tot_euler += (unsigned long long)(euler - e0);
                    ++steps;
                    ++used;
                    ++tot_steps;
                }
                if (status != GRAY_RAY_ACTIVE || yield) {
                    st_d4(v.X, id, y[0], y[1], y[2], y[3]);
                    st_d4(v.K, id, y[4], y[5], y[6], y[7]);
                    if (status != GRAY_RAY_ACTIVE)
                        st_d4(v.F, id, fin[0], fin[1], fin[2], fin[3]);
                    v.S0[id] = make_int4(status, steps, euler, remaps);
                    v.S1[id] = make_int4(n64, epoch, used, 0);
                    has = false;
                }
            }
        }
    }
    warp_stats<double>(A, lane, tot_steps, tot_euler, 0ull);
}

// The zone's arithmetic T: double, or double-single (ds) on the FP32 pipe.
// Conversions from and to a compensated single-precision pair (the true value
// is hi - c) and to a float.
template <typename T> struct ZoneArith;
template <> struct ZoneArith<double> {
    static __device__ __forceinline__ double from_pair(float hi, float c) { return (double)hi - (double)c; }
    static __device__ __forceinline__ void to_pair(double v, float &hi, float &c)
    {
        hi = (float)v;
        c = (float)((double)hi - v);
    }
    static __device__ __forceinline__ float to_float(double v) { return (float)v; }
};
template <> struct ZoneArith<ds> {
    static __device__ __forceinline__ ds from_pair(float hi, float c) { return ds_fast(hi, -c); }
    static __device__ __forceinline__ void to_pair(ds v, float &hi, float &c)
    {
        hi = v.hi;
        c = -v.lo;
    }
    static __device__ __forceinline__ float to_float(ds v) { return v.hi; }
};

// Zone kernel of GRAY_FP32_KAHAN_SEL64: the rays of the hand-off list, in
// extended precision T (double, or double-single on the single-precision
// pipe: GRAY_ZONE_DS) while r < r_demote (= r_promote + r_sw).  RETURN = true
// (first zone pass): double only; a ray that climbs out is stored as a
// compensated single pair and appended to the return list R, which the next
// single-precision pass drains at full occupancy (this kernel holds no
// single-precision state and fits three blocks per SM).  RETURN = false (last
// zone pass): a ray that climbs out continues in compensated single precision
// here, switching back below r_promote, so every handed-off ray finishes.
// The switches are exact one way (hi - lo to T) and a rounding the other way
// (T to hi, lo; exact for double-single), the same in both forms, so a ray's
// arithmetic does not depend on which pass runs it.
template <bool RETURN, typename T>
__global__ void __launch_bounds__(128, RETURN ? 3 : 1) zone_kernel(TraceArgs A)
{
    using Z = ZoneArith<T>;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const StateView &v = A.v;
    StepOpt<T> Od;
    Od.h_frac = T(A.h_frac);
    Od.h_min = T(A.h_min);
    Od.eps_xi = T(A.eps_xi);
    Od.step_rule = A.step_rule;
    Od.stop_equator = A.stop_equator;
    StepOpt<float> Of;
    Of.h_frac = (float)A.h_frac;
    Of.h_min = (float)A.h_min;
    Of.eps_xi = (float)A.eps_xi;
    Of.step_rule = A.step_rule;
    Of.stop_equator = A.stop_equator;
    const int64_t n = (int64_t)*(volatile unsigned long long *)&A.ws->handoff;
    const int epoch = *A.epoch_dev;

    bool has = false, exhausted = false, dbl = true;
    int64_t id = 0;
    T yd[8], cz[8], find[4];
    float yf[8], cf[8], finf[4];
    Hole<T> Hd;
    Hole<float> Hf;
    Geo<T> gd;
    Geo<float> gf;
    T r_demote = T(INFINITY);
    const T r_sw = T(A.r_sw), cap_frac = T(A.cap_frac), r_esc_frac = T(A.r_esc_frac);
    int steps = 0, euler = 0, remaps = 0, n64 = 0, used = 0;
    unsigned long long tot_steps = 0, tot_euler = 0, tot_fp64 = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m)
        cz[m] = T(0.0);

    for (;;) {
        const bool stop = cancelled(A, lane); // gray_cancel, as in trace32_kernel
        if (stop)
            exhausted = true;
        while (!exhausted) {
            const unsigned idle = __ballot_sync(FULL, !has);
            if (idle == 0)
                break;
            const int cnt = __popc(idle);
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if (lane == leader)
                base = atomicAdd(&A.ws->head, (unsigned long long)cnt);
            base = __shfl_sync(FULL, base, leader);
            if (!has) {
                const int64_t slot = (int64_t)base + __popc(idle & ((1u << lane) - 1u));
                if (slot < n) {
                    const int64_t my = (int64_t)v.L[slot];
                    const int4 s0 = v.S0[my];
                    if (s0.x == GRAY_RAY_ACTIVE) {
                        const int4 s1 = v.S1[my];
                        has = true;
                        dbl = true;
                        id = my;
                        steps = s0.y;
                        euler = s0.z;
                        remaps = s0.w;
                        n64 = s1.x;
                        used = (s1.y == epoch) ? s1.z : 0;
                        if constexpr (sizeof(T) == 8 && !std::is_same<T, ds>::value) {
                            const d4 p = ld_d4(v.P, my);
                            Hd = make_hole(p.x, p.y, p.z, A.cap_frac, A.r_esc_frac, A.r_sw);
                        } else {
                            const float2 lows = *(const float2 *)&v.P[my].w;
                            Hd = make_hole_ds(v.PF0[my], v.PF1[my], lows, cap_frac, r_esc_frac, r_sw);
                        }
                        if (!RETURN)
                            Hf = make_hole_f(v.PF0[my], v.PF1[my], (float)A.cap_frac, (float)A.r_esc_frac,
                                             (float)A.r_sw);
                        r_demote = Hd.r_promote + r_sw;
                        if (s1.w & FLAG_DOUBLE_REPR) {
                            // exact double state parked in the four single planes (IEEE-double zone)
                            const double2 q0 = ((const double2 *)v.X)[my], q1 = ((const double2 *)v.K)[my];
                            const double2 q2 = ((const double2 *)v.CX)[my], q3 = ((const double2 *)v.CK)[my];
                            const double q[8] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y, q3.x, q3.y};
#pragma unroll
                            for (int m = 0; m < 8; ++m) {
                                float hi, c;
                                ZoneArith<double>::to_pair(q[m], hi, c);
                                yd[m] = std::is_same<T, ds>::value ? Z::from_pair(hi, c) : T(q[m]);
                            }
                        } else {
                            const float4 X = ld_f4(v.X, my), K = ld_f4(v.K, my);
                            const float4 CX = ld_f4(v.CX, my), CK = ld_f4(v.CK, my);
                            yd[0] = Z::from_pair(X.x, CX.x); yd[1] = Z::from_pair(X.y, CX.y);
                            yd[2] = Z::from_pair(X.z, CX.z); yd[3] = Z::from_pair(X.w, CX.w);
                            yd[4] = Z::from_pair(K.x, CK.x); yd[5] = Z::from_pair(K.y, CK.y);
                            yd[6] = Z::from_pair(K.z, CK.z); yd[7] = Z::from_pair(K.w, CK.w);
                        }
                        gd = geometry(Hd, yd[1], yd[2]);
                    }
                }
            }
            if ((int64_t)base + cnt >= n)
                exhausted = true;
        }
        if (!__any_sync(FULL, has))
            break;

        for (int k = 0; k < A.refill; ++k) {
            bool ret = false; // this lane's ray climbed out and goes to the return list
            if (has) {
                int status = GRAY_RAY_ACTIVE;
                bool yield = false, stepped = true;
                if (steps >= A.max_steps) {
                    status = GRAY_RAY_STEP_CAP;
                    for (int m = 0; m < 4; ++m)
                        find[m] = dbl ? yd[m] : Z::from_pair(yf[m], cf[m]);
                } else if (stop || (A.budget > 0 && used >= A.budget)) {
                    yield = true;
                } else if (dbl && yd[1] >= r_demote) {
                    // climb out of the zone: back to a compensated single pair
                    stepped = false;
                    if (RETURN) {
                        float hi[8], lo[8];
#pragma unroll
                        for (int m = 0; m < 8; ++m)
                            Z::to_pair(yd[m], hi[m], lo[m]);
                        st_f4(v.X, id, hi[0], hi[1], hi[2], hi[3]);
                        st_f4(v.K, id, hi[4], hi[5], hi[6], hi[7]);
                        st_f4(v.CX, id, lo[0], lo[1], lo[2], lo[3]);
                        st_f4(v.CK, id, lo[4], lo[5], lo[6], lo[7]);
                        v.S0[id] = make_int4(GRAY_RAY_ACTIVE, steps, euler, remaps);
                        v.S1[id] = make_int4(n64, epoch, used, 0);
                        has = false;
                        ret = true;
                    } else {
#pragma unroll
                        for (int m = 0; m < 8; ++m)
                            Z::to_pair(yd[m], yf[m], cf[m]);
                        gf = geometry(Hf, yf[1], yf[2], -cf[1], -cf[2]);
                        dbl = false;
                    }
                } else if (!RETURN && !dbl && yf[1] - cf[1] < Hf.r_promote) {
                    stepped = false;
#pragma unroll
                    for (int m = 0; m < 8; ++m)
                        yd[m] = Z::from_pair(yf[m], cf[m]);
                    gd = geometry(Hd, yd[1], yd[2]);
                    dbl = true;
                } else {
                    const int e0 = euler;
                    if (RETURN || dbl) {
                        status = step_once<T, false, true>(Hd, Od, yd, cz, gd, find, euler, remaps);
                        ++n64;
                        ++tot_fp64;
                    } else {
                        status = step_once<float, true>(Hf, Of, yf, cf, gf, finf, euler, remaps, (const float2 *)&v.P[id].w);
                        for (int m = 0; m < 4; ++m)
                            find[m] = Z::from_pair(finf[m], 0.0f);
                    }
                    tot_euler += (unsigned long long)(euler - e0);
                    ++steps;
                    ++used;
                    ++tot_steps;
                }
                if (stepped && (status != GRAY_RAY_ACTIVE || yield)) {
                    int flags = 0;
                    if constexpr (!std::is_same<T, ds>::value) {
                        if (yield && dbl) {
                            // park the exact double state; the ray resumes in double
                            ((double2 *)v.X)[id] = make_double2(yd[0], yd[1]);
                            ((double2 *)v.K)[id] = make_double2(yd[2], yd[3]);
                            ((double2 *)v.CX)[id] = make_double2(yd[4], yd[5]);
                            ((double2 *)v.CK)[id] = make_double2(yd[6], yd[7]);
                            flags = FLAG_DOUBLE_MODE | FLAG_DOUBLE_REPR;
                        }
                    } else if (yield && dbl) {
                        flags = FLAG_DOUBLE_MODE; // a double-single state is a compensated pair: stored below
                    }
                    if (!(flags & FLAG_DOUBLE_REPR)) {
                        float hi[8], lo[8];
#pragma unroll
                        for (int m = 0; m < 8; ++m) {
                            if (dbl) {
                                Z::to_pair(yd[m], hi[m], lo[m]);
                            } else {
                                hi[m] = yf[m];
                                lo[m] = cf[m];
                            }
                        }
                        st_f4(v.X, id, hi[0], hi[1], hi[2], hi[3]);
                        st_f4(v.K, id, hi[4], hi[5], hi[6], hi[7]);
                        st_f4(v.CX, id, lo[0], lo[1], lo[2], lo[3]);
                        st_f4(v.CK, id, lo[4], lo[5], lo[6], lo[7]);
                        if (status != GRAY_RAY_ACTIVE)
                            st_f4(v.F, id, Z::to_float(find[0]), Z::to_float(find[1]), Z::to_float(find[2]),
                                  Z::to_float(find[3]));
                    }
                    v.S0[id] = make_int4(status, steps, euler, remaps);
                    v.S1[id] = make_int4(n64, epoch, used, flags);
                    has = false;
                }
            }
            if (RETURN) {
                int rank;
                const unsigned long long rb = warp_count(&A.ws->demoted, ret, lane, &rank);
                if (ret)
                    v.R[rb + rank] = (int)id;
            }
        }
    }
    warp_stats<double>(A, lane, tot_steps, tot_euler, tot_fp64, true);
}

// Mark rays as empty slots (never traced, never counted as active).
__global__ void clear_kernel(StateView v, int64_t first, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    v.S0[first + i] = make_int4(GRAY_RAY_EMPTY, 0, 0, 0);
    v.S1[first + i] = make_int4(0, 0, 0, 0);
}

// ACTIVE rays of each range (first, count): one block per range.
// Per range of rays (one block each): the number of ACTIVE rays and the
// steps all of them have taken, written to out[2 k] and out[2 k + 1].  A
// range is clipped to the buffer [0, n) (ranges may live in device memory,
// where the host cannot check them).
__global__ void range_stats_kernel(const int4 *S0, int64_t n, const long long *ranges, unsigned long long *out)
{
    long long first = ranges[2 * blockIdx.x], len = ranges[2 * blockIdx.x + 1];
    if (first < 0) {
        len += first;
        first = 0;
    }
    if (len > n - first)
        len = n - first;
    unsigned long long act = 0, steps = 0;
    for (long long i = threadIdx.x; i < len; i += blockDim.x) {
        const int4 s0 = S0[first + i];
        act += (s0.x == GRAY_RAY_ACTIVE);
        steps += (unsigned long long)(s0.x == GRAY_RAY_EMPTY ? 0 : s0.y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        act += __shfl_xor_sync(0xffffffffu, act, off);
        steps += __shfl_xor_sync(0xffffffffu, steps, off);
    }
    __shared__ unsigned long long part[2][32];
    if ((threadIdx.x & 31) == 0) {
        part[0][threadIdx.x >> 5] = act;
        part[1][threadIdx.x >> 5] = steps;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0, u = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t += part[0][w];
            u += part[1][w];
        }
        out[2 * blockIdx.x] = t;
        out[2 * blockIdx.x + 1] = u;
    }
}

// Rays still ACTIVE (for the per-call statistics).
__global__ void count_active_kernel(const int4 *S0, int64_t n, unsigned long long *out)
{
    unsigned long long mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mine += (S0[i].x == GRAY_RAY_ACTIVE);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        mine += __shfl_xor_sync(0xffffffffu, mine, off);
    if ((threadIdx.x & 31) == 0 && mine)
        atomicAdd(out, mine);
}

// --------------------------------------------------------------------------
// Planning: longest-first order of the rays of a set of images
// --------------------------------------------------------------------------
//
// A ray's cost (its number of steps) varies by an order of magnitude across
// an image (rays grazing a pole or the photon orbit take longest), and a
// persistent queue finishes only when its last long ray does; a long ray
// taken from the queue late therefore sets the length of the whole launch.
// gray_plan traces a sparse probe grid first (every stride-th pixel in both
// directions, with a small step budget), predicts each pixel's cost from the
// probes of its cell, and writes a queue of the image rays in descending
// predicted cost (a counting sort over PLAN_BUCKETS buckets).  The probe rays
// keep the progress they made.  A ray's result does not depend on its place
// in the queue.

// Buckets span predicted costs 0 .. 9 budget (a probe that spent its whole
// budget on Euler redos costs budget + 8 budget), about 3.5 steps wide at a
// 400-step budget: crawling rays are ordered by how hard they crawl, not
// lumped into one top bucket (measured: 8.06 -> 8.00 ms single-precision
// pass against 64 buckets over 0 .. 2 budget).
constexpr int PLAN_BUCKETS = 1024;
// aux layout: [0] unused, [1 ..] histogram, [1 + PLAN_BUCKETS ..] bucket offsets
constexpr int AUX_HIST = 1, AUX_OFF = 1 + PLAN_BUCKETS, AUX_WORDS = 1 + 2 * PLAN_BUCKETS;
// one more word after the planning words: the call epoch (never cleared)
constexpr int AUX_EPOCH = AUX_WORDS, AUX_CANCEL = AUX_WORDS + 1, AUX_ALLOC = AUX_WORDS + 2;

// Start a new call: epochs run 1 .. 2^31 - 2 (0 marks a ray no call touched).
__global__ void bump_epoch_kernel(unsigned long long *aux)
{
    int *e = (int *)&aux[AUX_EPOCH];
    *e = (*e % 0x7ffffffe) + 1;
}

__device__ __forceinline__ int image_of(const ImageDev *imgs, int n_images, int64_t i)
{
    int lo = 0, hi = n_images - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].first <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The probe rays of the planning pass (every stride-th pixel of every stride-th
// row of each image), one thread per probe: its queue entry, and with `setup`
// its initial state as setup_images_kernel writes it.  Probe q of the call
// lies in the last image with probe_first <= q.
__global__ void probe_rays_kernel(const ImageDev *imgs, int n_images, int64_t n_probes, int64_t first_ray,
                                  int stride, int *order, StateView v, int prec, int setup)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_probes)
        return;
    int lo = 0, hi = n_images - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].probe_first <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ImageDev im = imgs[lo];
    const int64_t per_row = (im.nx + stride - 1) / stride;
    const int64_t k = q - im.probe_first, row = (k / per_row) * stride, col = (k % per_row) * stride;
    const int64_t i = im.first + row * im.nx + col;
    order[q] = (int)(first_ray + i);
    if (setup) {
        double alpha, beta;
        image_point(im, row, col, alpha, beta);
        double y[8];
        initial_state_sc(im.M, im.a, im.r_obs, im.si, im.ci, alpha, beta, y);
        store_initial(v, prec, first_ray + i, y, im.a, im.M, im.r_obs, im.hc);
    }
}

// Predicted cost of pixel i: the largest probe cost among the 4 x 4 probes
// around its probe cell (the cell's corners and one ring beyond, so that thin
// long-ray features between probes are not missed); a probe that finished
// costs its steps, one that did not costs its steps plus eight per Euler redo
// (a ray crawling past a pole on redos is a long one).
__device__ __forceinline__ int plan_bucket(const ImageDev *imgs, int n_images, int64_t i, int64_t first_ray,
                                           int stride, int budget, const int4 *S0)
{
    const ImageDev im = imgs[image_of(imgs, n_images, i)];
    const int64_t p = i - im.first, row = p / im.nx, col = p - row * im.nx;
    const int64_t r0 = row - row % stride, c0 = col - col % stride;
    float cost = 0.0f;
    for (int dr = -1; dr < 3; ++dr)
        for (int dc = -1; dc < 3; ++dc) {
            const int64_t rr = r0 + dr * stride, cc = c0 + dc * stride;
            if (rr < 0 || cc < 0 || rr >= im.ny || cc >= im.nx)
                continue;
            const int4 q = S0[first_ray + im.first + rr * im.nx + cc];
            const float c = (q.x == GRAY_RAY_ACTIVE) ? (float)q.y + 8.0f * (float)q.z : (float)q.y;
            cost = fmaxf(cost, c);
        }
    int b = (int)(cost * ((float)PLAN_BUCKETS / 9.0f) / (float)budget);
    return b < 0 ? 0 : (b >= PLAN_BUCKETS ? PLAN_BUCKETS - 1 : b);
}

__global__ void plan_hist_kernel(const ImageDev *imgs, int n_images, int64_t total, int64_t first_ray, int stride,
                                 int budget, const int4 *S0, unsigned long long *aux)
{
    __shared__ unsigned int h[PLAN_BUCKETS];
    for (int k = threadIdx.x; k < PLAN_BUCKETS; k += blockDim.x)
        h[k] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total)
        atomicAdd(&h[plan_bucket(imgs, n_images, i, first_ray, stride, budget, S0)], 1u);
    __syncthreads();
    for (int k = threadIdx.x; k < PLAN_BUCKETS; k += blockDim.x)
        if (h[k])
            atomicAdd(&aux[AUX_HIST + k], (unsigned long long)h[k]);
}

// Offsets for descending buckets: one block of PLAN_BUCKETS threads, an
// inclusive scan (Hillis-Steele) over the buckets in descending order.
__global__ void __launch_bounds__(PLAN_BUCKETS) plan_scan_kernel(unsigned long long *aux)
{
    __shared__ unsigned long long v[2][PLAN_BUCKETS];
    const int t = threadIdx.x;                       // position in descending order
    const int b = PLAN_BUCKETS - 1 - t;              // bucket
    v[0][t] = aux[AUX_HIST + b];
    __syncthreads();
    int cur = 0;
    for (int d = 1; d < PLAN_BUCKETS; d <<= 1) {
        v[cur ^ 1][t] = v[cur][t] + (t >= d ? v[cur][t - d] : 0ull);
        cur ^= 1;
        __syncthreads();
    }
    aux[AUX_OFF + b] = v[cur][t] - aux[AUX_HIST + b]; // exclusive
}

// Neighbouring pixels mostly share a bucket: the lanes of a warp with the
// same bucket take their queue positions with one atomic (match + popc).
__global__ void plan_scatter_kernel(const ImageDev *imgs, int n_images, int64_t total, int64_t first_ray, int stride,
                                    int budget, const int4 *S0, unsigned long long *aux, int *order)
{
    const unsigned FULL = 0xffffffffu;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < total;
    const int b = valid ? plan_bucket(imgs, n_images, i, first_ray, stride, budget, S0) : -1;
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(FULL, b);
    const int leader = __ffs(peers) - 1;
    unsigned long long base = 0;
    if (valid && lane == leader)
        base = atomicAdd(&aux[AUX_OFF + b], (unsigned long long)__popc(peers));
    base = __shfl_sync(FULL, base, leader);
    if (valid)
        order[base + __popc(peers & ((1u << lane) - 1u))] = (int)(first_ray + i);
}

// --------------------------------------------------------------------------
// Read-out
// --------------------------------------------------------------------------

__device__ void load_state_double(const StateView &v, int prec, int64_t i, double *y, double *fin)
{
    if (prec == GRAY_FP64) {
        const d4 X = ld_d4(v.X, i), K = ld_d4(v.K, i), F = ld_d4(v.F, i);
        y[0] = X.x; y[1] = X.y; y[2] = X.z; y[3] = X.w;
        y[4] = K.x; y[5] = K.y; y[6] = K.z; y[7] = K.w;
        fin[0] = F.x; fin[1] = F.y; fin[2] = F.z; fin[3] = F.w;
    } else {
        const float4 X = ld_f4(v.X, i), K = ld_f4(v.K, i), F = ld_f4(v.F, i);
        fin[0] = F.x; fin[1] = F.y; fin[2] = F.z; fin[3] = F.w;
        if (prec == GRAY_FP32_KAHAN_SEL64 && (v.S1[i].w & FLAG_DOUBLE_REPR)) {
            const double2 q0 = ((const double2 *)v.X)[i], q1 = ((const double2 *)v.K)[i];
            const double2 q2 = ((const double2 *)v.CX)[i], q3 = ((const double2 *)v.CK)[i];
            y[0] = q0.x; y[1] = q0.y; y[2] = q1.x; y[3] = q1.y;
            y[4] = q2.x; y[5] = q2.y; y[6] = q3.x; y[7] = q3.y;
            return;
        }
        float4 CX = make_float4(0, 0, 0, 0), CK = CX;
        if (prec != GRAY_FP32) {
            CX = ld_f4(v.CX, i);
            CK = ld_f4(v.CK, i);
        }
        y[0] = (double)X.x - CX.x; y[1] = (double)X.y - CX.y; y[2] = (double)X.z - CX.z; y[3] = (double)X.w - CX.w;
        y[4] = (double)K.x - CK.x; y[5] = (double)K.y - CK.y; y[6] = (double)K.z - CK.z; y[7] = (double)K.w - CK.w;
        fin[0] = F.x; fin[1] = F.y; fin[2] = F.z; fin[3] = F.w;
    }
}

__global__ void render_kernel(StateView v, int prec, int64_t first, int64_t n, int kind, void *out)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n)
        return;
    const int64_t i = first + j;
    double y[8], fin[4];
    load_state_double(v, prec, i, y, fin);
    const int4 s0 = v.S0[i];
    if (kind == GRAY_RENDER_PIXELS64) {
        gray_pixel64 px;
        px.r = fin[1];
        px.theta = fin[2];
        px.phi = fin[3];
        px.status = s0.x;
        px.steps = s0.y;
        ((gray_pixel64 *)out)[j] = px;
    } else if (kind == GRAY_RENDER_PIXELS32) {
        gray_pixel32 px;
        px.r = (float)fin[1];
        px.theta = (float)fin[2];
        px.phi = (float)fin[3];
        px.status = s0.x;
        ((gray_pixel32 *)out)[j] = px;
    } else if (kind == GRAY_RENDER_RECORD) {
        double *o = (double *)out + 17 * j;
        o[0] = s0.x;
        o[1] = s0.y;
        o[2] = s0.z;
        o[3] = s0.w;
        for (int m = 0; m < 4; ++m)
            o[4 + m] = fin[m];
        for (int m = 0; m < 8; ++m)
            o[8 + m] = y[m];
        o[16] = v.S1[i].x;
    } else { // GRAY_RENDER_INVARIANTS, in double from the stored state
        const d4 p = ld_d4(v.P, i);
        const Hole<double> H = make_hole(p.x, p.y, p.z, 1.0, 1.0, 0.0);
        double s, c;
        sincos(y[2], &s, &c);
        const MetricPieces<double> m = metric_pieces(H, y[1], s, c);
        const double kt = y[4], kr = y[5], kh = y[6], kp = y[7];
        const double E = -(m.gtt * kt + m.gtp * kp);
        const double L = m.gtp * kt + m.gpp * kp;
        const double kth_low = m.gthth * kh;
        const double Q = kth_low * kth_low + c * c * (-H.a * H.a * E * E + L * L / (s * s));
        const double N = m.gtt * kt * kt + 2.0 * m.gtp * kt * kp + m.grr * kr * kr + m.gthth * kh * kh + m.gpp * kp * kp;
        double *o = (double *)out + 4 * j;
        o[0] = E;
        o[1] = L;
        o[2] = Q;
        o[3] = N;
    }
}

// Shadow moments: counts and the sums of the captured pixels' column and row
// indices per image, accumulated as 64-bit integers (exact, independent of
// the order of the atomics) directly in the caller's output records, then
// turned into area, radius and centroid.
__global__ void shadow_accum_kernel(StateView v, int64_t first, const ImageDev *imgs, int n_images, int64_t total,
                                    gray_shadow_info *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total)
        return;
    int lo = 0, hi = n_images - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].first <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ImageDev im = imgs[lo];
    const int64_t p = i - im.first;
    const int64_t row = p / im.nx, col = p - row * im.nx;
    const int st = v.S0[first + i].x;
    gray_shadow_info *o = out + lo;
    if (st == GRAY_RAY_CAPTURED) {
        atomicAdd((unsigned long long *)&o->n_captured, 1ull);
        atomicAdd((unsigned long long *)&o->alpha_c, (unsigned long long)col);
        atomicAdd((unsigned long long *)&o->beta_c, (unsigned long long)row);
    } else if (st == GRAY_RAY_ESCAPED) {
        atomicAdd((unsigned long long *)&o->n_escaped, 1ull);
    } else {
        atomicAdd((unsigned long long *)&o->n_other, 1ull);
    }
}

__global__ void shadow_final_kernel(const ImageDev *imgs, int n_images, gray_shadow_info *out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_images)
        return;
    gray_shadow_info s = out[k];
    const ImageDev im = imgs[k];
    const double cell = fabs(im.da * im.db);
    const double sum_col = (double)*(const unsigned long long *)&out[k].alpha_c;
    const double sum_row = (double)*(const unsigned long long *)&out[k].beta_c;
    s.area = (double)s.n_captured * cell;
    s.radius = sqrt(s.area / 3.14159265358979323846);
    if (s.n_captured > 0) {
        const double nc = (double)s.n_captured;
        s.alpha_c = im.a0 + (sum_col / nc + 0.5) * im.da;
        s.beta_c = im.b0 + (sum_row / nc + 0.5) * im.db;
    } else {
        s.alpha_c = 0.0;
        s.beta_c = 0.0;
    }
    out[k] = s;
}

// --------------------------------------------------------------------------
// Photon-ring metrics of polar images (Sec. 4, Eqs. 6-10)
// --------------------------------------------------------------------------

struct RingDev {
    long long first;     // first ray of the image relative to the call's first ray
    long long first_row; // first boundary row of the image
    int nx, ny;
    double R0, dR, th0, dth;
};

constexpr int RING_BLOCK = 256;
constexpr int RING_PER_THREAD = 16;
constexpr int RING_TILE = RING_BLOCK * RING_PER_THREAD;

// (score, k) packed so that the larger key has the larger score and, among
// equal scores, the smaller k (0 <= k < 2^31).
__device__ __forceinline__ long long ring_key(long long score, int k)
{
    return score * 4294967296LL + (long long)(4294967295u - (unsigned)k);
}

// One block per angle row.  The row's statuses are staged tile by tile in
// shared memory with coalesced loads; each thread owns 16 consecutive rays
// of a tile, a block scan gives the captured count before them, and each
// thread walks its rays tracking the best boundary k (the largest
// 2 C(k) - k, ties to the smallest k).  Boundary, captured count, rays on
// the wrong side and open rows go to the row's image with integer atomics.
__global__ void __launch_bounds__(RING_BLOCK) ring_rows_kernel(const int4 *S0, int64_t first_ray,
                                                                const RingDev *imgs, int n_images,
                                                                double *boundary, gray_ring_info *out)
{
    __shared__ unsigned char cap[RING_TILE];
    __shared__ int s_cnt[RING_BLOCK / 32];
    __shared__ long long s_key[RING_BLOCK / 32];
    const long long row = blockIdx.x;
    int lo = 0, hi = n_images - 1;
    while (lo < hi) { // last image with first_row <= row
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].first_row <= row)
            lo = mid;
        else
            hi = mid - 1;
    }
    const RingDev im = imgs[lo];
    const int64_t base = first_ray + im.first + (row - im.first_row) * (int64_t)im.nx;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long carry = 0;                 // captured rays before the tile
    long long best = ring_key(0, 0);     // k = 0: nothing inside
    for (int t0 = 0; t0 < im.nx; t0 += RING_TILE) {
        const int len = min(RING_TILE, im.nx - t0);
        for (int e = tid; e < len; e += RING_BLOCK)
            cap[e] = (unsigned char)(S0[base + t0 + e].x == GRAY_RAY_CAPTURED);
        __syncthreads();
        const int e0 = tid * RING_PER_THREAD, e1 = min(e0 + RING_PER_THREAD, len);
        int cnt = 0;
        for (int e = e0; e < e1; ++e)
            cnt += cap[e];
        // block exclusive scan of cnt
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += v;
        }
        if (lane == 31)
            s_cnt[warp] = incl;
        __syncthreads();
        int before = 0, tile_total = 0;
        for (int w = 0; w < RING_BLOCK / 32; ++w) {
            if (w < warp)
                before += s_cnt[w];
            tile_total += s_cnt[w];
        }
        long long C = carry + before + (incl - cnt);
        long long mine = best;
        for (int e = e0; e < e1; ++e) {
            C += cap[e];
            const int k = t0 + e + 1;
            const long long key = ring_key(2 * C - k, k);
            mine = key > mine ? key : mine;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long v = __shfl_xor_sync(0xffffffffu, mine, o);
            mine = v > mine ? v : mine;
        }
        if (lane == 0)
            s_key[warp] = mine;
        __syncthreads();
        for (int w = 0; w < RING_BLOCK / 32; ++w)
            best = s_key[w] > best ? s_key[w] : best;
        carry += tile_total;
        __syncthreads(); // cap, s_cnt and s_key are rewritten by the next tile
    }
    if (tid == 0) {
        const int k = (int)(4294967295u - (unsigned)(best & 0xffffffffLL));
        const long long score = (best - (long long)(4294967295u - (unsigned)k)) / 4294967296LL;
        const long long Ck = (score + k) / 2;
        boundary[row] = __dadd_rn(im.R0, __dmul_rn((double)k, im.dR)); // no contraction: R0 + k dR as written
        gray_ring_info *o = out + lo;
        atomicAdd((unsigned long long *)&o->n_captured, (unsigned long long)carry);
        atomicAdd((unsigned long long *)&o->n_wrong, (unsigned long long)((k - Ck) + (carry - Ck)));
        if (k == 0 || k == im.nx)
            atomicAdd(&o->n_open, 1);
    }
}

// Eqs. 6-8 from each image's boundary rows, one thread per image, in a fixed
// order: extremes of alpha_0 = R_b cos(vartheta), centre, then trapezoidal
// means over the rows' angles of R and of (R - <R>)^2.
__global__ void ring_final_kernel(const RingDev *imgs, int n_images, const double *boundary, gray_ring_info *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_images)
        return;
    const RingDev im = imgs[k];
    const double *Rb = boundary + im.first_row;
    double a_min = 0.0, a_max = 0.0;
    for (int j = 0; j < im.ny; ++j) {
        double sn, cs;
        sincos(im.th0 + (double)j * im.dth, &sn, &cs);
        const double al = Rb[j] * cs;
        a_min = (j == 0 || al < a_min) ? al : a_min;
        a_max = (j == 0 || al > a_max) ? al : a_max;
    }
    const double c = 0.5 * (a_min + a_max);
    double sum = 0.0, wsum = 0.0;
    for (int j = 0; j < im.ny; ++j) {
        double sn, cs;
        sincos(im.th0 + (double)j * im.dth, &sn, &cs);
        const double R = sqrt((Rb[j] * cs - c) * (Rb[j] * cs - c) + (Rb[j] * sn) * (Rb[j] * sn));
        const double w = (im.ny > 1 && (j == 0 || j == im.ny - 1)) ? 0.5 : 1.0;
        sum += w * R;
        wsum += w;
    }
    const double R_mean = sum / wsum;
    double var = 0.0;
    for (int j = 0; j < im.ny; ++j) {
        double sn, cs;
        sincos(im.th0 + (double)j * im.dth, &sn, &cs);
        const double R = sqrt((Rb[j] * cs - c) * (Rb[j] * cs - c) + (Rb[j] * sn) * (Rb[j] * sn));
        const double w = (im.ny > 1 && (j == 0 || j == im.ny - 1)) ? 0.5 : 1.0;
        var += w * (R - R_mean) * (R - R_mean);
    }
    gray_ring_info *o = out + k;
    o->D = fabs(c);
    o->R_mean = R_mean;
    o->A = 2.0 * sqrt(var / wsum);
    o->alpha_min = a_min;
    o->alpha_max = a_max;
    o->n_rows = im.ny;
}

// --------------------------------------------------------------------------
// Headless view: Boyer-Lindquist -> Cartesian -> camera -> point sprites
// (the interactive mode of Sec. 2, Fig. 1, without a graphics API)
// --------------------------------------------------------------------------

struct CamDev {
    double e[3], s[3], u[3], f[3]; // eye and the camera's right, up, forward unit vectors
    double k, cx, cy;              // pixels per unit (per unit of x/z in perspective), image centre
    double sprite;
    int width, height, ortho, mask;
};

__global__ void fill_kernel(unsigned *p, int64_t n, unsigned value)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        p[i] = value;
}

// Deposit one sprite at image position (x, y) with depth z.
template <typename T>
__device__ void deposit(const CamDev &c, T x, T y, T z, unsigned *count, float *depth)
{
    const T rad = (T)c.sprite;
    int i0, i1, j0, j1;
    if (rad <= T(0)) {
        i0 = i1 = (int)floor(x);
        j0 = j1 = (int)floor(y);
    } else {
        i0 = (int)ceil(x - rad - T(0.5));
        i1 = (int)floor(x + rad - T(0.5));
        j0 = (int)ceil(y - rad - T(0.5));
        j1 = (int)floor(y + rad - T(0.5));
    }
    i0 = max(i0, 0);
    j0 = max(j0, 0);
    i1 = min(i1, c.width - 1);
    j1 = min(j1, c.height - 1);
    const int zbits = __float_as_int((float)z);
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) {
            if (rad > T(0)) {
                const T dx = (T)i + T(0.5) - x, dy = (T)j + T(0.5) - y;
                if (!(dx * dx + dy * dy <= rad * rad))
                    continue;
            }
            const int64_t q = (int64_t)j * c.width + i;
            atomicAdd(count + q, 1u);
            if (depth)
                atomicMin((int *)depth + q, zbits); // positive floats order as their bits
        }
}

// One thread per ray: position (current state if active, final point if
// finished) -> Cartesian -> camera -> sprite, in T (double for FP64 buffers).
template <typename T>
__global__ void splat_kernel(StateView v, int prec, int64_t first, int64_t n, CamDev c, unsigned *count, float *depth)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n)
        return;
    const int64_t i = first + j;
    const int st = v.S0[i].x;
    if (st < 0 || st > 30 || !((c.mask >> st) & 1))
        return;
    T r, th, ph;
    if (prec == GRAY_FP64) {
        const d4 X = st == GRAY_RAY_ACTIVE ? ld_d4(v.X, i) : ld_d4(v.F, i);
        r = (T)X.y;
        th = (T)X.z;
        ph = (T)X.w;
    } else if (st != GRAY_RAY_ACTIVE) {
        const float4 F = ld_f4(v.F, i);
        r = (T)F.y;
        th = (T)F.z;
        ph = (T)F.w;
    } else if (prec == GRAY_FP32_KAHAN_SEL64 && (v.S1[i].w & FLAG_DOUBLE_REPR)) {
        const double2 q0 = ((const double2 *)v.X)[i], q1 = ((const double2 *)v.K)[i];
        r = (T)q0.y;
        th = (T)q1.x;
        ph = (T)q1.y;
    } else {
        const float4 X = ld_f4(v.X, i);
        float4 C = make_float4(0.f, 0.f, 0.f, 0.f);
        if (prec != GRAY_FP32)
            C = ld_f4(v.CX, i);
        r = (T)X.y - (T)C.y;
        th = (T)X.z - (T)C.z;
        ph = (T)X.w - (T)C.w;
    }
    const T a = (T)ld_d4(v.P, i).x;
    T sth, cth, sph, cph;
    fsincos(th, &sth, &cth);
    fsincos(ph, &sph, &cph);
    const T rho = sqrt(r * r + a * a);
    const T dx = rho * sth * cph - (T)c.e[0], dy = rho * sth * sph - (T)c.e[1], dz = r * cth - (T)c.e[2];
    const T x = dx * (T)c.s[0] + dy * (T)c.s[1] + dz * (T)c.s[2];
    const T y = dx * (T)c.u[0] + dy * (T)c.u[1] + dz * (T)c.u[2];
    const T z = dx * (T)c.f[0] + dy * (T)c.f[1] + dz * (T)c.f[2];
    if (!(z > T(0)))
        return;
    T px, py;
    if (c.ortho) {
        px = (T)c.cx + (T)c.k * x;
        py = (T)c.cy - (T)c.k * y;
    } else {
        px = (T)c.cx + (T)c.k * x / z;
        py = (T)c.cy - (T)c.k * y / z;
    }
    // off-image positions whose sprite cannot reach the image are skipped
    // before any conversion to int
    const T reach = (T)c.sprite + T(1);
    if (!(px > -reach && px < (T)c.width + reach && py > -reach && py < (T)c.height + reach))
        return;
    deposit<T>(c, px, py, z, count, depth);
}

// --------------------------------------------------------------------------
// Unit evaluations for parity tests
// --------------------------------------------------------------------------

template <typename T>
__global__ void eval_kernel(int what, const double *in, int64_t n, double *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    if (what == GRAY_EVAL_CHRISTOFFEL) {
        const double *q = in + 4 * i;
        const Hole<T> H = cast_hole<T>(make_hole(q[1], q[0], 1.0, 1.0, 1.0, 0.0));
        T G[64];
        christoffel_closed_form<T>(H, (T)q[2], (T)q[3], G);
        for (int m = 0; m < 64; ++m)
            out[64 * i + m] = (double)G[m];
    } else if (what == GRAY_EVAL_RHS) {
        const double *q = in + 10 * i;
        const Hole<T> H = cast_hole<T>(make_hole(q[1], q[0], 1.0, 1.0, 1.0, 0.0));
        T y[8];
        for (int m = 0; m < 8; ++m)
            y[m] = (T)q[2 + m];
        T acc[4];
        geodesic_accel<T>(H, y[1], y[2], y[4], y[5], y[6], y[7], acc);
        for (int m = 0; m < 4; ++m) {
            out[8 * i + m] = (double)y[4 + m];
            out[8 * i + 4 + m] = (double)acc[m];
        }
    } else if (what == GRAY_EVAL_INITIAL) {
        const double *q = in + 6 * i;
        double y[8];
        initial_state(q[0], q[1], q[2], q[3], q[4], q[5], y);
        for (int m = 0; m < 8; ++m)
            out[8 * i + m] = y[m];
    } else if (what == GRAY_EVAL_SINCOS) {
        T sv, cv;
        fsincos((T)in[i], &sv, &cv);
        out[2 * i] = (double)sv;
        out[2 * i + 1] = (double)cv;
    } else if (what == GRAY_EVAL_RECIP) {
        out[2 * i] = (double)recip((T)in[i]);
        out[2 * i + 1] = (double)recip_approx((T)in[i]);
    } else if (what == GRAY_EVAL_SINCOS_DS) {
        if constexpr (sizeof(T) == 4) {
            ds sv, cv;
            ds_sincos((float)in[i], sv, cv);
            out[2 * i] = (double)sv.hi + (double)sv.lo;
            out[2 * i + 1] = (double)cv.hi + (double)cv.lo;
        }
    } else if (what == GRAY_EVAL_NORM) {
        if constexpr (sizeof(T) == 4) {
            const double *q = in + 10 * i;
            const double M = q[0], a = q[1];
            float y1[8], c1[8];
            for (int m = 0; m < 8; ++m) {
                y1[m] = (float)q[2 + m];
                c1[m] = (float)((double)y1[m] - q[2 + m]);
            }
            float c8[8];
            hole_constants_f(a, M, 1000.0, c8);
            const Hole<float> H = make_hole_f(make_float4(c8[0], c8[1], c8[2], c8[3]),
                                              make_float4(c8[4], c8[5], c8[6], c8[7]), 1.0f, 1.0f, 0.0f);
            const Geo<float> g = geometry(H, y1[1], y1[2], -c1[1], -c1[2]);
            const float eps = 1e-3f;
            bool amb;
            const bool redo = xi_fails_flag(H, g, y1, eps, amb);
            const NormF nf = null_norm_f(H, g, y1);
            const float4 aM = make_float4(H.a, (float)(a - (double)(float)a), H.M, (float)(M - (double)(float)M));
            float iS;
            const ds nd = null_norm_ds(y1, c1, aM, iS);
            out[6 * i] = (double)nd.hi + (double)nd.lo;
            out[6 * i + 1] = (double)nf.norm;
            out[6 * i + 2] = (double)nf.size;
            out[6 * i + 3] = amb ? 1.0 : 0.0;
            out[6 * i + 4] = redo ? 1.0 : 0.0;
            out[6 * i + 5] = xi_fails_ds(y1, c1, aM, eps) ? 1.0 : 0.0;
        }
    } else if (what == GRAY_EVAL_XI) {
        const double *q = in + 10 * i;
        const Hole<T> H = cast_hole<T>(make_hole(q[1], q[0], 1.0, 1.0, 1.0, 0.0));
        T y[8];
        for (int m = 0; m < 8; ++m)
            y[m] = (T)q[2 + m];
        out[i] = (double)xi_eq4<T>(H, y);
    }
}

// --------------------------------------------------------------------------
// FMA-chain microbenchmark: the non-tensor FP32 / FP64 FMA rate that bounds
// the tracer (the denominators of its roofline), measured rather than taken
// from unit counts.  Each thread runs PEAK_CHAINS independent chains
// x <- x * m + b (contracting towards b / (1 - m), so nothing overflows);
// the chains hide the FMA latency and the sums go to a sink so the compiler
// keeps every FMA.
// --------------------------------------------------------------------------

constexpr int PEAK_CHAINS = 8;

template <typename T> __global__ void fma_peak_kernel(int64_t iters, T *sink)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const T m = T(0.9999995), b = T(1e-7);
    T x[PEAK_CHAINS];
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j)
        x[j] = T(1) + T(j) * T(1e-3) + T(threadIdx.x) * T(1e-6);
#pragma unroll 1
    for (int64_t i = 0; i < iters; i += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int j = 0; j < PEAK_CHAINS; ++j)
                x[j] = fma(x[j], m, b);
        }
    }
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j)
        acc += x[j];
    sink[tid] = acc;
}

// --------------------------------------------------------------------------
// Host helpers
// --------------------------------------------------------------------------

int cuda_err(cudaError_t e) { return e == cudaSuccess ? GRAY_OK : GRAY_ECUDA; }

// The constant table of ds_sincos on the current device, filled once per
// device (from the host: sin and cos of j/32 in double, split into the
// nearest float and the float nearest to the remainder).  A synchronous copy,
// so every later launch sees it; done at context creation (before any
// stream capture) and by gray_eval.
constexpr int kMaxTableDevices = 256;
std::atomic<int> g_sincos_table_ready[kMaxTableDevices];

int ensure_sincos_table()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxTableDevices)
        return GRAY_ECUDA;
    if (g_sincos_table_ready[dev].load(std::memory_order_acquire))
        return GRAY_OK;
    float4 t[2 * SINCOS_TABLE_HALF];
    for (int k = 0; k < 2 * SINCOS_TABLE_HALF; ++k) {
        const double x = (double)(k - SINCOS_TABLE_HALF) * 0.03125;
        const double sv = std::sin(x), cv = std::cos(x);
        const float sh = (float)sv, ch = (float)cv;
        t[k] = make_float4(sh, (float)(sv - (double)sh), ch, (float)(cv - (double)ch));
    }
    if (cudaMemcpyToSymbol(c_sincos_table, t, sizeof t) != cudaSuccess)
        return GRAY_ECUDA;
    g_sincos_table_ready[dev].store(1, std::memory_order_release);
    return GRAY_OK;
}

int check_launch()
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cuda_err(cudaGetLastError());
}

bool finite_all(std::initializer_list<double> xs)
{
    for (double x : xs)
        if (!std::isfinite(x))
            return false;
    return true;
}

int validate_options(const gray_options *o)
{
    if (!o)
        return GRAY_EINVAL;
    if (o->precision < GRAY_FP64 || o->precision > GRAY_FP32_KAHAN_SEL64)
        return GRAY_EINVAL;
    if (o->step_rule != GRAY_STEP_BENCH && o->step_rule != GRAY_STEP_EQ2)
        return GRAY_EINVAL;
    if (o->max_steps < 1)
        return GRAY_EINVAL;
    if (o->block != 0 && (o->block < 32 || o->block > 1024 || o->block % 32 != 0))
        return GRAY_EINVAL;
    if (o->blocks_per_sm < 0 || o->blocks_per_sm > 64 || o->refill < 0 || o->refill > 100000)
        return GRAY_EINVAL;
    if (o->launch != GRAY_LAUNCH_PERSISTENT && o->launch != GRAY_LAUNCH_ONE_PER_THREAD)
        return GRAY_EINVAL;
    if (o->stop_equator != 0 && o->stop_equator != 1)
        return GRAY_EINVAL;
    if ((o->zone_arith != GRAY_ZONE_DS && o->zone_arith != GRAY_ZONE_FP64) || o->reserved != 0)
        return GRAY_EINVAL;
    if (!finite_all({o->h_frac, o->h_min, o->cap_frac, o->eps_xi, o->r_esc_frac, o->r_sw}))
        return GRAY_EINVAL;
    if (!(o->h_frac > 0) || !(o->h_min > 0) || !(o->cap_frac >= 1.0) || !(o->eps_xi > 0) ||
        !(o->r_esc_frac > 0) || !(o->r_sw >= 0))
        return GRAY_EINVAL;
    return GRAY_OK;
}

int validate_image(const gray_image &im)
{
    if (!finite_all({im.a, im.M, im.r_obs, im.incl, im.alpha0, im.alpha1, im.beta0, im.beta1}))
        return GRAY_EINVAL;
    if (!(im.M >= 0) || !(im.r_obs > 0) || im.nx < 1 || im.ny < 1)
        return GRAY_EINVAL;
    if (im.M > 0 && !(std::fabs(im.a) < im.M))
        return GRAY_EINVAL;
    if (im.incl < 0 || im.incl > 3.14159265358979323846)
        return GRAY_EINVAL;
    if (im.reserved != 0)
        return GRAY_EINVAL;
    if (im.grid == GRAY_GRID_POLAR) {
        if (!(im.alpha0 >= 0) || !(im.alpha1 > im.alpha0) || (im.ny > 1 && !(im.beta1 != im.beta0)))
            return GRAY_EINVAL;
    } else if (im.grid == GRAY_GRID_CARTESIAN) {
        if (!(im.alpha1 != im.alpha0) || !(im.beta1 != im.beta0))
            return GRAY_EINVAL;
    } else {
        return GRAY_EINVAL;
    }
    return GRAY_OK;
}

int check_state(const gray_ctx *ctx, const void *state, size_t state_bytes, int64_t n_state)
{
    // ray indices are 32-bit in the queues (2^31 rays would need ~390 GB)
    if (!ctx || !state || n_state < 0 || n_state > 0x7fffffff)
        return GRAY_EINVAL;
    if (state_bytes < gray_state_bytes(n_state, ctx->opt.precision))
        return GRAY_EINVAL;
    return GRAY_OK;
}

unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// Device description of one (validated) image whose rays start `first` rays
// into the call's range.
ImageDev image_dev(const gray_image &im, int64_t first)
{
    ImageDev d;
    d.a = im.a;
    d.M = im.M;
    d.r_obs = im.r_obs;
    d.incl = im.incl;
    d.si = std::sin(im.incl);
    d.ci = std::cos(im.incl);
    d.a0 = im.alpha0;
    d.da = (im.alpha1 - im.alpha0) / im.nx;
    d.b0 = im.beta0;
    if (im.grid == GRAY_GRID_POLAR)
        d.db = im.ny > 1 ? (im.beta1 - im.beta0) / (im.ny - 1) : 0.0;
    else
        d.db = (im.beta1 - im.beta0) / im.ny;
    d.first = first;
    d.nx = im.nx;
    d.ny = im.ny;
    d.grid = im.grid;
    d.probe_first = 0;
    hole_constants_f(im.a, im.M, im.r_obs, d.hc);
    return d;
}

std::vector<ImageDev> image_table(const gray_image *images, int n_images, int64_t &total)
{
    std::vector<ImageDev> t((size_t)n_images);
    total = 0;
    for (int k = 0; k < n_images; ++k) {
        t[(size_t)k] = image_dev(images[k], total);
        total += (int64_t)images[k].nx * images[k].ny;
    }
    return t;
}

// Copy a small host table to the device on `stream` through a temporary
// buffer that is freed after the stream reaches it.
int upload_table(const void *host, size_t bytes, cudaStream_t s, void **dev)
{
    *dev = nullptr;
    if (cudaMallocAsync(dev, bytes, s) != cudaSuccess)
        return GRAY_ECUDA;
    if (cudaMemcpyAsync(*dev, host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return GRAY_ECUDA;
    return GRAY_OK;
}

} // namespace

// ==========================================================================
// C ABI
// ==========================================================================

extern "C" {

void gray_default_options(gray_options *o)
{
    if (!o)
        return;
    std::memset(o, 0, sizeof *o);
    o->precision = GRAY_FP64;
    o->step_rule = GRAY_STEP_BENCH;
    o->max_steps = 100000;
    o->block = 0;
    o->blocks_per_sm = 0;
    o->refill = 0;
    o->launch = GRAY_LAUNCH_PERSISTENT;
    o->zone_arith = GRAY_ZONE_DS;
    o->h_frac = 1.0 / 32.0;
    o->h_min = 1e-3;
    o->cap_frac = 1.01;
    o->eps_xi = 1e-3;
    o->r_esc_frac = 1.0;
    o->r_sw = 0.0;
}

size_t gray_state_bytes(int64_t n, int32_t precision)
{
    if (n < 0 || precision < GRAY_FP64 || precision > GRAY_FP32_KAHAN_SEL64)
        return 0;
    return make_layout(n, precision).total;
}

int gray_create(gray_ctx **ctx, const gray_options *opt)
{
    if (!ctx)
        return GRAY_EINVAL;
    *ctx = nullptr;
    int rc = validate_options(opt);
    if (rc)
        return rc;
    gray_ctx *c = new (std::nothrow) gray_ctx;
    if (!c)
        return GRAY_ENOMEM;
    c->opt = *opt;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return GRAY_ECUDA;
    }
    if (cudaMalloc((void **)&c->ws, sizeof(Workspace)) != cudaSuccess) {
        delete c;
        return GRAY_ENOMEM;
    }
    if (cudaMallocHost((void **)&c->ws_host, sizeof(Workspace)) != cudaSuccess) {
        cudaFree(c->ws);
        delete c;
        return GRAY_ENOMEM;
    }
    if (cudaMalloc((void **)&c->aux, AUX_ALLOC * sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(c->ws);
        cudaFreeHost(c->ws_host);
        delete c;
        return GRAY_ENOMEM;
    }
    if (cudaMemset(c->aux, 0, AUX_ALLOC * sizeof(unsigned long long)) != cudaSuccess) {
        gray_destroy(c);
        return GRAY_ECUDA;
    }
    if (cudaStreamCreateWithFlags(&c->cancel_stream, cudaStreamNonBlocking) != cudaSuccess) {
        gray_destroy(c);
        return GRAY_ECUDA;
    }
    if (ensure_sincos_table() != GRAY_OK) {
        gray_destroy(c);
        return GRAY_ECUDA;
    }
    std::memset(c->ws_host, 0, sizeof(Workspace));
    *ctx = c;
    return GRAY_OK;
}

void gray_destroy(gray_ctx *ctx)
{
    if (!ctx)
        return;
    for (int k = 0; k < 6; ++k)
        if (ctx->ev[k])
            cudaEventDestroy(ctx->ev[k]);
    if (ctx->fork)
        cudaEventDestroy(ctx->fork);
    if (ctx->join)
        cudaEventDestroy(ctx->join);
    if (ctx->side)
        cudaStreamDestroy(ctx->side);
    cudaFree(ctx->ws);
    cudaFree(ctx->aux);
    if (ctx->cancel_stream)
        cudaStreamDestroy(ctx->cancel_stream);
    cudaFreeHost(ctx->ws_host);
    delete ctx;
}

int gray_setup(gray_ctx *ctx, const gray_image *images, int32_t n_images, void *state, size_t state_bytes,
               int64_t n_state, int64_t first_ray, void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (!images || n_images < 1 || first_ray < 0)
        return GRAY_EINVAL;
    for (int k = 0; k < n_images; ++k)
        if ((rc = validate_image(images[k])))
            return rc;
    int64_t total = 0;
    std::vector<ImageDev> t = image_table(images, n_images, total);
    if (first_ray + total > n_state)
        return GRAY_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    void *dimg = nullptr;
    if ((rc = upload_table(t.data(), t.size() * sizeof(ImageDev), s, &dimg)))
        return rc;
    StateView v = make_view(state, n_state, ctx->opt.precision);
    setup_images_kernel<<<grid_for(total, 256), 256, 0, s>>>((const ImageDev *)dimg, n_images, total, first_ray, v,
                                                           ctx->opt.precision);
    rc = check_launch();
    cudaError_t e = cudaFreeAsync(dimg, s);
    if (rc)
        return rc;
    return cuda_err(e);
}

int gray_setup_rays(gray_ctx *ctx, const double *rays, int64_t n, double M, void *state, size_t state_bytes,
                    int64_t n_state, int64_t first_ray, void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (n < 0 || first_ray < 0 || first_ray + n > n_state || !std::isfinite(M) || M < 0)
        return GRAY_EINVAL;
    if (n == 0)
        return GRAY_OK;
    if (!rays)
        return GRAY_EINVAL;
    StateView v = make_view(state, n_state, ctx->opt.precision);
    setup_rays_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(rays, n, M, first_ray, v,
                                                                        ctx->opt.precision);
    return check_launch();
}

} // extern "C"

namespace {

TraceArgs make_trace_args(gray_ctx *ctx, void *state, int64_t n_state, int64_t step_budget)
{
    const gray_options &o = ctx->opt;
    TraceArgs A;
    A.v = make_view(state, n_state, o.precision);
    A.n = n_state;
    A.order = nullptr;
    A.n_queue = n_state;
    A.n_queue_dev = nullptr;
    A.budget = step_budget;
    A.max_steps = o.max_steps;
    A.refill = o.refill > 0 ? o.refill : 16;
    A.step_rule = o.step_rule;
    A.epoch_dev = (const int *)&ctx->aux[AUX_EPOCH];
    A.h_frac = o.h_frac;
    A.h_min = o.h_min;
    A.eps_xi = o.eps_xi;
    A.cap_frac = o.cap_frac;
    A.r_esc_frac = o.r_esc_frac;
    A.r_sw = o.r_sw;
    A.ws = ctx->ws;
    A.cancel = (const int *)&ctx->aux[AUX_CANCEL];
    A.one_per_thread = o.launch == GRAY_LAUNCH_ONE_PER_THREAD;
    A.stop_equator = o.stop_equator;
    A.zone_return = 0;
    return A;
}

// Persistent grid: resident blocks per SM x SMs, never more blocks than work.
unsigned persistent_grid(const gray_ctx *ctx, const void *kernel, int block, int64_t work)
{
    int per_sm = ctx->opt.blocks_per_sm;
    if (per_sm <= 0) {
        per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    int64_t want = (int64_t)per_sm * ctx->num_sms;
    const int64_t need = (work + block - 1) / block;
    if (want > need)
        want = need;
    return (unsigned)(want > 0 ? want : 1);
}

// One single- or double-precision pass over the queue of A (no zone kernel).
// A persistent single-precision pass; the probe pass takes the uncapped
// instantiation.
template <int MODE>
void launch_trace32(const gray_ctx *ctx, const TraceArgs &A, int64_t work, int block, bool probe, cudaStream_t s)
{
    if (probe)
        trace32_kernel<MODE, 168>
            <<<persistent_grid(ctx, (const void *)trace32_kernel<MODE, 168>, block, work), block, 0, s>>>(A);
    else
        trace32_kernel<MODE><<<persistent_grid(ctx, (const void *)trace32_kernel<MODE>, block, work), block, 0, s>>>(A);
}

// probe: the planner's probe pass (the uncapped instantiation).
int launch_pass(gray_ctx *ctx, const TraceArgs &A, int64_t work, cudaStream_t s, bool probe = false)
{
    if (A.one_per_thread && ctx->opt.precision != GRAY_FP64) {
        // the paper's launch (Eq. 1): n_grid = floor((n - 1) / n_block) + 1
        // blocks of n_block = 64 threads, one ray per thread, no refill
        const int nb = ctx->opt.block > 0 ? ctx->opt.block : 64;
        const unsigned grid = (unsigned)((work - 1) / nb + 1);
        switch (ctx->opt.precision) {
        case GRAY_FP32:
            trace32_kernel<GRAY_FP32><<<grid, nb, 0, s>>>(A);
            break;
        case GRAY_FP32_KAHAN:
            trace32_kernel<GRAY_FP32_KAHAN><<<grid, nb, 0, s>>>(A);
            break;
        default:
            trace32_kernel<GRAY_FP32_KAHAN_SEL64><<<grid, nb, 0, s>>>(A);
            break;
        }
        return check_launch();
    }
    const int block = ctx->opt.block > 0 ? ctx->opt.block : 128;
    switch (ctx->opt.precision) {
    case GRAY_FP64:
        // the double kernels are built for 128-thread blocks (their launch
        // bounds); the tunable block size is the single-precision pass's
        trace64_kernel<<<persistent_grid(ctx, (const void *)trace64_kernel, 128, work), 128, 0, s>>>(A);
        break;
    case GRAY_FP32:
        launch_trace32<GRAY_FP32>(ctx, A, work, block, probe, s);
        break;
    case GRAY_FP32_KAHAN:
        launch_trace32<GRAY_FP32_KAHAN>(ctx, A, work, block, probe, s);
        break;
    default:
        launch_trace32<GRAY_FP32_KAHAN_SEL64>(ctx, A, work, block, probe, s);
        break;
    }
    return check_launch();
}

} // namespace

extern "C" {

int gray_trace(gray_ctx *ctx, void *state, size_t state_bytes, int64_t n_state, const int32_t *order, int64_t n_order,
               int64_t step_budget, int64_t *n_active_host, int64_t *stats_host, void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (order ? n_order < 0 : n_order != 0)
        return GRAY_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(ctx->ws, 0, sizeof(Workspace), s) != cudaSuccess)
        return GRAY_ECUDA;
    bump_epoch_kernel<<<1, 1, 0, s>>>(ctx->aux);
    if ((rc = check_launch()))
        return rc;
    TraceArgs A = make_trace_args(ctx, state, n_state, step_budget);
    if (order) {
        A.order = order;
        A.n_queue = n_order;
    }
    const int64_t work = order ? n_order : n_state;
    ctx->ev_used[0] = ctx->ev_used[1] = false;
    if (n_state > 0 && work > 0) {
        if (ctx->timing) {
            cudaEventRecord(ctx->ev[0], s);
            ctx->ev_used[0] = true;
        }
        if ((rc = launch_pass(ctx, A, work, s)))
            return rc;
        if (ctx->timing)
            cudaEventRecord(ctx->ev[1], s);
        if (ctx->opt.precision == GRAY_FP32_KAHAN_SEL64) {
            // 1. the rays the single pass handed off, in the zone's arithmetic;
            //    those that climb out go to the return list (all counts stay
            //    on the device); 2. a single-precision pass over the return
            //    list; 3. its hand-offs, in the zone's arithmetic with a
            //    single-precision tail.
            const int block = 128; // the zone kernels' launch bounds
            // rays spend only a few steps in the zone: refill lanes often
            TraceArgs Z = A;
            Z.refill = 1;
            Z.zone_return = 1;
            TraceArgs B = A;
            B.order = A.v.R;
            B.n_queue_dev = &ctx->ws->demoted;
            if (ctx->timing) {
                cudaEventRecord(ctx->ev[2], s);
                ctx->ev_used[1] = true;
            }
            if (cudaMemsetAsync(&ctx->ws->head, 0, sizeof(unsigned long long), s) != cudaSuccess)
                return GRAY_ECUDA;
            // one block per SM: the double pipe is shared by the SM and a warp
            // instruction holds it whatever its active lanes, so few warps,
            // each draining many zone rays, waste the fewest pipe cycles on
            // partly filled warps (measured: 1.95 ms at three blocks per SM,
            // 1.53 ms at one, 2.2 ms with 64-thread blocks)
            if (ctx->opt.zone_arith == GRAY_ZONE_FP64)
                zone_kernel<true, double><<<(unsigned)ctx->num_sms, block, 0, s>>>(Z);
            else
                zone_kernel<true, ds><<<(unsigned)ctx->num_sms, block, 0, s>>>(Z);
            if ((rc = check_launch()))
                return rc;
            // the hand-off list is consumed: pass B appends to it from 0
            if (cudaMemsetAsync(&ctx->ws->head, 0, sizeof(unsigned long long), s) != cudaSuccess ||
                cudaMemsetAsync(&ctx->ws->handoff, 0, sizeof(unsigned long long), s) != cudaSuccess)
                return GRAY_ECUDA;
            if ((rc = launch_pass(ctx, B, work, s)))
                return rc;
            if (cudaMemsetAsync(&ctx->ws->head, 0, sizeof(unsigned long long), s) != cudaSuccess)
                return GRAY_ECUDA;
            Z.zone_return = 0;
            if (ctx->opt.zone_arith == GRAY_ZONE_FP64)
                zone_kernel<false, double>
                    <<<persistent_grid(ctx, (const void *)zone_kernel<false, double>, block, work), block, 0, s>>>(Z);
            else
                zone_kernel<false, ds>
                    <<<persistent_grid(ctx, (const void *)zone_kernel<false, ds>, block, work), block, 0, s>>>(Z);
            if ((rc = check_launch()))
                return rc;
            if (ctx->timing)
                cudaEventRecord(ctx->ev[3], s);
        }
    }
    if (!n_active_host && !stats_host)
        return 1;
    if (n_state > 0) {
        count_active_kernel<<<grid_for(n_state, 256) < 1024 ? grid_for(n_state, 256) : 1024, 256, 0, s>>>(
            A.v.S0, n_state, &ctx->ws->active);
        if ((rc = check_launch()))
            return rc;
    }
    // the cancel flag as the passes ended, into the workspace's last word
    if (cudaMemcpyAsync(&ctx->ws->cancel, &ctx->aux[AUX_CANCEL], sizeof(unsigned long long),
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ctx->ws_host, ctx->ws, sizeof(Workspace), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GRAY_ECUDA;
    const Workspace &w = *ctx->ws_host;
    if (n_active_host)
        *n_active_host = (int64_t)w.active;
    if (stats_host) {
        stats_host[0] = (int64_t)w.steps;
        stats_host[1] = (int64_t)w.euler;
        stats_host[2] = (int64_t)w.fp64;
        stats_host[3] = (int64_t)w.active;
    }
    if ((int)w.cancel != 0)
        return GRAY_ECANCEL;
    return w.active ? 1 : 0;
}

} // extern "C"

namespace {

// Argument checks shared by gray_plan and gray_setup_plan; fills the image
// table and its ray count.
int plan_args(gray_ctx *ctx, void *state, size_t state_bytes, int64_t n_state, const gray_image *images,
              int32_t n_images, int64_t first_ray, int32_t probe_stride, int32_t probe_budget, int32_t *order,
              size_t order_bytes, std::vector<ImageDev> &t, int64_t &total, int64_t &n_probes)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (!images || n_images < 1 || first_ray < 0 || !order || probe_stride < 1 || probe_stride > 65536 ||
        probe_budget < 1)
        return GRAY_EINVAL;
    for (int k = 0; k < n_images; ++k)
        if ((rc = validate_image(images[k])))
            return rc;
    t = image_table(images, n_images, total);
    if (first_ray + total > n_state || order_bytes < sizeof(int32_t) * (size_t)total)
        return GRAY_EINVAL;
    // each image's probes: ceil(nx / stride) per probe row, ceil(ny / stride) rows
    n_probes = 0;
    for (int k = 0; k < n_images; ++k) {
        t[(size_t)k].probe_first = (int)n_probes;
        n_probes += (int64_t)((images[k].nx + probe_stride - 1) / probe_stride) *
                    ((images[k].ny + probe_stride - 1) / probe_stride);
    }
    return GRAY_OK;
}

// The planning passes on stream s (image table `im` already on the device):
// 1. the probe list (written into the order buffer; with setup_probes the
// probe rays are set up in the same pass), 2. the probes traced under the
// probe budget, 3. predicted cost -> bucket histogram -> descending offsets
// -> queue.  Only the probe rays' states are read.
int plan_passes(gray_ctx *ctx, void *state, int64_t n_state, int32_t n_images, const ImageDev *im, int64_t total,
                int64_t n_probes, int64_t first_ray, int32_t probe_stride, int32_t probe_budget, int32_t *order,
                bool setup_probes, cudaStream_t s)
{
    int rc;
    if (cudaMemsetAsync(ctx->aux, 0, AUX_WORDS * sizeof(unsigned long long), s) != cudaSuccess ||
        cudaMemsetAsync(ctx->ws, 0, sizeof(Workspace), s) != cudaSuccess)
        return GRAY_ECUDA;
    const StateView v = make_view(state, n_state, ctx->opt.precision);
    probe_rays_kernel<<<grid_for(n_probes, 128), 128, 0, s>>>(im, n_images, n_probes, first_ray, probe_stride, order,
                                                             v, ctx->opt.precision, setup_probes ? 1 : 0);
    if ((rc = check_launch()))
        return rc;
    bump_epoch_kernel<<<1, 1, 0, s>>>(ctx->aux);
    if ((rc = check_launch()))
        return rc;
    TraceArgs A = make_trace_args(ctx, state, n_state, probe_budget);
    A.order = order;
    A.n_queue = n_probes;
    ctx->ev_used[2] = false;
    if (ctx->timing) {
        cudaEventRecord(ctx->ev[4], s);
        ctx->ev_used[2] = true;
    }
    if ((rc = launch_pass(ctx, A, n_probes, s, true)))
        return rc;
    if (ctx->timing)
        cudaEventRecord(ctx->ev[5], s);
    plan_hist_kernel<<<grid_for(total, 256), 256, 0, s>>>(im, n_images, total, first_ray, probe_stride, probe_budget,
                                                         v.S0, ctx->aux);
    if ((rc = check_launch()))
        return rc;
    plan_scan_kernel<<<1, PLAN_BUCKETS, 0, s>>>(ctx->aux);
    if ((rc = check_launch()))
        return rc;
    plan_scatter_kernel<<<grid_for(total, 256), 256, 0, s>>>(im, n_images, total, first_ray, probe_stride,
                                                            probe_budget, v.S0, ctx->aux, order);
    return check_launch();
}

} // namespace

extern "C" {

int gray_plan(gray_ctx *ctx, void *state, size_t state_bytes, int64_t n_state, const gray_image *images,
              int32_t n_images, int64_t first_ray, int32_t probe_stride, int32_t probe_budget, int32_t *order,
              size_t order_bytes, void *stream)
{
    std::vector<ImageDev> t;
    int64_t total = 0, n_probes = 0;
    int rc = plan_args(ctx, state, state_bytes, n_state, images, n_images, first_ray, probe_stride, probe_budget,
                       order, order_bytes, t, total, n_probes);
    if (rc)
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    void *dimg = nullptr;
    if ((rc = upload_table(t.data(), t.size() * sizeof(ImageDev), s, &dimg)))
        return rc;
    rc = plan_passes(ctx, state, n_state, n_images, (const ImageDev *)dimg, total, n_probes, first_ray, probe_stride,
                     probe_budget, order, false, s);
    cudaError_t e = cudaFreeAsync(dimg, s);
    if (rc)
        return rc;
    return cuda_err(e);
}

int gray_setup_plan(gray_ctx *ctx, const gray_image *images, int32_t n_images, void *state, size_t state_bytes,
                    int64_t n_state, int64_t first_ray, int32_t probe_stride, int32_t probe_budget, int32_t *order,
                    size_t order_bytes, void *stream)
{
    std::vector<ImageDev> t;
    int64_t total = 0, n_probes = 0;
    int rc = plan_args(ctx, state, state_bytes, n_state, images, n_images, first_ray, probe_stride, probe_budget,
                       order, order_bytes, t, total, n_probes);
    if (rc)
        return rc;
    int least = 0, greatest = 0;
    if (!ctx->side && (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
                       cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, greatest) != cudaSuccess))
        return GRAY_ECUDA;
    if ((!ctx->fork && cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) != cudaSuccess) ||
        (!ctx->join && cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming) != cudaSuccess))
        return GRAY_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    void *dimg = nullptr;
    if ((rc = upload_table(t.data(), t.size() * sizeof(ImageDev), s, &dimg)))
        return rc;
    const ImageDev *im = (const ImageDev *)dimg;
    StateView v = make_view(state, n_state, ctx->opt.precision);
    // the probe rays' set-up and the planning passes on the context's
    // high-priority stream, after everything queued so far on the caller's
    // stream (the image table); meanwhile the other rays' set-up (bound by
    // the double-precision pipe) fills the SMs that the probe pass (few,
    // latency-bound warps) leaves free
    {
        if (cudaEventRecord(ctx->fork, s) != cudaSuccess || cudaStreamWaitEvent(ctx->side, ctx->fork, 0) != cudaSuccess) {
            rc = GRAY_ECUDA;
        } else {
            rc = plan_passes(ctx, state, n_state, n_images, im, total, n_probes, first_ray, probe_stride, probe_budget,
                             order, true, ctx->side);
            const bool joined = cudaEventRecord(ctx->join, ctx->side) == cudaSuccess;
            if (!rc) {
                setup_images_kernel<<<grid_for(total, 256), 256, 0, s>>>(im, n_images, total, first_ray, v,
                                                                       ctx->opt.precision, probe_stride, 0);
                rc = check_launch();
            }
            // the caller's stream resumes only after the plan as well; if it
            // cannot wait for it, nothing on the side stream may outlive the
            // image table freed below
            if (!joined || cudaStreamWaitEvent(s, ctx->join, 0) != cudaSuccess) {
                cudaStreamSynchronize(ctx->side);
                if (!rc)
                    rc = GRAY_ECUDA;
            }
        }
    }
    cudaError_t e = cudaFreeAsync(dimg, s);
    if (rc)
        return rc;
    return cuda_err(e);
}

int gray_cancel(gray_ctx *ctx, int32_t on)
{
    if (!ctx)
        return GRAY_EINVAL;
    // a 4-byte word of the aux buffer (device memory), through the context's
    // non-blocking stream: it runs beside a trace in flight on any stream
    if (cudaMemsetAsync(&ctx->aux[AUX_CANCEL], 0, sizeof(unsigned long long), ctx->cancel_stream) != cudaSuccess ||
        (on && cudaMemsetAsync(&ctx->aux[AUX_CANCEL], 1, 1, ctx->cancel_stream) != cudaSuccess) ||
        cudaStreamSynchronize(ctx->cancel_stream) != cudaSuccess)
        return GRAY_ECUDA;
    return GRAY_OK;
}

int gray_set_timing(gray_ctx *ctx, int32_t on)
{
    if (!ctx)
        return GRAY_EINVAL;
    if (on && !ctx->ev[0])
        for (int k = 0; k < 6; ++k)
            if (cudaEventCreate(&ctx->ev[k]) != cudaSuccess)
                return GRAY_ECUDA;
    ctx->timing = on != 0;
    return GRAY_OK;
}

int gray_timings(gray_ctx *ctx, double *ms_host, int64_t *zone_steps_host)
{
    if (!ctx || !ms_host)
        return GRAY_EINVAL;
    for (int k = 0; k < 3; ++k) {
        ms_host[k] = -1.0;
        if (!ctx->timing || !ctx->ev_used[k])
            continue;
        float ms = 0.0f;
        if (cudaEventSynchronize(ctx->ev[2 * k + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, ctx->ev[2 * k], ctx->ev[2 * k + 1]) != cudaSuccess)
            return GRAY_ECUDA;
        ms_host[k] = ms;
    }
    if (zone_steps_host) {
        if (cudaMemcpy(ctx->ws_host, ctx->ws, sizeof(Workspace), cudaMemcpyDeviceToHost) != cudaSuccess)
            return GRAY_ECUDA;
        *zone_steps_host = (int64_t)ctx->ws_host->zone_steps;
    }
    return GRAY_OK;
}

int gray_clear(gray_ctx *ctx, void *state, size_t state_bytes, int64_t n_state, int64_t first_ray, int64_t n,
               void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (n < 0 || first_ray < 0 || first_ray + n > n_state)
        return GRAY_EINVAL;
    if (n == 0)
        return GRAY_OK;
    StateView v = make_view(state, n_state, ctx->opt.precision);
    clear_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(v, first_ray, n);
    return check_launch();
}

int gray_count_active(gray_ctx *ctx, const void *state, size_t state_bytes, int64_t n_state, const int64_t *ranges,
                      int32_t n_ranges, int64_t *counts, void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (n_ranges < 0 || (n_ranges > 0 && (!ranges || !counts)))
        return GRAY_EINVAL;
    for (int k = 0; k < n_ranges; ++k)
        if (ranges[2 * k] < 0 || ranges[2 * k + 1] < 0 || ranges[2 * k] + ranges[2 * k + 1] > n_state)
            return GRAY_EINVAL;
    if (n_ranges == 0)
        return GRAY_OK;
    cudaStream_t s = (cudaStream_t)stream;
    void *dr = nullptr, *dc = nullptr;
    if ((rc = upload_table(ranges, 2 * sizeof(int64_t) * (size_t)n_ranges, s, &dr)))
        return rc;
    if (cudaMallocAsync(&dc, 2 * sizeof(unsigned long long) * (size_t)n_ranges, s) != cudaSuccess) {
        cudaFreeAsync(dr, s);
        return GRAY_ECUDA;
    }
    StateView v = make_view((void *)state, n_state, ctx->opt.precision);
    range_stats_kernel<<<(unsigned)n_ranges, 256, 0, s>>>(v.S0, n_state, (const long long *)dr,
                                                          (unsigned long long *)dc);
    rc = check_launch();
    if (!rc && cudaMemcpy2DAsync(counts, sizeof(int64_t), dc, 2 * sizeof(int64_t), sizeof(int64_t), (size_t)n_ranges,
                                 cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = GRAY_ECUDA;
    cudaFreeAsync(dr, s);
    cudaFreeAsync(dc, s);
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess)
        rc = GRAY_ECUDA;
    return rc;
}

int gray_range_stats(gray_ctx *ctx, const void *state, size_t state_bytes, int64_t n_state, const int64_t *ranges,
                     int32_t n_ranges, int64_t *out, void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (n_ranges < 0 || (n_ranges > 0 && (!ranges || !out)))
        return GRAY_EINVAL;
    if (n_ranges == 0)
        return GRAY_OK;
    StateView v = make_view((void *)state, n_state, ctx->opt.precision);
    range_stats_kernel<<<(unsigned)n_ranges, 256, 0, (cudaStream_t)stream>>>(v.S0, n_state, (const long long *)ranges,
                                                                             (unsigned long long *)out);
    return check_launch();
}

int gray_render(gray_ctx *ctx, const void *state, size_t state_bytes, int64_t n_state, int64_t first_ray, int64_t n,
                int32_t kind, void *out, size_t out_bytes, void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (n < 0 || first_ray < 0 || first_ray + n > n_state)
        return GRAY_EINVAL;
    size_t per;
    switch (kind) {
    case GRAY_RENDER_PIXELS64: per = sizeof(gray_pixel64); break;
    case GRAY_RENDER_PIXELS32: per = sizeof(gray_pixel32); break;
    case GRAY_RENDER_RECORD: per = 17 * sizeof(double); break;
    case GRAY_RENDER_INVARIANTS: per = 4 * sizeof(double); break;
    default: return GRAY_EINVAL;
    }
    if (n == 0)
        return GRAY_OK;
    if (!out || out_bytes < per * (size_t)n)
        return GRAY_EINVAL;
    StateView v = make_view((void *)state, n_state, ctx->opt.precision);
    render_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(v, ctx->opt.precision, first_ray, n, kind, out);
    return check_launch();
}

int gray_shadow(gray_ctx *ctx, const void *state, size_t state_bytes, int64_t n_state, int64_t first_ray,
                const gray_image *images, int32_t n_images, gray_shadow_info *out, size_t out_bytes, void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (!images || n_images < 1 || first_ray < 0 || !out || out_bytes < sizeof(gray_shadow_info) * (size_t)n_images)
        return GRAY_EINVAL;
    for (int k = 0; k < n_images; ++k)
        if ((rc = validate_image(images[k])) || images[k].grid != GRAY_GRID_CARTESIAN)
            return GRAY_EINVAL;
    int64_t total = 0;
    std::vector<ImageDev> t = image_table(images, n_images, total);
    if (first_ray + total > n_state)
        return GRAY_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    void *dimg = nullptr;
    if ((rc = upload_table(t.data(), t.size() * sizeof(ImageDev), s, &dimg)))
        return rc;
    if (cudaMemsetAsync(out, 0, sizeof(gray_shadow_info) * (size_t)n_images, s) != cudaSuccess)
        return GRAY_ECUDA;
    StateView v = make_view((void *)state, n_state, ctx->opt.precision);
    shadow_accum_kernel<<<grid_for(total, 256), 256, 0, s>>>(v, first_ray, (const ImageDev *)dimg, n_images, total,
                                                            out);
    if ((rc = check_launch()))
        return rc;
    shadow_final_kernel<<<grid_for(n_images, 128), 128, 0, s>>>((const ImageDev *)dimg, n_images, out);
    rc = check_launch();
    cudaError_t e = cudaFreeAsync(dimg, s);
    if (rc)
        return rc;
    return cuda_err(e);
}

int gray_ring(gray_ctx *ctx, const void *state, size_t state_bytes, int64_t n_state, int64_t first_ray,
              const gray_image *images, int32_t n_images, gray_ring_info *out, size_t out_bytes, double *boundary,
              size_t boundary_bytes, void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (!images || n_images < 1 || first_ray < 0 || !out || out_bytes < sizeof(gray_ring_info) * (size_t)n_images)
        return GRAY_EINVAL;
    std::vector<RingDev> t((size_t)n_images);
    int64_t total = 0, rows = 0;
    for (int k = 0; k < n_images; ++k) {
        const gray_image &im = images[k];
        if ((rc = validate_image(im)) || im.grid != GRAY_GRID_POLAR)
            return GRAY_EINVAL;
        const ImageDev d = image_dev(im, total);
        RingDev &r = t[(size_t)k];
        r.first = total;
        r.first_row = rows;
        r.nx = im.nx;
        r.ny = im.ny;
        r.R0 = d.a0;
        r.dR = d.da;
        r.th0 = d.b0;
        r.dth = d.db;
        total += (int64_t)im.nx * im.ny;
        rows += im.ny;
    }
    if (first_ray + total > n_state || rows > 0x7fffffff)
        return GRAY_EINVAL;
    if (boundary && boundary_bytes < sizeof(double) * (size_t)rows)
        return GRAY_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // one stream-ordered scratch block: the image table, then (without a
    // caller buffer) the boundary rows
    const size_t table_bytes = (sizeof(RingDev) * t.size() + 255) & ~(size_t)255;
    const size_t scratch = table_bytes + (boundary ? 0 : sizeof(double) * (size_t)rows);
    void *dmem = nullptr;
    if (cudaMallocAsync(&dmem, scratch, s) != cudaSuccess)
        return GRAY_ECUDA;
    const RingDev *dimg = (const RingDev *)dmem;
    double *rb = boundary ? boundary : (double *)((char *)dmem + table_bytes);
    if (cudaMemcpyAsync(dmem, t.data(), sizeof(RingDev) * t.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(out, 0, sizeof(gray_ring_info) * (size_t)n_images, s) != cudaSuccess) {
        cudaFreeAsync(dmem, s);
        return GRAY_ECUDA;
    }
    const StateView v = make_view((void *)state, n_state, ctx->opt.precision);
    ring_rows_kernel<<<(unsigned)rows, RING_BLOCK, 0, s>>>(v.S0, first_ray, dimg, n_images, rb, out);
    rc = check_launch();
    if (!rc) {
        ring_final_kernel<<<grid_for(n_images, 128), 128, 0, s>>>(dimg, n_images, rb, out);
        rc = check_launch();
    }
    cudaError_t e = cudaFreeAsync(dmem, s);
    if (rc)
        return rc;
    return cuda_err(e);
}

int gray_splat(gray_ctx *ctx, const void *state, size_t state_bytes, int64_t n_state, int64_t first_ray, int64_t n,
               const gray_camera *cam, uint32_t *count, float *depth, size_t image_bytes, void *stream)
{
    int rc = check_state(ctx, state, state_bytes, n_state);
    if (rc)
        return rc;
    if (!cam || !count || first_ray < 0 || n < 0 || first_ray + n > n_state)
        return GRAY_EINVAL;
    if (!finite_all({cam->eye[0], cam->eye[1], cam->eye[2], cam->look[0], cam->look[1], cam->look[2], cam->up[0],
                     cam->up[1], cam->up[2], cam->fov, cam->half_height, cam->sprite}))
        return GRAY_EINVAL;
    if (cam->width < 1 || cam->height < 1 || (int64_t)cam->width * cam->height >= ((int64_t)1 << 31))
        return GRAY_EINVAL;
    if (!(cam->fov >= 0.0) || !(cam->fov < 3.14159265358979323846) || !(cam->sprite >= 0.0) ||
        !(cam->sprite <= 64.0) || (cam->fov == 0.0 && !(cam->half_height > 0.0)))
        return GRAY_EINVAL;
    const int64_t npix = (int64_t)cam->width * cam->height;
    if (image_bytes < sizeof(uint32_t) * (size_t)npix)
        return GRAY_EINVAL;
    CamDev c;
    double f[3], s3[3], u[3];
    for (int m = 0; m < 3; ++m)
        f[m] = cam->look[m] - cam->eye[m];
    const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0.0))
        return GRAY_EINVAL;
    for (int m = 0; m < 3; ++m)
        f[m] /= fl;
    s3[0] = f[1] * cam->up[2] - f[2] * cam->up[1];
    s3[1] = f[2] * cam->up[0] - f[0] * cam->up[2];
    s3[2] = f[0] * cam->up[1] - f[1] * cam->up[0];
    const double sl = std::sqrt(s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2]);
    if (!(sl > 1e-12))
        return GRAY_EINVAL; // up parallel to the viewing direction
    for (int m = 0; m < 3; ++m)
        s3[m] /= sl;
    u[0] = s3[1] * f[2] - s3[2] * f[1];
    u[1] = s3[2] * f[0] - s3[0] * f[2];
    u[2] = s3[0] * f[1] - s3[1] * f[0];
    for (int m = 0; m < 3; ++m) {
        c.e[m] = cam->eye[m];
        c.s[m] = s3[m];
        c.u[m] = u[m];
        c.f[m] = f[m];
    }
    c.ortho = cam->fov == 0.0;
    c.k = c.ortho ? 0.5 * cam->height / cam->half_height : 0.5 * cam->height / std::tan(0.5 * cam->fov);
    c.cx = 0.5 * cam->width;
    c.cy = 0.5 * cam->height;
    c.sprite = cam->sprite;
    c.width = cam->width;
    c.height = cam->height;
    c.mask = cam->status_mask;
    cudaStream_t st = (cudaStream_t)stream;
    if (cam->clear) {
        if (cudaMemsetAsync(count, 0, sizeof(uint32_t) * (size_t)npix, st) != cudaSuccess)
            return GRAY_ECUDA;
        if (depth) {
            fill_kernel<<<grid_for(npix, 256), 256, 0, st>>>((unsigned *)depth, npix, 0x7f800000u);
            if ((rc = check_launch()))
                return rc;
        }
    }
    if (n == 0)
        return GRAY_OK;
    const StateView v = make_view((void *)state, n_state, ctx->opt.precision);
    if (ctx->opt.precision == GRAY_FP64)
        splat_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(v, ctx->opt.precision, first_ray, n, c, count, depth);
    else
        splat_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(v, ctx->opt.precision, first_ray, n, c, count, depth);
    return check_launch();
}

int gray_eval(int32_t what, int32_t precision, const double *in, int64_t n, double *out, void *stream)
{
    if (what < GRAY_EVAL_CHRISTOFFEL || what > GRAY_EVAL_NORM || n < 0)
        return GRAY_EINVAL;
    if (precision != GRAY_FP64 && precision != GRAY_FP32)
        return GRAY_EINVAL;
    if (what >= GRAY_EVAL_SINCOS_DS && precision != GRAY_FP32)
        return GRAY_EINVAL; // the double-single evaluations exist in single precision only
    if (n == 0)
        return GRAY_OK;
    if (!in || !out)
        return GRAY_EINVAL;
    if (ensure_sincos_table() != GRAY_OK)
        return GRAY_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == GRAY_FP64)
        eval_kernel<double><<<grid_for(n, 128), 128, 0, s>>>(what, in, n, out);
    else
        eval_kernel<float><<<grid_for(n, 128), 128, 0, s>>>(what, in, n, out);
    return check_launch();
}

int gray_fma_peak(int32_t precision, int32_t blocks, int32_t threads, int64_t iters, void *sink, size_t sink_bytes,
                  void *stream)
{
    if (precision != GRAY_FP64 && precision != GRAY_FP32)
        return GRAY_EINVAL;
    if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 8 || iters % 8 != 0)
        return GRAY_EINVAL;
    const size_t per = precision == GRAY_FP64 ? sizeof(double) : sizeof(float);
    if (!sink || sink_bytes < per * (size_t)blocks * (size_t)threads)
        return GRAY_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == GRAY_FP64)
        fma_peak_kernel<double><<<blocks, threads, 0, s>>>(iters, (double *)sink);
    else
        fma_peak_kernel<float><<<blocks, threads, 0, s>>>(iters, (float *)sink);
    return check_launch();
}

// ---- setup without allocation ---------------------------------------------
// The image table of gray_setup_noalloc lives in this file-scope device
// array; host code reaches it only through the address that
// cudaGetSymbolAddress returns for the current device (cached per device).
static __device__ __align__(256) ImageDev g_noalloc_images[GRAY_NOALLOC_MAX_IMAGES];

namespace {
constexpr int kMaxDevices = 256;
std::atomic<void *> g_noalloc_addr[kMaxDevices];
} // namespace

int gray_setup_noalloc(int32_t precision, const gray_image *images, int32_t n_images, void *state,
                       size_t state_bytes, int64_t n_state, int64_t first_ray, void *stream)
{
    if (precision < GRAY_FP64 || precision > GRAY_FP32_KAHAN_SEL64)
        return GRAY_EINVAL;
    // ray indices are 32-bit in the work queues, as in gray_setup
    if (!images || n_images < 1 || n_images > GRAY_NOALLOC_MAX_IMAGES || !state || n_state < 0 ||
        n_state > 0x7fffffff || first_ray < 0)
        return GRAY_EINVAL;
    if (state_bytes < gray_state_bytes(n_state, precision))
        return GRAY_EINVAL;
    int rc;
    int64_t total = 0;
    for (int k = 0; k < n_images; ++k) {
        if ((rc = validate_image(images[k])))
            return rc;
        total += (int64_t)images[k].nx * images[k].ny;
    }
    if (first_ray + total > n_state)
        return GRAY_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return GRAY_ECUDA;
    void *table = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!table) {
        if (cudaGetSymbolAddress(&table, g_noalloc_images) != cudaSuccess || !table)
            return GRAY_ECUDA;
        g_noalloc_addr[dev].store(table, std::memory_order_release);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Fill the table in chunks through a small stack buffer: a copy from
    // pageable memory has consumed its source when cudaMemcpyAsync returns.
    constexpr int kChunk = 64;
    ImageDev chunk[kChunk];
    int64_t first = 0;
    for (int k0 = 0; k0 < n_images; k0 += kChunk) {
        const int m = (n_images - k0) < kChunk ? (n_images - k0) : kChunk;
        for (int j = 0; j < m; ++j) {
            const gray_image &im = images[k0 + j];
            chunk[j] = image_dev(im, first);
            first += (int64_t)im.nx * im.ny;
        }
        if (cudaMemcpyAsync((ImageDev *)table + k0, chunk, sizeof(ImageDev) * (size_t)m, cudaMemcpyHostToDevice,
                            s) != cudaSuccess)
            return GRAY_ECUDA;
    }
    StateView v = make_view(state, n_state, precision);
    setup_images_kernel<<<grid_for(total, 256), 256, 0, s>>>((const ImageDev *)table, n_images, total, first_ray, v,
                                                           precision);
    return check_launch();
}

const char *gray_strerror(int code)
{
    switch (code) {
    case GRAY_OK: return "success";
    case 1: return "rays remain active after the step budget";
    case GRAY_EINVAL: return "invalid argument";
    case GRAY_ECUDA: return "CUDA runtime error";
    case GRAY_ENOMEM: return "out of memory";
    case GRAY_ECANCEL: return "trace cancelled by gray_cancel";
    default: return "unknown error code";
    }
}

int64_t gray_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

} // extern "C"
