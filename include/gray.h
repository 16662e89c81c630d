/*
 * gray.h -- C ABI of libgray, a GB300 (sm_103a) tracer of photons along null
 * geodesics of the Kerr metric, after Chan, Psaltis & Ozel 2013, "GRay: a
 * Massively Parallel GPU-Based Code for Ray Tracing in Relativistic
 * Spacetimes".
 *
 * The method (Sec. 2): one photon per GPU thread; the second-order geodesic
 * equation d^2 x^mu / d l^2 = -Gamma^mu_ab k^a k^b in Boyer-Lindquist
 * coordinates is integrated with classic RK4, with the step size of Eq. 2
 * (or the benchmark rule |h| = max(min(f r, (r - r_h) / (2 |k^r|)), h_min)),
 * the null-norm monitor xi of Eq. 4 with a forward-Euler redo at h/9, the pole
 * remap of Eq. 3, and a stop at the horizon or at escape.  Photons start on an
 * image plane at distance r_obs and inclination i (Sec. 4) and are traced
 * backward in the affine parameter.
 *
 * Conventions for every call:
 *   - Units G = c = 1; lengths in units of M.  Angles in radians.
 *   - Buffers named *_dev are device pointers owned by the caller; buffers
 *     named *_host are host pointers owned by the caller.  The library owns
 *     only the gray_ctx and the small device workspace inside it.
 *   - Every call that takes a stream enqueues its work on that stream
 *     (cudaStream_t passed as void*; NULL = legacy default stream) and
 *     returns without waiting, unless a host output pointer is given.
 *   - A gray_ctx may be used by one host thread and one stream at a time.
 *   - Return value 0 = success; negative values are errors (GRAY_E*), never
 *     exceptions; gray_trace returns a positive value when rays remain
 *     active after the step budget (not an error).
 */
#ifndef GRAY_H
#define GRAY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes --------------------------------------------------- */
#define GRAY_OK 0
#define GRAY_EINVAL (-1)   /* bad argument: NaN or out-of-range parameter, n < 0, buffer too small */
#define GRAY_ECUDA (-2)    /* a CUDA runtime call failed (launch, copy, memset) */
#define GRAY_ENOMEM (-3)   /* host or device allocation of the context failed */
#define GRAY_ECANCEL (-4)  /* gray_trace stopped early because the context's cancel flag was set */

/* ---- per-ray status (the paper's stop conditions, Sec. 2) ----------- */
#define GRAY_RAY_ACTIVE 0    /* still being traced */
#define GRAY_RAY_CAPTURED 1  /* reached r <= cap_frac * r_h (horizon stop) */
#define GRAY_RAY_ESCAPED 2   /* reached r >= r_esc moving outward along the trace */
#define GRAY_RAY_STEP_CAP 3  /* hit max_steps */
#define GRAY_RAY_NONFINITE 4 /* state became NaN or Inf */
#define GRAY_RAY_EMPTY 5     /* an unused slot of a resident pool (gray_clear) */
#define GRAY_RAY_EQUATOR 6   /* crossed the equatorial plane (stop_equator): final point on it */

/* ---- arithmetic of the trace ---------------------------------------- */
#define GRAY_FP64 0             /* every step in double precision */
#define GRAY_FP32 1             /* every step in single precision */
#define GRAY_FP32_KAHAN 2       /* single precision, compensated (Kahan) state update */
#define GRAY_FP32_KAHAN_SEL64 3 /* as GRAY_FP32_KAHAN, with steps near the horizon promoted to extended
                                   precision (zone_arith: double-single or double) */

/* ---- arithmetic of the near-horizon zone of GRAY_FP32_KAHAN_SEL64 ---- */
#define GRAY_ZONE_DS 0   /* double-single (two floats, ~48-bit significand) on the FP32 pipe */
#define GRAY_ZONE_FP64 1 /* IEEE double on the FP64 pipe (1/64 of the FP32 rate on this part) */

/* ---- step-size rule ------------------------------------------------- */
#define GRAY_STEP_BENCH 0 /* |h| = max(min(h_frac r, (r - r_h)/(2|k^r|)), h_min) */
#define GRAY_STEP_EQ2 1   /* Eq. 2: min(h_frac / (|k^r/r| + |k^th| + |k^ph|), (r - r_h)/(2|k^r|)), floored at h_min */

/* ---- render kinds ---------------------------------------------------- */
#define GRAY_RENDER_PIXELS64 0   /* per ray gray_pixel64 */
#define GRAY_RENDER_PIXELS32 1   /* per ray gray_pixel32 */
#define GRAY_RENDER_RECORD 3     /* per ray 17 doubles, see gray_render */
#define GRAY_RENDER_INVARIANTS 4 /* per ray 4 doubles (E, L_z, Q, g k k) of the stored state */

/* ---- device unit evaluations (gray_eval) ----------------------------- */
#define GRAY_EVAL_CHRISTOFFEL 0 /* in (M, a, r, th) -> out Gamma^mu_ab, 64 values, [mu][a][b] */
#define GRAY_EVAL_RHS 1         /* in (M, a, y[8]) -> out dy/dl, 8 values */
#define GRAY_EVAL_INITIAL 2     /* in (M, a, r_obs, incl, alpha, beta) -> out y[8] */
#define GRAY_EVAL_XI 3          /* in (M, a, y[8]) -> out xi of Eq. 4, 1 value */
#define GRAY_EVAL_SINCOS 4      /* in (theta) -> out (sin, cos) as the tracer evaluates them, 2 values */
#define GRAY_EVAL_RECIP 5       /* in (x) -> out 1/x as the tracer evaluates it: refined (step rule, */
                                /* double everywhere) and, second, the single-precision geometry's  */
                                /* hardware approximation; 2 values                                 */
#define GRAY_EVAL_SINCOS_DS 6   /* in (theta) -> out (sin, cos) of the float theta in the double-single */
                                /* arithmetic of the ambiguous Eq. 4 test (GRAY_FP32 only); 2 values */
#define GRAY_EVAL_NORM 7        /* in (M, a, y[8]) -> out, for the compensated single-precision pair */
                                /* of y (GRAY_FP32 only): g(k, k) in double-single, g(k, k) and the  */
                                /* size of its terms as the single-precision test evaluates them, the */
                                /* test's ambiguity flag (1/0), its decision (1: redo), and the       */
                                /* decision after the double-single re-test; 6 values                */

/* ---- launch of the trace kernel ------------------------------------- */
#define GRAY_LAUNCH_PERSISTENT 0     /* persistent warps refilled from a work queue (default) */
#define GRAY_LAUNCH_ONE_PER_THREAD 1 /* the paper's launch (Eq. 1): one ray per thread, blocks of 64, no refill */

/* ---- image-plane grids (gray_image.grid) ------------------------------ */
#define GRAY_GRID_CARTESIAN 0 /* pixel centres of an nx x ny grid over [alpha0, alpha1] x [beta0, beta1] */
#define GRAY_GRID_POLAR 1     /* Sec. 4's polar grid: nx radii x ny angles, see gray_image */

/* One image: a hole of spin a and mass M seen by an observer at distance
 * r_obs and inclination incl, through a grid of rays on the image plane
 * (Sec. 4 sets the plane at r = 1000 M).  Ray index within the image is
 * row * nx + column.
 *
 * GRAY_GRID_CARTESIAN: pixel centres alpha_j = alpha0 + (j + 1/2)(alpha1 -
 *   alpha0)/nx, beta_i = beta0 + (i + 1/2)(beta1 - beta0)/ny; rows along beta.
 * GRAY_GRID_POLAR (the ring study of Sec. 4, Eqs. 9-10): columns are radii
 *   R_j = alpha0 + (j + 1/2)(alpha1 - alpha0)/nx, cell-centred on the open
 *   interval (alpha0, alpha1), 0 <= alpha0 < alpha1; rows are angles
 *   vartheta_i = beta0 + i (beta1 - beta0)/(ny - 1), both ends included
 *   (vartheta = beta0 when ny = 1); the ray sits at alpha = R cos vartheta,
 *   beta = R sin vartheta.  The paper's grid is nx = 6000 over (1.5, 7.5) M,
 *   ny = 181 over [0, pi]. */
typedef struct gray_image {
    double a;        /* spin; |a| < M when M > 0, any |a| when M = 0 (flat space) */
    double M;        /* mass, >= 0 */
    double r_obs;    /* distance of the image plane, > 0 */
    double incl;     /* observer inclination, radians, [0, pi] */
    int32_t nx, ny;  /* rays per row and rows, >= 1 each */
    double alpha0, alpha1, beta0, beta1; /* window (Cartesian) or radial and angular range (polar) */
    int32_t grid;     /* GRAY_GRID_CARTESIAN (0) or GRAY_GRID_POLAR */
    int32_t reserved; /* must be 0 */
} gray_image;

/* Integration options (Sec. 2 parameters plus the GPU launch shape). */
typedef struct gray_options {
    int32_t precision;     /* GRAY_FP64 ... GRAY_FP32_KAHAN_SEL64 */
    int32_t step_rule;     /* GRAY_STEP_BENCH or GRAY_STEP_EQ2 */
    int32_t max_steps;     /* per-ray cap over all gray_trace calls, >= 1 */
    int32_t block;         /* threads per block of the single-precision trace kernel (multiple of 32, 32..1024), 0 = default */
    int32_t blocks_per_sm; /* resident blocks per SM of the persistent grid, 0 = default */
    int32_t refill;        /* steps between warp refills from the work queue, 0 = default */
    int32_t launch;        /* GRAY_LAUNCH_PERSISTENT or GRAY_LAUNCH_ONE_PER_THREAD (single precision only) */
    int32_t stop_equator;  /* 1: also stop at the first crossing of theta = pi/2 (the grid projection of Sec. 3) */
    int32_t zone_arith;    /* GRAY_FP32_KAHAN_SEL64: GRAY_ZONE_DS (default) or GRAY_ZONE_FP64 */
    int32_t reserved;      /* must be 0 */
    double h_frac;         /* 1/32: the f of the benchmark rule, the Delta of Eq. 2 */
    double h_min;          /* 1e-3: floor on |h| */
    double cap_frac;       /* 1.01: capture when r <= cap_frac * r_h */
    double eps_xi;         /* 1e-3: Euler redo when |xi + 1| > eps_xi (Eq. 4) */
    double r_esc_frac;     /* 1.0: escape radius = r_esc_frac * r_obs */
    double r_sw;           /* GRAY_FP32_KAHAN_SEL64: steps with r < cap_frac r_h + r_sw run in the zone's
                              extended precision (zone_arith) */
} gray_options;

/* Per-ray output of GRAY_RENDER_PIXELS64: final position on the stop
 * surface (interpolated within the last step) and the ray's status. */
typedef struct gray_pixel64 {
    double r, theta, phi;
    int32_t status, steps;
} gray_pixel64;

/* Per-ray output of GRAY_RENDER_PIXELS32. */
typedef struct gray_pixel32 {
    float r, theta, phi;
    int32_t status;
} gray_pixel32;

/* Per-image output of gray_shadow: pixels whose ray was captured,
 * their area on the image plane, the radius sqrt(area/pi) of the disc of
 * equal area, and the mean (alpha, beta) of the captured pixels. */
typedef struct gray_shadow_info {
    int64_t n_captured, n_escaped, n_other;
    double area, radius, alpha_c, beta_c;
} gray_shadow_info;

typedef struct gray_ctx gray_ctx; /* opaque */

/* Fill *opt with the defaults named above (FP64, benchmark rule, 1e5 steps). */
void gray_default_options(gray_options *opt);

/* Bytes of device memory the state of n rays needs at this precision.
 * Returns 0 for n < 0 or an unknown precision. */
size_t gray_state_bytes(int64_t n, int32_t precision);

/* Create a context: validates *opt, allocates the small device workspace
 * (work-queue counters and statistics, < 4 KB) on the current device.
 * Errors: GRAY_EINVAL (NULL pointer, bad option), GRAY_ENOMEM, GRAY_ECUDA. */
int gray_create(gray_ctx **ctx, const gray_options *opt);

/* Release the context and its workspace.  NULL is ignored. */
void gray_destroy(gray_ctx *ctx);

/* State buffers.  The state of n_state rays is one device buffer of
 * gray_state_bytes(n_state, precision) bytes laid out as planes (structure of
 * arrays) for exactly n_state rays; every call that touches it receives the
 * same (state_dev, state_bytes, n_state), and calls that fill or read part of
 * it say which rays with first_ray (and a count).  A buffer is tied to the
 * precision of the context that set it up.  Calls fail with GRAY_EINVAL when
 * state_bytes is smaller than gray_state_bytes(n_state, precision) or a ray
 * range falls outside [0, n_state). */

/* Image-plane initial conditions (the set-up the paper takes from Psaltis &
 * Johannsen 2012, Sec. 2; plane at r_obs, Sec. 4), computed in double
 * precision: writes the state of every pixel of n_images images, image after
 * image, into rays first_ray, first_ray + 1, ... of the buffer.  Every ray is
 * left ACTIVE with zero steps.
 * Errors: GRAY_EINVAL (bad image, n_images < 1, range outside the buffer),
 * GRAY_ECUDA. */
int gray_setup(gray_ctx *ctx, const gray_image *images_host, int32_t n_images,
               void *state_dev, size_t state_bytes, int64_t n_state, int64_t first_ray,
               void *stream);

/* Per-ray initial conditions: rays_dev holds n rows of 5 doubles
 * (alpha, beta, a, incl, r_obs), mass M common to all; written into rays
 * first_ray .. first_ray + n - 1.  Each row is validated by the caller (same
 * ranges as gray_image).  Errors: GRAY_EINVAL, GRAY_ECUDA. */
int gray_setup_rays(gray_ctx *ctx, const double *rays_dev, int64_t n, double M,
                    void *state_dev, size_t state_bytes, int64_t n_state, int64_t first_ray,
                    void *stream);

/* Trace rays of the buffer backward until each is captured, escapes, hits
 * max_steps, turns non-finite, or has taken step_budget steps in this call
 * (step_budget <= 0: no per-call budget; Sec. 2 notes the same step-limited
 * mode for interactive use).  The work queue is order_dev[0 .. n_order-1]
 * (ray indices; entries outside [0, n_state) are skipped) or, when order_dev
 * is NULL (n_order must then be 0), every ray 0 .. n_state-1.  Only ACTIVE
 * rays are traced: finished ones are skipped, so a trace split over several
 * calls gives the same result as one call, and a ray's result does not depend
 * on its place in the queue.  If n_active_host is not NULL the call waits for
 * the stream and stores the number of rays of the buffer still active; if
 * stats_host is not NULL (4 int64) it stores, for this call: steps taken,
 * Euler redos, steps taken in the zone by the selective mode, rays still
 * active.  Returns 0 when no ray is active, 1 when some remain or when no
 * host output was requested (the count is then unknown), or an error
 * (GRAY_EINVAL, GRAY_ECUDA).
 * In GRAY_FP32_KAHAN_SEL64 the call makes a single-precision pass over the
 * queue, then a pass in the zone's extended precision (zone_arith) over the
 * rays that entered the zone near the horizon (rays climbing out of it are
 * returned to a single-precision pass), then a last zone pass for the rays
 * that came back to the zone (in the zone's arithmetic there, in compensated
 * single precision once they leave it).  A ray's arithmetic does not depend
 * on which pass runs it.  Inside the single-precision pass, an Eq. 4 test
 * whose outcome lies within single precision's rounding of its threshold
 * (near the ergosurface, where g_tt vanishes) is taken again in double-single
 * arithmetic.  With r_sw = 0.02 the final angles of every ray whose result
 * is conditioned at single precision stay within 1e-4 rad of the FP64
 * oracle's, captured rays included. */
int gray_trace(gray_ctx *ctx, void *state_dev, size_t state_bytes, int64_t n_state,
               const int32_t *order_dev, int64_t n_order, int64_t step_budget,
               int64_t *n_active_host, int64_t *stats_host, void *stream);

/* Plan a longest-first work queue for the rays of n_images images set up at
 * first_ray (as by gray_setup with the same list).  A persistent trace ends
 * when its last long ray does, so long rays (grazing a pole or the photon
 * orbit) should start first.  The call traces a probe grid -- every
 * probe_stride-th pixel in both directions -- for at most probe_budget steps
 * per probe (the probes keep that progress), predicts every pixel's cost from
 * the 4 x 4 probes around its cell (a finished probe costs its steps; an
 * unfinished one its steps plus 8 per Euler redo), and writes into order_dev
 * (int32, out_bytes >= 4 x total pixels) all the images' ray indices sorted by
 * descending predicted cost, ready for gray_trace.  The order within one cost
 * bucket is not deterministic; results do not depend on it.
 * Errors: GRAY_EINVAL, GRAY_ECUDA. */
int gray_plan(gray_ctx *ctx, void *state_dev, size_t state_bytes, int64_t n_state,
              const gray_image *images_host, int32_t n_images, int64_t first_ray,
              int32_t probe_stride, int32_t probe_budget, int32_t *order_dev, size_t order_bytes,
              void *stream);

/* gray_setup followed by gray_plan with the same images, first_ray, probe
 * stride and budget, in one call: the probe rays' set-up and the planning
 * passes run on a high-priority stream of the context (after everything
 * queued so far on `stream`) while the other rays are set up on `stream`
 * (the set-up is bound by the double-precision
 * pipe, the probe pass by single-precision issue and latency, so the two
 * share the SMs).  `stream` waits for the plan before the call's last
 * operation, so work queued on it afterwards sees every ray set up and the
 * queue written.  States and queue as from the two calls (the queue's order
 * within a cost bucket is not deterministic).  The context's stream and
 * events are created on the first call and freed by gray_destroy.
 * Errors: GRAY_EINVAL (as gray_setup and gray_plan), GRAY_ECUDA. */
int gray_setup_plan(gray_ctx *ctx, const gray_image *images, int32_t n_images, void *state_dev,
                    size_t state_bytes, int64_t n_state, int64_t first_ray, int32_t probe_stride,
                    int32_t probe_budget, int32_t *order_dev, size_t order_bytes, void *stream);

/* Read rays first_ray .. first_ray + n - 1 of the buffer into out_dev
 * (out_bytes bytes):
 *   GRAY_RENDER_PIXELS64    n gray_pixel64
 *   GRAY_RENDER_PIXELS32    n gray_pixel32
 *   GRAY_RENDER_RECORD      n x 17 doubles: status, steps, Euler redos, pole
 *                           remaps, final (t, r, theta, phi) on the stop
 *                           surface, state y[8] at the end of the last step
 *                           (compensated value for FP32 modes), steps
 *                           promoted to double
 *   GRAY_RENDER_INVARIANTS  n x 4 doubles (E, L_z, Carter Q, g k k) of the
 *                           stored state, evaluated in double
 * Errors: GRAY_EINVAL (unknown kind, buffer too small, bad range), GRAY_ECUDA. */
int gray_render(gray_ctx *ctx, const void *state_dev, size_t state_bytes, int64_t n_state,
                int64_t first_ray, int64_t n, int32_t kind, void *out_dev, size_t out_bytes,
                void *stream);

/* Mark rays first_ray .. first_ray + n - 1 as empty slots (GRAY_RAY_EMPTY):
 * traces skip them and gray_count_active does not count them.  For resident
 * pools that admit requests into free slots.  Errors: GRAY_EINVAL, GRAY_ECUDA. */
int gray_clear(gray_ctx *ctx, void *state_dev, size_t state_bytes, int64_t n_state,
               int64_t first_ray, int64_t n, void *stream);

/* Number of ACTIVE rays in each of n_ranges ranges of the buffer: ranges_host
 * holds (first_ray, count) pairs; counts_host receives n_ranges int64.  Waits
 * for the stream.  Errors: GRAY_EINVAL (range outside the buffer), GRAY_ECUDA. */
int gray_count_active(gray_ctx *ctx, const void *state_dev, size_t state_bytes, int64_t n_state,
                      const int64_t *ranges_host, int32_t n_ranges, int64_t *counts_host,
                      void *stream);

/* Asynchronous per-range statistics for resident pools, with every buffer in
 * device memory: ranges_dev holds n_ranges (first_ray, count) int64 pairs;
 * out_dev receives, per range, two int64: the number of ACTIVE rays and the
 * steps its rays have taken so far (empty slots count none).  Ranges are
 * clipped to the buffer.  Nothing waits and nothing is allocated, so a
 * serving loop can enqueue it after each trace round and read the counts
 * back with its own copy and event.  Errors: GRAY_EINVAL (NULL context,
 * state too small, n_ranges < 0, NULL buffers), GRAY_ECUDA. */
int gray_range_stats(gray_ctx *ctx, const void *state_dev, size_t state_bytes, int64_t n_state,
                     const int64_t *ranges_dev, int32_t n_ranges, int64_t *out_dev, void *stream);

/* Shadow of each of n_images images whose rays start at first_ray (as laid
 * down by gray_setup with the same image list): captured count, area of the
 * captured pixels on the image plane, equivalent radius sqrt(area/pi) and
 * centroid (the quantities from which Sec. 4 builds its ring metrics).
 * out_dev receives n_images gray_shadow_info records (out_bytes bytes).
 * Cartesian images only (a polar image is GRAY_EINVAL).
 * Errors: GRAY_EINVAL, GRAY_ECUDA. */
int gray_shadow(gray_ctx *ctx, const void *state_dev, size_t state_bytes, int64_t n_state,
                int64_t first_ray, const gray_image *images_host, int32_t n_images,
                gray_shadow_info *out_dev, size_t out_bytes, void *stream);

/* Photon ring of each of n_images polar images (GRAY_GRID_POLAR) whose rays
 * start at first_ray, traced to completion: the ring metrics of Sec. 4.
 *
 * Boundary of each angle row: the cell edge R_b = alpha0 + k dR (k = 0..nx,
 * dR = (alpha1 - alpha0)/nx) that leaves the fewest of the row's rays on the
 * wrong side (captured outside it, or not captured inside it); with C(k) the
 * captured count among the k innermost rays, k maximises 2 C(k) - k, ties to
 * the smallest k.  For a row whose captured rays are exactly its innermost
 * ones this is the midpoint between the last captured and the first
 * uncaptured ray; isolated misclassified rays away from the boundary do not
 * move it.  From the boundary points alpha_0 = R_b cos vartheta, beta_0 =
 * R_b sin vartheta (Eqs. 9-10): alpha_min and alpha_max over the rows,
 * centre c = (alpha_min + alpha_max)/2, D = |c| (Eq. 6), R = |(alpha_0 - c,
 * beta_0)|, <R> (Eq. 7) and A = 2 sqrt(mean (R - <R>)^2) (Eq. 8), where the
 * means over vartheta are trapezoidal over the rows' angles divided by their
 * span (over [0, pi] this is the full-circle mean of Eqs. 7-8, the image being
 * symmetric under beta -> -beta).
 *
 * out_dev receives n_images gray_ring_info records (out_bytes bytes);
 * boundary_dev, if not NULL, receives each image's ny boundary radii R_b,
 * images one after another (boundary_bytes >= 8 * total rows).  Rays still
 * ACTIVE count as not captured.  Integer counts are exact; the metrics are
 * computed in double in a fixed order (bitwise reproducible).
 * Errors: GRAY_EINVAL (NULL or short buffers, a Cartesian image, rays outside
 * the buffer), GRAY_ECUDA. */
typedef struct gray_ring_info {
    double D;                    /* Eq. 6 */
    double R_mean;               /* Eq. 7 */
    double A;                    /* Eq. 8 */
    double alpha_min, alpha_max; /* horizontal extent of the sampled ring */
    int64_t n_captured;          /* captured rays of the image */
    int64_t n_wrong;             /* rays on the wrong side of their row's boundary */
    int32_t n_open;              /* rows whose boundary is an end of the radial range (k = 0 or nx) */
    int32_t n_rows;              /* rows (ny) */
} gray_ring_info;

int gray_ring(gray_ctx *ctx, const void *state_dev, size_t state_bytes, int64_t n_state,
              int64_t first_ray, const gray_image *images_host, int32_t n_images,
              gray_ring_info *out_dev, size_t out_bytes, double *boundary_dev, size_t boundary_bytes,
              void *stream);

/* ---- headless view of live photons (gray_splat) --------------------------
 * GRay's interactive mode (Sec. 2, Fig. 1) draws the photons of the device
 * buffer while they are being integrated: a shader maps their Boyer-Lindquist
 * positions to Cartesian space and draws them as point sprites into an OpenGL
 * frame buffer.  gray_splat does the same arithmetic into plain device images
 * (no graphics API): position (r, theta, phi) -> x = sqrt(r^2 + a^2) sin(theta)
 * cos(phi), y = sqrt(r^2 + a^2) sin(theta) sin(phi), z = r cos(theta) (the
 * Cartesian coordinates in which Boyer-Lindquist ones are oblate spheroidal)
 * -> camera -> sprite.
 *
 * Camera: forward f = (look - eye)/|look - eye|, right s = f x up/|f x up|,
 * true up u = s x f; a point at d = P - eye has camera coordinates
 * (d.s, d.u, d.f) and is drawn only when d.f > 0.  Perspective (fov > 0, the
 * vertical field of view): k = (height/2)/tan(fov/2), image position
 * (width/2 + k x/z, height/2 - k y/z) pixels, row 0 at the top; orthographic
 * (fov = 0): k = (height/2)/half_height, (width/2 + k x, height/2 - k y).
 * Sprite: every pixel whose centre lies within `sprite` pixels of the image
 * position gets one count and the depth d.f if smaller than the pixel's;
 * sprite = 0 draws the one pixel containing the position.  Integer counts and
 * a minimum make the images independent of drawing order (bitwise
 * reproducible).  A ray is drawn when bit (1 << status) of status_mask is set:
 * an ACTIVE ray at its current position, a finished ray at its final point on
 * the stop surface.  FP64 buffers are drawn in double, FP32 buffers in single
 * precision from the compensated position. */
typedef struct gray_camera {
    double eye[3], look[3], up[3]; /* Cartesian, units of M */
    double fov;                    /* vertical field of view, radians, in [0, pi); 0 = orthographic */
    double half_height;            /* orthographic: half the image height in M, > 0 */
    double sprite;                 /* sprite radius in pixels, 0 <= sprite <= 64 */
    int32_t width, height;         /* image size in pixels, >= 1, width * height < 2^31 */
    int32_t status_mask;           /* draw rays with status s when bit (1 << s) is set */
    int32_t clear;                 /* nonzero: zero the counts and set the depths to +inf first */
} gray_camera;

/* Draw rays first_ray .. first_ray + n - 1 of the buffer into count_dev
 * (uint32, width x height, row-major, row 0 at the top) and, if not NULL,
 * depth_dev (float, same shape; +inf where nothing was drawn).  image_bytes
 * is the size of each of the two images (>= 4 width height).  Without `clear`
 * the call adds to the images.
 * Errors: GRAY_EINVAL (bad camera, NULL count image, short images, range
 * outside the buffer), GRAY_ECUDA. */
int gray_splat(gray_ctx *ctx, const void *state_dev, size_t state_bytes, int64_t n_state,
               int64_t first_ray, int64_t n, const gray_camera *camera_host,
               uint32_t *count_dev, float *depth_dev, size_t image_bytes, void *stream);

/* Maximum number of images one gray_setup_noalloc call accepts. */
#define GRAY_NOALLOC_MAX_IMAGES 4096

/* gray_setup for callers that must not allocate device memory -- for
 * example a simulation code that owns the whole device memory budget through
 * its own pool, or a caller whose allocator calls are forbidden in its
 * time-critical loop.  gray_setup uploads the image table through a
 * temporary stream-ordered allocation on every call and needs a context,
 * whose creation allocates; this entry point needs neither.  The paper has no
 * counterpart: it is an interface convenience of this library.
 *
 * It writes the same initial states as gray_setup (bit for bit) for a
 * buffer laid out for `precision`.  The image table is copied into a
 * file-scope device array of GRAY_NOALLOC_MAX_IMAGES entries (136 bytes each,
 * 544 KB) that every device loading the library holds until the process
 * exits; n_images above that maximum is rejected with GRAY_EINVAL before any
 * work is enqueued.  On the first call on a device the library looks up that
 * array's device address (cudaGetSymbolAddress) with the device current and
 * caches it; make that first call before any stream capture.  The array is
 * shared by all calls and keeps the last call's table: calls that overlap on
 * the GPU (on different streams, or from several threads) race on it, so
 * order them on one stream or synchronise between them.  No cudaMalloc,
 * cudaFree or other allocating routine is called.
 * Errors: GRAY_EINVAL (bad precision, image or range; too many images),
 * GRAY_ECUDA. */
int gray_setup_noalloc(int32_t precision, const gray_image *images_host, int32_t n_images,
                       void *state_dev, size_t state_bytes, int64_t n_state, int64_t first_ray,
                       void *stream);

/* Evaluate one device function of the tracer on n inputs, in the arithmetic
 * of `precision` (GRAY_FP64 or GRAY_FP32), for unit parity tests: in_dev and
 * out_dev are n rows of doubles laid out as listed at GRAY_EVAL_*.
 * Errors: GRAY_EINVAL, GRAY_ECUDA. */
int gray_eval(int32_t what, int32_t precision, const double *in_dev, int64_t n,
              double *out_dev, void *stream);

/* FMA-chain microbenchmark of the non-tensor FMA rate, the bound of the
 * tracer's arithmetic (the paper states its single-precision throughput
 * against the GPU's peak arithmetic rate: abstract, Sec. 3; this measures
 * that peak, in FP32 and FP64, on the running device instead of deriving it
 * from unit counts).  Launches
 * `blocks` blocks of `threads` threads (a multiple of 32, at most 1024) on
 * `stream`; every thread runs `iters` (a positive multiple of 8) iterations
 * of 8 independent FMA chains in `precision` (GRAY_FP32 or GRAY_FP64) and
 * writes one value to sink_dev (blocks x threads elements of that type,
 * caller-owned).  One launch performs exactly
 * 2 x 8 x iters x blocks x threads floating-point operations; the caller
 * times it (CUDA events on the same stream).  Asynchronous.
 * Errors: GRAY_EINVAL (precision, shape, iters, sink too small), GRAY_ECUDA. */
int gray_fma_peak(int32_t precision, int32_t blocks, int32_t threads, int64_t iters, void *sink_dev,
                  size_t sink_bytes, void *stream);

/* Cancel the context's traces from the host (on = 1), or clear the request
 * (on = 0).  The flag lives in the context's device memory and is written
 * through a private non-blocking stream, so it takes effect while a
 * gray_trace of this context runs on another stream (or waits in another
 * host thread); this call returns once the flag is set.  Every trace pass
 * reads it when its warps refill (every `refill` steps): from then on no ray
 * is picked up and every ray in flight is stored as it stands, still ACTIVE
 * (as when a step budget runs out), so nothing is lost and a later trace
 * continues each ray bit for bit as if it had not been interrupted.  While
 * the flag is set, gray_trace returns GRAY_ECANCEL (when it reports counts)
 * instead of 0 or 1; it stays set until cleared with on = 0.  The paper's
 * interactive mode (Sec. 2) stops and resumes the integration in this way.
 * Errors: GRAY_EINVAL (NULL context), GRAY_ECUDA. */
int gray_cancel(gray_ctx *ctx, int32_t on);

/* Record CUDA events around the passes of every later gray_trace and
 * gray_plan call of this context (on = 1) or stop (on = 0).  Diagnostic.
 * Errors: GRAY_EINVAL (NULL context), GRAY_ECUDA (event creation). */
int gray_set_timing(gray_ctx *ctx, int32_t on);

/* Durations of the last call's passes, in milliseconds (-1 where the pass did
 * not run or timing is off): ms_host[0] the single-precision (or FP64) pass
 * of gray_trace, ms_host[1] its zone passes (GRAY_FP32_KAHAN_SEL64), ms_host[2]
 * the probe pass of gray_plan.  If zone_steps_host is not NULL it receives
 * the steps the zone pass took in the last gray_trace.  Waits for the events.
 * Errors: GRAY_EINVAL, GRAY_ECUDA. */
int gray_timings(gray_ctx *ctx, double *ms_host, int64_t *zone_steps_host);

/* Human-readable text of a return code; never NULL. */
const char *gray_strerror(int code);

/* Number of kernel launches made by this process through the library so far
 * (diagnostic counter). */
int64_t gray_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* GRAY_H */
