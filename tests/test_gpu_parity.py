"""GPU parity: the CUDA tracer, called through the C ABI, against the FP64 CPU
oracle on the same seeded inputs -- unit evaluations, the Schwarzschild
image, the grid projection, and the properties every launch shape, queue
order and call split must keep.  The acceptance of whole Kerr images and of
the mixed per-ray stream against the oracle is in test_gpu_acceptance.py.

Tolerances (pixels within 0.05 M of the analytic critical curve excluded,
where rays are chaotic):
  * FP64 path: same status and step count; final angles within 1e-9
    relative (|d| <= 1e-9 max(1, |ref|));
  * FP32 paths: classification agreement >= 99.99 %; final theta, phi within
    1e-4 rad.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import parity as P
import theory as T
from paper_1303_5057_gb300 import gray
from paper_1303_5057_gb300 import inputs as I

pytestmark = pytest.mark.gpu

M = 1.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1303_5057_gb300 import build
    build.build()
    gray.lib()
    oracle.lib()
    torch.cuda.init()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def trace_image(im, opt, step_budget=0):
    tr = gray.Tracer(opt, im.n)
    tr.setup([im])
    inv0 = tr.invariants()
    rc, n_active, stats = tr.trace(step_budget)
    rec = tr.records()
    inv1 = tr.invariants()
    tr.close()
    return rec, inv0, inv1, stats


def oracle_image(im, max_steps, step_rule=oracle.STEP_BENCH):
    rays = oracle.image_rays(im.a, im.incl, im.r_obs, im.nx, im.ny, im.alpha0, im.alpha1, im.beta0, im.beta1)
    return rays, oracle.trace_many(rays, oracle.Options(M=im.M, max_steps=max_steps, step_rule=step_rule))


# ------------------------------------------------------------ unit parity ---

def _points(n=512, seed=7):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-0.999, 0.999, n)
    r = np.exp(rng.uniform(np.log(1.05), np.log(2000.0), n)) * (1 + np.sqrt(1 - a * a))
    th = rng.uniform(0.02, math.pi - 0.02, n)
    return a, r, th


@pytest.mark.parametrize("prec,tol", [(gray.FP64, 1e-12), (gray.FP32, 2e-5)])
def test_closed_form_christoffel_matches_general_formula(prec, tol):
    a, r, th = _points()
    inp = np.stack([np.full_like(a, M), a, r, th], axis=1)
    got = gray.gray_eval(gray.EVAL_CHRISTOFFEL, prec, dev(inp)).cpu().numpy().reshape(-1, 4, 4, 4)
    for k in range(len(a)):
        G = oracle.christoffel(M, a[k], r[k], th[k])
        scale = np.abs(G).max()
        assert np.abs(got[k] - G).max() <= tol * scale, (k, a[k], r[k], th[k])


@pytest.mark.parametrize("prec,tol", [(gray.FP64, 1e-11), (gray.FP32, 5e-5)])
def test_geodesic_rhs_matches_oracle(prec, tol):
    a, r, th = _points(seed=11)
    rng = np.random.default_rng(3)
    k = rng.normal(size=(len(a), 4))
    k[:, 0] = np.abs(k[:, 0]) * 3 + 1
    y = np.zeros((len(a), 8))
    y[:, 1], y[:, 2] = r, th
    y[:, 4:] = k
    inp = np.concatenate([np.stack([np.full_like(a, M), a], axis=1), y], axis=1)
    got = gray.gray_eval(gray.EVAL_RHS, prec, dev(inp)).cpu().numpy()
    for i in range(len(a)):
        ref = oracle.rhs(M, a[i], y[i])
        # terms of the contraction can cancel: compare against the size of the terms
        G = oracle.christoffel(M, a[i], r[i], th[i])
        terms = np.einsum("mab,a,b->m", np.abs(G), np.abs(k[i]), np.abs(k[i]))
        assert np.all(np.abs(got[i, 4:] - ref[4:]) <= tol * (terms + 1e-300)), i
        assert np.all(got[i, :4] == y[i, 4:].astype(np.float32 if prec == gray.FP32 else np.float64))


def test_initial_conditions_match_oracle():
    rng = np.random.default_rng(5)
    n = 400
    inp = np.stack([np.full(n, M), rng.uniform(-0.99, 0.99, n), rng.choice([1e3, 1e4], n),
                    rng.uniform(0, math.pi, n), rng.uniform(-15, 15, n), rng.uniform(-15, 15, n)], axis=1)
    got = gray.gray_eval(gray.EVAL_INITIAL, gray.FP64, dev(inp)).cpu().numpy()
    for i in range(n):
        ref = oracle.initial(*inp[i])
        assert np.allclose(got[i], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("prec,tol", [(gray.FP64, 1e-12), (gray.FP32, 1e-4)])
def test_xi_matches_oracle(prec, tol):
    rng = np.random.default_rng(9)
    rows = []
    for _ in range(200):
        a = rng.uniform(-0.99, 0.99)
        y = oracle.initial(M, a, 1000.0, rng.uniform(0.1, 3.0), rng.uniform(-9, 9), rng.uniform(-9, 9))
        y[5] *= 1 + rng.uniform(-0.01, 0.01)
        rows.append(np.concatenate([[M, a], y]))
    inp = np.array(rows)
    got = gray.gray_eval(gray.EVAL_XI, prec, dev(inp)).cpu().numpy()[:, 0]
    for i in range(len(rows)):
        ref = oracle.xi(M, inp[i, 1], inp[i, 2:])
        assert abs(got[i] - ref) <= tol * max(1.0, abs(ref))


def test_single_precision_sincos_error_bound():
    """The single-precision sin/cos the tracer evaluates, against double sin/cos
    of the same float argument: both within 4 ulp of themselves (relative, so
    1/sin and cot stay accurate near both poles and cos near the equator)."""
    rng = np.random.default_rng(4)
    th = np.concatenate([rng.uniform(-math.pi / 2, 1.5 * math.pi, 20000),
                         np.geomspace(1e-7, 1e-1, 200), math.pi - np.geomspace(1e-6, 1e-1, 200),
                         [0.0, math.pi / 2, math.pi, -1.0, 5.0, -3.0, 40.0]]).astype(np.float32).astype(np.float64)
    got = gray.gray_eval(gray.EVAL_SINCOS, gray.FP32, dev(th[:, None])).cpu().numpy()
    s_ref, c_ref = np.sin(th), np.cos(th)
    for k, ref in ((0, s_ref), (1, c_ref)):
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(got[:, k] - ref) <= 4 * ulp + 1e-45), k


@pytest.mark.parametrize("prec,ulps", [(gray.FP64, 2.0), (gray.FP32, 2.0)])
def test_reciprocal_error_bound(prec, ulps):
    """The tracer's reciprocals against the exact quotient of the same
    argument, over the magnitudes the tracer meets (Sigma Delta sin theta
    from ~1e-12 near a pole at the horizon to ~1e13 far out) and both signs:
    the refined one (hardware approximation + Newton-Raphson: one step in
    single, two in double) within `ulps`; the single-precision geometry's
    plain hardware approximation within 2 ulp (in double the two are the
    same function)."""
    rng = np.random.default_rng(6)
    x = np.concatenate([np.geomspace(1e-12, 1e13, 4000), -np.geomspace(1e-6, 1e6, 500),
                        rng.uniform(0.5, 2.0, 4000), [1.0, 3.0, 7.0, 1e-3]])
    if prec == gray.FP32:
        x = x.astype(np.float32).astype(np.float64)
    got = gray.gray_eval(gray.EVAL_RECIP, prec, dev(x[:, None])).cpu().numpy()
    ref = 1.0 / x
    if prec == gray.FP32:
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    else:
        ulp = np.spacing(np.abs(ref))
        assert np.array_equal(got[:, 0], got[:, 1])
    assert np.all(np.abs(got[:, 0] - ref) <= ulps * ulp)
    assert np.all(np.abs(got[:, 1] - ref) <= 2 * ulp)


def test_double_single_sincos_error_bound():
    """The double-single sin/cos of the ambiguous-test path (a table of sin
    and cos at multiples of 1/32 and angle addition with short series),
    against double sin/cos of the same float argument: within 2e-13 over the
    angles the tracer meets (theta in [-1, 4.5], the poles, the equator,
    multiples of pi/2)."""
    rng = np.random.default_rng(12)
    th = np.concatenate([rng.uniform(-1.0, 4.5, 20000), np.geomspace(1e-9, 0.5, 300),
                         math.pi - np.geomspace(1e-7, 0.5, 300), math.pi / 2 + np.linspace(-1e-3, 1e-3, 101),
                         [0.0, math.pi / 2, math.pi, 3 * math.pi / 2, -math.pi / 4, 3 * math.pi / 4]])
    th = th.astype(np.float32).astype(np.float64)
    got = gray.gray_eval(gray.EVAL_SINCOS_DS, gray.FP32, dev(th[:, None])).cpu().numpy()
    assert np.abs(got[:, 0] - np.sin(th)).max() <= 2e-13
    assert np.abs(got[:, 1] - np.cos(th)).max() <= 2e-13


def _compensated_states(n_rays=40, seed=13):
    """States (M, a, y) along oracle trajectories near the hole (r < 30), and
    the same states with k^r moved so that the null norm sits within a
    relative 1e-2 ... 1e-6 of the Eq. 4 threshold (the decisions the
    double-single re-test exists for)."""
    rng = np.random.default_rng(seed)
    o = oracle.Options(max_steps=10000)
    rows = []
    for _ in range(n_rays):
        a = rng.uniform(0.0, 0.999)
        y = oracle.initial(M, a, 1000.0, rng.uniform(0.05, 1.55), *rng.uniform(-8, 8, 2))
        r_h = oracle.horizon(M, a)
        for step in range(3000):
            h = oracle.step_size(o, r_h, y)
            y1, k1 = oracle.rk4(M, a, y, h)
            if abs(oracle.xi(M, a, y1) + 1) > 1e-3:
                y1 = y + (h / 9) * k1
            y, _ = oracle.remap(y1)
            if y[1] <= 1.01 * r_h or (y[1] >= 1000 and h * y[5] > 0):
                break
            if y[1] < 30 and step % 5 == 0:
                rows.append(np.concatenate([[M, a], y]))
                g = oracle.metric(M, a, y[1], y[2])
                rest = oracle.null_norm(M, a, y) - g[1, 1] * y[5] ** 2
                for rel in (1e-2, -1e-2, 1e-4, -1e-4, 1e-6, -1e-6):
                    target = 1e-3 * abs(g[0, 0]) * y[4] ** 2 * (1 + rel)
                    kr2 = (target - rest) / g[1, 1]
                    if kr2 > 0:
                        z = y.copy()
                        z[5] = math.copysign(math.sqrt(kr2), y[5])
                        rows.append(np.concatenate([[M, a], z]))
    return np.array(rows)


def test_ambiguous_eq4_test_is_retaken_in_double_single():
    """The Eq. 4 test of the compensated single-precision path, on compensated
    states of oracle trajectories and on states placed 1e-2 ... 1e-6 (relative)
    from its threshold: the double-single null norm matches the oracle's
    double one (of the state hi - lo) to 1e-10 of its terms; the single-
    precision norm stays within half the ambiguity band (2^-21 of its terms)
    of it, so every single-precision decision that could differ from the
    double one is flagged; the decision after the re-test equals the double
    decision wherever the norm is farther from the threshold than 1e-6 of it
    and 1e-9 of its terms."""
    rows = _compensated_states()
    got = gray.gray_eval(gray.EVAL_NORM, gray.FP32, dev(rows)).cpu().numpy()
    n_true = np.empty(len(rows))
    thr = np.empty(len(rows))
    for i, q in enumerate(rows):
        y = q[2:].astype(np.float32).astype(np.float64)
        lo = (y - q[2:]).astype(np.float32).astype(np.float64)
        yt = y - lo  # the compensated pair's exact value
        n_true[i] = oracle.null_norm(q[0], q[1], yt)
        thr[i] = 1e-3 * abs(oracle.metric(q[0], q[1], yt[1], yt[2])[0, 0]) * yt[4] ** 2
    size = got[:, 2]
    assert np.all(np.abs(got[:, 0] - n_true) <= 1e-10 * size)
    assert np.all(np.abs(got[:, 1] - n_true) <= 2.0 ** -21 * size)
    fails_true = ~(np.abs(n_true) <= thr)
    differ = (got[:, 4] == 1) != fails_true
    assert np.all(got[differ, 3] == 1)  # every differing single-precision decision is flagged
    clear = np.abs(np.abs(n_true) - thr) > np.maximum(1e-6 * thr, 1e-9 * size)
    assert np.all((got[clear, 5] == 1) == fails_true[clear])
    assert np.sum(got[:, 3] == 1) > 50  # the near-threshold states do exercise the re-test


# ------------------------------------------------------------- whole rays ---

def test_schwarzschild_64x64_fp64_matches_oracle():
    """Schwarzschild, i = 60 deg, 64 x 64 over [-10, 10]^2, FP64, cap 1e5."""
    wl = I.schwarzschild_64()
    im = wl.images[0]
    rec, _, _, stats = trace_image(im, gray.Options(precision=gray.FP64, max_steps=wl.max_steps))
    rays, ref = oracle_image(im, wl.max_steps)
    far = P.band_mask((rays[:, 0], rays[:, 1]), im.a, im.incl)
    assert P.class_agreement(rec, ref, far)[1] == 0
    c = P.compare(rec, ref, far & ((ref[:, 0] == oracle.CAPTURED) | (ref[:, 0] == oracle.ESCAPED)))
    assert c["status_disagree"] == 0 and c["max_rel"] <= 1e-9, c
    assert np.all(rec[far, 1] == ref[far, 1]) and np.all(rec[far, 2] == ref[far, 2])
    assert stats[0] == int(rec[:, 1].sum())


@pytest.mark.parametrize("a,incl_deg", [(0.95, 60.0), (0.0, 0.0), (0.95, 0.0)])
def test_grid_projection_matches_oracle(a, incl_deg):
    """Sec. 3 grid projection: each pixel's ray stops where it first crosses
    the equatorial plane; FP64 reproduces the oracle's status and crossing
    point (r, phi) to 1e-9; compensated FP32 with the double zone to 1e-4."""
    im = I.Image(a=a, incl=math.radians(incl_deg), nx=40, ny=36, alpha0=-12, alpha1=12, beta0=-12, beta1=12)
    rays = oracle.image_rays(im.a, im.incl, im.r_obs, im.nx, im.ny, im.alpha0, im.alpha1, im.beta0, im.beta1)
    ref = oracle.trace_many(rays, oracle.Options(max_steps=20000, stop_equator=1))
    far = P.band_mask((rays[:, 0], rays[:, 1]), a, max(im.incl, 1e-3))
    rec64, _, _, _ = trace_image(im, gray.Options(precision=gray.FP64, max_steps=20000, stop_equator=1))
    assert np.mean(ref[:, 0] == oracle.EQUATOR) > 0.5
    same = rec64[:, 0] == ref[:, 0]
    assert same[far].all()
    eq = same & (ref[:, 0] == oracle.EQUATOR)
    assert np.abs(rec64[eq, 5] - ref[eq, 5]).max() <= 1e-9 * np.abs(ref[eq, 5]).max()
    assert np.abs(P.wrap(rec64[eq, 7] - ref[eq, 7])).max() <= 1e-9
    assert np.all(rec64[eq, 6] == np.float64(math.pi / 2))
    rec32, _, _, _ = trace_image(im, gray.Options(precision=gray.FP32_KAHAN_SEL64, max_steps=20000, r_sw=0.02,
                                                  stop_equator=1))
    # single precision: every ray outside the band that the oracle resolves
    # (not chaotic, and its crossing conditioned at single precision, as in
    # the acceptance tests) keeps its status, crossing radius and phi
    R = P.Reference(rays, oracle.Options(max_steps=20000, stop_equator=1), far)
    settled = far & ~R.chaotic
    assert np.all(rec32[settled, 0] == ref[settled, 0])
    sel = R.compared("single") & (ref[:, 0] == oracle.EQUATOR)
    assert sel.sum() >= 0.9 * (far & (ref[:, 0] == oracle.EQUATOR)).sum(), R.census()
    rel = np.abs(rec32[sel, 5] - ref[sel, 5]) / ref[sel, 5]
    assert rel.max() <= 1e-4
    assert np.abs(P.wrap(rec32[sel, 7] - ref[sel, 7])).max() <= 1e-4


def test_trace_split_over_calls_equals_one_call():
    """Resumable tracing (the step-limited mode of Sec. 2): many calls with a
    small per-call budget give bit-identical records to one call."""
    im = I.Image(a=0.7, incl=math.radians(40.0), nx=20, ny=17)
    for prec in (gray.FP64, gray.FP32_KAHAN_SEL64):
        opt = gray.Options(precision=prec, max_steps=5000, r_sw=0.5, refill=3)
        one, _, _, _ = trace_image(im, opt)
        tr = gray.Tracer(opt, im.n)
        tr.setup([im])
        calls = 0
        while True:
            rc, n_active, stats = tr.trace(step_budget=37)
            calls += 1
            if n_active == 0:
                break
            assert calls < 1000
        many = tr.records()
        tr.close()
        assert calls > 5
        assert np.array_equal(one, many)


@pytest.mark.parametrize("n", [1, 31, 33, 1000])
def test_ragged_sizes(n):
    """Ray counts that are not multiples of the warp or block."""
    rng = np.random.default_rng(n)
    rays = np.stack([rng.uniform(-9, 9, n), rng.uniform(-9, 9, n), rng.uniform(0, 0.99, n),
                     rng.uniform(0.1, 1.5, n), np.full(n, 1000.0)], axis=1)
    tr = gray.Tracer(gray.Options(precision=gray.FP64, max_steps=20000), n)
    tr.setup_rays(dev(rays))
    rc, n_active, _ = tr.trace()
    rec = tr.records()
    tr.close()
    assert rc == 0 and n_active == 0
    # every ray outside its own 0.05 M band and not chaotic keeps the
    # oracle's status; the double-conditioned ones its final angles to 1e-9
    # with identical step counts
    R = P.Reference(rays, oracle.Options(max_steps=20000), P.per_ray_far(rays[:, :4]), single=False,
                    double=True)
    ref = R.ref
    settled = R.far & ~R.chaotic
    assert np.all(rec[settled, 0] == ref[settled, 0])
    sel = R.compared("double")
    assert sel.sum() >= 0.9 * settled.sum(), R.census("double")
    assert P.rel_move(rec, ref)[sel].max(initial=0.0) <= 1e-9
    assert np.all(rec[sel, 1] == ref[sel, 1])


def test_empty_and_degenerate():
    tr = gray.Tracer(gray.Options(precision=gray.FP64), 0)
    rc, n_active, stats = tr.trace()
    assert rc == 0 and n_active == 0 and stats[0] == 0
    tr.close()
    # flat space (M = 0): no capture, straight lines, same as the oracle
    im = I.Image(a=0.0, incl=1.0, nx=9, ny=7, M=0.0, alpha0=2.0, alpha1=9.0, beta0=1.0, beta1=8.0)
    rec, _, _, _ = trace_image(im, gray.Options(precision=gray.FP64))
    rays, ref = oracle_image(im, 100000)
    assert np.all(rec[:, 0] == oracle.ESCAPED) and np.all(ref[:, 0] == oracle.ESCAPED)
    assert np.abs(rec[:, 6] - ref[:, 6]).max() < 1e-10
    # the step cap: status 3 and the same state as the oracle after max_steps steps
    im2 = I.Image(a=0.5, incl=0.7, nx=4, ny=4)
    rec, _, _, _ = trace_image(im2, gray.Options(precision=gray.FP64, max_steps=25))
    rays2, ref2 = oracle_image(im2, 25)
    assert np.all(rec[:, 0] == oracle.STEP_CAP) and np.all(rec[:, 1] == 25)
    assert np.allclose(rec[:, 8:16], ref2[:, 8:16], rtol=1e-12, atol=1e-9)
    # a polar observer (i = 0): pixel centres avoid the axis itself
    im3 = I.Image(a=0.9, incl=0.0, nx=6, ny=6)
    rec3, _, _, _ = trace_image(im3, gray.Options(precision=gray.FP64, max_steps=20000))
    _, ref3 = oracle_image(im3, 20000)
    assert np.array_equal(rec3[:, 0], ref3[:, 0])


@pytest.mark.parametrize("prec", [gray.FP64, gray.FP32_KAHAN, gray.FP32_KAHAN_SEL64])
def test_planned_order_gives_identical_results(prec):
    """gray_plan's longest-first queue is a permutation of the image's rays,
    puts the predicted-long rays first, and tracing in that order (probes
    first) gives bit-identical records to tracing in natural order."""
    ims = [I.Image(a=0.99, incl=math.radians(90.0), nx=48, ny=40), I.Image(a=0.4, incl=0.3, nx=17, ny=23)]
    n = sum(im.n for im in ims)
    opt = gray.Options(precision=prec, max_steps=10000, r_sw=0.02)
    ref = gray.Tracer(opt, n)
    ref.setup(ims)
    ref.trace()
    want = ref.records()
    ref.close()
    tr = gray.Tracer(opt, n + 5)
    tr.setup(ims, first_ray=5)
    order = tr.plan(ims, first_ray=5, probe_stride=4, probe_budget=150)
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(5, 5 + n))
    rc, n_active, _ = tr.trace(order=order)
    got = tr.records(first_ray=5, n=n)
    tr.close()
    assert rc == 1 and n_active == 5  # the five rays before first_ray were never set up, nor traced
    assert np.array_equal(want, got)


@pytest.mark.parametrize("stride", [1, 4, 100])
def test_fused_plan_sets_up_and_queues_every_ray_for_any_stride(stride):
    """gray_setup_plan with images of very different sizes (one pixel, a
    ragged 7 x 3 and 40 x 33) and probe strides from 1 (every pixel a probe)
    to beyond every image's side (one probe per image): the queue is a
    permutation of the rays, and the planned trace (probes set up and traced
    on the planning stream, the other rays set up beside them) equals
    gray_setup + a natural-order trace bit for bit."""
    ims = [I.Image(a=0.9, incl=1.0, nx=1, ny=1, alpha0=3.0, alpha1=3.5, beta0=1.0, beta1=1.5),
           I.Image(a=0.5, incl=0.7, nx=7, ny=3), I.Image(a=0.99, incl=1.5, nx=40, ny=33)]
    n = sum(im.n for im in ims)
    opt = gray.Options(precision=gray.FP32_KAHAN_SEL64, max_steps=10000, r_sw=0.02)
    ref = gray.Tracer(opt, n)
    ref.setup(ims)
    ref.trace()
    want = ref.records()
    ref.close()
    tr = gray.Tracer(opt, n + 2)
    order = tr.setup_plan(ims, first_ray=2, probe_stride=stride, probe_budget=60)
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(2, 2 + n))
    tr.trace(order=order)
    assert np.array_equal(tr.records(first_ray=2, n=n), want)
    tr.close()


@pytest.mark.parametrize("prec", [gray.FP32_KAHAN, gray.FP32_KAHAN_SEL64])
def test_one_ray_per_thread_launch_equals_persistent(prec):
    """The paper's launch (Eq. 1: one ray per thread, blocks of 64) and the
    persistent refilling queue compute each ray identically."""
    im = I.Image(a=0.9, incl=1.2, nx=37, ny=31)
    a, _, _, _ = trace_image(im, gray.Options(precision=prec, max_steps=10000, r_sw=0.02))
    b, _, _, _ = trace_image(im, gray.Options(precision=prec, max_steps=10000, r_sw=0.02,
                                              launch=gray.LAUNCH_ONE_PER_THREAD))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [gray.FP64, gray.FP32_KAHAN_SEL64])
@pytest.mark.parametrize("shape", [dict(block=64), dict(block=256), dict(block=256, refill=32),
                                   dict(blocks_per_sm=2, refill=4)])
def test_launch_shape_does_not_change_results(prec, shape):
    """Every launch shape the autotuner may pick is accepted by every pass
    (the double passes keep their own block size) and gives the same bits."""
    im = I.Image(a=0.9, incl=math.radians(75.0), nx=37, ny=29)
    ref, _, _, _ = trace_image(im, gray.Options(precision=prec, max_steps=20000, r_sw=0.02))
    got, _, _, _ = trace_image(im, gray.Options(precision=prec, max_steps=20000, r_sw=0.02, **shape))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", [gray.FP32_KAHAN_SEL64, gray.FP64])
def test_setup_plan_equals_setup_then_plan(prec):
    """The fused call (non-probe set-up on a side stream, overlapping the
    probe pass) leaves every state as gray_setup + gray_plan do, queues the
    same rays, and the traces that follow agree bit for bit."""
    ims = [I.Image(a=0.9, incl=1.1, nx=41, ny=23), I.Image(a=-0.5, incl=0.4, nx=17, ny=30)]
    n = sum(im.n for im in ims)
    opt = gray.Options(precision=prec, max_steps=10000, r_sw=0.02)
    out = []
    for fused in (False, True):
        tr = gray.Tracer(opt, n + 3)
        if fused:
            order = tr.setup_plan(ims, first_ray=3, probe_stride=5, probe_budget=120)
        else:
            tr.setup(ims, first_ray=3)
            order = tr.plan(ims, first_ray=3, probe_stride=5, probe_budget=120)
        after_plan = tr.records(first_ray=3, n=n)
        o = np.sort(order.cpu().numpy())
        tr.trace(order=order)
        out.append((after_plan, o, tr.records(first_ray=3, n=n)))
        tr.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[1][1], np.arange(3, 3 + n))
    assert np.array_equal(out[0][2], out[1][2])


def test_plan_puts_long_rays_first():
    """On a 256^2 image of the a = 0.99, i = 90 deg workload, the rays that
    take over 1000 steps sit in the first fifth of the planned queue."""
    im = I.kerr_1024(256).images[0]
    opt = gray.Options(precision=gray.FP32_KAHAN, max_steps=10000)
    tr = gray.Tracer(opt, im.n)
    tr.setup([im])
    order = tr.plan([im], probe_stride=4, probe_budget=400).cpu().numpy()
    tr.trace()
    steps = tr.records()[:, 1]
    tr.close()
    pos = np.empty(im.n, dtype=np.int64)
    pos[order] = np.arange(im.n)
    long = steps > 1000
    assert long.sum() > 100
    assert np.median(pos[long]) < 0.2 * im.n


def test_order_restricts_the_trace_to_listed_rays():
    im = I.Image(a=0.5, incl=1.0, nx=16, ny=16)
    tr = gray.Tracer(gray.Options(precision=gray.FP32_KAHAN, max_steps=10000), im.n)
    tr.setup([im])
    sub = torch.arange(0, im.n, 3, dtype=torch.int32, device="cuda")
    rc, n_active, _ = tr.trace(order=sub)
    rec = tr.records()
    tr.close()
    traced = np.zeros(im.n, dtype=bool)
    traced[::3] = True
    assert np.all(rec[traced, 0] != gray.ACTIVE) and np.all(rec[~traced, 0] == gray.ACTIVE)
    assert n_active == (~traced).sum()


def test_batched_images_equal_separate_images():
    """Several (a, i) images set up in one call and traced in one launch give
    the same records as each image alone."""
    ims = [I.Image(a=0.3, incl=0.4, nx=13, ny=9), I.Image(a=0.95, incl=1.4, nx=7, ny=11),
           I.Image(a=0.0, incl=1.0, nx=16, ny=16)]
    opt = gray.Options(precision=gray.FP32_KAHAN_SEL64, max_steps=10000, r_sw=0.5)
    tr = gray.Tracer(opt, sum(im.n for im in ims))
    tr.setup(ims)
    tr.trace()
    allrec = tr.records()
    sh = tr.shadow(ims)
    tr.close()
    off = 0
    for k, im in enumerate(ims):
        alone, _, _, _ = trace_image(im, opt)
        assert np.array_equal(alone, allrec[off:off + im.n])
        cap = alone[:, 0] == oracle.CAPTURED
        al, be = oracle.pixel_centres(im.nx, im.ny, im.alpha0, im.alpha1, im.beta0, im.beta1)
        assert sh[k]["n_captured"] == cap.sum()
        cell = (im.alpha1 - im.alpha0) / im.nx * (im.beta1 - im.beta0) / im.ny
        assert sh[k]["area"] == pytest.approx(cap.sum() * cell)
        if cap.any():
            assert sh[k]["alpha_c"] == pytest.approx(al[cap].mean(), abs=1e-9)
            assert sh[k]["beta_c"] == pytest.approx(be[cap].mean(), abs=1e-9)
        off += im.n
