"""Batching, graph replay, autotuning and the serving loop on the GPU."""
import math

import numpy as np
import pytest
import torch

from paper_1303_5057_gb300 import batch, gray, serve, tune
from paper_1303_5057_gb300 import inputs as I

pytestmark = pytest.mark.gpu

OPT = gray.Options(precision=gray.FP32_KAHAN_SEL64, max_steps=10000, r_sw=0.02)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1303_5057_gb300 import build
    build.build()
    gray.lib()
    torch.cuda.init()


def test_shadow_sweep_matches_images_traced_one_by_one_and_graph_replay():
    ims = I.shadow_sweep(n_images=6, side_lo=24, side_hi=72).images
    sw = batch.ShadowSweep(ims, OPT, plan=True, probe_stride=4, probe_budget=200)
    sh, ms = sw.run()
    rec = sw.stats()
    off = 0
    for k, im in enumerate(ims):
        alone = gray.Tracer(OPT, im.n)
        alone.setup([im])
        alone.trace()
        want = alone.records()
        alone.close()
        assert np.array_equal(want, rec[off:off + im.n])
        assert sh[k]["n_captured"] == (want[:, 0] == gray.CAPTURED).sum()
        off += im.n
    sw.capture()
    sh2, _ = sw.run()
    assert np.array_equal(rec, sw.stats())
    assert np.array_equal(sh, sh2)
    sw.close()


def test_shadow_radius_of_schwarzschild_converges_to_3_sqrt_3():
    """a = 0: the shadow is the disc b < 3 sqrt 3; its pixel-counted area
    radius approaches 3 sqrt 3 within the pixel size."""
    im = I.Image(a=0.0, incl=math.radians(30.0), nx=160, ny=160, alpha0=-8, alpha1=8, beta0=-8, beta1=8)
    sw = batch.ShadowSweep([im], OPT, plan=False)
    sh, _ = sw.run()
    sw.close()
    assert abs(sh[0]["radius"] - 3 * math.sqrt(3)) < 16 / 160
    assert abs(sh[0]["alpha_c"]) < 0.01 and abs(sh[0]["beta_c"]) < 0.01


def test_autotuner_picks_valid_options(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tune.json"))
    ims = [I.Image(a=0.9, incl=1.2, nx=48, ny=48)]
    space = {"block": [64, 128], "blocks_per_sm": [0], "refill": [8, 32], "plan": [None, (4, 150)]}
    opt, plan, table = tune.autotune(ims, OPT, space=space)
    assert len(table) == 8 and opt.block in (64, 128) and opt.refill in (8, 32)
    opt2, plan2, _ = tune.autotune(ims, OPT, space=space)  # from the cache
    assert (opt2.block, opt2.refill, plan2) == (opt.block, opt.refill, plan)
    # every candidate computes the same rays
    recs = []
    for cand in (gray.Options(**{**OPT.__dict__, "block": 64, "refill": 8}), opt):
        tr = gray.Tracer(cand, ims[0].n)
        tr.setup(ims)
        tr.trace()
        recs.append(tr.records())
        tr.close()
    assert np.array_equal(recs[0], recs[1])


def test_clear_and_count_active():
    im = I.Image(a=0.5, incl=1.0, nx=10, ny=10)
    tr = gray.Tracer(OPT, 300)
    gray.gray_clear(tr.ctx, tr.state, 300, 0, 300)
    tr.setup([im], first_ray=100)
    assert gray.gray_count_active(tr.ctx, tr.state, 300, [(0, 100), (100, 100), (200, 100)]) == [0, 100, 0]
    tr.trace(step_budget=5)
    assert gray.gray_count_active(tr.ctx, tr.state, 300, [(100, 100)]) == [100]
    # the asynchronous form: ranges and results in device memory, clipped to the buffer
    ranges = torch.tensor([0, 100, 100, 100, 150, 400, -50, 120], dtype=torch.int64, device="cuda")
    out = torch.full((8,), -1, dtype=torch.int64, device="cuda")
    gray.gray_range_stats(tr.ctx, tr.state, 300, ranges, out)
    got = out.cpu().numpy()
    assert list(got[0::2]) == [0, 100, 50, 0]
    assert got[3] == 5 * 100 and got[5] == 5 * 50 and got[1] == 0 and got[7] == 0
    rc, n_active, _ = tr.trace()
    assert rc == 0 and n_active == 0
    rec = tr.records()
    assert np.all(rec[:100, 0] == gray.EMPTY) and np.all(rec[200:, 0] == gray.EMPTY)
    gray.gray_range_stats(tr.ctx, tr.state, 300, ranges, out)
    got = out.cpu().numpy()
    assert list(got[0::2]) == [0, 0, 0, 0] and got[3] == rec[100:200, 1].sum()
    tr.close()


@pytest.mark.parametrize("plan_min_rays", [None, 0])
def test_serving_result_is_the_same_alone_and_in_the_mix(plan_min_rays):
    """Continuous batching: requests admitted into a pool too small for all
    of them at once, traced in budget-limited rounds together (two rounds
    enqueued ahead of the host; with plan_min_rays = 0 each request planned
    longest-first into the pool's queue), give exactly the image each gives
    when traced alone, and their step counts add up."""
    reqs = I.request_stream(1000.0, 12, sides=(16, 24, 32, 48))
    srv = serve.Server(OPT, capacity=4000, round_budget=64, plan_min_rays=plan_min_rays, probe_stride=3,
                       probe_budget=50)
    stats = srv.run(reqs, realtime=False)
    srv.close()
    assert len(stats.results) == 12 and stats.rounds > 3
    by_id = {r.rid: r for r in stats.results}
    steps = 0
    for q in reqs:
        tr = gray.Tracer(OPT, q.image.n)
        tr.setup([q.image])
        tr.trace()
        alone_rec = tr.records()
        tr.close()
        alone = serve.render_alone(q.image, OPT)
        mixed = by_id[q.rid].pixels
        assert np.array_equal(alone, mixed)
        assert by_id[q.rid].steps == alone_rec[:, 1].sum()
        steps += alone_rec[:, 1].sum()
    s = stats.summary()
    assert s["photon_steps"] == steps
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_cancel_stops_a_trace_and_the_trace_resumes_bit_for_bit():
    """gray_cancel from another host thread stops a trace in flight at its
    warps' next refill: the call returns GRAY_ECANCEL early with rays still
    active; after the flag is cleared the next trace finishes them, and the
    records equal those of a trace that was never interrupted."""
    import threading
    import time

    im = I.kerr_1024(512).images[0]
    opt = gray.Options(precision=gray.FP64, max_steps=10000)
    ref = gray.Tracer(opt, im.n)
    ref.setup([im])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, n_active, _ = ref.trace()
    full = time.perf_counter() - t0
    want = ref.records()
    ref.close()
    assert rc == 0 and n_active == 0 and full > 0.02

    tr = gray.Tracer(opt, im.n)
    tr.setup([im])
    torch.cuda.synchronize()
    out = {}

    def run():
        t1 = time.perf_counter()
        out["res"] = tr.trace()
        out["dt"] = time.perf_counter() - t1

    th = threading.Thread(target=run)
    th.start()
    time.sleep(min(0.005, full / 10))
    gray.gray_cancel(tr.ctx, True)
    th.join()
    rc, n_active, stats = out["res"]
    assert rc == gray.ECANCEL and n_active > 0
    assert out["dt"] < 0.8 * full
    # while the flag is set, a trace takes no step
    rc, n_again, stats = tr.trace()
    assert rc == gray.ECANCEL and n_again == n_active and stats[0] == 0
    gray.gray_cancel(tr.ctx, False)
    rc, n_active, _ = tr.trace()
    assert rc == 0 and n_active == 0
    assert np.array_equal(tr.records(), want)
    tr.close()


def test_cancel_in_the_selective_double_mode_resumes_bit_for_bit():
    """The same in compensated FP32 with the double zone: a cancelled call
    parks rays of both passes (single precision and the zone) as they stand."""
    im = I.Image(a=0.95, incl=1.3, nx=64, ny=64)
    opt = gray.Options(precision=gray.FP32_KAHAN_SEL64, max_steps=10000, r_sw=0.3, refill=2)
    ref = gray.Tracer(opt, im.n)
    ref.setup([im])
    ref.trace()
    want = ref.records()
    ref.close()
    tr = gray.Tracer(opt, im.n)
    tr.setup([im])
    rc, n1, _ = tr.trace(step_budget=150)   # part of the way, some rays inside the zone
    assert rc == 1 and n1 > 0
    gray.gray_cancel(tr.ctx, True)
    rc, n2, st = tr.trace()
    assert rc == gray.ECANCEL and n2 == n1 and st[0] == 0
    gray.gray_cancel(tr.ctx, False)
    rc, n3, _ = tr.trace()
    assert rc == 0 and n3 == 0
    assert np.array_equal(tr.records(), want)
    tr.close()
