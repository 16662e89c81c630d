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
