"""Benchmark of the Kerr photon tracer on one GB300 (or N replicas).

One step = one pass of the whole hot path over one image: image-plane set-up
(FP64), backward RK4 trace of every ray to capture or escape, and render of
the per-pixel results.  Workload: a = 0.99, i = 90 deg, r_obs = 1000 M,
1024 x 1024 pixels over [-10, 10]^2 M, compensated FP32 with double steps
near the horizon, at most 1e4 steps per ray.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead, on a bounded sample of the same workload.

Multi-GPU: rays are independent, so N GPUs run N independent replicas of the
workload (weak scaling, no collective on the data path); the timing is the
maximum over ranks and the value is the sum of the work of all ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "photon RK4 steps/s FP32 vs FP64, 1 GB300; p50/p99 image-request latency"
UNIT = "photon-steps/s"

# Algorithmic work of one step, counted on the closed-form source (FMA = 2
# flops, add/mul = 1; each divide and each sincos counted as 1 flop and listed
# apart): 4 right-hand sides x 109, stage states 37, RK4 combination 41, Eq. 4
# monitor 39, step rule 6 = 559.  The compensated (Kahan) state update adds 32
# flops of overhead that the roofline fraction does not credit.
F_STEP = 559
F_KAHAN = 32
# Special-function work per step: one full sin/cos (the step's end point), three
# by angle addition with short series (the interior stages, no SFU), and 13
# SFU reciprocals (three per geometry, plain, for four geometries; one in the
# step size, refined by a Newton-Raphson step), three more on a redone step.
# At 16 SFU results per clock per SM they alone would allow
# 152 x 16 x 2.070e9 / 13 = 3.9e11 steps/s, far above the FMA bound.
SPECIAL_PER_STEP = {"sincos_full": 1, "sincos_by_angle_addition": 3, "sfu_reciprocal": 13}
SFU_PER_CLK_PER_SM = 16
# Nominal FP32 non-tensor peak: 152 SMs x 128 FP32 lanes x 2 flop/FMA x
# 2.070 GHz (context; the roofline divides by the rate measured in the run).
SMS, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.070
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_GHZ / 1000.0
# DRAM bytes (read + write) of one launch of the dominant kernel (the
# single-precision pass of the 1024^2 image, planned queue), from ncu's
# dram__bytes_read.sum + dram__bytes_write.sum (one pass, full size):
# 1.42e8 read + 0.64e8 written.  The pass moves ~250 B per ray (state, stop
# point, status, per-ray constants, queue entry); part of what the set-up
# just wrote is still in L2.
TRAFFIC_BYTES = 2.06e8
# Nominal FP64 non-tensor peak at 2 FP64 lanes per SM (context only).
FP64_PEAK_TFLOPS = SMS * 2 * 2 * SM_MAX_GHZ / 1000.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gray", choices=["gray", "reference"])
    p.add_argument("--side", type=int, default=1024)
    p.add_argument("--precision", default=None,
                   help="fp64 | fp32 | fp32_kahan | fp32_kahan_sel64 (default: fp32_kahan for the ring study, "
                        "whose result is the capture map alone, else fp32_kahan_sel64)")
    p.add_argument("--r-sw", type=float, default=0.02)
    p.add_argument("--step-rule", default="bench", choices=["bench", "eq2"])
    p.add_argument("--block", type=int, default=0)
    p.add_argument("--blocks-per-sm", type=int, default=0)
    p.add_argument("--refill", type=int, default=0)
    p.add_argument("--no-plan", action="store_true")
    p.add_argument("--separate-setup", action="store_true",
                   help="planned queue: gray_setup then gray_plan instead of the fused gray_setup_plan")
    p.add_argument("--probe-stride", type=int, default=6)
    p.add_argument("--probe-budget", type=int, default=400)
    p.add_argument("--no-fp64-leg", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-rays", type=int, default=262144,
                   help="pixels of the CPU-baseline sample (~10 s on 16 cores); the reference arm takes 1/16 per step")
    p.add_argument("--workload", default="kerr1024",
                   choices=["kerr1024", "schwarzschild64", "mixed", "sweep", "serve", "projection", "rings", "view"])
    p.add_argument("--rays", type=int, default=1 << 22, help="mixed workload: rays")
    p.add_argument("--images", type=int, default=256, help="sweep workload: images")
    p.add_argument("--rates", default="10,30,100,300,1000", help="serve workload: req/s")
    p.add_argument("--requests", type=int, default=0,
                   help="serve workload: requests per rate (0: 60 s of arrivals, at least 200, at most 2000)")
    p.add_argument("--ring-nr", type=int, default=6000, help="rings workload: radii per angle")
    p.add_argument("--ring-nth", type=int, default=181, help="rings workload: angles")
    p.add_argument("--ring-out", default="", help="rings workload: write the per-image table here (JSON)")
    p.add_argument("--frame-steps", type=int, default=8, help="view workload: RK4 steps per frame")
    p.add_argument("--frame-out", default="", help="view workload: write one frame here (PGM)")
    p.add_argument("--no-serve", action="store_true", help="skip the serving leg of the default workload")
    p.add_argument("--no-peaks", action="store_true",
                   help="skip the FMA-chain peak measurement (the roofline then divides by the nominal peaks)")
    p.add_argument("--serve-rates", default="10,30", help="serving leg: Poisson arrival rates (req/s)")
    p.add_argument("--serve-seconds", type=float, default=20.0, help="serving leg: seconds of arrivals per rate")
    p.add_argument("--serve-saturation", type=int, default=240,
                   help="serving leg: requests offered at once to measure the saturated rate (0: skip)")
    return p.parse_args()


# ------------------------------------------------------------------ clocks ---

class ClockSampler:
    """nvidia-smi clock and throttle samples taken while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# ------------------------------------------------------ measured ALU peaks ---

def measure_alu_peaks(gray, torch, launches=24):
    """Non-tensor FP32 and FP64 FMA rates of this device from the library's
    FMA-chain microbenchmark (gray_fma_peak: 8 independent chains per thread,
    every SM filled with 2048 threads), timed with CUDA events on the
    launching stream, with the SM clock sampled while it runs.  Changes no
    GPU setting."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, threads = sms * 8, 256
    stream = torch.cuda.current_stream()
    out = {"sms": sms, "blocks": blocks, "threads": threads, "chains_per_thread": 8}
    for name, prec, iters, dt in (("fp32", gray.FP32, 1 << 17, torch.float32),
                                  ("fp64", gray.FP64, 1 << 11, torch.float64)):
        sink = torch.empty(blocks * threads, dtype=dt, device="cuda")
        gray.gray_fma_peak(prec, blocks, threads, iters, sink)  # warm-up
        torch.cuda.synchronize()
        clk = ClockSampler(torch.cuda.current_device())
        clk.start()
        time.sleep(0.25)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(launches)]
        flop = 0
        for a, b in ev:
            a.record(stream)
            flop = gray.gray_fma_peak(prec, blocks, threads, iters, sink)
            b.record(stream)
        torch.cuda.synchronize()
        c = clk.stop()
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        out[name] = {"tflops": flop / (ms / 1000.0) / 1e12, "ms_per_launch": ms, "flop_per_launch": flop,
                     "sm_mhz": c.get("sm_mhz"), "sm_max_mhz": c.get("sm_max_mhz"), "reasons": c.get("reasons")}
    return out


# ------------------------------------------------------------- CPU oracle ---

def cpu_sample_rays(im, n_sample):
    """A seeded, evenly spread subset of the image's pixels (alpha, beta)."""
    from oracle import oracle as O
    al, be = O.pixel_centres(im.nx, im.ny, im.alpha0, im.alpha1, im.beta0, im.beta1)
    n = al.size
    idx = np.unique(np.linspace(0, n - 1, min(n_sample, n)).astype(np.int64))
    rays = np.empty((idx.size, 5))
    rays[:, 0], rays[:, 1] = al[idx], be[idx]
    rays[:, 2], rays[:, 3], rays[:, 4] = im.a, im.incl, im.r_obs
    return rays


def cpu_oracle_rate(im, max_steps, step_rule, n_sample, threads=None):
    import oracle
    rays = cpu_sample_rays(im, n_sample)
    cores = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    out = oracle.trace_many(rays, oracle.Options(max_steps=max_steps, step_rule=step_rule), nthreads=cores)
    dt = time.perf_counter() - t0
    steps = float(out[:, 1].sum())
    return steps / dt, cores, rays.shape[0], steps, dt


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1303_5057_gb300 import inputs as I
    im = I.kerr_1024(args.side).images[0]
    rule = 1 if args.step_rule == "eq2" else 0
    per_step = max(256, args.cpu_rays // 16)
    for _ in range(args.warmup):
        cpu_oracle_rate(im, 10000, rule, per_step)
    rates, steps_all, t_all = [], 0.0, 0.0
    cores = os.cpu_count() or 1
    for _ in range(args.steps):
        r, cores, n, st, dt = cpu_oracle_rate(im, 10000, rule, per_step)
        rates.append(r)
        steps_all += st
        t_all += dt
    value = steps_all / t_all
    sample = "%d evenly spread pixels of the %dx%d image per step" % (per_step, args.side, args.side)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "kerr_a0.99_i90_%dx%d" % (args.side, args.side), "precision": "fp64 (oracle)",
                       "rays": args.side ** 2, "max_steps": 10000, "step_rule": args.step_rule},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------- other workloads (GPU) ---

def _timed(fn, repeats):
    import torch
    ts = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return min(ts), out


def run_schwarzschild64(args):
    """a = 0, i = 60 deg, 64 x 64, FP64 on the GPU against the FP64 oracle on
    the host cores (the whole image both ways)."""
    import torch
    import oracle
    from paper_1303_5057_gb300 import gray
    from paper_1303_5057_gb300 import inputs as I
    wl = I.schwarzschild_64()
    im = wl.images[0]
    tr = gray.Tracer(gray.Options(precision=gray.FP64, max_steps=wl.max_steps), im.n)

    def step():
        tr.setup([im])
        return tr.trace()[2]
    step()
    ms, st = _timed(step, max(3, args.steps))
    rays = oracle.image_rays(im.a, im.incl, im.r_obs, im.nx, im.ny, im.alpha0, im.alpha1, im.beta0, im.beta1)
    t0 = time.perf_counter()
    out = oracle.trace_many(rays, oracle.Options(max_steps=wl.max_steps))
    dt = time.perf_counter() - t0
    tr.close()
    print(json.dumps({"workload": wl.name, "metric": "photon RK4 steps/s", "unit": UNIT, "dtype": "f64",
                      "gpu": {"value": st[0] / (ms / 1000.0), "ms_per_image": ms, "steps": st[0]},
                      "cpu_oracle": {"value": float(out[:, 1].sum()) / dt, "s_per_image": dt,
                                     "cores": os.cpu_count()}}), flush=True)
    return 0


def run_mixed(args):
    """2^k rays, per-ray (alpha, beta, a, i), half near each ray's critical
    curve: the precision variants with the persistent refilling queue
    (compaction on) and with the paper's one-ray-per-thread launch (off)."""
    import torch
    from paper_1303_5057_gb300 import gray
    from paper_1303_5057_gb300 import inputs as I
    n = args.rays
    t0 = time.perf_counter()
    rays = torch.as_tensor(I.mixed_rays(n), device="cuda")
    gen_s = time.perf_counter() - t0
    res = {}
    variants = [("fp32", gray.FP32, gray.LAUNCH_PERSISTENT), ("fp32_kahan", gray.FP32_KAHAN, gray.LAUNCH_PERSISTENT),
                ("fp32_kahan_sel64", gray.FP32_KAHAN_SEL64, gray.LAUNCH_PERSISTENT),
                ("fp32_kahan_sel64_no_compaction", gray.FP32_KAHAN_SEL64, gray.LAUNCH_ONE_PER_THREAD)]
    for name, prec, launch in variants:
        tr = gray.Tracer(gray.Options(precision=prec, max_steps=10000, r_sw=args.r_sw, launch=launch), n)

        def step():
            tr.setup_rays(rays)
            return tr.trace()[2]
        step()
        ms, st = _timed(step, 2)
        tr.close()
        res[name] = {"value": st[0] / (ms / 1000.0), "ms": ms, "steps": st[0], "fp64_steps": st[2]}
    # plain FP64 on a 1/16 subset (1/64 of the FP32 rate)
    sub = rays[: max(1, n // 16)].contiguous()
    tr = gray.Tracer(gray.Options(precision=gray.FP64, max_steps=10000), sub.shape[0])

    def step64():
        tr.setup_rays(sub)
        return tr.trace()[2]
    ms, st = _timed(step64, 1)
    tr.close()
    res["fp64_subset_1_16"] = {"value": st[0] / (ms / 1000.0), "ms": ms, "steps": st[0]}
    print(json.dumps({"workload": "mixed_%d_rays" % n, "metric": "photon RK4 steps/s", "unit": UNIT,
                      "generation_s": gen_s, "variants": res}), flush=True)
    return 0


def run_sweep(args):
    """Batched shadow sweep: `images` (a, i) images of side U{64..1024} in one
    set-up, one plan, one persistent trace and one shadow reduction."""
    import torch
    from paper_1303_5057_gb300 import batch, gray
    from paper_1303_5057_gb300 import inputs as I
    wl = I.shadow_sweep(n_images=args.images)
    opt = gray.Options(precision=gray.FP32_KAHAN_SEL64, max_steps=10000, r_sw=args.r_sw,
                       block=args.block, blocks_per_sm=args.blocks_per_sm, refill=args.refill)
    sw = batch.ShadowSweep(wl.images, opt, plan=not args.no_plan, probe_stride=args.probe_stride,
                           probe_budget=args.probe_budget)
    sw.run()
    times = []
    for _ in range(max(1, min(args.steps, 3))):
        sh, ms = sw.run()
        times.append(ms)
    steps = int(sw.stats()[:, 1].sum())
    sw.close()
    ms = min(times)
    print(json.dumps({"workload": wl.name, "images": len(wl.images), "rays": wl.n_rays,
                      "metric": "photon RK4 steps/s", "unit": UNIT, "value": steps / (ms / 1000.0),
                      "ms_per_sweep": ms, "steps": steps,
                      "radius_range": [float(sh["radius"].min()), float(sh["radius"].max())],
                      "queue": "natural" if args.no_plan else "planned"}), flush=True)
    return 0


def run_serve(args):
    """Poisson arrivals of render requests (side in {32, ..., 2048}, a, i
    random), continuous batching over a resident pool; p50/p99 latency and
    photon-steps/s per arrival rate."""
    from paper_1303_5057_gb300 import gray, serve
    from paper_1303_5057_gb300 import inputs as I
    opt = gray.Options(precision=gray.FP32_KAHAN_SEL64, max_steps=10000, r_sw=args.r_sw)
    out = []
    for rate in [float(x) for x in args.rates.split(",")]:
        srv = serve.Server(opt, capacity=32 << 20, round_budget=4096)
        n_req = args.requests if args.requests > 0 else int(min(2000, max(200, 60.0 * rate)))
        reqs = I.request_stream(rate, n_req)
        st = srv.run(reqs, realtime=True, max_wall=180.0)
        srv.close()
        summ = st.summary()
        summ["rate_req_per_s"] = rate
        summ["offered"] = n_req
        out.append(summ)
        print(json.dumps({"workload": "serve", "rate": rate, **summ}), flush=True)
    return 0


def serving_leg(args, rates, seconds, saturation):
    """Serving (the request loop of serve.py): Poisson arrivals of render
    requests (side uniform over {32, ..., 2048}, a ~ U[0, 0.999], i ~ U[0, 90]
    deg, r_obs = 1000, compensated FP32 + zone) at each rate for `seconds` of
    arrivals, then `saturation` requests offered at once.  p50/p99 latency
    (arrival to image in host memory) and photon-steps/s per rate."""
    from paper_1303_5057_gb300 import gray, serve
    from paper_1303_5057_gb300 import inputs as I
    opt = gray.Options(precision=gray.FP32_KAHAN_SEL64, max_steps=10000, r_sw=args.r_sw)
    srv = serve.Server(opt, capacity=32 << 20, round_budget=4096)
    srv.run(I.request_stream(100.0, 6, seed_index=40), realtime=False)  # warm-up
    out = {"sides": "uniform over {32, 64, ..., 2048}", "pool_rays": 32 << 20, "round_budget": 4096,
           "planned": "requests of >= 65536 rays (probe stride 6, budget 400)",
           "precision": "fp32_kahan_sel64", "latency": "arrival to image in pinned host memory", "rates": []}
    for rate in rates:
        n_req = max(10, int(rate * seconds))
        st = srv.run(I.request_stream(rate, n_req), realtime=True, max_wall=seconds * 4 + 30.0)
        summ = st.summary()
        summ["rate_req_per_s"] = rate
        summ["offered"] = n_req
        out["rates"].append(summ)
    if saturation > 0:
        st = srv.run(I.request_stream(1000.0, saturation, seed_index=41), realtime=False)
        out["saturated"] = {**st.summary(), "offered_at_once": saturation}
    srv.close()
    return out


def run_projection(args):
    """Sec. 3 grid projection (a = 0.95, i = 60 deg, r = 1000 M, each ray stops
    on the equatorial plane): time per image against the number of geodesics,
    in FP64 (as the paper's Fig. 4) and in compensated FP32 with the double
    zone; the oracle on the host cores for the smaller images."""
    import torch
    import oracle
    from paper_1303_5057_gb300 import gray
    from paper_1303_5057_gb300 import inputs as I
    rows = []
    for side in (8, 16, 32, 64, 128, 256, 512, 1024):
        im = I.Image(a=0.95, incl=math.radians(60.0), nx=side, ny=side, alpha0=-15, alpha1=15, beta0=-15, beta1=15)
        row = {"geodesics": im.n}
        for name, prec in (("gpu_fp64", gray.FP64), ("gpu_fp32_kahan_sel64", gray.FP32_KAHAN_SEL64)):
            tr = gray.Tracer(gray.Options(precision=prec, max_steps=20000, r_sw=args.r_sw, stop_equator=1), im.n)
            out = torch.empty(16 * im.n, dtype=torch.uint8, device="cuda")

            def step():
                tr.setup([im])
                tr.trace(wait=False)
                tr.render(gray.RENDER_PIXELS32, out=out)
            step()
            ms, _ = _timed(step, 3)
            tr.close()
            row[name + "_ms"] = ms
        if im.n <= 16384:
            rays = oracle.image_rays(im.a, im.incl, im.r_obs, im.nx, im.ny, im.alpha0, im.alpha1, im.beta0, im.beta1)
            t0 = time.perf_counter()
            oracle.trace_many(rays, oracle.Options(max_steps=20000, stop_equator=1), nthreads=1)
            row["cpu_oracle_1core_ms"] = 1000.0 * (time.perf_counter() - t0)
        rows.append(row)
        print(json.dumps({"workload": "grid_projection_a0.95_i60", **row}), flush=True)
    return 0


def run_rings(args):
    """Sec. 4 ring study: 16 spins x 19 inclinations, each a polar image of
    ring-nr x ring-nth rays (3.3e8 rays at the paper's 6000 x 181), set up,
    planned, traced in one persistent launch (Eq. 2 step rule, compensated
    FP32 with double steps near the hole) and reduced to D, <R>, A per image.
    The timed region is the whole study, inputs generated on the device."""
    import torch
    from paper_1303_5057_gb300 import gray
    from paper_1303_5057_gb300 import inputs as I
    wl = I.ring_sweep(args.ring_nr, args.ring_nth)
    ims = wl.images
    opt = gray.Options(precision=gray.PRECISIONS[args.precision], step_rule=gray.STEP_EQ2, h_min=1e-9,
                       max_steps=100000, r_sw=args.r_sw, block=args.block, blocks_per_sm=args.blocks_per_sm,
                       refill=args.refill)
    tr = gray.Tracer(opt, wl.n_rays)
    rows = sum(im.ny for im in ims)
    order = torch.empty(wl.n_rays, dtype=torch.int32, device="cuda")
    info = torch.empty(gray.RING_DTYPE.itemsize * len(ims), dtype=torch.uint8, device="cuda")
    bnd = torch.empty(rows, dtype=torch.float64, device="cuda")
    gray.gray_set_timing(tr.ctx, True)
    launches0 = gray.gray_launch_count()

    def step():
        tr.setup(ims)
        q = order
        if not args.no_plan:
            q = tr.plan(ims, probe_stride=args.probe_stride, probe_budget=args.probe_budget, order=order)
        _, _, st = tr.trace(order=None if args.no_plan else q)
        gray.gray_ring(tr.ctx, tr.state, tr.n, ims, out=info, boundary=bnd)
        return st
    step()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    reps = max(1, min(args.steps, 2))
    launches1 = gray.gray_launch_count()
    ms, st = _timed(step, reps)
    launches = (gray.gray_launch_count() - launches1) // reps
    clk = clocks.stop()
    passes = gray.gray_timings(tr.ctx)
    r = gray.as_numpy(info, gray.RING_DTYPE)
    tr.close()
    table = [{"a": im.a, "incl_deg": round(math.degrees(im.incl), 6), "D": float(x["D"]), "R_mean": float(x["R_mean"]),
              "A": float(x["A"]), "n_wrong": int(x["n_wrong"]), "n_open": int(x["n_open"])}
             for im, x in zip(ims, r)]
    if args.ring_out:
        with open(args.ring_out, "w") as f:
            json.dump(table, f)
    print(json.dumps({"workload": wl.name, "images": len(ims), "rays": wl.n_rays,
                      "metric": "photon RK4 steps/s", "unit": UNIT, "value": st[0] / (ms / 1000.0),
                      "ms_per_study": ms, "steps": st[0], "fp64_steps": st[2], "euler": st[1],
                      "ns_per_photon_step": 1e6 * ms / st[0], "gpu_launches": launches,
                      "passes_ms": passes, "queue": "natural" if args.no_plan else "planned",
                      "R_mean_range": [float(r["R_mean"].min()), float(r["R_mean"].max())],
                      "A_max": float(r["A"].max()), "D_max": float(r["D"].max()),
                      "wrong_rays": int(r["n_wrong"].sum()), "open_rows": int(r["n_open"].sum()),
                      "precision": args.precision, "clocks": clk}), flush=True)
    return 0


def run_view(args):
    """The interactive mode of Sec. 2 (Fig. 1) headless: a plane-parallel grid
    of photons (1024^2, from r = 1000 M) falls onto an a = 0.999 hole; each
    frame advances every live photon by frame-steps RK4 steps (gray_trace with
    a step budget) and draws the live photons as sprites into a 1920 x 1080
    count image (gray_splat), until none is left."""
    import torch
    from paper_1303_5057_gb300 import gray
    from paper_1303_5057_gb300 import inputs as I
    im = I.Image(a=0.999, incl=math.radians(60.0), nx=args.side, ny=args.side)
    opt = gray.Options(precision=gray.PRECISIONS[args.precision], max_steps=10000, r_sw=args.r_sw)
    tr = gray.Tracer(opt, im.n)
    cam = gray.Camera(eye=(30.0, -22.0, 16.0), look=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), fov=math.radians(60.0),
                      sprite=1.0, width=1920, height=1080, status_mask=1 << gray.ACTIVE)
    count = torch.empty((cam.height, cam.width), dtype=torch.int32, device="cuda")
    depth = torch.empty((cam.height, cam.width), dtype=torch.float32, device="cuda")

    def run(record):
        tr.setup([im])
        torch.cuda.synchronize()
        frames, steps, ms_frames, ms_splat = 0, 0, [], []
        saved = False
        while True:
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            _, n_active, st = tr.trace(step_budget=args.frame_steps, wait=True)
            e[1].record()
            gray.gray_splat(tr.ctx, tr.state, tr.n, cam, count=count, depth=depth)
            e[2].record()
            torch.cuda.synchronize()
            frames += 1
            steps += st[0]
            ms_frames.append(e[0].elapsed_time(e[2]))
            ms_splat.append(e[1].elapsed_time(e[2]))
            if record and args.frame_out and not saved and frames == 24:
                img = count.cpu().numpy().view(np.uint32)
                g = np.clip(255.0 * np.log1p(img) / max(1.0, np.log1p(img.max())), 0, 255).astype(np.uint8)
                with open(args.frame_out, "wb") as f:
                    f.write(b"P5 %d %d 255\n" % (cam.width, cam.height))
                    f.write(g.tobytes())
                saved = True
            if n_active == 0:
                return frames, steps, ms_frames, ms_splat
    run(False)
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    launches0 = gray.gray_launch_count()
    t0 = time.perf_counter()
    frames, steps, ms_frames, ms_splat = run(True)
    wall = time.perf_counter() - t0
    launches = gray.gray_launch_count() - launches0
    clocks = clk.stop()
    tr.close()
    splat_med = statistics.median(ms_splat)
    # algorithmic bytes of one splat launch: S0 (16 B) of every ray, position
    # and compensation (32 B) and spin (32 B of the P plane) of each drawn ray
    print(json.dumps({"workload": "view_a0.999_i60_%dx%d_photons_1920x1080" % (args.side, args.side),
                      "metric": "frames/s", "unit": "frames/s", "value": frames / (sum(ms_frames) / 1000.0),
                      "frames": frames, "frame_steps": args.frame_steps, "photons": im.n,
                      "ms_per_frame_mean": sum(ms_frames) / frames, "ms_per_frame_max": max(ms_frames),
                      "splat_ms_median": splat_med, "photon_steps_per_s": steps / (sum(ms_frames) / 1000.0),
                      "wall_s": wall, "gpu_launches": launches, "precision": args.precision, "clocks": clocks}),
          flush=True)
    return 0


# --------------------------------------------------------------- GPU arm ---

def main():
    args = parse_args()
    if args.precision is None:
        args.precision = "fp32_kahan" if args.workload == "rings" else "fp32_kahan_sel64"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "kerr1024":
        import torch
        from paper_1303_5057_gb300 import build, gray
        torch.cuda.set_device(0)
        build.build()
        gray.lib()
        return {"schwarzschild64": run_schwarzschild64, "mixed": run_mixed, "sweep": run_sweep,
                "serve": run_serve, "projection": run_projection, "rings": run_rings,
                "view": run_view}[args.workload](args)

    import torch

    from paper_1303_5057_gb300 import build, gray
    from paper_1303_5057_gb300 import inputs as I

    from paper_1303_5057_gb300 import replicas
    me = replicas.from_env()
    world, rank = me.world, me.rank
    dist = replicas.init(me, "nccl")
    if dist is None:
        torch.cuda.set_device(0)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    gray.lib()

    prec = gray.PRECISIONS[args.precision]
    rule = gray.STEP_EQ2 if args.step_rule == "eq2" else gray.STEP_BENCH
    im = I.kerr_1024(args.side).images[0]
    n = im.n
    opt = gray.Options(precision=prec, max_steps=10000, r_sw=args.r_sw, step_rule=rule, block=args.block,
                       blocks_per_sm=args.blocks_per_sm, refill=args.refill)
    tr = gray.Tracer(opt, n)
    gray.gray_set_timing(tr.ctx, True)
    stream = torch.cuda.current_stream()
    out_dev = torch.empty(16 * n, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    order_buf = torch.empty(n, dtype=torch.int32, device="cuda")

    def setup_and_plan():
        # planned: set-up and plan in one call (the non-probe set-up overlaps
        # the probe pass); natural order: set-up alone
        if args.no_plan:
            tr.setup([im])
            return None
        if args.separate_setup:
            tr.setup([im])
            return tr.plan([im], probe_stride=args.probe_stride, probe_budget=args.probe_budget, order=order_buf)
        return tr.setup_plan([im], probe_stride=args.probe_stride, probe_budget=args.probe_budget, order=order_buf)

    def one_step():
        order = setup_and_plan()
        tr.trace(wait=False, order=order)
        tr.render(gray.RENDER_PIXELS32, out=out_dev)

    # warm-up; the last warm-up step also reads the step statistics
    for _ in range(max(args.warmup, 1)):
        one_step()
    _, _, stats = tr.trace(order=setup_and_plan())
    _, _, _, zone_steps = gray.gray_timings(tr.ctx)
    main_pass_steps = stats[0] - zone_steps  # steps of the dominant kernel (single-precision pass)
    rec = tr.records()
    steps_per_pass = int(rec[:, 1].sum())  # every step of the hot path, probe steps included
    fp64_steps = int(rec[:, 16].sum())
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(torch.cuda.current_device())
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = gray.gray_launch_count()
    pass_ms = []
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        e0, e1, e2, e3 = ev[k]
        e0.record(stream)
        order = setup_and_plan()
        e1.record(stream)
        tr.trace(wait=False, order=order)
        e2.record(stream)
        tr.render(gray.RENDER_PIXELS32, out=out_dev)
        e3.record(stream)
        pass_ms.append(gray.gray_timings(tr.ctx)[:3])  # events of this step's passes (waits for them)
    torch.cuda.synchronize()
    launches = gray.gray_launch_count() - launches0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(d) for a, b, c, d in ev]
    setup_plan_ms = [a.elapsed_time(b) for a, b, c, d in ev]  # set-up + plan (one call when planned)
    trace_ms = [b.elapsed_time(c) for a, b, c, d in ev]
    total_ms = replicas.max_over_ranks(dist, sum(step_ms), device="cuda")
    value = replicas.job_rate(steps_per_pass * args.steps, total_ms, world)
    main_ms = statistics.mean(p[0] for p in pass_ms)
    zone_ms = statistics.mean(p[1] for p in pass_ms) if pass_ms[0][1] >= 0 else None
    probe_ms = statistics.mean(p[2] for p in pass_ms) if pass_ms[0][2] >= 0 and not args.no_plan else None
    achieved = F_STEP * main_pass_steps / (main_ms / 1000.0) / 1e12

    # ---- end to end through the C ABI: host image table in, pixels out to pinned host ----
    host_out = torch.empty(16 * n, dtype=torch.uint8, pin_memory=True)
    e2e_ms = []
    for k in range(1 + max(1, min(args.steps, 5))):  # the first pass warms the pinned buffer up, untimed
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tr.trace(wait=False, order=setup_and_plan())
        tr.render(gray.RENDER_PIXELS32, out=out_dev)
        host_out.copy_(out_dev, non_blocking=True)
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    e2e_value = steps_per_pass / (statistics.mean(e2e_ms) / 1000.0) * world

    # ---- measured non-tensor FMA peaks (the roofline's denominators) ----
    peaks = measure_alu_peaks(gray, torch) if rank == 0 and not args.no_peaks else None
    fp32_peak = peaks["fp32"]["tflops"] if peaks else FP32_PEAK_TFLOPS
    fp64_peak = peaks["fp64"]["tflops"] if peaks else FP64_PEAK_TFLOPS

    # ---- plain FP64 GPU path on the same image (the speed reference), with
    # the same planned queue as the single-precision arm ----
    fp64 = None
    if not args.no_fp64_leg and rank == 0:
        tr64 = gray.Tracer(gray.Options(precision=gray.FP64, max_steps=10000, step_rule=rule), n)
        order64 = torch.empty(n, dtype=torch.int32, device="cuda")

        def plan64():
            if args.no_plan:
                tr64.setup([im])
                return None
            return tr64.setup_plan([im], probe_stride=args.probe_stride, probe_budget=args.probe_budget,
                                   order=order64)
        q = plan64()
        tr64.trace(order=q)
        q = plan64()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tr64.trace(wait=False, order=q)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        q = plan64()
        _, _, st64 = tr64.trace(order=q)
        tr64.close()
        fp64 = {"value": st64[0] / (ms64 / 1000.0), "unit": UNIT, "trace_ms": ms64,
                "queue": "natural" if args.no_plan else "planned (same probes as the single-precision arm)",
                "roofline_frac_fp64": F_STEP * st64[0] / (ms64 / 1000.0) / 1e12 / fp64_peak,
                "peak_tflops": fp64_peak, "peak_source": "measured FMA chain (gray_fma_peak)" if peaks else
                "nominal"}

    serving = None
    if not args.no_serve and rank == 0:
        serving = serving_leg(args, [float(x) for x in args.serve_rates.split(",") if x],
                              args.serve_seconds, args.serve_saturation)

    cpu = None
    if not args.no_cpu and rank == 0:
        rate, cores, ns, st, dt = cpu_oracle_rate(im, 10000, 1 if rule == gray.STEP_EQ2 else 0, args.cpu_rays)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d evenly spread pixels of the %dx%d image (%.0f steps, %.1f s)" % (
                   ns, args.side, args.side, st, dt)}
        # the same oracle on one core, on a 64x smaller sample
        rate1, _, ns1, st1, dt1 = cpu_oracle_rate(im, 10000, 1 if rule == gray.STEP_EQ2 else 0,
                                                  max(256, args.cpu_rays // 64), threads=1)
        cpu["single_thread"] = {"value": rate1, "unit": UNIT, "cores": 1,
                                "sample": "%d evenly spread pixels (%.0f steps, %.1f s)" % (ns1, st1, dt1)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "kerr_a0.99_i90_%dx%d" % (args.side, args.side), "precision": args.precision,
                       "rays": n, "max_steps": 10000, "step_rule": args.step_rule, "r_sw": args.r_sw,
                       "queue": "natural" if args.no_plan else "planned (probe stride %d, budget %d%s)" % (
                           args.probe_stride, args.probe_budget,
                           "; set-up, then plan" if args.separate_setup else
                           "; set-up fused with the plan, non-probe set-up overlapping the probe pass"),
                       "l2": "flushed between timed steps (256 MB write)"},
            "ns_per_photon_step": 1e9 / (value / world),
            "steps_per_pass": steps_per_pass, "fp64_steps_per_pass": fp64_steps,
            "setup_plan_ms": statistics.mean(setup_plan_ms), "trace_ms": statistics.mean(trace_ms),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak,
                         # the captured figure belongs to the default workload only
                         "traffic": TRAFFIC_BYTES if (args.side == 1024 and not args.no_plan
                                                      and args.precision == "fp32_kahan_sel64"
                                                      and args.step_rule == "bench" and args.r_sw == 0.02) else None,
                         "kernel": "trace32_kernel (single-precision pass)", "kernel_ms": main_ms,
                         "kernel_steps": main_pass_steps,
                         "peak_source": ("measured: FP32 FMA chains (gray_fma_peak) in this run, at the SM clock in "
                                         "measured_peaks" if peaks else "nominal 152 x 128 x 2 x 2.070 GHz"),
                         "peak_nominal": FP32_PEAK_TFLOPS,
                         "frac_with_kahan_update": achieved * (F_STEP + F_KAHAN) / F_STEP / fp32_peak,
                         "sfu_bound_steps_per_s": SMS * SFU_PER_CLK_PER_SM * SM_MAX_GHZ * 1e9
                         / SPECIAL_PER_STEP["sfu_reciprocal"],
                         "flop_per_step": F_STEP, "flop_per_step_with_kahan_update": F_STEP + F_KAHAN,
                         "special_per_step": SPECIAL_PER_STEP},
            "measured_peaks": peaks,
            "passes_ms": {"single": main_ms, "zone": zone_ms, "probe": probe_ms,
                          "zone_steps": zone_steps, "setup_plan_trace_render": total_ms / args.steps},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 72, "d2h_bytes_per_step": 16 * n},
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64_gpu": fp64,
            "serving": serving,
            "speedup_vs_fp64_gpu": (value / world) / fp64["value"] if fp64 else None,
        }
        print(json.dumps(line), flush=True)
    tr.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
