"""Autotuner for the launch shape of the tracer.

Searches the trace kernel's block size, resident blocks per SM, refill
interval (steps between warp refills, i.e. how often finished lanes are
compacted out) and the planning probe (stride, budget), timing each candidate
with CUDA events on a representative workload, and caches the winner per
(GPU name, precision, step rule) in a JSON file.  The tuned knobs change only
the launch and the queue order, never a ray's arithmetic, so results are the
same for every candidate (the tests check this for the launch options).
"""
from __future__ import annotations

import itertools
import json
import os
import time
from dataclasses import asdict, replace

from . import gray

CACHE = os.environ.get("GRAY_TUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "paper_1303_5057_gb300", "tune.json"))

DEFAULT_SPACE = {
    "block": [64, 128],
    "blocks_per_sm": [0, 4],
    "refill": [8, 16, 32],
    "plan": [None, (4, 400), (8, 500)],
}


def _key(opt: gray.Options):
    import torch
    return "%s|prec%d|rule%d" % (torch.cuda.get_device_name(), opt.precision, opt.step_rule)


def load_cache():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(data):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_candidate(images, opt: gray.Options, plan, repeats=2):
    """Best-of-`repeats` milliseconds of set-up + plan + trace of `images`."""
    import torch
    n = sum(int(im.nx) * int(im.ny) for im in images)
    tr = gray.Tracer(opt, n)
    order_buf = torch.empty(max(1, n), dtype=torch.int32, device="cuda")
    best = float("inf")
    try:
        for _ in range(repeats + 1):  # the first run warms up
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            tr.setup(images)
            order = tr.plan(images, probe_stride=plan[0], probe_budget=plan[1], order=order_buf) if plan else None
            tr.trace(wait=False, order=order)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
    finally:
        tr.close()
    return best


def autotune(images, opt: gray.Options, space=None, use_cache=True, budget_s=120.0, verbose=False):
    """Pick launch options for `opt` on `images`.  Returns (options, plan,
    table) where plan is None or (probe_stride, probe_budget) and table lists
    every candidate tried with its time."""
    key = _key(opt)
    cache = load_cache() if use_cache else {}
    if use_cache and key in cache:
        c = cache[key]
        return (replace(opt, block=c["block"], blocks_per_sm=c["blocks_per_sm"], refill=c["refill"]),
                tuple(c["plan"]) if c["plan"] else None, c.get("table", []))
    space = space or DEFAULT_SPACE
    t_start = time.perf_counter()
    table = []
    best = None
    for block, bps, refill, plan in itertools.product(space["block"], space["blocks_per_sm"], space["refill"],
                                                      space["plan"]):
        if time.perf_counter() - t_start > budget_s:
            break
        cand = replace(opt, block=block, blocks_per_sm=bps, refill=refill)
        try:
            ms = time_candidate(images, cand, plan)
        except gray.GrayError:
            continue  # a launch shape this kernel cannot take
        table.append({"block": block, "blocks_per_sm": bps, "refill": refill, "plan": plan, "ms": ms})
        if verbose:
            print(table[-1], flush=True)
        if best is None or ms < best[0]:
            best = (ms, cand, plan)
    if best is None:
        return opt, None, table
    _, cand, plan = best
    if use_cache:
        cache[key] = {"block": cand.block, "blocks_per_sm": cand.blocks_per_sm, "refill": cand.refill,
                      "plan": list(plan) if plan else None, "ms": best[0], "table": table}
        save_cache(cache)
    return cand, plan, table


def options_dict(opt: gray.Options):
    return asdict(opt)
