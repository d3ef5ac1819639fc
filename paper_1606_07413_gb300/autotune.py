"""Autotuner of the batched search (qcs_batch_*).

For a sample of the targets it times a few rounds of the real engine for
every candidate setting and keeps the best, in two stages:

1. the host-side batch parameters -- walks per job, walk steps per round, the
   cap on the distinguished fraction theta (``theta_min_bits``: theta <=
   2^-bits) and the merge-queue capacity -- by the jobs finished per second
   of GPU time, ties broken by walk steps per second;
2. for each qubit count n >= 3 in the sample, the walk kernel's launch shape
   (warps per CTA and resident CTAs per SM, ``qcs_launch_shapes``) together
   with the device layout of C^ (``c_layout``: int8 byte quads for dp4a or
   32-bit words for IMAD), by the time the same rounds take.  Shapes and
   layouts change neither the walks nor their results, so every trial of this
   stage does identical work and the fastest wins.

Every trial runs the same seeded jobs, so settings are compared on identical
inputs.
"""
from __future__ import annotations

import itertools
import time

import paper_1606_07413_gb300 as Q

DEFAULT_GRID = {
    "walks_per_job": (512, 2048),
    "steps_per_round": (16, 64),
    "theta_min_bits": (1, 3),
    "queue_capacity": (1 << 12, 1 << 16),
}
HOST_KEYS = tuple(DEFAULT_GRID)


def _trial(targets, setting, rounds, stream, table_log2, seed):
    shapes = setting.get("launch_shape", {})
    layouts = setting.get("c_layout", {})
    bp = Q.default_batch_params(max_jobs=len(targets), walks_per_job=setting["walks_per_job"],
                                steps_per_round=setting["steps_per_round"], table_log2=table_log2,
                                queue_capacity=setting["queue_capacity"], launch_shape=dict(shapes))
    probs = []
    with Q.Batch(bp, stream) as b:
        ids = []
        for i, t in enumerate(targets):
            p = Q.Problem.from_circuit(t["n"], t["gates"], t["t"],
                                       Q.default_params(t["n"], theta_min_bits=setting["theta_min_bits"],
                                                        c_layout=layouts.get(t["n"], 0), seed=seed + i))
            probs.append(p)
            ids.append(b.add(p))
        t0 = time.perf_counter()
        for _ in range(rounds):
            if b.round() == 0:
                break
        dt = time.perf_counter() - t0
        res = [b.poll(j) for j in ids]
    for p in probs:
        p.close()
    done = sum(r["status_name"] == "found" for r in res)
    steps = sum(r["steps"] for r in res)
    return {**setting, "seconds": dt, "found": done, "jobs_per_s": done / dt, "steps_per_s": steps / dt}


def tune_batch(targets, rounds: int = 8, grid: dict | None = None, stream=None, table_log2: int = 18,
               seed: int = 4242, shapes: bool = True):
    """Return (best setting, all trials) for the batched search of `targets`
    (dicts with n, t, gates as produced by workloads.batched_targets).  The
    best setting holds the host keys of the grid and, when `shapes` is true,
    "launch_shape" and "c_layout" as {n: choice} for every n >= 3 present."""
    grid = grid or DEFAULT_GRID
    keys = list(grid)
    trials = []
    for values in itertools.product(*(grid[k] for k in keys)):
        trials.append(_trial(targets, dict(zip(keys, values)), rounds, stream, table_log2, seed))
    top = max(trials, key=lambda r: (r["jobs_per_s"], r["steps_per_s"]))
    best = {k: top[k] for k in keys}
    if not shapes:
        return best, trials
    best["launch_shape"], best["c_layout"] = {}, {}
    for n in sorted({t["n"] for t in targets if t["n"] >= 3}):
        stage = []
        for shape, layout in itertools.product(range(len(Q.launch_shapes(n))), (0, 1)):
            setting = dict(best, launch_shape={**best["launch_shape"], n: shape},
                           c_layout={**best["c_layout"], n: layout})
            stage.append(_trial(targets, setting, rounds, stream, table_log2, seed))
        fastest = min(stage, key=lambda r: r["seconds"])
        best["launch_shape"][n] = fastest["launch_shape"][n]
        best["c_layout"][n] = fastest["c_layout"][n]
        trials += stage
    return best, trials


def tune_level_shape(n: int, make_problem, k: int, steps: int, stream=None, launches: int = 3):
    """Launch shape and C^ layout of the single-target level walk: for every
    (shape, layout) pair, make_problem(launch_shape=, c_layout=) gives a
    problem, whose level k is walked `launches` times by `steps` steps after
    one untimed launch; the pair with the most walk steps per second of
    kernel time wins (the walks are the same for every pair).  Returns (best
    {"launch_shape", "c_layout"}, trials)."""
    import torch

    trials = []
    layouts = (0, 1) if n >= 3 else (0,)
    for shape, layout in itertools.product(range(len(Q.launch_shapes(n))), layouts):
        prob = make_problem(launch_shape=shape, c_layout=layout)
        prob.level_begin(k, 0, 0, stream=stream)
        prob.level_walk(steps, stream)
        prob.level_rewalk(stream)
        prob.level_collect(stream)
        r0 = prob.poll()
        ms = 0.0
        for _ in range(launches):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            prob.level_walk(steps, stream)
            e1.record(stream)
            prob.level_rewalk(stream)
            prob.level_collect(stream)
            ms += e0.elapsed_time(e1)
        r1 = prob.poll()
        prob.close()
        trials.append({"launch_shape": shape, "c_layout": layout, "walk_ms": ms,
                       "walk_steps_per_s": (r1["steps"] - r0["steps"]) / (ms / 1e3)})
    top = max(trials, key=lambda r: r["walk_steps_per_s"])
    return {"launch_shape": top["launch_shape"], "c_layout": top["c_layout"]}, trials
