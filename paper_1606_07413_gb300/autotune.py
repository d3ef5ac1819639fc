"""Autotuner of the batched search (qcs_batch_*).

For a sample of the targets it times a few rounds of the real engine for every
candidate setting -- walks per job, walk steps per round, the cap on the
distinguished fraction theta (``theta_min_bits``: theta <= 2^-bits) and the
merge-queue capacity -- and keeps the setting that finishes the most jobs per
second of GPU time, breaking ties by walk steps per second.  Every trial runs
the same seeded jobs, so the settings are compared on identical work.
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


def _trial(targets, setting, rounds, stream, table_log2, seed):
    bp = Q.default_batch_params(max_jobs=len(targets), walks_per_job=setting["walks_per_job"],
                                steps_per_round=setting["steps_per_round"], table_log2=table_log2,
                                queue_capacity=setting["queue_capacity"])
    probs = []
    with Q.Batch(bp, stream) as b:
        ids = []
        for i, t in enumerate(targets):
            p = Q.Problem.from_circuit(t["n"], t["gates"], t["t"],
                                       Q.default_params(t["n"], theta_min_bits=setting["theta_min_bits"],
                                                        seed=seed + i))
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
               seed: int = 4242):
    """Return (best setting, all trials) for the batched search of `targets`
    (dicts with n, t, gates as produced by workloads.batched_targets)."""
    grid = grid or DEFAULT_GRID
    keys = list(grid)
    trials = []
    for values in itertools.product(*(grid[k] for k in keys)):
        trials.append(_trial(targets, dict(zip(keys, values)), rounds, stream, table_log2, seed))
    best = max(trials, key=lambda r: (r["jobs_per_s"], r["steps_per_s"]))
    return {k: best[k] for k in keys}, trials
