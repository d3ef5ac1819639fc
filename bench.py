#!/usr/bin/env python3
"""Benchmark of the deterministic-walk T-count search hot path on GB300.

Workload (the largest single-GPU configuration): n = 4 qubits, one seeded
target C0 R(P7)..R(P1), level k = 7 (three rotations per side, 255 chunks,
N = 2 x 255^4 = 8.5e9 walk points), 2^20 concurrent walks, 64-bit states,
distinguished fraction 2^-12, a 2^26-slot distinguished-point table.  One
bench step is one pass of the whole hot path over the batch: every walk
advances 64 walk steps (decode, exact half product hashed modulo Clifford,
distinguished-point test, table insert), the queued merges are re-walked and
classified on the device, and claw candidates are checked exactly on the host.

value   = walk steps per second over the timed steps (all ranks).
e2e     = the same metric through the public API (problem creation from the
          host gate list, qcs_run_walks, qcs_poll_collisions), with the bytes
          the library reports it copied each way.
Also reported: the roofline of the dominant kernel (contraction multiply-adds
against twice the measured dp4a rate, and issue slots from its ncu record),
the time to the optimal T-count of configurations 1-3 by the collision walk
alone and by the exhaustive pass, the n = 3 level-5 record, the batched and
serving workloads, and the CPU oracle timed on the host cores.

--impl reference times the CPU oracle (the reference arm of this build).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFG = 3
K_LEVEL = 7
STEPS_PER_LAUNCH = 64
# evaluations of f one merge's re-walk may take per bench step (0: none).
# The headline re-walks every merge of a step to its end within that step, so
# no classification work is carried past the timed steps; the budgeted,
# carried re-walk (params.rewalk_budget) is the library's option for long runs.
REWALK_BUDGET = 0
FLUSH_BYTES = 256 << 20
LEVELS = {1: 3, 2: 5, 3: 7}  # the level each configuration's construction T-count puts its claw on


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-T-count run")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and other-size runs")
    ap.add_argument("--batched-only", action="store_true",
                    help="only run the batched-search comparison (256 seeded targets), print its JSON and exit")
    ap.add_argument("--level-only", choices=["n2_level3", "n3_level5", "n4_level7"], default=None,
                    help="only time that single-target level launch (walk-kernel throughput), print its JSON and exit")
    ap.add_argument("--config3-walk", type=int, default=0, metavar="TABLE_LOG2",
                    help="only time the n = 4 seeded target's search by the collision walk alone with a "
                         "2^TABLE_LOG2-slot table, print its JSON and exit")
    ap.add_argument("--exhaustive-only", action="store_true",
                    help="only time one whole n = 4 level-7 exhaustive pass (no claw), print its JSON and exit")
    ap.add_argument("--adder-walk", type=int, default=0, metavar="TABLE_LOG2",
                    help="only time the 4-qubit full adder's search by the collision walk alone with a "
                         "2^TABLE_LOG2-slot table, print its JSON and exit")
    ap.add_argument("--sharded", action="store_true",
                    help="walk the headline level sharded by distinguished-point owner even on one rank "
                         "(the form N > 1 ranks always use; under torchrun)")
    ap.add_argument("--shape", type=int, default=0, help="launch shape of the --level-only walk kernel")
    ap.add_argument("--c-layout", type=int, default=0, help="C^ layout of the --level-only walk (0 int8, 1 words)")
    ap.add_argument("--theta-shapes", action="store_true",
                    help="only time one n = 4 level-7 walk launch (2^20 walks x 16 steps) of launch shapes 0 "
                         "and 3 at several distinguished fractions, print its JSON and exit")
    ap.add_argument("--tto-sweep", action="store_true",
                    help="only time the n = 4 seeded target's collision walk over a grid of table sizes and "
                         "distinguished fractions, print its JSON and exit")
    return ap.parse_args()


def workload_config(c, k=None, steps=None, rewalk_budget=None):
    k = K_LEVEL if k is None else k
    rewalk_budget = REWALK_BUDGET if rewalk_budget is None else rewalk_budget
    steps = STEPS_PER_LAUNCH if steps is None else steps
    return {
        "workload": f"n{c['n']}_t{c['t']}_level{k}_walks{c['walks']}_L{c['L']}_theta2^-{c['dtheta']}",
        "n_qubits": c["n"], "level_k": k, "chunks": 4 ** c["n"] - 1, "walks": c["walks"],
        "level_points": 2 * (4 ** c["n"] - 1) ** (k // 2) * ((4 ** c["n"] - 1) if k & 1 else 1),
        "steps_per_walk_per_step": steps, "state_bits": c["L"], "dp_bits": c["dtheta"],
        "rewalk_budget_per_step": rewalk_budget or "none (every merge re-walked in its own step)",
        "table_slots": 1 << c["table_log2"], "coefficients": "exact: int64 on the host, C^ as int8 byte quads on the device; fingerprints mod 2^16",
        "l2": f"flushed between steps ({FLUSH_BYTES >> 20} MiB write)",
        "parallelism": "one GPU (with N > 1: the level sharded over ranks by distinguished-point owner)",
    }


# ------------------------------------------------------------------ ncu records
# Per walk kernel, from ncu captures of the commands named in profiles/: DRAM
# traffic of one launch of the bench's workload (dram__bytes_read.sum +
# dram__bytes_write.sum) and warp instructions issued per walk step
# (smsp__inst_executed.sum / walk steps of the captured launch).  A record
# holds only for the kernel source it was captured on (hash of the walk
# kernel's source files, comments and layout removed); otherwise its figures
# are reported as null.
# Each n = 4 record: `ncu --set full` of `bench.py --level-only n4_level7
# --steps 2 --shape S` (2^20 walks x 16 steps; profiles/k_walks_n4_level7_walks1048576.md
# and profiles/k_walks_mma4_n4_level7_walks1048576.md).  The launch's DRAM
# traffic is the walk states and the staged tables, which do not grow with
# the steps, plus 32 bytes per distinguished point (0.5 MB at the headline's
# 64 steps), so the figure stands for the headline launch.
WALK_NCU = {
    "k_walks<4,3>": {"source_sha256_16": "80027283cc3dbf3c", "dram_bytes_per_launch": 34747136,
                     "warp_inst_per_step": 1073.2},
    "k_walks<4,0>": {"source_sha256_16": "80027283cc3dbf3c", "dram_bytes_per_launch": 35021312,
                     "warp_inst_per_step": 1937.6},
    # n = 3, level 5: `bench.py --level-only n3_level5 --steps 2`, one launch of 2^16 walks x 512 steps,
    # the launch of the n3_level5 record (profiles/k_walks_n3_level5_walks65536.md)
    "k_walks<3,0>": {"source_sha256_16": "80027283cc3dbf3c", "dram_bytes_per_launch": 2178304,
                     "warp_inst_per_step": 379.3},
}


def walk_source_hash() -> str:
    """Hash of the walk kernel's code (comments and layout removed, so that a
    comment edit does not count as a kernel change)."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in ("qcs_walk.cu", "qcs_internal.h"):
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1606_07413_gb300", "csrc", f)) as fh:
            text = fh.read()
        if f == "qcs_internal.h":
            # only the structures the walk kernels read (the rest is host-only)
            text = text[: text.index("// Exhaustive meet-in-the-middle pass over one level")]
        code = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def measured_tensor_tflops(sustained: bool = True):
    """Dense bf16 tensor throughput measured on the GB300s
    (MEASURED_PEAKS.json beside this file; the sustained figure for a kernel
    timed inside a long step), else the fallback figure.  f16 has the same
    nominal dense rate as bf16."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    try:
        with open(path) as f:
            return float(json.load(f)[key]), f"measured dense bf16 ({key}, MEASURED_PEAKS.json; f16 = bf16 nominal)"
    except (OSError, KeyError, ValueError):
        return (1700.0 if sustained else 1900.0), "fallback (no measured peaks file)"


def measured_hbm_gbs():
    """HBM copy bandwidth measured on the GB300s (MEASURED_PEAKS.json
    beside this file), else the fallback figure of one earlier measurement."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (no measured peaks file)"


def ncu_record(kernel: str):
    """The kernel's ncu record if it was captured on the current source, else None."""
    rec = WALK_NCU.get(kernel)
    if not rec or rec["source_sha256_16"] != walk_source_hash():
        return None
    return rec


def walk_roofline(kernel, n, w_steps, steps, walk_s, launches, dp4a_per_s, clock_mhz, num_sms, hmma_per_s=None):
    """Roofline of a walk kernel ("bound": "alu").  achieved = the W side's
    contraction multiply-adds (W-side steps x 2 d^2, d = 4^n - 1: 16-bit
    fingerprint weights times C^) per second of the kernel's CUDA-event time;
    peak = twice the measured dp4a rate (a dp4a makes four byte products, a
    16-bit-weight multiply-add needs two).  The issue-slot fraction takes the
    warp instructions per walk step from the kernel's ncu record against 4
    issue slots per SM per clock at the clock sampled during the run."""
    d = 4 ** n - 1
    achieved = w_steps * 2 * d * d / walk_s
    peak = 2 * dp4a_per_s
    rec = ncu_record(kernel)
    traffic = rec["dram_bytes_per_launch"] if rec else None
    hbm_peak, hbm_src = measured_hbm_gbs()
    hbm = None
    if traffic is not None:
        per_launch_s = walk_s / max(1, launches)
        hbm = {"achieved_gbs": traffic / per_launch_s / 1e9, "peak_gbs": hbm_peak,
               "frac": traffic / per_launch_s / 1e9 / hbm_peak, "peak_source": hbm_src}
    issue = None
    if rec and rec.get("warp_inst_per_step") and clock_mhz:
        issue_rate = rec["warp_inst_per_step"] * steps / walk_s
        issue_peak = num_sms * 4 * clock_mhz * 1e6
        issue = {"warp_inst_per_step": rec["warp_inst_per_step"], "achieved_per_s": issue_rate,
                 "peak_per_s": issue_peak, "frac": issue_rate / issue_peak,
                 "peak_source": f"{num_sms} SMs x 4 schedulers x {clock_mhz:.0f} MHz (median sampled SM clock)"}
    if kernel == "k_walks<4,3>":
        # The tensor-core shape: each 16-bit-weight multiply-add is two f16
        # byte-plane multiply-adds (4 flops) on the tensor cores, against the
        # measured dense f16/bf16 peak; beside it the same work against the
        # legacy mma.sync rate this kernel issues on, and the issue slots.
        peak_tf, peak_src = measured_tensor_tflops(sustained=True)
        flops = 4 * achieved
        mma_sync = None
        if hmma_per_s:
            mma_sync = {"achieved_mac_per_s": 2 * achieved, "peak_mac_per_s": hmma_per_s,
                        "frac": 2 * achieved / hmma_per_s,
                        "peak_source": "measured mma.sync m16n8k16 f16 -> f32 rate (qcs_peak_hmma, this run)"}
        return {"bound": "tensor", "unit": "TFLOP/s", "kernel": kernel,
                "achieved": flops / 1e12, "peak": peak_tf, "frac": flops / 1e12 / peak_tf,
                "peak_source": peak_src, "mma_sync": mma_sync,
                "dp4a_equivalent": {"achieved_gops": achieved / 1e9, "peak_gops": peak / 1e9, "frac": achieved / peak,
                                    "peak_source": "2 x measured dp4a rate (the other shapes' contraction pipe)"},
                "traffic": traffic, "traffic_unit": "bytes per launch", "hbm": hbm, "issue_slots": issue,
                "algorithmic_ops": f"2*d^2 = {2 * d * d} 16-bit-weight multiply-adds per W-side walk step, "
                                   "each two f16 byte-plane multiply-adds (4 flops) on the tensor cores"}
    return {"bound": "alu", "unit": "Gop/s", "kernel": kernel,
            "achieved": achieved / 1e9, "peak": peak / 1e9, "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "bytes per launch", "hbm": hbm, "issue_slots": issue,
            "peak_source": "2 x measured dp4a rate (qcs_peak_idp4a, this run: "
                           f"{dp4a_per_s / 1e9:.0f} G dp4a/s)",
            "algorithmic_ops": f"2*d^2 = {2 * d * d} 16-bit-weight multiply-adds per W-side walk step "
                               "(executed as two byte-plane dp4a per four multiply-adds)"}


# ------------------------------------------------------------------ ranks
def rank_seed(rank: int) -> int:
    """Walk seed of one rank.  Ranks are independent replicas of the level
    walk with disjoint pseudo-random walk families, so their steps add up and
    they never talk except to combine their timings."""
    return 0x5EED0000 + rank


def combine_ranks(t_local: float, units_local: float, world: int, dist=None, device="cpu"):
    """Whole-job timing over ranks: the slowest rank's time and all ranks' units."""
    import torch

    if world <= 1 or dist is None:
        return t_local, units_local
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ------------------------------------------------------------------ CPU oracle
def _oracle_worker(args):
    n, gates, k, chunk, L, states = args
    import oracle

    C = oracle.channel_from_circuit(n, gates)
    t0 = time.perf_counter()
    oracle.walk_step(C, k, chunk, 1, L, states)
    return len(states), time.perf_counter() - t0


def cpu_oracle_rate(budget_s: float, cfg: int = CFG, k: int = K_LEVEL):
    """Oracle walk steps/s on all host cores (spawned pool, one process per
    core) on a bounded sample of the configuration's level-k walk steps."""
    import multiprocessing as mp

    import oracle
    from paper_1606_07413_gb300 import workloads as W

    oracle.build()
    c = W.CONFIGS[cfg]
    gates, _ = W.config_target(cfg)
    cores = os.cpu_count() or 1
    xi = 4 ** c["n"] - 1
    # calibrate one process on a small batch
    _, dt = _oracle_worker((c["n"], gates, k, 3, c["L"], W.seeded_states(16, c["L"], 1)))
    per_step = max(dt / 16, 1e-7)
    per_core = max(16, int(budget_s / per_step / 4))  # about budget_s/4 of wall time per worker
    jobs = [(c["n"], gates, k, 1 + (i % xi), c["L"], W.seeded_states(per_core, c["L"], 100 + i))
            for i in range(cores)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        out = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    steps = sum(o[0] for o in out)
    busy = max(o[1] for o in out)
    return {"value": steps / busy, "unit": "walk_steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} oracle walk steps (n={c['n']}, level {k}, {c['L']}-bit states, seeded) in "
                      f"{cores} spawned processes, {busy:.1f}s of compute ({wall:.1f}s wall incl. start-up)"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        self.path = f"/tmp/qcs_clocks_{os.getpid()}.csv"
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ other workloads
def level_throughput(Q, W, torch, cfg, k, steps, stream, launches=3, alu_per_s=None, dp_bits=None, table_log2=None,
                     target=None, shape=0, c_layout=0):
    """Walk steps/s of one single-target level launch at a configured size
    (dp_bits / table_log2 override the configuration's theta and table;
    target = (n, t, seed) takes another seeded target of that size class),
    and the distinguished-point table's algorithmic traffic: one 16-byte
    exchange (read and write) per distinguished point, 24 bytes per queued
    merge."""
    c = W.CONFIGS[cfg]
    if target is None:
        gates, _ = W.config_target(cfg)
        k_max = c["k_max"]
    else:
        gates, _ = W.seeded_target(*target)
        k_max = k
    dpb = dp_bits or c["dtheta"]
    p = Q.default_params(c["n"], walks=c["walks"], state_bits=c["L"], dp_bits=dpb,
                         table_log2=table_log2 or min(c["table_log2"], 24), launch_shape=shape, c_layout=c_layout)
    prob = Q.Problem.from_circuit(c["n"], gates, k_max, p)
    prob.level_begin(k, 0, dpb, stream=stream)
    prob.level_walk(steps, stream); prob.level_rewalk(stream); prob.level_collect(stream)
    r0 = prob.poll()
    ms = []
    for _ in range(launches):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prob.level_walk(steps, stream)
        e1.record(stream)
        prob.level_rewalk(stream)
        prob.level_collect(stream)
        ms.append(e0.elapsed_time(e1))
    r1 = prob.poll()
    prob.close()
    d = 4 ** c["n"] - 1
    walk_s = sum(ms) / 1e3
    table_bytes = 32 * (r1["dps"] - r0["dps"]) + 24 * (r1["merges"] - r0["merges"])
    name = f"n{c['n']}_level{k}_walks{c['walks']}_L{c['L']}_theta2^-{dpb}"
    if target is not None:
        name += f"_target_n{target[0]}_t{target[1]}_seed{target[2]}"
    out = {"workload": name, "walk_steps_per_s": (r1["steps"] - r0["steps"]) / walk_s,
           "table_gbs": table_bytes / walk_s / 1e9, "launches": launches, "steps_per_walk_per_launch": steps,
           "walk_kernel_s": walk_s}
    if alu_per_s:  # multiply-adds per second at the contraction's peak
        out["alu_frac"] = (r1["w_steps"] - r0["w_steps"]) * 2 * d * d / walk_s / alu_per_s
    return out


def run_batched(Q, W, torch, stream, n_targets=256, mac_peak=None, min_seconds=1.0, repeats=3):
    """The batched workload: many seeded targets in one persistent launch per qubit
    count (one CUDA-graph replay per round) against the same jobs launched
    one target at a time, on identical work (the trajectories are
    deterministic, and each arm runs every job for the same rounds).  The
    rounds double until the batched arm takes at least min_seconds; each arm
    is then timed `repeats` times on fresh copies of the jobs."""
    from paper_1606_07413_gb300 import autotune

    targets = W.batched_targets(n_targets)
    t0 = time.perf_counter()
    best, trials = autotune.tune_batch(targets[:48], rounds=8, stream=stream)
    tune_s = time.perf_counter() - t0

    def mk(i, t):
        return Q.Problem.from_circuit(t["n"], t["gates"], t["t"],
                                      Q.default_params(t["n"], theta_min_bits=best["theta_min_bits"], seed=1000 + i,
                                                       c_layout=best["c_layout"].get(t["n"], 0)))

    def bp(J):
        return Q.default_batch_params(max_jobs=J, walks_per_job=best["walks_per_job"],
                                      steps_per_round=best["steps_per_round"], table_log2=18,
                                      queue_capacity=best["queue_capacity"], launch_shape=best["launch_shape"])

    def batched(rounds):
        probs = [mk(i, t) for i, t in enumerate(targets)]
        with Q.Batch(bp(len(targets)), stream) as b:
            ids = [b.add(p) for p in probs]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(rounds):
                b.round()
            secs = time.perf_counter() - t0
            res = [b.poll(j) for j in ids]
        for p in probs:
            p.close()
        return secs, res

    def one_at_a_time(rounds):
        secs = 0.0
        res = []
        for i, t in enumerate(targets):
            p = mk(i, t)
            with Q.Batch(bp(1), stream) as b:
                j = b.add(p)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(rounds):
                    b.round()
                secs += time.perf_counter() - t0
                res.append(b.poll(j))
            p.close()
        return secs, res

    rounds = 12
    while True:
        secs, res = batched(rounds)
        if secs >= min_seconds or rounds >= 4096:
            break
        rounds *= 2
    b_secs = [secs] + [batched(rounds)[0] for _ in range(repeats - 1)]
    o_runs = [one_at_a_time(rounds) for _ in range(repeats)]
    o_secs = [r[0] for r in o_runs]
    fev = sum(r["steps"] + r["rewalk_steps"] for r in res)
    fev_one = sum(r["steps"] + r["rewalk_steps"] for r in o_runs[0][1])
    walk = sum(r["steps"] for r in res)
    imad = sum(r["w_steps"] * 2 * (4 ** t["n"] - 1) ** 2 for r, t in zip(res, targets))
    tts = sorted(r["seconds"] for r in res if r["status_name"] == "found")
    q = lambda f: tts[min(len(tts) - 1, int(f * len(tts)))] if tts else None
    bs, os_ = statistics.median(b_secs), statistics.median(o_secs)
    return {
        "workload": f"{n_targets} seeded targets, n~U{{2,3,4}}, T-count~U{{3..7}}, {rounds} rounds per job",
        "autotuned": {**best, "launch_shape": {str(k): v for k, v in best["launch_shape"].items()},
                      "c_layout": {str(k): v for k, v in best["c_layout"].items()}},
        "autotune_seconds": tune_s, "autotune_trials": len(trials),
        "batched_fevals_per_s": fev / bs, "one_target_fevals_per_s": fev_one / os_,
        "batched_walk_steps_per_s": walk / bs, "one_target_walk_steps_per_s": walk / os_,
        "speedup": os_ / bs, "speedup_min_max": [min(o_secs) / max(b_secs), max(o_secs) / min(b_secs)],
        "batched_s": b_secs, "one_target_s": o_secs, "repeats": repeats,
        "identical_work": fev == fev_one,
        "contraction_ops_per_s_batched": imad / bs,
        "contraction_alu_frac_batched": (imad / bs / mac_peak) if mac_peak else None,
        "alu_peak_note": "contraction multiply-adds of all jobs against twice the measured dp4a rate",
        "found": len(tts), "time_to_tcount_p50_s": q(0.5), "time_to_tcount_p99_s": q(0.99),
        "graph": "each batched round is one CUDA-graph replay",
    }


def perm_unitary(perm):
    """The permutation matrix of a basis-state permutation, as Z[omega]
    coefficients (4 int64 per entry) over sqrt2^0."""
    d = len(perm)
    u = np.zeros((d, d, 4), np.int64)
    for c, r in enumerate(perm):
        u[r, c, 0] = 1
    return u


def table1_circuits(Q, W, stream, trials=10):
    """Time to the optimal T-count of the paper's named circuits.  Toffoli,
    Fredkin, Peres and OR (Table 1; published means 25.9870 s, 25.0031 s,
    25.4931 s and 24.1854 s on 4096 Blue Gene/Q cores, context only: other
    hardware): each trial is a full ladder from sde = 2 through the public
    API with its own walk seed.  The 4-qubit full adder (Sec. 5.3; the
    paper's first synthesis took 12.5 hours on 4096 cores): one deterministic
    ladder settled by the exhaustive pass alone (every level exact);
    `--adder-walk` times the walk alone."""
    targets = W.permutation_targets()
    paper = {"toffoli": 25.9870, "fredkin": 25.0031, "peres": 25.4931, "quantum_or": 24.1854}
    out = {}
    for name in ("toffoli", "fredkin", "peres", "quantum_or"):
        _, perm = targets[name]
        secs, tcs = [], []
        for t in range(trials):
            p = Q.Problem.from_unitary(3, perm_unitary(perm), 0, 7, Q.default_params(3, seed=0x7AB1E + t))
            t0 = time.perf_counter()
            p.run_walks(stream=stream)
            r = p.wait(600_000)
            secs.append(time.perf_counter() - t0)
            tcs.append(r["t_count"])
            p.close()
        out[name] = {"t_counts": sorted(set(tcs)), "mean_s": float(np.mean(secs)), "sd_s": float(np.std(secs)),
                     "trials": trials, "paper_mean_s_4096_bgq_cores": paper[name]}
    out["adder"] = dict(time_to_optimal(Q, W, stream, 3, "exhaustive", unitary=perm_unitary(targets["adder"][1])),
                        paper_first_synthesis_s_4096_bgq_cores=12.5 * 3600)
    return out


# table of the collision walk for time-to-optimal runs per configuration:
# (table_log2, queue_log2); the level-7 walk at n = 4 gets 16 GiB of table
TTO_TABLES = {1: (16, 20), 2: (22, 20), 3: (28, 24)}


def time_to_optimal(Q, W, stream, cfg, mode="walk", table_log2=None, queue_log2=None, limit_s=900, unitary=None,
                    dp_bits=None, seed=None):
    """Time to the optimal T-count of a configuration's seeded target (or of
    the given n-qubit unitary, Z[omega] coefficients over sqrt2^0), through
    the public API (qcs_create_problem_circuit, qcs_run_walks, qcs_wait).
    mode "walk": the collision search alone (no exhaustive pass) with a
    2^table_log2-slot table (16 bytes a slot) and theta from the Appendix
    policy (or fixed at 2^-dp_bits); mode "exhaustive": every level settled
    by the exhaustive pass alone."""
    c = W.CONFIGS[cfg]
    n = c["n"]
    gates, _ = W.config_target(cfg)
    tl, ql = TTO_TABLES[cfg]
    table_log2 = table_log2 or tl
    queue_log2 = queue_log2 or ql
    if mode == "exhaustive":
        p = Q.default_params(n, exhaustive_first=1, exhaustive_log2=34)
    else:
        extra = {"theta_policy": 0, "dp_bits": dp_bits} if dp_bits else {}
        if seed is not None:
            extra["seed"] = seed
        p = Q.default_params(n, table_log2=table_log2, queue_capacity=1 << queue_log2, exhaustive_log2=0, **extra)
    t0 = time.perf_counter()
    if unitary is None:
        prob = Q.Problem.from_circuit(n, gates, c["k_max"], p)
    else:
        prob = Q.Problem.from_unitary(n, unitary, 0, c["k_max"], p)
    prob.run_walks(stream=stream)
    r = prob.wait(int(limit_s * 1000))
    if r["timed_out"]:
        prob.cancel()
        r = prob.wait(60_000)
        r["status_name"] = "time_limit"
    secs = time.perf_counter() - t0
    sde = prob.sde
    prob.close()
    out = {"mode": mode, "seconds": secs, "status": r["status_name"], "t_count": r["t_count"], "sde": r["sde"],
           "walk_steps": r["steps"], "rewalk_steps": r["rewalk_steps"], "merges": r["merges"],
           "claws": r["claws"], "false_hash": r["false_hash"], "exhaustive_points": r["cert_points"],
           "certified_levels": r["certified_levels"]}
    if mode == "walk":
        k = r["t_count"] if r["t_count"] > 0 else c["k_max"]
        plan = Q.plan_level(n, k, p)
        out.update(table_slots=1 << table_log2, dp_bits=plan["dp_bits"], theta=2.0 ** -plan["dp_bits"],
                   walks=plan["walks"], steps_per_launch=plan["steps"], level_points=plan["points"],
                   walk_steps_over_level_points=r["steps"] / plan["points"],
                   levels=f"{sde}..{k}", theta_rule="fixed" if dp_bits else "Appendix optimum sqrt(2w/N), "
                                                                          "at most 1/2")
    return out


def exhaustive_level_pass(Q, W, stream, n=4, k=7, t=9, seed=4009):
    """One whole exhaustive pass over level k of a seeded n-qubit target whose
    sde is t > k, so no claw exists and every point is evaluated: the worst
    case of the pass at the n = 4 seven-factor target's level (k = 7: 255^3 stored points,
    255^4 streamed)."""
    gates, _ = W.seeded_target(n, t, seed)
    with Q.Problem.from_circuit(n, gates, max(k, t), Q.default_params(n, exhaustive_log2=34)) as prob:
        t0 = time.perf_counter()
        has = prob.certify_level(k, stream=stream)
        secs = time.perf_counter() - t0
        r = prob.poll()
    return {"workload": f"n{n}_level{k}_exhaustive (seeded target of sde {r['sde']}, no claw)",
            "seconds": secs, "points": r["cert_points"], "points_per_s": r["cert_points"] / secs,
            "has_claw": bool(has), "certified_levels": r["certified_levels"]}


def serving_stats(polls, deadline_s):
    """Latency over every request of the stream: a request answered in time
    counts with its latency, one that missed its deadline (dropped in the
    queue, or stopped while running) counts at the deadline and is censored
    (its true time to an answer is longer)."""
    lat = []
    for p in polls:
        if p["status"] == "found":
            lat.append((p["latency"], False))
        else:
            lat.append((deadline_s, True))
    lat.sort()
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))] if lat else (None, False)
    answered = sorted(v for v, cens in lat if not cens)
    qa = lambda f: answered[min(len(answered) - 1, int(f * len(answered)))] if answered else None
    misses = {}
    for p in polls:
        if p["status"] != "found":
            key = f"n{p['n']}_t{p['k_max']}"
            misses[key] = misses.get(key, 0) + 1
    return {"p50_all_s": q(0.5)[0], "p50_all_censored": q(0.5)[1], "p99_all_s": q(0.99)[0],
            "p99_all_censored": q(0.99)[1], "miss_rate": sum(c for _, c in lat) / max(1, len(lat)),
            "misses_by_class": dict(sorted(misses.items())), "answered_p50_s": qa(0.5), "answered_p99_s": qa(0.99),
            "note": "p50/p99 over all requests; a missed request counts at the deadline (censored)"}


def run_serving(Q, W, torch, stream, tuned, n_requests=2000, rate=50.0, budget_bytes=16 << 30,
                deadline_s=10.0, drain_s=15.0, cert_points_log2=24):
    """The serving workload: a Poisson stream of seeded targets replayed in real time
    into the continuous-batching server; latency is arrival to answer, and
    the deadline counts from arrival too."""
    from paper_1606_07413_gb300 import serve

    times, targets = W.poisson_arrivals(n_requests, rate)
    bp = Q.default_batch_params(max_jobs=512, walks_per_job=tuned["walks_per_job"],
                                steps_per_round=tuned["steps_per_round"], table_log2=18,
                                queue_capacity=tuned["queue_capacity"],
                                launch_shape={int(k): v for k, v in tuned.get("launch_shape", {}).items()},
                                cert_points_log2=cert_points_log2)
    layouts = {int(k): v for k, v in tuned.get("c_layout", {}).items()}
    # serving policy: every level of at most 2^32 V + W points (all levels of
    # this stream, n = 4 level 7 included) is settled by the exact pass
    policy = {"theta_min_bits": tuned["theta_min_bits"], "exhaustive_first": 1, "exhaustive_log2": 32}
    with serve.Server(bp, budget_bytes, stream=stream, deadline_s=deadline_s,
                      params_for=lambda n: Q.default_params(n, c_layout=layouts.get(n, 0), **policy)) as srv:
        rids, wall = serve.replay_stream(srv, times, targets, time_limit_s=float(times[-1]) + drain_s)
        polls = [srv.poll(r) for r in rids]
        fevals, rounds, peak, cert_points = srv.fevals, srv.rounds, srv.peak_used, srv.cert_points
    status = {}
    for p in polls:
        status[p["status"]] = status.get(p["status"], 0) + 1
    offered = {}
    for t in targets:
        key = f"n{t['n']}_t{t['t']}"
        offered[key] = offered.get(key, 0) + 1
    span = float(times[-1])
    return {
        "workload": f"{n_requests} seeded targets, Poisson arrivals at {rate}/s, n~U{{2,3,4}}, T-count~U{{3..7}}",
        **serving_stats(polls, deadline_s), "status_counts": status,
        "offered_per_s_by_class": {k: v / span for k, v in sorted(offered.items())},
        "fevals_per_s": fevals / wall, "exhaustive_points_per_s": cert_points / wall, "wall_s": wall, "rounds": rounds, "memory_budget_bytes": budget_bytes,
        "peak_admitted_bytes": peak, "deadline_s": deadline_s,
        "policy": dict(policy, cert_points_log2=cert_points_log2,
                       note="exhaustive pass first on every level of at most 2^32 V + W points (n = 4 level 7: "
                            "4.2e9 points, a 512 MiB key table held by its job and reserved at admission); a round "
                            f"runs at most 2^{cert_points_log2} points of the passes, oldest job first; a request "
                            "still queued at its deadline is dropped unanswered"),
    }


# ------------------------------------------------------------------ GPU arm
def timed_level(Q, torch, prob, stream, k, dp_bits, steps, warmup, launches, flush):
    """`warmup` untimed then `launches` timed bench steps of one level: the
    walk launch, the re-walk and the host collect, each step bracketed by
    CUDA events on the launching stream (L2 flushed before each step,
    outside the events).  Returns (step ms list, walk-kernel ms list, result
    before, result after)."""
    with torch.cuda.stream(stream):
        prob.level_begin(k, version=0, dp_bits=dp_bits, stream=stream)
        for _ in range(warmup):
            prob.level_walk(steps, stream)
            prob.level_rewalk(stream)
            prob.level_collect(stream)
    torch.cuda.synchronize()
    r0 = prob.poll()
    step_ms, walk_ms = [], []
    split = {"walk_ms": 0.0, "rewalk_ms": 0.0, "collect_ms": 0.0}
    with torch.cuda.stream(stream):
        for _ in range(launches):
            flush.zero_()  # evict L2 between steps (outside the timed events)
            e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            e0.record(stream)
            prob.level_walk(steps, stream)
            e1.record(stream)
            prob.level_rewalk(stream)
            e2.record(stream)
            prob.level_collect(stream)  # synchronizes and checks claw candidates on the host
            e3.record(stream)
            e3.synchronize()
            step_ms.append(e0.elapsed_time(e3))
            walk_ms.append(e0.elapsed_time(e1))
            split["walk_ms"] += e0.elapsed_time(e1)
            split["rewalk_ms"] += e1.elapsed_time(e2)
            split["collect_ms"] += e2.elapsed_time(e3)
    torch.cuda.synchronize()
    timed_level.split = {k: v / max(1, launches) for k, v in split.items()}
    return step_ms, walk_ms, r0, prob.poll()


def timed_sharded_level(Q, torch, prob, stream, k, dp_bits, steps, warmup, launches, flush, walks, dev):
    """The level walked by every rank with distinguished points exchanged
    with their owner ranks (DP-owner sharding, paper_1606_07413_gb300.shard):
    `warmup` untimed then `launches` timed rounds (walk, bin, all-to-all,
    insert, re-walk, collect), each bracketed by CUDA events on the launching
    stream.  Returns (round ms list, walk-kernel ms list, result before, result
    after, points lost to a full outbox)."""
    import torch.distributed as dist

    from paper_1606_07413_gb300 import shard

    world = dist.get_world_size()
    cap = 4 * max(1 << 16, (walks * steps) >> max(0, dp_bits - 2))  # 16 x the expected points, at least 2^18
    eng = shard.DeviceEngine(prob, dev, cap, world, stream)
    lvl = shard.ShardedLevel(eng, walks)
    with torch.cuda.stream(stream):
        lvl.begin(k, 0, dp_bits)
        for _ in range(warmup):
            lvl.round(steps)
    torch.cuda.synchronize()
    r0 = prob.poll()
    step_ms, walk_ms = [], []
    with torch.cuda.stream(stream):
        for _ in range(launches):
            flush.zero_()
            e0, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lvl.round(steps)
            e3.record(stream)
            e3.synchronize()
            step_ms.append(e0.elapsed_time(e3))
    torch.cuda.synchronize()
    return step_ms, walk_ms, r0, prob.poll(), lvl.lost


def e2e_run(Q, torch, cfg_c, gates, k, steps_per_launch, launches, stream, seed, shape):
    """The headline metric through the public API: problem creation from the
    host gate list (uploads C^ and its tables), qcs_run_walks with a step
    budget of `launches` bench steps, and the per-launch reads of the
    counters and queued candidates; the byte counts are the ones the library
    reports it copied."""
    c = cfg_c
    budget = launches * c["walks"] * steps_per_launch
    pe = Q.default_params(c["n"], walks=c["walks"], state_bits=c["L"], dp_bits=c["dtheta"],
                          table_log2=c["table_log2"], theta_policy=0, version_factor=0,
                          steps_per_launch=steps_per_launch, budget_factor=1 << 20, stop_on_claw=0,
                          exhaustive_log2=0, seed=seed, launch_shape=shape["launch_shape"],
                          c_layout=shape["c_layout"], rewalk_budget=REWALK_BUDGET)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pb = Q.Problem.from_circuit(c["n"], gates, k, pe)
    pb.run_walks(step_budget=budget, stream=stream)
    re = pb.wait(600_000)
    t_e2e = time.perf_counter() - t0
    pb.close()
    n_launch = max(re["launches"], 1)
    return {"value": re["steps"] / t_e2e, "unit": "walk_steps/s",
            "h2d_bytes_per_step": re["h2d_bytes"] / n_launch, "d2h_bytes_per_step": re["d2h_bytes"] / n_launch,
            "h2d_bytes": re["h2d_bytes"], "d2h_bytes": re["d2h_bytes"], "steps": re["steps"],
            "seconds": t_e2e, "launches": n_launch,
            "path": "qcs_create_problem_circuit + qcs_run_walks + qcs_poll_collisions/qcs_wait; bytes as counted "
                    "by the library (C^ and its tables up, counters and queued candidates down)"}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1606_07413_gb300 as Q
    from paper_1606_07413_gb300 import build as B
    from paper_1606_07413_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    sharded = world > 1 or args.sharded
    if sharded:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_base = cpu_oracle_rate(args.cpu_seconds)  # before any GPU work in this process

    B.build()
    c = W.CONFIGS[CFG]
    gates, _ = W.config_target(CFG)
    # replicas of one level would each need their own walk seed; the sharded
    # level (N > 1) walks one level over all ranks with one seed
    params = Q.default_params(c["n"], walks=c["walks"], state_bits=c["L"], dp_bits=c["dtheta"],
                              table_log2=c["table_log2"], seed=rank_seed(0), rewalk_budget=REWALK_BUDGET)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # measured integer-ALU peaks: IMAD (the 32-bit contraction) and dp4a
    # (the byte-plane contraction, n >= 3 with C^ in int8)
    Q.measure_int_peak("imad", 8, 512)
    imad_per_s, _ = Q.measure_int_peak("imad", 8, 4096)
    dp4a_per_s, _ = Q.measure_int_peak("idp4a", 8, 4096)
    hmma_per_s, _ = Q.measure_int_peak("hmma", 4, 512)

    # launch shape and C^ layout of the level walk, chosen by the autotuner on
    # this level (the walks are the same under every choice)
    from paper_1606_07413_gb300 import autotune

    def tune_problem(**kw):
        pt = Q.default_params(c["n"], walks=c["walks"], state_bits=c["L"], dp_bits=c["dtheta"], table_log2=24,
                              seed=rank_seed(rank), **kw)
        return Q.Problem.from_circuit(c["n"], gates, K_LEVEL, pt)

    shape, shape_trials = autotune.tune_level_shape(c["n"], tune_problem, K_LEVEL, 16, stream)
    params.launch_shape, params.c_layout = shape["launch_shape"], shape["c_layout"]
    prob = Q.Problem.from_circuit(c["n"], gates, K_LEVEL, params)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t_wall = time.perf_counter()
    lost = None
    if sharded:
        # one level over every rank, distinguished points exchanged with their owners
        step_ms, walk_ms, r0, r1, lost = timed_sharded_level(Q, torch, prob, stream, K_LEVEL, c["dtheta"],
                                                             STEPS_PER_LAUNCH, args.warmup, args.steps, flush,
                                                             c["walks"], dev)
    else:
        step_ms, walk_ms, r0, r1 = timed_level(Q, torch, prob, stream, K_LEVEL, c["dtheta"], STEPS_PER_LAUNCH,
                                               args.warmup, args.steps, flush)
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    prob.close()
    steps_done = r1["steps"] - r0["steps"]
    w_steps = r1["w_steps"] - r0["w_steps"]
    t_local = sum(step_ms) / 1e3
    t_all, steps_all = combine_ranks(t_local, float(steps_done), world, dist if world > 1 else None, dev)
    value = steps_all / t_all
    walk_s = sum(walk_ms) / 1e3 if walk_ms else t_local  # sharded rounds time the whole round
    roof = walk_roofline(f"k_walks<{c['n']},{shape['launch_shape']}>", c["n"], w_steps, steps_done, walk_s,
                         args.steps, dp4a_per_s, clk.get("sm_mhz"), num_sms, hmma_per_s)
    roof["walk_kernel_share"] = walk_s / t_local
    step_split = getattr(timed_level, "split", None) if not sharded else None
    roof["imad_measured_gops"] = imad_per_s / 1e9

    e2e = None
    extra = {}
    if rank == 0:
        e2e = e2e_run(Q, torch, c, gates, K_LEVEL, STEPS_PER_LAUNCH, args.steps, stream, 0xE2E, shape)
        # the other workloads run once, on one GPU (N > 1 holds every GPU only for the sharded headline)
        if not args.no_tts and world == 1:
            extra["tto_walk_cfg1"] = time_to_optimal(Q, W, stream, 1, "walk")
            extra["tto_walk_cfg2"] = time_to_optimal(Q, W, stream, 2, "walk")
            extra["tto_walk_cfg3"] = time_to_optimal(Q, W, stream, 3, "walk", limit_s=300)
            extra["tto_exhaustive_cfg2"] = time_to_optimal(Q, W, stream, 2, "exhaustive")
            extra["tto_exhaustive_cfg3"] = time_to_optimal(Q, W, stream, 3, "exhaustive")
        if not args.no_extra and world == 1:
            c2 = W.CONFIGS[2]
            g2, _ = W.config_target(2)
            p2 = Q.default_params(c2["n"], walks=c2["walks"], state_bits=c2["L"], dp_bits=c2["dtheta"],
                                  table_log2=c2["table_log2"], seed=rank_seed(rank))
            prob2 = Q.Problem.from_circuit(c2["n"], g2, 5, p2)
            s2, w2, q0, q1 = timed_level(Q, torch, prob2, stream, 5, c2["dtheta"], 512, 3, 20, flush)
            prob2.close()
            st2 = q1["steps"] - q0["steps"]
            extra["n3_level5"] = {
                "config": workload_config(c2, 5, 512, 0), "walk_steps_per_s": st2 / (sum(s2) / 1e3),
                "ms_per_step": sum(s2) / len(s2),
                "roofline": walk_roofline("k_walks<3,0>", 3, q1["w_steps"] - q0["w_steps"], st2, sum(w2) / 1e3, 20,
                                          dp4a_per_s, clk.get("sm_mhz"), num_sms)}
            batched = run_batched(Q, W, torch, stream, mac_peak=2 * dp4a_per_s)
            extra.update({
                "batched": batched,
                "serving": run_serving(Q, W, torch, stream, batched["autotuned"]),
                "table1_circuits": table1_circuits(Q, W, stream),
                "n4_level7_exhaustive_pass": exhaustive_level_pass(Q, W, stream),
                "n2_level3": level_throughput(Q, W, torch, 1, 3, 512, stream, alu_per_s=imad_per_s),
                # the table at its busiest: half the points distinguished
                "n3_level5_theta_half": level_throughput(Q, W, torch, 2, 5, 64, stream, alu_per_s=2 * dp4a_per_s,
                                                         dp_bits=1, table_log2=26),
                # targets whose reduced C^ leaves int8: the 32-bit word contraction (IMAD; n = 4 reads C^
                # through L2), against the measured IMAD rate
                "c32_n3_level5": level_throughput(Q, W, torch, 2, 5, 512, stream, alu_per_s=imad_per_s,
                                                  target=(3, 19, 4019)),
                "c32_n4_level7": level_throughput(Q, W, torch, 3, 7, 16, stream, alu_per_s=imad_per_s,
                                                  target=(4, 15, 4015)),
            })

    if rank == 0:
        line = {
            "metric": "walk_steps_per_sec", "value": value, "unit": "walk_steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_all * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded target C0.R(P7)..R(P1), n=4)",
            "config": dict(workload_config(c), launch_shape=Q.launch_shapes(c["n"])[shape["launch_shape"]],
                           c_layout=["int8 byte quads (dp4a)", "32-bit words (IMAD)"][shape["c_layout"]]),
            "autotuned_level_shape": shape_trials, "roofline": roof, "cpu_baseline": cpu_base, "e2e": e2e, "clocks": clk,
            "gpu_launches": (5 if sharded else 2) * args.steps, "wall_s": wall,
            "step_split_ms": dict(step_split or {}, note="per bench step: walk kernel; re-walk kernel and the "
                                                         "reads of its results; host wait and exact checks of "
                                                         "claw candidates"),
            "headline_counts": {k: r1[k] - r0[k] for k in ("steps", "w_steps", "dps", "merges", "claws",
                                                            "false_hash", "robin_hood", "rewalk_steps")},
        }
        if sharded:
            line["config"]["parallelism"] = (f"DP-owner sharding over {world} ranks: one level, every rank walks "
                                             f"{c['walks']} walks and owns a hash share of the distinguished points "
                                             "(all-to-all exchange per round)")
            line["points_lost_to_outbox"] = lost
        line.update(extra)
        print(json.dumps(line))
    if sharded:
        dist.destroy_process_group()


def run_reference(args):
    """The CPU oracle, as it stands, on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1606_07413_gb300 import workloads as W

    c = W.CONFIGS[CFG]
    per = max(args.cpu_seconds / max(args.steps + args.warmup, 1), 2.0)
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(per)
        if i >= args.warmup:
            vals.append(r)
    value = statistics.median(v["value"] for v in vals)
    base = dict(vals[-1])
    base["value"] = value
    line = {"metric": "walk_steps_per_sec", "value": value, "unit": "walk_steps/s", "impl": "reference",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded target C0.R(P7)..R(P1), n=4)", "config": workload_config(c),
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "walk_steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_level_only(args):
    import torch

    import paper_1606_07413_gb300 as Q
    from paper_1606_07413_gb300 import build as B
    from paper_1606_07413_gb300 import workloads as W

    B.build()
    stream = torch.cuda.Stream()
    cfg, k, steps = {"n2_level3": (1, 3, 512), "n3_level5": (2, 5, 512), "n4_level7": (3, 7, 16)}[args.level_only]
    Q.measure_int_peak("imad", 8, 512)
    peak = Q.measure_int_peak("imad" if cfg == 1 else "idp4a", 8, 4096)[0] * (1 if cfg == 1 else 2)
    print(json.dumps({args.level_only: level_throughput(Q, W, torch, cfg, k, steps, stream, launches=args.steps,
                                                        alu_per_s=peak, shape=args.shape, c_layout=args.c_layout)}))


def run_batched_only(args):
    import torch

    import paper_1606_07413_gb300 as Q
    from paper_1606_07413_gb300 import build as B
    from paper_1606_07413_gb300 import workloads as W

    B.build()
    Q.measure_int_peak("idp4a", 8, 512)
    peak = 2 * Q.measure_int_peak("idp4a", 8, 4096)[0]
    print(json.dumps({"batched": run_batched(Q, W, torch, torch.cuda.Stream(), mac_peak=peak)}))


def run_config3_walk(args):
    import torch

    import paper_1606_07413_gb300 as Q
    from paper_1606_07413_gb300 import build as B
    from paper_1606_07413_gb300 import workloads as W

    B.build()
    stream = torch.cuda.Stream()
    if args.adder_walk:
        u = perm_unitary(W.permutation_targets()["adder"][1])
        print(json.dumps({"adder_time_to_optimal": time_to_optimal(Q, W, stream, 3, "walk", args.adder_walk,
                                                                  unitary=u)}))
    else:
        print(json.dumps({"tto_walk_cfg3": time_to_optimal(Q, W, stream, 3, "walk", args.config3_walk)}))


def run_tto_sweep(args):
    """The n = 4 seeded target's collision walk over table sizes w and
    distinguished fractions theta (the Appendix's steps per collision,
    N theta / w + 2 / theta, against measured time)."""
    import torch

    import paper_1606_07413_gb300 as Q
    from paper_1606_07413_gb300 import build as B
    from paper_1606_07413_gb300 import workloads as W

    B.build()
    stream = torch.cuda.Stream()
    out = []
    # each (table, theta) with three walk seeds: one seeded trajectory is a
    # single draw of a random search's time
    for table_log2, dp_bits in ((28, None), (30, None), (30, 2), (32, None)):
        for seed in (0x2545F4914F6CDD1D, 11, 12):
            r = time_to_optimal(Q, W, stream, 3, "walk", table_log2, limit_s=240, dp_bits=dp_bits, seed=seed)
            r["seed"] = seed
            out.append(r)
            print(json.dumps(r), file=sys.stderr)
    print(json.dumps({"tto_walk_cfg3_sweep": out}))


def run_theta_shapes(args):
    """Walk steps/s of the dp4a shape (0) and the tensor-core shape (3) at
    theta = 2^-2, 2^-4, 2^-8 and 2^-12 (one warm-up and four timed 16-step
    launches of 2^20 walks at n = 4, level 7)."""
    import torch

    import paper_1606_07413_gb300 as Q
    from paper_1606_07413_gb300 import build as B
    from paper_1606_07413_gb300 import workloads as W

    B.build()
    stream = torch.cuda.Stream()
    out = {}
    for dp_bits in (2, 4, 8, 12):
        for shape in (0, 3):
            r = level_throughput(Q, W, torch, 3, 7, 16, stream, launches=4, dp_bits=dp_bits, shape=shape)
            out[f"theta2^-{dp_bits}_shape{shape}"] = r["walk_steps_per_s"]
    print(json.dumps({"n4_level7_theta_shapes": out}))


def run_exhaustive_only(args):
    import torch

    import paper_1606_07413_gb300 as Q
    from paper_1606_07413_gb300 import build as B
    from paper_1606_07413_gb300 import workloads as W

    B.build()
    print(json.dumps({"n4_level7_exhaustive_pass": exhaustive_level_pass(Q, W, torch.cuda.Stream())}))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.exhaustive_only:
        run_exhaustive_only(a)
    elif a.tto_sweep:
        run_tto_sweep(a)
    elif a.theta_shapes:
        run_theta_shapes(a)
    elif a.config3_walk or a.adder_walk:
        run_config3_walk(a)
    elif a.level_only:
        run_level_only(a)
    elif a.batched_only:
        run_batched_only(a)
    else:
        run_ours(a)
