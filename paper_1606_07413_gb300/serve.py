"""Serving loop: continuous batching of synthesis requests on one GPU.

Requests (a target and its k_max) arrive at any time.  Between two rounds of
the batched search (qcs_batch_*) the server admits waiting requests while a
job slot and enough device memory for the job's walk states, distinguished-
point table and merge queue are free, then runs one round for every admitted
job, so new work overlaps on the device with the work already there.  A job
may settle a level by the exhaustive pass, which holds a key table until the
pass ends (a round runs a bounded share of the passes, oldest job first), so
each job is admitted with room for its largest such table.  A job
leaves the batch as soon as it has its answer (or passes its deadline) and
its memory is released for the next request.  Times are measured from each
request's arrival to its answer, and so is the deadline: a request still
waiting when its deadline passes is dropped without running, so that the
GPU's time goes to requests that can still be answered in time.
"""
from __future__ import annotations

import collections
import concurrent.futures
import os
import time

import numpy as np

import paper_1606_07413_gb300 as Q


def exhaustive_table_bytes(params, n: int | None = None, k_max: int | None = None) -> int:
    """Key table of the largest exhaustive level pass a request may run under
    these search parameters (16 bytes a slot).  The pass stores the xi^h
    points of its smaller side (xi = 4^n - 1, h = floor(k/2)) in a power-of-two
    table of at least twice as many slots and at least 1024, and runs only on
    levels 2..k_max of at most 2^exhaustive_log2 V + W points.  Without n and
    k_max: the bound 16 x 2^exhaustive_log2 over every level size."""
    e = int(getattr(params, "exhaustive_log2", 0) or 0)
    if e <= 0:
        return 0
    if n is None or k_max is None:
        return 16 << max(e, 10)
    xi = 4 ** int(n) - 1
    most = 0
    for k in range(2, int(k_max) + 1):
        stored = xi ** (k // 2)
        if stored + stored * (xi if k & 1 else 1) > 1 << e:
            continue
        slots = 1024
        while slots < 2 * stored:
            slots <<= 1
        most = max(most, 16 * slots)
    return most


class Request:
    __slots__ = ("rid", "n", "gates", "k_max", "params", "t_arrival", "t_admit", "t_done", "prob", "slot",
                 "bytes", "table_bytes", "status", "result", "future")

    def __init__(self, rid, n, gates, k_max, params, t_arrival):
        self.rid, self.n, self.gates, self.k_max, self.params = rid, n, gates, k_max, params
        self.t_arrival, self.t_admit, self.t_done = t_arrival, None, None
        self.prob, self.slot, self.bytes, self.table_bytes = None, None, 0, 0
        self.status, self.result, self.future = "queued", None, None


class Server:
    def __init__(self, batch_params: Q.BatchParams, memory_budget: int, stream=None, deadline_s: float | None = None,
                 clock=time.perf_counter, params_for=None):
        """params_for(n) gives the search parameters of an n-qubit request
        that comes without its own (default: Q.default_params(n))."""
        self.batch = Q.Batch(batch_params, stream)
        self.params_for = params_for or Q.default_params
        self.slots = batch_params.max_jobs
        self.budget, self.used = int(memory_budget), 0
        self.deadline = deadline_s
        self.clock = clock
        self.waiting = collections.deque()
        self.running = {}
        self.requests = {}
        self.rounds = 0
        self.fevals = 0
        self.cert_points = 0
        self.next_id = 0
        self.peak_used = 0
        # the exact host set-up of a target (channel representation, upload)
        # runs on worker threads so that it overlaps the rounds
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1))

    # ---- client side ----------------------------------------------------
    def submit(self, n, gates, k_max, params: Q.Params | None = None, t_arrival: float | None = None) -> int:
        rid = self.next_id
        self.next_id += 1
        r = Request(rid, n, np.asarray(gates, np.int32), k_max, params,
                    self.clock() if t_arrival is None else t_arrival)
        p = params or self.params_for(n)
        r.table_bytes = exhaustive_table_bytes(p, n, k_max) if p is not None else 0
        r.future = self.pool.submit(Q.Problem.from_circuit, n, r.gates, k_max, p)
        self.requests[rid] = r
        self.waiting.append(r)
        return rid

    def poll(self, rid: int) -> dict:
        r = self.requests[rid]
        out = {"status": r.status, "n": r.n, "k_max": r.k_max, "t_arrival": r.t_arrival, "t_admit": r.t_admit,
               "t_done": r.t_done}
        if r.result is not None:
            out.update(t_count=r.result["t_count"], paulis=r.result["paulis"], steps=r.result["steps"],
                       latency=r.t_done - r.t_arrival)
        return out

    # ---- server side ----------------------------------------------------
    def _expired(self, r, now) -> bool:
        return self.deadline is not None and now - r.t_arrival > self.deadline

    def _drop_expired(self):
        """Requests whose deadline passed while they waited leave unanswered."""
        now = self.clock()
        keep = collections.deque()
        for r in self.waiting:
            if self._expired(r, now):
                r.status, r.t_done = "deadline", now
                r.future.add_done_callback(lambda f: f.result().close())
            else:
                keep.append(r)
        self.waiting = keep

    def _admit(self, block: bool = False):
        """Admit waiting requests in arrival order while job slots are free.
        A request that does not fit the free memory, or whose set-up is
        still running, is passed over for now and later ones that fit are
        admitted (backfilling), so one large job waiting for memory does not
        hold back small ones; it keeps its place in the order."""
        self._drop_expired()
        kept = collections.deque()
        while self.waiting and len(self.running) < self.slots:
            r = self.waiting.popleft()
            if not r.future.done() and not (block and not self.running):
                kept.append(r)  # its set-up is still running
                continue
            prob = r.future.result()
            need = self.batch.job_bytes(prob) + r.table_bytes
            if self.used + need > self.budget and self.running:
                kept.append(r)  # does not fit now: wait for memory, let later ones try
                continue
            try:
                slot = self.batch.add(prob)
            except Q.QcsError as e:
                if e.code != Q.ERR_BUSY:
                    raise
                kept.append(r)
                break  # every job slot of the batch is taken (also by jobs added directly)
            r.prob, r.bytes, r.slot = prob, need, slot
            r.t_admit = self.clock()
            r.status = "running"
            self.used += need
            self.peak_used = max(self.peak_used, self.used)
            self.running[r.slot] = r
        kept.extend(self.waiting)
        self.waiting = kept

    def _finish(self, r, status, result):
        r.status, r.result, r.t_done = status, result, self.clock()
        self.fevals += result["steps"] + result["rewalk_steps"]
        self.cert_points += result.get("cert_points", 0)
        self.batch.remove(r.slot)
        r.prob.close()
        r.prob = None
        self.used -= r.bytes
        del self.running[r.slot]

    def step(self) -> int:
        """Admit, run one round, harvest; returns the number of running jobs."""
        self._admit(block=True)
        if not self.running:
            return 0
        self.batch.round()
        self.rounds += 1
        now = self.clock()
        for slot, r in list(self.running.items()):
            res = self.batch.poll(slot)
            if res["status_name"] != "searching":
                self._finish(r, res["status_name"], res)
            elif self._expired(r, now):
                self._finish(r, "deadline", res)
        return len(self.running)

    def idle(self) -> bool:
        return not self.waiting and not self.running

    def close(self):
        for r in list(self.running.values()):
            self.batch.remove(r.slot)
            r.prob.close()
        self.running.clear()
        for r in self.waiting:
            p = r.future.result()
            p.close()
        self.waiting.clear()
        self.pool.shutdown()
        self.batch.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def replay_stream(server: Server, arrivals, targets, time_limit_s: float):
    """Feed a timed stream (arrival offsets in seconds) into the server in
    real time; returns the per-request latencies of the answered ones and the
    wall time."""
    t0 = server.clock()
    order = list(zip(arrivals, targets))
    i = 0
    rids = []
    while True:
        now = server.clock() - t0
        while i < len(order) and order[i][0] <= now:
            a, t = order[i]
            rids.append(server.submit(t["n"], t["gates"], t["t"], t_arrival=t0 + a))
            i += 1
        busy = server.step()
        if i == len(order) and server.idle():
            break
        if server.clock() - t0 > time_limit_s:
            break
        if not busy and i < len(order):
            time.sleep(max(0.0, min(0.002, order[i][0] - (server.clock() - t0))))
    wall = server.clock() - t0
    return rids, wall
