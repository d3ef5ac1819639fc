"""The autotuner's selection logic on CPU (paper_1606_07413_gb300.autotune):
against a fake batch engine with a known cost model, it must time every
setting of the grid on the same jobs and keep the one that finishes the most
jobs per second, breaking ties by walk steps per second."""
import itertools

import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import autotune


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


CLOCK = FakeClock()


class FakeProblem:
    def __init__(self, n, gates, k, params):
        self.n = n

    def close(self):
        pass


class FakeBatch:
    """A job needs `need` rounds, fewer with more walks; a round costs time
    in proportion to the walks and steps it runs."""

    def __init__(self, bp, stream=None):
        self.bp = bp
        self.jobs = []
        self.rounds = 0

    def add(self, p):
        self.jobs.append(p)
        return len(self.jobs) - 1

    def round(self):
        self.rounds += 1
        CLOCK.t += 1e-6 * self.bp.walks_per_job * self.bp.steps_per_round * len(self.jobs)
        return len(self.jobs)

    def _need(self):
        return max(1, 40000 // (self.bp.walks_per_job * self.bp.steps_per_round))

    def poll(self, j):
        done = self.rounds >= self._need()
        return {"status_name": "found" if done else "searching",
                "steps": self.rounds * self.bp.walks_per_job * self.bp.steps_per_round}

    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(Q, "Batch", FakeBatch)
    monkeypatch.setattr(Q.Problem, "from_circuit", classmethod(lambda cls, *a: FakeProblem(*a)))
    monkeypatch.setattr(autotune.time, "perf_counter", CLOCK)


def test_tuner_times_every_setting_and_keeps_the_fastest(fake):
    targets = [{"n": 2, "t": 3, "gates": [[0, 0, 0]]} for _ in range(4)]
    grid = {"walks_per_job": (512, 2048), "steps_per_round": (16, 64), "theta_min_bits": (1,),
            "queue_capacity": (4096,)}
    best, trials = autotune.tune_batch(targets, rounds=8, grid=grid, shapes=False)
    assert len(trials) == 4
    seen = {(t["walks_per_job"], t["steps_per_round"]) for t in trials}
    assert seen == set(itertools.product((512, 2048), (16, 64)))
    key = lambda t: (t["jobs_per_s"], t["steps_per_s"])
    top = max(trials, key=key)
    assert best == {k: top[k] for k in grid}
    # in this cost model only settings that finish within 8 rounds find jobs
    for t in trials:
        need = max(1, 40000 // (t["walks_per_job"] * t["steps_per_round"]))
        assert (t["found"] > 0) == (need <= 8)


class ShapedBatch(FakeBatch):
    """Round time depends on the launch shape of each qubit count present and
    on the C^ layout of its jobs: n = 3 is fastest with shape 2 and int8
    quads, n = 4 with shape 1 and 32-bit words."""

    COST = {2: [1.0], 3: [3.0, 2.5, 1.0, 4.0], 4: [5.0, 4.0, 6.0, 4.5]}

    def add(self, p):
        p.layout = p.params_layout
        return super().add(p)

    def round(self):
        self.rounds += 1
        for p in self.jobs:
            shape = self.bp.launch_shape[p.n - 1]
            base = self.COST[p.n][shape]
            fast_layout = 0 if p.n == 3 else 1
            CLOCK.t += 1e-3 * base * (1.0 if p.layout == fast_layout else 1.5)
        return len(self.jobs)


def test_tuner_picks_each_qubit_counts_fastest_shape_and_layout(monkeypatch):
    class P(FakeProblem):
        def __init__(self, n, gates, k, params):
            super().__init__(n, gates, k, params)
            self.params_layout = params.c_layout

    monkeypatch.setattr(Q, "Batch", ShapedBatch)
    monkeypatch.setattr(Q.Problem, "from_circuit", classmethod(lambda cls, *a: P(*a)))
    monkeypatch.setattr(autotune.time, "perf_counter", CLOCK)
    targets = [{"n": n, "t": 3, "gates": [[0, 0, 0]]} for n in (2, 3, 4, 3)]
    grid = {"walks_per_job": (512,), "steps_per_round": (16,), "theta_min_bits": (1,), "queue_capacity": (4096,)}
    best, trials = autotune.tune_batch(targets, rounds=4, grid=grid)
    assert best["launch_shape"] == {3: 2, 4: 1} and best["c_layout"] == {3: 0, 4: 1}
    # one host trial, then every (shape, layout) pair of n = 3 (4 x 2) and n = 4 (4 x 2)
    assert len(trials) == 1 + 8 + 8
    assert [s["shape"] for s in Q.launch_shapes(3)] == [0, 1, 2, 3]
