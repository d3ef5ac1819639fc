"""The batched search (qcs_batch_*): many targets in one persistent launch per
qubit count, each round one CUDA-graph replay.  Every job must reach the
optimal T-count the oracle fixes, with an exactly verified decomposition, and
a job's walks must be the same alone and in a mix (its trajectories depend
only on its own seed and level plan)."""
import numpy as np
import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    from paper_1606_07413_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def small_params(**over):
    return Q.default_batch_params(max_jobs=16, walks_per_job=512, steps_per_round=32, table_log2=16,
                                  queue_capacity=1 << 14, **over)


def run_to_end(batch, max_rounds=400):
    for _ in range(max_rounds):
        if batch.round() == 0:
            return True
    return False


@pytest.mark.parametrize("budget", [0, 3, 64])
def test_batch_reaches_optimal_tcounts(orc, dev, budget):
    # budget: evaluations of f a re-walk may take per round (0: no bound);
    # a re-walk that runs out resumes in the next round
    cases = []
    g1, _ = W.config_target(1)
    cases.append((2, g1, 3))
    g2, _ = W.config_target(2)
    cases.append((3, g2, 5))
    cases.append((1, np.asarray([(W.OP_T, 0, 0)], np.int32), 3))                  # T-count 1 (level 1)
    cases.append((2, W.clifford_word(np.random.default_rng(1), 2, 30), 3))        # Clifford (level 0)
    for s in (71, 72):
        gs, _ = W.seeded_target(2, 2, s)
        cases.append((2, gs, 3))
    probs, jobs = [], []
    with Q.Batch(small_params(rewalk_budget=budget), torch.cuda.Stream()) as batch:
        for n, gates, kmax in cases:
            p = Q.Problem.from_circuit(n, gates, kmax, Q.default_params(n))
            probs.append(p)
            jobs.append(batch.add(p))
        assert run_to_end(batch, 4000)
        for (n, gates, kmax), j in zip(cases, jobs):
            r = batch.poll(j)
            C = orc.channel_from_circuit(n, gates)
            if n == 3:
                want = 5  # sde 5 = construction count
                assert orc.sde(C) == 5
            else:
                want, _ = orc.mitm_tcount(C, kmax)
            assert r["status_name"] == "found" and r["t_count"] == want, (n, r)
            assert orc.verify(C, r["paulis"])
    for p in probs:
        p.close()


def toffoli_unitary():
    u = np.zeros((8, 8, 4), np.int64)
    for c in range(8):
        u[c ^ (4 if (c & 3) == 3 else 0), c, 0] = 1
    return u


def _walk_counts(others, rounds, graph=1, seed=7):
    """(steps, w_steps, dps, abandoned, level, status) of a probe job after
    `rounds` rounds: Toffoli with k_max 6 walks levels 2..6 and can never
    finish (its optimum is 7), so its walks stay deterministic."""
    probs = []
    with Q.Batch(small_params(use_graph=graph), torch.cuda.Stream()) as batch:
        probe = Q.Problem.from_unitary(3, toffoli_unitary(), 0, 6, Q.default_params(3, seed=seed))
        probs.append(probe)
        ids = [batch.add(probe)]
        for i, (n, gates, kmax) in enumerate(others):
            p = Q.Problem.from_circuit(n, gates, kmax, Q.default_params(n, seed=seed + 1 + i))
            probs.append(p)
            ids.append(batch.add(p))
        for _ in range(rounds):
            batch.round()
        r = batch.poll(ids[0])
    for p in probs:
        p.close()
    return r["steps"], r["w_steps"], r["dps"], r["abandoned"], r["k"], r["status_name"]


def test_job_walks_are_the_same_alone_and_in_a_mix(dev):
    others = [(2, W.seeded_target(2, 3, 900 + i)[0], 3) for i in range(5)]
    others.append((3, W.config_target(2)[0], 5))
    alone = _walk_counts([], 12)
    mixed = _walk_counts(others, 12)
    assert alone == mixed
    assert alone[0] > 0 and alone[5] == "searching" and alone[4] > 2


def test_graph_and_direct_rounds_agree(dev):
    assert _walk_counts([], 8, graph=1) == _walk_counts([], 8, graph=0)


def test_jobs_join_and_leave_between_rounds(orc, dev):
    g1, _ = W.config_target(1)
    g2, _ = W.config_target(2)
    with Q.Batch(small_params(), torch.cuda.Stream()) as batch:
        p_slow = Q.Problem.from_unitary(3, toffoli_unitary(), 0, 6, Q.default_params(3))  # never finishes
        j_slow = batch.add(p_slow)
        batch.round()
        p_fast = Q.Problem.from_circuit(2, g1, 3, Q.default_params(2))
        j_fast = batch.add(p_fast)
        for _ in range(200):
            batch.round()
            if batch.poll(j_fast)["status_name"] != "searching":
                break
        r = batch.poll(j_fast)
        t_exact, _ = orc.mitm_tcount(orc.channel_from_circuit(2, g1), 3)
        assert r["status_name"] == "found" and r["t_count"] == t_exact
        batch.remove(j_slow)
        assert batch.round() == 0
        with pytest.raises(Q.QcsError):
            batch.poll(j_slow)
        p_slow.close()
        p_fast.close()


@pytest.mark.parametrize("share", [0, 10])
def test_batch_exhaustive_first_settles_levels_without_walking(orc, dev, share):
    # share: log2 of the exhaustive-pass points a round may run (0: every
    # pass to its end in its round); with 2^10 a pass spans many rounds, its
    # job parked (not walked) meanwhile, and the answers are the same
    cases = [(2, W.seeded_target(2, t, 400 + t)[0], t) for t in (3, 4, 5)]
    cases.append((3, W.seeded_target(3, 4, 404)[0], 4))
    probs, jobs = [], []
    with Q.Batch(small_params(cert_points_log2=share), torch.cuda.Stream()) as batch:
        for n, gates, kmax in cases:
            p = Q.Problem.from_circuit(n, gates, kmax, Q.default_params(n, exhaustive_first=1))
            probs.append(p)
            jobs.append(batch.add(p))
        rounds = 0
        while batch.round() > 0:
            rounds += 1
            assert rounds < 2000
        assert rounds == 0 if share == 0 else rounds > 4
        for (n, gates, kmax), j in zip(cases, jobs):
            r = batch.poll(j)
            C = orc.channel_from_circuit(n, gates)
            assert r["status_name"] == "found" and orc.verify(C, r["paulis"])
            assert r["steps"] == 0
            if n == 2:
                assert r["t_count"] == orc.mitm_tcount(C, kmax)[0]
    for p in probs:
        p.close()
