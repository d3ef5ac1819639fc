"""Serving (continuous batching): requests that arrive while others run are
admitted as slots and memory free up, run on the device together with the
work already there, and get the same answer (optimal T-count, exactly
verified decomposition) as when served alone."""
import numpy as np
import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import serve
from paper_1606_07413_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    from paper_1606_07413_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def params(J=8):
    return Q.default_batch_params(max_jobs=J, walks_per_job=512, steps_per_round=16, table_log2=16,
                                  queue_capacity=4096)


def toffoli():
    u = np.zeros((8, 8, 4), np.int64)
    for c in range(8):
        u[c ^ (4 if (c & 3) == 3 else 0), c, 0] = 1
    return u


def small_targets(count, seed=300):
    out = []
    for i in range(count):
        n = 2 if i % 3 else 3
        gates, _ = W.seeded_target(n, 2 + i % 3, seed + i)
        out.append((n, gates, 2 + i % 3))
    return out


def serve_all(srv, reqs, max_steps=2000):
    for _ in range(max_steps):
        srv.step()
        if srv.idle():
            return True
    return False


def test_requests_join_a_running_batch_and_match_the_oracle(orc, dev):
    with serve.Server(params(), memory_budget=1 << 34, stream=torch.cuda.Stream()) as srv:
        # a long job (Toffoli below its optimum never finishes) keeps the device busy
        slow = Q.Problem.from_unitary(3, toffoli(), 0, 6, Q.default_params(3))
        slow_slot = srv.batch.add(slow)
        srv.batch.round()
        rids = [srv.submit(n, g, k) for n, g, k in small_targets(9)]
        for _ in range(3000):
            srv.step()
            if all(srv.poll(r)["status"] not in ("queued", "running") for r in rids):
                break
        for (n, g, k), rid in zip(small_targets(9), rids):
            res = srv.poll(rid)
            C = orc.channel_from_circuit(n, g)
            t_exact, _ = orc.mitm_tcount(C, k)
            assert res["status"] == "found" and res["t_count"] == t_exact, (n, k, res)
            assert orc.verify(C, res["paulis"])
            assert res["latency"] > 0
        assert srv.batch.poll(slow_slot)["status_name"] == "searching"  # overlapped, still running
        srv.batch.remove(slow_slot)
        slow.close()


def peak_concurrency(polls):
    """Most requests in flight at once, from their admit and done times (a
    job admitted and finished within one round still counts)."""
    return max(sum(1 for s in polls if s["t_admit"] <= r["t_admit"] < s["t_done"]) for r in polls)


def test_admission_respects_slots_and_memory(dev):
    with serve.Server(params(J=8), memory_budget=1, stream=torch.cuda.Stream()) as srv:
        # a budget below one job admits exactly one job at a time
        rids = [srv.submit(n, g, k) for n, g, k in small_targets(5, seed=500)]
        for _ in range(3000):
            srv.step()
            assert len(srv.running) <= 1
            if srv.idle():
                break
        polls = [srv.poll(r) for r in rids]
        assert srv.idle() and all(p["status"] == "found" for p in polls)
        assert peak_concurrency(polls) == 1
    with serve.Server(params(J=2), memory_budget=1 << 34, stream=torch.cuda.Stream()) as srv:
        # two job slots: two requests run together, never three
        rids = [srv.submit(n, g, k) for n, g, k in small_targets(6, seed=600)]
        for _ in range(3000):
            srv.step()
            assert len(srv.running) <= 2
            if srv.idle():
                break
        polls = [srv.poll(r) for r in rids]
        assert srv.idle() and all(p["status"] == "found" for p in polls)
        assert peak_concurrency(polls) == 2


def test_same_answer_alone_and_in_the_mix(orc, dev):
    n, g, k = 3, W.config_target(2)[0], 5
    C = orc.channel_from_circuit(n, g)
    with serve.Server(params(), memory_budget=1 << 34, stream=torch.cuda.Stream()) as srv:
        rid = srv.submit(n, g, k)
        assert serve_all(srv, [rid])
        alone = srv.poll(rid)
    with serve.Server(params(J=16), memory_budget=1 << 34, stream=torch.cuda.Stream()) as srv:
        others = [srv.submit(nn, gg, kk) for nn, gg, kk in small_targets(12, seed=700)]
        rid = srv.submit(n, g, k)
        others += [srv.submit(nn, gg, kk) for nn, gg, kk in small_targets(6, seed=800)]
        assert serve_all(srv, others + [rid])
        mixed = srv.poll(rid)
    assert alone["status"] == mixed["status"] == "found"
    assert alone["t_count"] == mixed["t_count"] == 5
    assert orc.verify(C, alone["paulis"]) and orc.verify(C, mixed["paulis"])


def test_deadline_releases_the_slot(dev):
    clock = [0.0]
    with serve.Server(params(J=1), memory_budget=1 << 34, stream=torch.cuda.Stream(), deadline_s=5.0,
                      clock=lambda: clock[0]) as srv:
        rid = srv.submit(3, np.zeros((0, 3), np.int32), 0)  # the identity: T-count 0, settles at once
        srv.step()
        assert srv.poll(rid)["status"] == "found" and srv.poll(rid)["t_count"] == 0
        slow = srv.submit(4, W.config_target(3)[0], 7)  # level 7 of n = 4 takes far longer than the deadline
        srv.step()
        assert srv.poll(slow)["status"] == "running"
        clock[0] += 10.0
        srv.step()
        assert srv.poll(slow)["status"] == "deadline"
        assert srv.idle() and srv.used == 0
