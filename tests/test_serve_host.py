"""Host logic of the serving loop (paper_1606_07413_gb300.serve) on CPU: a
fake batch engine stands in for the device, so admission by memory and job
slots, arrival order, deadlines and full-batch handling are checked without a
GPU."""
import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import serve


class FakeProblem:
    def __init__(self, n, gates, k_max, params):
        self.n, self.k_max, self.closed = n, k_max, False
        self.rounds_needed = int(gates[0][0])  # encoded by the test

    def close(self):
        self.closed = True


class FakeBatch:
    """Job slots; a job finishes after its rounds_needed rounds."""

    def __init__(self, params, stream=None):
        self.max_jobs = params.max_jobs
        self.jobs = {}
        self.added = []
        self.busy_once = False

    def job_bytes(self, prob):
        return 100 * prob.n

    def add(self, prob):
        if self.busy_once:
            self.busy_once = False
            raise Q.QcsError(Q.ERR_BUSY, "qcs_batch_add")
        free = [s for s in range(self.max_jobs) if s not in self.jobs]
        if not free:
            raise Q.QcsError(Q.ERR_BUSY, "qcs_batch_add")
        self.jobs[free[0]] = [prob, 0]
        self.added.append(prob)
        return free[0]

    def remove(self, slot):
        del self.jobs[slot]

    def round(self):
        for j in self.jobs.values():
            j[1] += 1
        return len(self.jobs)

    def poll(self, slot):
        prob, r = self.jobs[slot]
        done = r >= prob.rounds_needed
        return {"status_name": "found" if done else "searching", "t_count": prob.k_max if done else -1,
                "paulis": [1] * prob.k_max if done else [], "steps": 10 * r, "rewalk_steps": r}

    def close(self):
        pass


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(Q, "Batch", FakeBatch)
    monkeypatch.setattr(Q.Problem, "from_circuit", classmethod(lambda cls, *a: FakeProblem(*a)))
    monkeypatch.setattr(Q, "default_params", lambda n, **kw: None)


def bparams(J):
    p = Q.BatchParams()
    p.max_jobs = J
    return p


def test_admission_follows_memory_slots_and_arrival_order(fake):
    clock = Clock()
    with serve.Server(bparams(3), memory_budget=450, clock=clock) as srv:
        # n = 2 jobs take 200 bytes each: at most two fit the budget at once
        rids = [srv.submit(2, [[3 + i, 0, 0]], 2) for i in range(5)]
        peak_running = 0
        for _ in range(100):
            clock.t += 0.01
            srv.step()
            peak_running = max(peak_running, len(srv.running))
            assert srv.used <= 450
            if srv.idle():
                break
        assert srv.idle() and peak_running == 2 and srv.peak_used == 400
        admits = [srv.poll(r)["t_admit"] for r in rids]
        assert admits == sorted(admits)  # first come, first admitted
        assert all(srv.poll(r)["status"] == "found" for r in rids)
        assert srv.fevals == sum(10 * (3 + i) + (3 + i) for i in range(5))


def test_a_single_job_larger_than_the_budget_still_runs_alone(fake):
    with serve.Server(bparams(2), memory_budget=100, clock=Clock()) as srv:
        rid = srv.submit(4, [[2, 0, 0]], 3)  # 400 bytes > budget
        for _ in range(10):
            srv.step()
        assert srv.poll(rid)["status"] == "found"


def test_deadline_ends_a_job_and_frees_its_memory(fake):
    clock = Clock()
    with serve.Server(bparams(2), memory_budget=10_000, deadline_s=1.0, clock=clock) as srv:
        slow = srv.submit(3, [[1000, 0, 0]], 5)
        fast = srv.submit(2, [[2, 0, 0]], 3)
        for r in srv.requests.values():  # both set-ups done before the simulated clock runs
            r.future.result()
        for _ in range(30):
            clock.t += 0.1
            srv.step()
        assert srv.poll(slow)["status"] == "deadline"
        assert srv.poll(fast)["status"] == "found"
        assert srv.used == 0 and not srv.running


def test_a_full_batch_leaves_the_request_queued(fake):
    with serve.Server(bparams(2), memory_budget=10_000, clock=Clock()) as srv:
        srv.batch.busy_once = True  # the batch refuses the next add once
        rid = srv.submit(2, [[2, 0, 0]], 3)
        srv.step()
        assert srv.poll(rid)["status"] == "queued"
        for _ in range(5):
            srv.step()
        assert srv.poll(rid)["status"] == "found"


def test_admission_keeps_room_for_each_jobs_exhaustive_key_table(fake):
    """A job may hold the key table of an exhaustive pass across rounds:
    admission counts each admitted job with its largest such table (16 bytes
    x 2^exhaustive_log2 at most without the request's qubit count)."""
    from types import SimpleNamespace

    assert serve.exhaustive_table_bytes(SimpleNamespace(exhaustive_log2=10)) == 16 << 10
    assert serve.exhaustive_table_bytes(SimpleNamespace(exhaustive_log2=0)) == 0
    assert serve.exhaustive_table_bytes(None) == 0
    table = 16 << 10
    for budget, most in ((2 * table + 450, 2), (table + 250, 1)):
        clock = Clock()
        with serve.Server(bparams(4), memory_budget=budget, clock=clock,
                          params_for=lambda n: SimpleNamespace(exhaustive_log2=10)) as srv:
            rids = [srv.submit(2, [[3, 0, 0]], 2) for _ in range(4)]
            peak = 0
            for _ in range(100):
                clock.t += 0.01
                srv.step()
                peak = max(peak, len(srv.running))
                assert not srv.running or srv.used <= budget or len(srv.running) == 1
                if srv.idle():
                    break
            assert srv.idle() and peak == most
            assert all(srv.poll(r)["status"] == "found" for r in rids)



def test_a_request_whose_deadline_passes_in_the_queue_never_runs(fake):
    """The deadline counts from arrival: a request still queued behind a long
    job when its deadline passes is dropped without being added to the batch."""
    clock = Clock()
    with serve.Server(bparams(1), memory_budget=10_000, deadline_s=1.0, clock=clock) as srv:
        long_job = srv.submit(3, [[1000, 0, 0]], 5)
        queued = srv.submit(2, [[2, 0, 0]], 3)
        for r in srv.requests.values():
            r.future.result()
        for _ in range(30):
            clock.t += 0.1
            srv.step()
        assert srv.poll(long_job)["status"] == "deadline"
        assert srv.poll(queued)["status"] == "deadline" and srv.poll(queued)["t_admit"] is None
        assert len(srv.batch.added) == 1 and srv.idle()


def test_exhaustive_table_is_sized_for_the_requests_largest_eligible_level():
    """xi^h stored points in a power-of-two table of at least twice as many
    slots: n = 4 level 7 stores 255^3 points in 2^25 slots (512 MiB); a level
    beyond 2^exhaustive_log2 points does not count."""
    from types import SimpleNamespace

    p32, p26 = SimpleNamespace(exhaustive_log2=32), SimpleNamespace(exhaustive_log2=26)
    assert serve.exhaustive_table_bytes(p32, 4, 7) == 16 << 25
    assert serve.exhaustive_table_bytes(p26, 4, 7) == 16 << 25  # level 6: 2 x 255^3 points, same table
    assert serve.exhaustive_table_bytes(p26, 4, 5) == 16 << 17  # level 5: 255^2 stored
    assert serve.exhaustive_table_bytes(p32, 2, 3) == 16 << 10
    assert serve.exhaustive_table_bytes(SimpleNamespace(exhaustive_log2=0), 4, 7) == 0


def test_a_request_waiting_for_memory_does_not_hold_back_smaller_ones(fake):
    """Backfilling: with room for one n = 4 job (400 bytes) or two n = 2 jobs,
    a second n = 4 request waits for memory while the n = 2 requests behind
    it are admitted; it keeps its place and runs once memory frees."""
    clock = Clock()
    with serve.Server(bparams(4), memory_budget=650, clock=clock) as srv:
        big1 = srv.submit(4, [[3, 0, 0]], 3)
        big2 = srv.submit(4, [[3, 0, 0]], 3)
        small = [srv.submit(2, [[1, 0, 0]], 2) for _ in range(2)]
        for r in srv.requests.values():
            r.future.result()
        clock.t += 0.01
        srv.step()
        assert srv.poll(big1)["status"] == "running" and srv.poll(big2)["status"] == "queued"
        assert all(srv.poll(r)["status"] in ("running", "found") for r in small[:1])
        for _ in range(20):
            clock.t += 0.01
            srv.step()
        assert all(srv.poll(r)["status"] == "found" for r in (big1, big2, *small))
        assert srv.poll(small[0])["t_admit"] < srv.poll(big2)["t_admit"]
