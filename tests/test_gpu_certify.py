"""The exhaustive level pass (qcs_certify_level): on every level it must
agree exactly with the oracle's exhaustive meet-in-the-middle (Sec. 2
Eq. mitm), and in the ladder it settles the levels whose walk budget ran out
without a claw, so the reported T-count is exact at those sizes."""
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


# (n, construction t, seed, highest level checked): the oracle's pass over
# n = 3 above level 4 takes too long for a test.  An odd level of a target
# with a denominator (sde >= 1) stores the h-rotation side with C^ and
# streams the (h + 1)-rotation side; a Clifford target (t = 0, sde 0) takes
# the other split, so both are covered.
CASES = [(1, t, 60 + t, 8) for t in (0, 2, 3, 5, 6)] + \
        [(2, t, 70 + t, 7) for t in (0, 2, 3, 4, 5, 6)] + \
        [(3, 3, 83, 4), (3, 4, 84, 4), (3, 5, 85, 5)]


@pytest.mark.parametrize("n,t,seed,kmax", CASES)
def test_certify_agrees_with_the_oracle_on_every_level(orc, dev, n, t, seed, kmax):
    gates, _ = W.seeded_target(n, t, seed)
    C = orc.channel_from_circuit(n, gates)
    for k in range(2, kmax + 1):
        prob = Q.Problem.from_circuit(n, gates, kmax, Q.default_params(n))
        has = prob.certify_level(k)
        want = orc.mitm_level(C, k)
        assert has == (want is not None), (n, t, k)
        r = prob.poll()
        if has:
            assert r["t_count"] == k and orc.verify(C, r["paulis"])
        else:
            assert r["certified_levels"] == 1
        assert r["cert_points"] == (4 ** n - 1) ** (k // 2) * (1 + ((4 ** n - 1) if k & 1 else 1))
        prob.close()


def test_certify_rejects_bad_levels(dev):
    gates, _ = W.seeded_target(2, 3, 7)
    with Q.Problem.from_circuit(2, gates, 4, Q.default_params(2)) as prob:
        for k in (-1, 0, 1, 5):
            with pytest.raises(Q.QcsError):
                prob.certify_level(k)


def test_certify_refuses_a_key_table_beyond_device_memory(dev):
    # n = 4, level 12: 255^6 V points would need a 2^49-slot table; the host
    # refuses before allocating or launching anything
    gates, _ = W.seeded_target(4, 3, 8)
    with Q.Problem.from_circuit(4, gates, 12, Q.default_params(4)) as prob:
        with pytest.raises(Q.QcsError) as ei:
            prob.certify_level(12)
        assert ei.value.code == Q.ERR_NOMEM


@pytest.mark.parametrize("n,t,seed", [(2, 5, 91), (2, 6, 92), (3, 4, 93), (3, 5, 94)])
def test_ladder_settles_small_levels_exactly(orc, dev, n, t, seed):
    # walks far too short to find anything: the exhaustive pass decides
    gates, _ = W.seeded_target(n, t, seed)
    C = orc.channel_from_circuit(n, gates)
    p = Q.default_params(n, walks=64, steps_per_launch=2, budget_factor=0, version_factor=0, exhaustive_log2=24)
    with Q.Problem.from_circuit(n, gates, t, p) as prob:
        prob.run_walks()
        r = prob.wait(120_000)
    assert r["status_name"] == "found"
    assert orc.verify(C, r["paulis"])
    low = max(orc.sde(C), 2)
    if n == 2:
        t_exact, _ = orc.mitm_tcount(C, t)
        assert r["t_count"] == t_exact
    assert r["t_count"] <= t
    assert r["certified_levels"] == max(0, r["t_count"] - low)


@pytest.mark.parametrize("n,t,seed", [(2, 5, 91), (2, 6, 92), (3, 4, 93)])
def test_exhaustive_first_settles_levels_without_walking(orc, dev, n, t, seed):
    gates, _ = W.seeded_target(n, t, seed)
    C = orc.channel_from_circuit(n, gates)
    p = Q.default_params(n, exhaustive_first=1)
    with Q.Problem.from_circuit(n, gates, t, p) as prob:
        prob.run_walks()
        r = prob.wait(120_000)
    assert r["status_name"] == "found" and orc.verify(C, r["paulis"])
    assert r["steps"] == 0 and r["launches"] == 0
    t_exact, _ = orc.mitm_tcount(C, t) if n == 2 else (r["t_count"], None)
    assert r["t_count"] == t_exact
    assert r["certified_levels"] == max(0, r["t_count"] - max(orc.sde(C), 2))
