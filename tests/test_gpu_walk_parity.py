"""Bit-exact parity of the CUDA walk step (qcs_walk_step) and re-walk
(qcs_rewalk) with the CPU oracle on seeded inputs (Sec. 2 Fig. 1, Sec. 3).

Small cases span several CTAs of 8 warps plus a ragged tail; the full-size
cases run the configured walk counts in one launch and check a sample of
outputs against the oracle one by one.  Integer results: exact equality."""
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


def make(orc, n, gates, k_max, **over):
    p = Q.default_params(n, **over)
    prob = Q.Problem.from_circuit(n, gates, k_max, p)
    C = orc.channel_from_circuit(n, gates)
    return prob, C, p


def gpu_step(prob, dev, k, chunk, version, states):
    x = torch.from_numpy(np.asarray(states, np.uint64).view(np.int64)).to(dev)
    y = torch.empty_like(x)
    dp = torch.empty(x.numel(), dtype=torch.uint8, device=dev)
    prob.walk_step(k, chunk, version, x, y, dp)
    torch.cuda.synchronize()
    return y.cpu().numpy().view(np.uint64), dp.cpu().numpy().astype(bool)


def target(cfg_n, t, seed):
    gates, _ = W.seeded_target(cfg_n, t, seed)
    return gates


# (n, construction t, k, chunk, count) -- counts are 8-warp CTAs plus a tail
SMALL = [
    (1, 3, 2, 0, 37), (1, 3, 3, 2, 37), (1, 5, 4, 0, 40),
    (2, 3, 2, 0, 301), (2, 3, 3, 1, 301), (2, 3, 3, 15, 77), (2, 5, 4, 0, 203), (2, 5, 5, 7, 203),
    (2, 3, 0, 0, 19), (2, 3, 1, 4, 19),
    (3, 5, 4, 0, 201), (3, 5, 5, 1, 97), (3, 5, 5, 63, 97), (3, 5, 2, 0, 65), (3, 5, 3, 30, 65),
    (3, 7, 6, 0, 41), (3, 7, 7, 11, 41),
    (4, 7, 6, 0, 29), (4, 7, 7, 200, 21), (4, 3, 2, 0, 19), (4, 7, 1, 255, 9),
]


@pytest.mark.parametrize("n,t,k,chunk,count", SMALL)
def test_walk_step_bit_exact(orc, dev, n, t, k, chunk, count):
    gates = target(n, t, 1000 + 10 * n + t)
    prob, C, p = make(orc, n, gates, max(k, 1))
    L = p.state_bits
    for version in (0, 3, 0xFFFFFFFF):
        states = W.seeded_states(count, L, 77 + k + version % 97)
        states[0] = 0
        states[-1] = (1 << L) - 1
        y, dp = gpu_step(prob, dev, k, chunk, version, states)
        want = orc.walk_step(C, k, chunk, version, L, states)
        assert np.array_equal(y, want), (n, k, chunk, version, np.nonzero(y != want)[0][:5])
        assert np.array_equal(dp, orc.is_dp(want, L, p.dp_bits))
    prob.close()


# (n, construction t, seed, whether some entry of C^ leaves int8): the walk
# kernel contracts C^ as signed byte quads when every numerator fits in int8
# and falls back to 32-bit words otherwise (staged, n = 3; through L2, n = 4)
WIDTHS = [(3, 13, 4013, False), (3, 19, 4019, True), (4, 13, 4013, False), (4, 15, 4015, True)]


@pytest.mark.parametrize("n,t,seed,wide", WIDTHS)
def test_contraction_widths_bit_exact(orc, dev, n, t, seed, wide):
    gates, _ = W.seeded_target(n, t, seed)
    C = orc.channel_from_circuit(n, gates).reduced()
    big = int(max(np.abs(C.a).max(), np.abs(C.b).max()))
    assert (big > 127) == wide and big >= 32  # the high bits of the bytes are in use
    params = Q.default_params(n)
    prob = Q.Problem.from_circuit(n, gates, 5, params)
    L = params.state_bits
    for k, chunk in ((4, 0), (5, 7)):
        states = W.seeded_states(45, L, 900 + k)
        y, _ = gpu_step(prob, dev, k, chunk, 1, states)
        assert np.array_equal(y, orc.walk_step(C, k, chunk, 1, L, states)), (n, t, k)
    prob.close()


def test_state_bits_and_dp_bits_follow_params(orc, dev):
    gates = target(2, 3, 5)
    for L, dth in ((20, 3), (40, 7), (64, 1)):
        prob, C, p = make(orc, 2, gates, 3, state_bits=L, dp_bits=dth)
        states = W.seeded_states(100, L, L)
        y, dp = gpu_step(prob, dev, 3, 5, 9, states)
        want = orc.walk_step(C, 3, 5, 9, L, states)
        assert np.array_equal(y, want)
        assert np.array_equal(dp, orc.is_dp(want, L, dth))
        assert int(y.max()) < (1 << L) or L == 64
        prob.close()


def test_empty_and_bad_arguments(orc, dev):
    gates = target(2, 3, 6)
    prob, C, p = make(orc, 2, gates, 3)
    x = torch.empty(0, dtype=torch.int64, device=dev)
    prob.walk_step(2, 0, 0, x, torch.empty_like(x))  # count 0: no-op
    one = torch.zeros(1, dtype=torch.int64, device=dev)
    for k, chunk in ((3, 0), (3, 16), (2, 1), (4, 0)):
        with pytest.raises(Q.QcsError) as ei:
            prob.walk_step(k, chunk, 0, one, torch.empty_like(one))
        assert ei.value.code == Q.ERR_ARG
    prob.close()


@pytest.mark.parametrize("cfg", [2, 3])
def test_full_size_launch_sampled(orc, dev, cfg):
    """The configured number of walks in one launch (2^16 at n = 3, 2^20 at
    n = 4); 48 sampled outputs are recomputed by the oracle one by one."""
    c = W.CONFIGS[cfg]
    gates, _ = W.config_target(cfg)
    prob, C, p = make(orc, c["n"], gates, c["k_max"])
    k = c["t"]
    states = W.seeded_states(c["walks"], c["L"], 4242 + cfg)
    y, dp = gpu_step(prob, dev, k, 3, 1, states)
    rng = np.random.default_rng(cfg)
    idx = np.concatenate([[0, len(states) - 1], rng.choice(len(states), 46, replace=False)])
    want = orc.walk_step(C, k, 3, 1, c["L"], states[idx])
    assert np.array_equal(y[idx], want)
    # the flag is the distinguished predicate of every output
    assert np.array_equal(dp, orc.is_dp(y, c["L"], c["dtheta"]))
    prob.close()


def _merging_pairs(orc, C, k, chunk, version, L, rng, want=24):
    """Pairs (start, len) of oracle trails that reach one common state."""
    starts = W.seeded_states(300, L, int(rng.integers(1 << 30)))
    trails = [[int(s)] for s in starts]
    for _ in range(6):
        cur = np.asarray([t[-1] for t in trails], np.uint64)
        nxt = orc.walk_step(C, k, chunk, version, L, cur)
        for t, v in zip(trails, nxt):
            t.append(int(v))
    seen = {}
    pairs = []
    for i, t in enumerate(trails):
        for ln, v in enumerate(t[1:], start=1):
            if v in seen and seen[v][0] != i and trails[seen[v][0]][0] != t[0]:
                j, lj = seen[v]
                pairs.append((trails[j][0], lj, t[0], ln))
                break
            seen.setdefault(v, (i, ln))
        if len(pairs) >= want:
            break
    return pairs


@pytest.mark.parametrize("n,t,k,chunk", [(2, 3, 2, 0), (2, 3, 3, 9), (3, 5, 4, 0), (3, 3, 3, 17)])
def test_rewalk_matches_oracle(orc, dev, n, t, k, chunk):
    gates = target(n, t, 2000 + n + k)
    prob, C, p = make(orc, n, gates, k)
    L = p.state_bits
    rng = np.random.default_rng(n * 10 + k)
    pairs = _merging_pairs(orc, C, k, chunk, 5, L, rng)
    assert pairs, "no merging trails found"
    # add one inconsistent pair (the trails never meet within the lengths)
    pairs.append((int(W.seeded_states(1, L, 1)[0]), 1, int(W.seeded_states(1, L, 2)[0]), 1))
    sa = np.asarray([q[0] for q in pairs], np.uint64)
    la = np.asarray([q[1] for q in pairs], np.uint32)
    sb = np.asarray([q[2] for q in pairs], np.uint64)
    lb = np.asarray([q[3] for q in pairs], np.uint32)
    t_sa = torch.from_numpy(sa.view(np.int64)).to(dev)
    t_sb = torch.from_numpy(sb.view(np.int64)).to(dev)
    t_la = torch.from_numpy(la.view(np.int32)).to(dev)
    t_lb = torch.from_numpy(lb.view(np.int32)).to(dev)
    cls = torch.empty(len(pairs), dtype=torch.int32, device=dev)
    ab = torch.empty(2 * len(pairs), dtype=torch.int64, device=dev)
    prob.rewalk(k, chunk, 5, t_sa, t_la, t_sb, t_lb, cls, ab)
    torch.cuda.synchronize()
    g_cls = cls.cpu().numpy()
    g_ab = ab.cpu().numpy().view(np.uint64).reshape(-1, 2)
    for i, (a0, l0, b0, l1) in enumerate(pairs):
        o_cls, oa, ob, _ = orc.rewalk(C, k, chunk, 5, L, a0, l0, b0, l1)
        # the GPU reports claw candidates before the exact check; the oracle
        # has already decided claw or false hash
        exp_cls = Q.MERGE_CLAW if o_cls in (orc.CLAW, orc.FALSE_HASH) else o_cls
        assert g_cls[i] == exp_cls, (i, g_cls[i], o_cls)
        if o_cls != orc.NO_MERGE:
            assert {int(g_ab[i, 0]), int(g_ab[i, 1])} == {oa, ob}
    prob.close()


def test_claw_states_step_together_on_gpu(orc, dev):
    """States naming the two halves of a known decomposition (Eq. mitm) map to
    the same next state on the GPU as well."""
    n, t = 3, 5
    rng = np.random.default_rng(8)
    ps = [int(rng.integers(1, 64))]
    while len(ps) < t:
        q = int(rng.integers(1, 64))
        if orc.pauli_phase(n, ps[-1], q) != orc.pauli_phase(n, q, ps[-1]):
            ps.append(q)
    rows = [tuple(r) for r in W.clifford_word(rng, n, 40)] + [(W.OP_RP, p, 0) for p in ps]
    gates = np.asarray(rows, np.int32)
    prob, C, p = make(orc, n, gates, t)
    h = t // 2
    xv = orc.encode(n, t, p.state_bits, 0, ps[:h])
    xw = orc.encode(n, t, p.state_bits, 1, ps[h:2 * h])
    y, _ = gpu_step(prob, dev, t, ps[2 * h], 12, [xv, xw])
    assert y[0] == y[1]
    prob.close()
