"""The walk kernel the benchmark times, at the benchmark's size and launch
shape (n = 3, level 5, 2^16 walks, 512 steps per walk in one launch,
theta = 2^-10), checked against the oracle.  qcs_level_walk_static runs that
kernel on caller-owned walk states, so every walk's trail can be read back:
its current state must be the oracle's f applied `len` times to the trail's
start, with the trail's chunk (Sec. 3 trails; Sec. 2 f), bit-exactly."""
import numpy as np
import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bench_launch_trajectories_match_the_oracle(orc):
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    c = W.CONFIGS[2]
    gates, _ = W.config_target(2)
    k, version, steps = c["t"], 1, 512
    params = Q.default_params(3, walks=c["walks"], state_bits=c["L"], dp_bits=c["dtheta"], table_log2=18)
    C = orc.channel_from_circuit(3, gates)
    with Q.Problem.from_circuit(3, gates, k, params) as prob:
        ws = torch.zeros(4 * c["walks"], dtype=torch.int64, device=dev)
        merges = torch.zeros(3 * 65536, dtype=torch.int64, device=dev)
        counts = torch.zeros(8, dtype=torch.int64, device=dev)
        prob.level_walk_static(k, version, c["dtheta"], 1, ws, steps, merges, counts)
        torch.cuda.synchronize()
        st = ws.cpu().numpy().view(np.uint64).reshape(-1, 4)
        got = counts.cpu().numpy().astype(np.uint64)
    assert int(got[0]) == c["walks"] * steps
    # walk record: start, cur, len | chunk << 32, seq | pad << 32
    lens = (st[:, 2] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    chunks = (st[:, 2] >> np.uint64(32)).astype(np.int64)
    assert np.all((chunks >= 1) & (chunks <= 63)) and np.all(lens <= steps)
    rng = np.random.default_rng(2)
    idx = list(rng.choice(c["walks"], 14, replace=False)) + [0, c["walks"] - 1]
    for i in idx:
        x = np.array([st[i, 0]], np.uint64)
        for _ in range(int(lens[i])):
            x = orc.walk_step(C, k, int(chunks[i]), version, c["L"], x)
        assert x[0] == st[i, 1], (i, int(lens[i]))


def test_headline_launch_trajectories_match_the_oracle(orc):
    """The headline kernel at the headline's size: n = 4, level 7, 2^20 walks,
    one launch of 64 steps, theta = 2^-12, on the tensor-core launch shape
    (3) and the dp4a one (0) from the same trail starts.  Every walk record
    is bit-identical between the two, and sampled walks' states equal the
    oracle's f iterated from their trail starts."""
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    c = W.CONFIGS[3]
    gates, _ = W.config_target(3)
    k, version, steps = c["t"], 1, 64
    C = orc.channel_from_circuit(4, gates)
    records = {}
    for shape in (3, 0):
        params = Q.default_params(4, walks=c["walks"], state_bits=c["L"], dp_bits=c["dtheta"], table_log2=18,
                                  launch_shape=shape)
        with Q.Problem.from_circuit(4, gates, k, params) as prob:
            ws = torch.zeros(4 * c["walks"], dtype=torch.int64, device=dev)
            merges = torch.zeros(3 * 65536, dtype=torch.int64, device=dev)
            counts = torch.zeros(8, dtype=torch.int64, device=dev)
            prob.level_walk_static(k, version, c["dtheta"], 1, ws, steps, merges, counts)
            torch.cuda.synchronize()
            records[shape] = (ws.cpu().numpy().view(np.uint64).reshape(-1, 4), counts.cpu().numpy()[:4].tolist())
            del ws, merges, counts
    st, cnt = records[3]
    assert np.array_equal(st, records[0][0]) and cnt == records[0][1]
    assert cnt[0] == c["walks"] * steps and cnt[2] > 0
    lens = (st[:, 2] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    chunks = (st[:, 2] >> np.uint64(32)).astype(np.int64)
    assert np.all((chunks >= 1) & (chunks <= 255)) and np.all(lens <= steps)
    rng = np.random.default_rng(4)
    idx = list(rng.choice(c["walks"], 6, replace=False)) + [0, c["walks"] - 1]
    for i in idx:
        x = np.array([st[i, 0]], np.uint64)
        for _ in range(int(lens[i])):
            x = orc.walk_step(C, k, int(chunks[i]), version, c["L"], x)
        assert x[0] == st[i, 1], (i, int(lens[i]))
