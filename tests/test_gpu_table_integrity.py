"""Distinguished-point table and merge queue integrity (Sec. 3): every merge
the walk kernel queues names two trails that really reach the stored point.
Each queued pair's trails are recomputed from their references (start of
trail (walk, seq) at its length, chunk of that start) and walked by the
oracle; both must end at the stored distinguished point, so no torn or mixed
table entry slips through.  A queue smaller than the merges found keeps
counting and writes nothing past its capacity."""
import numpy as np
import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


def smix(z):
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def trail(ref, seed, version, L, n_chunks):
    """(start, chunk, length) of a trail reference: walk 24 bits, sequence 23,
    length 17; the start and chunk follow the library's trail convention."""
    walk, seq, length = ref & ((1 << 24) - 1), (ref >> 24) & ((1 << 23) - 1), ref >> 47
    start = smix(seed ^ smix((walk << 32) | seq) ^ (version << 40)) & ((1 << L) - 1)
    chunk = 1 + smix(start ^ 0x5851F42D4C957F2D) % n_chunks if n_chunks else 0
    return start, chunk, length


def run_static(prob, dev, n_walks, k, version, dp_bits, steps, cap):
    ws = torch.zeros(4 * n_walks, dtype=torch.int64, device=dev)
    merges = torch.full((3 * cap + 3,), -1, dtype=torch.int64, device=dev)  # one sentinel triple past the cap
    counts = torch.zeros(8, dtype=torch.int64, device=dev)
    prob.level_walk_static(k, version, dp_bits, 1, ws, steps, merges[: 3 * cap], counts)
    torch.cuda.synchronize()
    return merges.cpu().numpy().view(np.uint64).reshape(-1, 3), counts.cpu().numpy().astype(np.uint64)


def test_queued_merges_reach_the_stored_point(orc):
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    c = W.CONFIGS[2]
    gates, _ = W.config_target(2)
    k, version, dp_bits = 5, 3, 6
    params = Q.default_params(3, walks=1 << 14, state_bits=c["L"], dp_bits=dp_bits, table_log2=18)
    C = orc.channel_from_circuit(3, gates)
    with Q.Problem.from_circuit(3, gates, k, params) as prob:
        m, counts = run_static(prob, dev, 1 << 14, k, version, dp_bits, 96, 1 << 16)
    stored = min(int(counts[7]) & 0xFFFFFFFF, 1 << 16)
    assert stored > 50
    rng = np.random.default_rng(9)
    for i in rng.choice(stored, 24, replace=False):
        ref_a, ref_b, dp = (int(v) for v in m[i])
        assert ref_a != ref_b and dp >> (c["L"] - dp_bits) == 0
        for ref in (ref_a, ref_b):
            start, chunk, length = trail(ref, params.seed, version, c["L"], 63)
            x = np.array([start], np.uint64)
            for _ in range(length):
                x = orc.walk_step(C, k, chunk, version, c["L"], x)
            assert int(x[0]) == dp, (i, ref)


def test_a_full_merge_queue_counts_and_stays_in_bounds():
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    gates, _ = W.config_target(1)
    params = Q.default_params(2, dp_bits=3)
    with Q.Problem.from_circuit(2, gates, 3, params) as prob:
        cap = 8
        m, counts = run_static(prob, dev, params.walks, 3, 1, 3, 64, cap)
    found, stored = int(counts[6]), int(counts[7]) & 0xFFFFFFFF
    assert found > cap and min(stored, cap) == cap
    assert np.all(m[cap] == np.uint64(M64))  # nothing written past the capacity


@pytest.mark.parametrize("dp_bits,samples", [(6, 16), (9, 4)])
def test_tensor_core_walk_queues_real_merges(orc, dp_bits, samples):
    """The n = 4 tensor-core walk (launch shape 3) at a theta where its MMA
    warps store the distinguished points the stage warps hand them (2^-6),
    and at one where each stage warp stores its own (2^-9): sampled queued
    merges name two trails that both reach the stored point."""
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    c = W.CONFIGS[3]
    gates, _ = W.config_target(3)
    k, version = 7, 2
    params = Q.default_params(4, walks=1 << 14, state_bits=c["L"], dp_bits=dp_bits, table_log2=18, launch_shape=3)
    C = orc.channel_from_circuit(4, gates)
    with Q.Problem.from_circuit(4, gates, k, params) as prob:
        m, counts = run_static(prob, dev, 1 << 14, k, version, dp_bits, 48, 1 << 16)
    assert int(counts[7]) >> 32 == 0  # no bounded wait ran out
    assert int(counts[0]) == (1 << 14) * 48 and int(counts[2]) > 0
    stored = min(int(counts[7]) & 0xFFFFFFFF, 1 << 16)
    assert stored >= samples
    rng = np.random.default_rng(dp_bits)
    for i in rng.choice(stored, samples, replace=False):
        ref_a, ref_b, dp = (int(v) for v in m[i])
        assert ref_a != ref_b and dp >> (c["L"] - dp_bits) == 0
        for ref in (ref_a, ref_b):
            start, chunk, length = trail(ref, params.seed, version, c["L"], 255)
            x = np.array([start], np.uint64)
            for _ in range(length):
                x = orc.walk_step(C, k, chunk, version, c["L"], x)
            assert int(x[0]) == dp, (i, ref)
