"""qcs_level_walk_static -- the walk for callers that cannot allocate device
memory (code captured into CUDA graphs, memory owned by a framework's caching
allocator, loops that cannot take cudaMalloc's synchronisation) -- must
compute what the allocating entry points qcs_level_begin + qcs_level_walk
compute.  The per-walk trails are deterministic, so the walk-step, W-step,
distinguished-point and abandoned-trail counts agree exactly, on two calls in
a row.  (Which merges the table reports depends on the order in which warps
reach it, so those are only checked for validity.)"""
import numpy as np
import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K, VERSION, DP_BITS, STEPS = 3, 2, 4, 24


def _collect_deltas(prob, before):
    prob.level_rewalk()
    r = prob.level_collect()
    keys = ("steps", "w_steps", "dps", "abandoned")
    return r, [r[k] - before.get(k, 0) for k in keys]


def test_static_walk_matches_allocating_walk_on_two_calls():
    from paper_1606_07413_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    dev = torch.device("cuda:0")
    gates, _ = W.config_target(1)
    params = Q.default_params(2)
    assert params.table_log2 <= 18
    n_walks = params.walks

    with Q.Problem.from_circuit(2, gates, 3, params) as ref, Q.Problem.from_circuit(2, gates, 3, params) as fix:
        walk_states = torch.zeros(4 * n_walks, dtype=torch.int64, device=dev)
        merges = torch.zeros(3 * 65536, dtype=torch.int64, device=dev)
        counts = torch.zeros(8, dtype=torch.int64, device=dev)

        ref.level_begin(K, VERSION, DP_BITS)
        before = {}
        for call in range(2):
            ref.level_walk(STEPS)
            before_res, want = _collect_deltas(ref, before)
            before = before_res

            fix.level_walk_static(K, VERSION, DP_BITS, 1 if call == 0 else 0, walk_states, STEPS, merges, counts)
            torch.cuda.synchronize()
            got = counts.cpu().numpy().astype(np.uint64)
            assert [int(v) for v in got[:4]] == want, (call, got[:4], want)
            assert int(got[0]) == n_walks * STEPS

            # every stored merge names two different trails that reached one
            # distinguished point (top d_theta of the 32 state bits zero)
            stored = min(int(got[7]) & 0xFFFFFFFF, merges.numel() // 3)
            assert stored <= int(got[6])
            m = merges[: 3 * stored].cpu().numpy().view(np.uint64).reshape(-1, 3)
            assert np.all(m[:, 0] != m[:, 1])
            assert np.all((m[:, 2] >> np.uint64(32 - DP_BITS)) == 0)


def test_static_walk_rejects_tables_beyond_its_size():
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    gates, _ = W.config_target(1)
    big = Q.default_params(2, table_log2=19)
    with Q.Problem.from_circuit(2, gates, 3, big) as prob:
        ws = torch.zeros(4 * 64, dtype=torch.int64, device=dev)
        merges = torch.zeros(3 * 16, dtype=torch.int64, device=dev)
        counts = torch.zeros(8, dtype=torch.int64, device=dev)
        with pytest.raises(Q.QcsError) as ei:
            prob.level_walk_static(K, VERSION, DP_BITS, 1, ws, STEPS, merges, counts)
        assert ei.value.code == Q.ERR_ARG
