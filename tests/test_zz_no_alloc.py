"""qcs_level_walk_static -- the walk for callers that cannot allocate device
memory (memory owned by a framework's caching allocator or a fixed arena,
loops that cannot take cudaMalloc's synchronisation) -- must compute what the
allocating entry points qcs_level_begin + qcs_level_walk compute, and must
leave the device's free memory unchanged once its first call has set it up.  The per-walk trails are deterministic, so the walk-step, W-step,
distinguished-point and abandoned-trail counts agree exactly, on two calls in
a row.  (Which merges the table reports depends on the order in which warps
reach it, so those are only checked for validity.)"""
import json
import os
import subprocess
import sys

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

            free0 = torch.cuda.mem_get_info(dev)[0]
            fix.level_walk_static(K, VERSION, DP_BITS, 1 if call == 0 else 0, walk_states, STEPS, merges, counts)
            torch.cuda.synchronize()
            if call > 0:  # the first call may load the library's device module and its static table
                assert torch.cuda.mem_get_info(dev)[0] == free0
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


# A fresh process whose first call of the entry point continues caller-made
# walk states (begin = 0): the static table must then already read as empty.
_FIRST_CALL = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import workloads as W
gates, _ = W.config_target(2)
dev = torch.device("cuda:0")
torch.cuda.set_device(dev)
with Q.Problem.from_circuit(3, gates, 5, Q.default_params(3, table_log2=18)) as prob:
    n_walks, L = 4096, 48
    x = W.seeded_states(n_walks, L, 77).view(np.int64)
    ws = np.zeros((n_walks, 4), np.int64)  # {start, cur, len | chunk << 32, seq | pad << 32}
    ws[:, 0] = x
    ws[:, 1] = x
    walk_states = torch.from_numpy(ws.reshape(-1)).to(dev)
    merges = torch.zeros(3 * 65536, dtype=torch.int64, device=dev)
    counts = torch.zeros(8, dtype=torch.int64, device=dev)
    prob.level_walk_static(4, 1, 4, 0, walk_states, 32, merges, counts)
    torch.cuda.synchronize()
    print(json.dumps([int(v) for v in counts.cpu().numpy()]))
"""


def test_first_call_on_a_device_sees_an_empty_table():
    """Level 4 of the n = 3 seeded target has 2 x 63^2 points, so its few
    hundred distinguished points are reached by thousands of trails: most
    inserts meet their own point again, but the first insert into each slot
    must find the slot empty.  A table that started zero-filled would count
    every insert as overwriting point 0 (overwritten + duplicates + merges ==
    distinguished points)."""
    from paper_1606_07413_gb300 import build

    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _FIRST_CALL, root], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    c = json.loads(out.stdout.strip().splitlines()[-1])
    assert c[0] == 4096 * 32
    assert c[2] > 1000, c
    met_occupied = c[4] + c[5] + c[6]
    assert 0 < c[2] - met_occupied <= 2 * 63 * 63, c
