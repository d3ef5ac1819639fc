"""Every launch shape of the walk kernel (warps per CTA, resident CTAs per SM)
and both device layouts of C^ (int8 byte quads for dp4a, 32-bit words for
IMAD) evaluate the same walks: after one launch from the same trail starts,
every walk's state record is bit-identical across them, the counters agree,
and sampled walks equal the oracle's f iterated from their trail starts
(Sec. 3 trails; Sec. 2 f).  Also: the bytes a problem reports it copied
between host and device are the ones its uploads and launches move."""
import numpy as np
import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (config, level, walks, steps, d_theta): several CTAs of every shape, trails
# that reach distinguished points and restart within the launch
CASES = [(2, 5, 1 << 14, 64, 6), (3, 7, 1 << 13, 8, 3)]


@pytest.mark.parametrize("cfg,k,walks,steps,dpb", CASES)
def test_every_shape_and_layout_walks_the_same_trails(orc, cfg, k, walks, steps, dpb):
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    c = W.CONFIGS[cfg]
    n = c["n"]
    gates, _ = W.config_target(cfg)
    shapes = Q.launch_shapes(n)
    assert len(shapes) >= 3 and shapes[0]["shape"] == 0
    runs = {}
    for sh in shapes:
        for layout in (0, 1):
            p = Q.default_params(n, walks=walks, table_log2=18, launch_shape=sh["shape"], c_layout=layout)
            with Q.Problem.from_circuit(n, gates, k, p) as prob:
                ws = torch.zeros(4 * walks, dtype=torch.int64, device=dev)
                merges = torch.zeros(3 * 65536, dtype=torch.int64, device=dev)
                counts = torch.zeros(8, dtype=torch.int64, device=dev)
                prob.level_walk_static(k, 1, dpb, 1, ws, steps, merges, counts)
                torch.cuda.synchronize()
                runs[(sh["shape"], layout)] = (ws.cpu().numpy().view(np.uint64).reshape(-1, 4),
                                               counts.cpu().numpy()[:4].tolist())
    ref_ws, ref_counts = runs[(0, 0)]
    assert ref_counts[0] == walks * steps and ref_counts[2] > 0  # trails did reach distinguished points
    for key, (ws, counts) in runs.items():
        assert np.array_equal(ws, ref_ws), key
        assert counts == ref_counts, key
    C = orc.channel_from_circuit(n, gates)
    lens = (ref_ws[:, 2] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    chunks = (ref_ws[:, 2] >> np.uint64(32)).astype(np.int64)
    rng = np.random.default_rng(cfg)
    for i in list(rng.choice(walks, 5, replace=False)) + [walks - 1]:
        x = np.array([ref_ws[i, 0]], np.uint64)
        for _ in range(int(lens[i])):
            x = orc.walk_step(C, k, int(chunks[i]), 1, c["L"], x)
        assert x[0] == ref_ws[i, 1], (i, int(lens[i]))


def test_reported_copies_match_the_uploads_and_reads():
    """A second n = 3 problem (the shared stage tables are already on the
    device) uploads C^ as 64 x 64 (a, b) words, the 64 fingerprint weights,
    the rotation masks (a 16-bit word per Pauli and lane, 32 lanes) and, with
    every entry in int8, the byte quads; each walk launch reads back the 16 counters and
    three queue heads, plus 24 bytes per claw candidate."""
    from paper_1606_07413_gb300 import build

    build.build()
    c = W.CONFIGS[2]
    gates, _ = W.config_target(2)
    D, lanes = 64, 32
    want_up = D * D * 8 + D * 8 + D * lanes * 2 + D * D // 2 * 4
    with Q.Problem.from_circuit(3, gates, 5, Q.default_params(3, walks=4096)) as first:
        pass
    with Q.Problem.from_circuit(3, gates, 5, Q.default_params(3, walks=4096)) as prob:
        assert prob.poll()["h2d_bytes"] == want_up
        prob.level_begin(5, 0, 6)
        launches = 3
        for _ in range(launches):
            prob.level_walk(32)
            prob.level_rewalk()
            r = prob.level_collect()
        checked = r["claws"] + r["false_hash"]  # the host stops checking a launch's list at its first claw
        assert r["h2d_bytes"] == want_up
        read_cands = r["d2h_bytes"] - launches * (16 * 8 + 3 * 4)
        assert read_cands % 24 == 0 and read_cands // 24 >= checked
    with Q.Problem.from_circuit(3, gates, 5, Q.default_params(3, walks=4096, c_layout=1)) as wide:
        assert wide.poll()["h2d_bytes"] == want_up - D * D // 2 * 4  # no byte quads


def test_carried_rewalks_account_for_every_merge():
    """With a per-launch re-walk budget (params.rewalk_budget), a merge whose
    re-walk (Sec. 3, Fig. 2) does not finish in its launch resumes in the
    next one: after every launch, the merges queued so far are exactly the
    ones classified plus the ones carried (level 4 of the n = 3 seeded
    target has no claw, so every candidate is checked and counted), and the
    walk itself is the same as without the budget."""
    from paper_1606_07413_gb300 import build

    build.build()
    gates, _ = W.config_target(2)
    runs = {}
    for budget in (0, 4):
        p = Q.default_params(3, walks=4096, rewalk_budget=budget)
        with Q.Problem.from_circuit(3, gates, 5, p) as prob:
            prob.level_begin(4, 2, 4)
            seen_carried = 0
            hist = []
            for _ in range(5):
                prob.level_walk(48)
                prob.level_rewalk()
                r = prob.level_collect()
                classified = r["robin_hood"] + r["trivial"] + r["same_side"] + r["claws"] + r["false_hash"] + \
                    r["no_merge"]
                assert r["queue_overflow"] == 0 and r["claws"] == 0
                assert classified + r["rewalk_carried"] == r["merges"], (budget, r)
                seen_carried = max(seen_carried, r["rewalk_carried"])
                hist.append((r["steps"], r["dps"], r["merges"]))
            runs[budget] = (hist, seen_carried)
    assert runs[0][1] == 0 and runs[4][1] > 0
    assert runs[0][0] == runs[4][0]  # same walks, distinguished points and merges


@pytest.mark.parametrize("walks,steps,dpb", [(1, 3, 3), (23, 1, 3), (25, 5, 3), (48, 2, 12), (49, 7, 3),
                                             (97, 4, 12), (1000, 9, 3)])
def test_tensor_core_walk_ragged_launches(walks, steps, dpb):
    """The n = 4 tensor-core walk (launch shape 3) at ragged and tiny sizes.
    The cases cover fewer walks than one set (24), a half-empty second set, a
    group boundary (48) and single steps.  Both instantiations run: the one
    whose MMA warps store the distinguished points (theta = 2^-3) and the
    plain one (2^-12).  Every walk's record and the order-independent
    counters equal the dp4a shape's, and no bounded wait runs out."""
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    gates, _ = W.config_target(3)
    runs = {}
    for shape in (0, 3):
        p = Q.default_params(4, walks=walks, table_log2=16, launch_shape=shape)
        with Q.Problem.from_circuit(4, gates, 7, p) as prob:
            ws = torch.zeros(4 * walks, dtype=torch.int64, device=dev)
            merges = torch.zeros(3 * 4096, dtype=torch.int64, device=dev)
            counts = torch.zeros(8, dtype=torch.int64, device=dev)
            prob.level_walk_static(7, 1, dpb, 1, ws, steps, merges, counts)
            torch.cuda.synchronize()
            c = counts.cpu().numpy()
            runs[shape] = (ws.cpu().numpy(), c[:4].tolist(), int(c[7]) >> 32)
    assert runs[3][2] == 0
    assert runs[0][1][0] == walks * steps
    assert np.array_equal(runs[3][0], runs[0][0])
    assert runs[3][1] == runs[0][1]


def test_static_walk_rejects_an_empty_launch():
    """n_walks = 0 is an argument error, not an empty launch."""
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    gates, _ = W.config_target(3)
    with Q.Problem.from_circuit(4, gates, 7, Q.default_params(4, walks=64, table_log2=16)) as prob:
        ws = torch.zeros(0, dtype=torch.int64, device=dev)
        merges = torch.zeros(3, dtype=torch.int64, device=dev)
        counts = torch.zeros(8, dtype=torch.int64, device=dev)
        with pytest.raises(Q.QcsError):
            prob.level_walk_static(7, 1, 6, 1, ws, 4, merges, counts)
