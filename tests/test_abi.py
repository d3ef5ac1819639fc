"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/qcs.h declares, and its exact host paths
(verification, input validation) agree with the oracle."""
import os
import re

import numpy as np
import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import workloads as W
from paper_1606_07413_gb300 import build as B


@pytest.fixture(scope="module")
def qlib():
    B.build()
    return Q.lib()


def declared_symbols():
    hdr = open(B.os.path.join(B.INCLUDE, "qcs.h")).read()
    return sorted(set(re.findall(r"QCS_API\s+[^;(]*?\b(qcs_[a-z_]+)\s*\(", hdr, flags=re.S)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["qcs_create_problem", "qcs_create_problem_channel", "qcs_run_walks", "qcs_poll_collisions",
                 "qcs_verify_decomposition", "qcs_walk_step", "qcs_destroy_problem", "qcs_strerror"]:
        assert must in names


def test_library_exports_every_declared_symbol(qlib):
    import subprocess

    out = subprocess.check_output(["nm", "-D", "--defined-only", B.LIB]).decode()
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for name in declared_symbols():
        assert name in exported, name
        assert hasattr(qlib, name)
    # nothing but the ABI leaks out
    assert all(s.startswith("qcs_") for s in exported if not s.startswith("_"))


def test_strerror_and_defaults(qlib):
    for code in range(0, -10, -1):
        assert Q.strerror(code)
    for n, L in ((2, 32), (3, 48), (4, 64)):
        p = Q.default_params(n)
        assert p.state_bits == L and p.walks >= 4096


def test_verify_decomposition_host_exact(qlib, orc):
    gates, _ = W.config_target(1)
    u, e = orc.unitary_from_circuit(2, gates)
    C = orc.channel_from_circuit(2, gates)
    t, p = orc.mitm_tcount(C, 3)
    assert Q.verify_decomposition(2, u, e, p)
    bad = list(p)
    bad[-1] = bad[-1] % 15 + 1
    assert not Q.verify_decomposition(2, u, e, bad)
    assert not Q.verify_decomposition(2, u, e, [])


def test_verify_agrees_with_oracle_on_random_sequences(qlib, orc):
    rng = np.random.default_rng(4)
    for trial in range(20):
        n = 2 if trial % 2 else 3
        ps = [int(v) for v in rng.integers(1, 4 ** n, size=3)]
        rows = [tuple(r) for r in W.clifford_word(rng, n, 20)] + [(W.OP_RP, p, 0) for p in ps]
        u, e = orc.unitary_from_circuit(n, np.asarray(rows, np.int32))
        C = orc.channel_from_circuit(n, np.asarray(rows, np.int32))
        cand = ps if trial % 3 else [int(v) for v in rng.integers(1, 4 ** n, size=3)]
        assert Q.verify_decomposition(n, u, e, cand) == orc.verify(C, cand)


def test_verify_agrees_with_oracle_at_four_qubits(qlib, orc):
    """The library's exact host verification (Eq. tcount_synthesis: D^ must
    be a signed permutation) on 4-qubit targets with up to seven rotations,
    against the oracle: the true decomposition, a reordered one and a
    corrupted one."""
    rng = np.random.default_rng(44)
    for t in (4, 7):
        ps = [int(v) for v in rng.integers(1, 256, size=t)]
        rows = [tuple(r) for r in W.clifford_word(rng, 4, 30)] + [(W.OP_RP, p, 0) for p in ps]
        u, e = orc.unitary_from_circuit(4, np.asarray(rows, np.int32))
        C = orc.channel_from_circuit(4, np.asarray(rows, np.int32))
        bad = list(ps)
        bad[t // 2] = bad[t // 2] % 255 + 1
        for cand in (ps, ps[::-1], bad):
            assert Q.verify_decomposition(4, u, e, cand) == orc.verify(C, cand)
        assert Q.verify_decomposition(4, u, e, ps)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_channel_from_unitary_agrees_with_the_oracle(qlib, orc, n):
    """qcs_channel_from_unitary (the library's exact host channel, Sec. 4.1)
    equals the oracle's on Clifford+T circuits, reduced to the sde."""
    rng = np.random.default_rng(70 + n)
    for t in (0, 3):
        ps = [int(v) for v in rng.integers(1, 4 ** n, size=t)]
        rows = [tuple(r) for r in W.clifford_word(rng, n, 30)] + [(W.OP_RP, p, 0) for p in ps]
        u, e = orc.unitary_from_circuit(n, np.asarray(rows, np.int32))
        a, b, E = Q.channel_from_unitary(n, u, e)
        C = orc.channel_from_unitary(n, u, e)
        assert orc.Chan(n, a, b, E).equals(C) and E == orc.sde(C)
    with pytest.raises(Q.QcsError) as ei:
        Q.channel_from_unitary(n, np.zeros((1 << n, 1 << n, 4), np.int64), 0)
    assert ei.value.code == Q.ERR_NOT_UNITARY


def test_create_problem_rejects_bad_input_before_any_device_work(qlib):
    d = 4
    u = np.zeros((d, d, 4), np.int64)
    for i in range(d):
        u[i, i, 0] = 1
    u[0, 1, 0] = 1  # not unitary
    with pytest.raises(Q.QcsError) as ei:
        Q.Problem.from_unitary(2, u, 0, 3)
    assert ei.value.code == Q.ERR_NOT_UNITARY
    with pytest.raises(Q.QcsError) as ei:
        Q.Problem.from_circuit(5, [(W.OP_H, 0, 0)], 3)
    assert ei.value.code == Q.ERR_ARG
    with pytest.raises(Q.QcsError) as ei:
        Q.Problem.from_circuit(2, [(W.OP_CNOT, 0, 0)], 3)
    assert ei.value.code == Q.ERR_ARG
    with pytest.raises(Q.QcsError) as ei:
        Q.Problem.from_circuit(2, [(W.OP_H, 0, 0)], 16)
    assert ei.value.code == Q.ERR_ARG
    p = Q.default_params(2, dp_bits=40)  # d_theta >= L
    with pytest.raises(Q.QcsError) as ei:
        Q.Problem.from_circuit(2, [(W.OP_H, 0, 0)], 3, p)
    assert ei.value.code == Q.ERR_ARG
    # a channel that is not orthogonal
    D = 16
    a = np.eye(D, dtype=np.int64)
    a[3, 4] = 1
    with pytest.raises(Q.QcsError) as ei:
        Q.Problem.from_channel(2, a, np.zeros_like(a), 0, 3)
    assert ei.value.code == Q.ERR_NOT_UNITARY


def test_verify_rejects_bad_arguments(qlib):
    u = np.zeros((4, 4, 4), np.int64)
    for i in range(4):
        u[i, i, 0] = 1
    with pytest.raises(Q.QcsError):
        Q.verify_decomposition(2, u, 0, [16])
    assert Q.verify_decomposition(2, u, 0, [])


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes mirrors of qcs_params, qcs_result and qcs_batch_params must
    # have the header's field offsets and sizes (compiled here with gcc)
    import ctypes
    import subprocess

    structs = {"qcs_params": Q.Params, "qcs_result": Q.Result, "qcs_batch_params": Q.BatchParams}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qcs.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-I", inc, str(src), "-o", str(exe)])
    got = {}
    for ln in subprocess.check_output([str(exe)]).decode().splitlines():
        cname, field, val = ln.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_level_plan_follows_the_appendix_rule(qlib):
    # theta_policy 1: theta = 2^-d, d = max(theta_min_bits, round(log2 sqrt(N / 2w)))
    import math

    for n, k, tl in ((2, 3, 16), (3, 5, 22), (3, 7, 18), (4, 6, 26), (4, 7, 26), (4, 7, 30), (4, 8, 20)):
        p = Q.default_params(n, table_log2=tl, dp_bits=30 if n == 4 else 20)
        pl = Q.plan_level(n, k, p)
        xi = 4 ** n - 1
        N = 2 * xi ** (k // 2) * (xi if k & 1 else 1)
        w = 2 ** tl
        assert pl["points"] == N
        if N <= 2 * w:
            assert pl["dp_bits"] == p.theta_min_bits
        else:
            assert abs(pl["dp_bits"] - 0.5 * math.log2(N / (2 * w))) <= 0.5
        theta = 2.0 ** -pl["dp_bits"]
        steps_per_launch = pl["walks"] * pl["steps"]
        # a launch stays within one function version, trails of 4/theta fit
        assert steps_per_launch <= max(p.version_factor * N, pl["walks"] * min(p.steps_per_launch, 4 / theta))
        # expected merges per launch fit half the queue
        stored = min(1.0, w / (theta * N))
        assert steps_per_launch * theta * stored <= p.queue_capacity / 2 or pl["steps"] == 1
        # the level's budget and at least four versions
        assert pl["min_launches"] * steps_per_launch >= p.budget_factor * N
        assert pl["min_launches"] >= 4 * pl["launches_per_version"]


def test_level_plan_fixed_theta_and_bad_arguments(qlib):
    p = Q.default_params(3, theta_policy=0, dp_bits=10)
    assert Q.plan_level(3, 5, p)["dp_bits"] == 10
    for n, k in ((0, 4), (5, 4), (3, 1), (3, 16)):
        with pytest.raises(Q.QcsError):
            Q.plan_level(n, k, p)
