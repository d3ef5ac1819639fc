"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper it pins and the outside fact used:
textbook matrices and conjugation tables, closed forms, algebraic invariants,
floating-point evaluations through numpy's Kronecker products, and brute force
on tiny instances.  A plausible slip in the oracle (a dropped sqrt2, a wrong
sign or phase, a transposed product, a wrong half-split order) fails at least
one of them.
"""

import numpy as np
import pytest

from paper_1606_07413_gb300 import workloads as W

R2 = np.sqrt(2.0)
w8 = np.exp(1j * np.pi / 4)

# textbook one-qubit matrices
I2 = np.eye(2, dtype=complex)
SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
SZ = np.array([[1, 0], [0, -1]], dtype=complex)
GH = np.array([[1, 1], [1, -1]], dtype=complex) / R2
GS = np.diag([1, 1j])
GT = np.diag([1, w8])


def kron_pauli(n, code):
    """P(code) as a Kronecker product of textbook Paulis; qubit q is bit q of
    the basis index (the most significant factor is qubit n-1)."""
    x, z = code >> n, code & ((1 << n) - 1)
    table = {(0, 0): I2, (0, 1): SZ, (1, 0): SX, (1, 1): SY}
    m = np.eye(1, dtype=complex)
    for q in reversed(range(n)):
        m = np.kron(m, table[((x >> q) & 1, (z >> q) & 1)])
    return m


def embed(n, q, g):
    m = np.eye(1, dtype=complex)
    for t in reversed(range(n)):
        m = np.kron(m, g if t == q else I2)
    return m


def float_unitary(n, gates):
    """Unitary of a gate list from textbook gate matrices (numpy, complex128)."""
    d = 1 << n
    U = np.eye(d, dtype=complex)
    for op, a, b in np.asarray(gates).reshape(-1, 3):
        if op == W.OP_CNOT:
            G = np.zeros((d, d), complex)
            for c in range(d):
                G[c ^ (((c >> a) & 1) << b), c] = 1
        elif op == W.OP_RP:
            P = kron_pauli(n, int(a))
            G = 0.5 * (1 + w8) * np.eye(d) + 0.5 * (1 - w8) * P
        else:
            g = {W.OP_H: GH, W.OP_S: GS, W.OP_T: GT, W.OP_X: SX, W.OP_Z: SZ,
                 W.OP_SDG: GS.conj(), W.OP_TDG: GT.conj()}[int(op)]
            G = embed(n, int(a), g)
        U = G @ U
    return U


def float_channel(n, U):
    """C[i][j] = Tr(P_i U P_j U^dagger) / 2^n over Kronecker Paulis: with
    A_j = U P_j U^dagger, Tr(P_i A_j) = sum_ab P_i[b, a] A_j[a, b]."""
    D = 4 ** n
    Ps = np.stack([kron_pauli(n, j) for j in range(D)])
    A = np.einsum("ab,jbc,dc->jad", U, Ps, U.conj())
    return np.einsum("iba,jab->ij", Ps, A).real / 2 ** n


def random_circuit(rng, n, length, t_gates=True):
    rows = []
    ops = [W.OP_H, W.OP_S, W.OP_T] if t_gates else [W.OP_H, W.OP_S]
    for _ in range(length):
        kind = int(rng.integers(len(ops) + (1 if n > 1 else 0)))
        if kind < len(ops):
            rows.append((ops[kind], int(rng.integers(n)), 0))
        else:
            c, t = rng.choice(n, 2, replace=False)
            rows.append((W.OP_CNOT, int(c), int(t)))
    return np.asarray(rows, np.int32).reshape(-1, 3)


# ---------------------------------------------------------------- Paulis (Sec. 4.1)

@pytest.mark.parametrize("n", [1, 2])
def test_pauli_product_phase_matches_kronecker_matrices(orc, n):
    """P(p) P(q) = i^lambda P(p^q) with lambda from textbook matrix products."""
    D = 4 ** n
    for p in range(D):
        for q in range(D):
            lhs = kron_pauli(n, p) @ kron_pauli(n, q)
            lam = orc.pauli_phase(n, p, q)
            assert np.allclose(lhs, (1j ** lam) * kron_pauli(n, p ^ q)), (p, q)


def test_unitary_builder_matches_textbook_gates(orc):
    rng = np.random.default_rng(3)
    for n in (1, 2, 3):
        gates = random_circuit(rng, n, 40)
        gates = np.concatenate([gates, np.asarray([(W.OP_RP, int(rng.integers(1, 4 ** n)), 0)], np.int32)])
        u, e = orc.unitary_from_circuit(n, gates)
        exact = (u[..., 0] + u[..., 1] * w8 + u[..., 2] * w8 ** 2 + u[..., 3] * w8 ** 3) / R2 ** e
        assert np.allclose(exact, float_unitary(n, gates))


# ------------------------------------------------------- channel representation (Sec. 4.1)

def test_channel_of_H_S_CNOT_follow_textbook_conjugation_tables(orc):
    # n = 1 codes: I=0, Z=1, X=2, Y=3
    H = orc.channel_from_circuit(1, [(W.OP_H, 0, 0)]).values()
    assert np.allclose(H, [[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, -1]])  # X<->Z, Y->-Y
    S = orc.channel_from_circuit(1, [(W.OP_S, 0, 0)]).values()
    assert np.allclose(S[:, 2], [0, 0, 0, 1])   # S X S^dag = Y
    assert np.allclose(S[:, 3], [0, 0, -1, 0])  # S Y S^dag = -X
    assert np.allclose(S[:, 1], [0, 1, 0, 0])   # Z fixed
    # CNOT with control qubit 0, target qubit 1 (n = 2; code = x << 2 | z)
    C = orc.channel_from_circuit(2, [(W.OP_CNOT, 0, 1)]).values()

    def code(x, z):
        return (x << 2) | z

    assert C[code(0b11, 0), code(0b01, 0)] == pytest.approx(1)  # X_c -> X_c X_t
    assert C[code(0b10, 0), code(0b10, 0)] == pytest.approx(1)  # X_t -> X_t
    assert C[code(0, 0b11), code(0, 0b10)] == pytest.approx(1)  # Z_t -> Z_c Z_t
    assert C[code(0, 0b01), code(0, 0b01)] == pytest.approx(1)  # Z_c -> Z_c


def test_T_closed_form(orc):
    """R(Z) on one qubit is T; T X T^dag = (X + Y)/sqrt2 and T Y T^dag = (Y - X)/sqrt2."""
    T = orc.channel_from_circuit(1, [(W.OP_T, 0, 0)])
    assert T.equals(orc.rhat(1, 1))
    v = T.values()
    assert np.allclose(v[:, 2], [0, 0, 1 / R2, 1 / R2])
    assert np.allclose(v[:, 3], [0, 0, -1 / R2, 1 / R2])
    assert np.allclose(v[:, 1], [0, 1, 0, 0])
    assert T.reduced().E == 1


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_channel_matches_float_trace_over_kronecker_paulis(orc, n):
    rng = np.random.default_rng(10 + n)
    for _ in range(3 if n < 4 else 1):
        gates = random_circuit(rng, n, 30 if n < 4 else 16)
        C = orc.channel_from_circuit(n, gates)
        assert np.allclose(C.values(), float_channel(n, float_unitary(n, gates)), atol=1e-9)


@pytest.mark.parametrize("n", [2, 3])
def test_channel_is_a_homomorphism(orc, n):
    """(UV)^ = U^ V^ (used implicitly when the paper writes Eq. tcount_synthesis in channel form)."""
    rng = np.random.default_rng(20 + n)
    for _ in range(2):
        g1 = random_circuit(rng, n, 25)
        g2 = random_circuit(rng, n, 25)
        both = orc.channel_from_circuit(n, np.concatenate([g1, g2]))  # g1 acts first
        prod = orc.channel_from_circuit(n, g2) @ orc.channel_from_circuit(n, g1)
        assert both.equals(prod)
        swapped = orc.channel_from_circuit(n, g1) @ orc.channel_from_circuit(n, g2)
        assert not both.equals(swapped)


# ------------------------------------------------------------ R^(P) (Sec. 4.1)

@pytest.mark.parametrize("n", [1, 2, 3])
def test_rhat_columns_equal_trace_definition(orc, n):
    for p in range(1, 4 ** n):
        assert orc.rhat(n, p).equals(orc.rhat_trace(n, p)), p


@pytest.mark.parametrize("n", [1, 2, 3])
def test_rhat_invariants(orc, n):
    ident = orc.identity(n)
    rng = np.random.default_rng(30 + n)
    for p in rng.choice(np.arange(1, 4 ** n), size=min(8, 4 ** n - 1), replace=False):
        R, Rt = orc.rhat(n, int(p)), orc.rhat(n, int(p), transpose=True)
        assert (R @ Rt).equals(ident)                   # orthogonal
        assert Rt.equals(orc.Chan(n, R.a.T.copy(), R.b.T.copy(), R.E))
        R2m = R @ R
        assert orc.is_clifford(R2m) and not orc.is_clifford(R)  # R^2 Clifford, R not
        R8 = R2m @ R2m
        R8 = R8 @ R8
        assert R8.equals(ident)                          # R^8 = I
        # at most two nonzeros per column, and exactly half the columns are split
        nz = (R.a != 0) | (R.b != 0)
        assert nz.sum(axis=0).max() <= 2
        assert (nz.sum(axis=0) == 2).sum() == 4 ** n // 2


def test_rp_gate_channel_equals_rhat(orc):
    for n in (1, 2, 3, 4):
        for p in (1, 4 ** n - 1, 5 % (4 ** n - 1) + 1):
            assert orc.channel_from_circuit(n, [(W.OP_RP, p, 0)]).equals(orc.rhat(n, p))


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_rhat_equals_the_float_channel_of_the_rotation(orc, n):
    """Sec. 4.1: R(P) = e^(i pi/8) exp(-i pi P/8) = ((1 + w) I + (1 - w) P) / 2
    with w = e^(i pi/4), built here from Kronecker Paulis; its channel,
    evaluated in floating point over the trace definition, equals the
    oracle's exact R^(P) and (as the transpose) R^(P)^T."""
    rng = np.random.default_rng(60 + n)
    ps = {1, 4 ** n - 1} | {int(v) for v in rng.integers(1, 4 ** n, size=6)}
    d = 1 << n
    for p in sorted(ps):
        R = 0.5 * (1 + w8) * np.eye(d) + 0.5 * (1 - w8) * kron_pauli(n, p)
        F = float_channel(n, R)
        assert np.allclose(orc.rhat(n, p).values(), F, atol=1e-12)
        assert np.allclose(orc.rhat(n, p, transpose=True).values(), F.T, atol=1e-12)


# ------------------------------------------------------ canonical form modulo Clifford

@pytest.mark.parametrize("n", [2, 3])
def test_canonical_form_and_walk_hash_are_clifford_invariant(orc, n):
    rng = np.random.default_rng(40 + n)
    gates, _ = W.seeded_target(n, 3, 99 + n)
    C = orc.channel_from_circuit(n, gates)
    for _ in range(3):
        Dc = orc.channel_from_circuit(n, W.clifford_word(rng, n, 60))
        CD = C @ Dc
        assert orc.same_coset(C, CD)
        assert orc.matrix_hash(C, 4, 0, 5, 48) == orc.matrix_hash(CD, 4, 0, 5, 48)
    # a different coset: multiply by one more rotation
    other = C @ orc.rhat(n, 3)
    assert not orc.same_coset(C, other)
    assert orc.matrix_hash(C, 4, 0, 5, 48) != orc.matrix_hash(other, 4, 0, 5, 48)


def test_walk_hash_is_a_function_of_the_column_multiset(orc):
    """The hash sees the product only through the multiset of its sign-folded
    non-identity column fingerprints: any signed permutation of the columns
    Q >= 1 keeps it (a Clifford is one such), and a repeated column counts
    with its multiplicity (two matrices whose multisets differ only in which
    column is doubled hash apart, which an accumulation that cancels pairs
    would miss)."""
    rng = np.random.default_rng(77)
    gates, _ = W.seeded_target(2, 3, 5)
    C = orc.channel_from_circuit(2, gates)
    D = C.a.shape[0]
    h0 = orc.matrix_hash(C, 4, 0, 5, 64)
    for _ in range(3):
        perm = np.concatenate([[0], 1 + rng.permutation(D - 1)])
        sgn = np.concatenate([[1], rng.choice([-1, 1], size=D - 1)])
        M = orc.Chan(2, C.a[:, perm] * sgn, C.b[:, perm] * sgn, C.E)
        assert orc.matrix_hash(M, 4, 0, 5, 64) == h0
    assert not np.array_equal(np.abs(C.a[:, 1]), np.abs(C.a[:, 2]))
    a1, b1, a2, b2 = C.a.copy(), C.b.copy(), C.a.copy(), C.b.copy()
    a1[:, 2], b1[:, 2] = C.a[:, 1], C.b[:, 1]  # column 1 twice, column 2 gone
    a2[:, 1], b2[:, 1] = C.a[:, 2], C.b[:, 2]  # column 2 twice, column 1 gone
    h1 = orc.matrix_hash(orc.Chan(2, a1, b1, C.E), 4, 0, 5, 64)
    h2 = orc.matrix_hash(orc.Chan(2, a2, b2, C.E), 4, 0, 5, 64)
    assert len({h0, h1, h2}) == 3


def test_hash_depends_on_version_and_tag(orc):
    gates, _ = W.seeded_target(2, 3, 5)
    C = orc.channel_from_circuit(2, gates)
    h = {orc.matrix_hash(C, 4, c, v, 64) for v in range(3) for c in range(3)}
    assert len(h) == 9


# --------------------------------------------------------------- T-count (Sec. 4.1)

def test_tcount_of_single_T_is_one(orc):
    C = orc.channel_from_circuit(1, [(W.OP_T, 0, 0)])
    assert orc.mitm_tcount(C, 3)[0] == 1
    assert orc.brute_tcount(C, 3)[0] == 1


def test_tcount_of_clifford_is_zero(orc):
    rng = np.random.default_rng(7)
    for n in (1, 2, 3):
        C = orc.channel_from_circuit(n, W.clifford_word(rng, n, 80))
        assert orc.is_clifford(C) and orc.sde(C) == 0
        assert orc.mitm_tcount(C, 2)[0] == 0


def test_rotation_squared_is_clifford(orc):
    for p in (1, 6, 15):
        C = orc.channel_from_circuit(2, [(W.OP_RP, p, 0), (W.OP_RP, p, 0)])
        assert orc.mitm_tcount(C, 2)[0] == 0
        assert orc.brute_tcount(C, 2)[0] == 0


def test_every_single_rotation_has_tcount_one(orc):
    for p in range(1, 16):
        C = orc.channel_from_circuit(2, [(W.OP_RP, p, 0), (W.OP_H, 1, 0), (W.OP_CNOT, 1, 0)])
        t, paulis = orc.mitm_tcount(C, 2)
        assert t == 1 and orc.verify(C, paulis)


def test_mitm_matches_brute_force_on_tiny_instances(orc):
    """Exhaustive MITM (Eq. mitm) agrees with brute force over all products (Sec. 3)."""
    rng = np.random.default_rng(11)
    seen = set()
    for trial in range(10):
        t = int(rng.integers(1, 4))
        # repeated or commuting factors make some instances collapse below t
        ps = [int(v) for v in rng.integers(1, 16, size=t)]
        if trial % 3 == 0 and t >= 2:
            ps[1] = ps[0]
        rows = [(W.OP_RP, p, 0) for p in ps] + [tuple(r) for r in W.clifford_word(rng, 2, 30)]
        C = orc.channel_from_circuit(2, np.asarray(rows, np.int32))
        tb, pb = orc.brute_tcount(C, 3)
        tm, pm = orc.mitm_tcount(C, 3)
        assert tb == tm and tm <= t
        assert orc.sde(C) <= tm
        assert orc.verify(C, pm) and orc.verify(C, pb)
        seen.add(tm)
    assert len(seen) >= 2


def _perm_unitary(perm):
    d = len(perm)
    u = np.zeros((d, d, 4), np.int64)
    for c, r in enumerate(perm):
        u[r, c, 0] = 1
    return u


def test_full_adder_is_a_toffoli_between_cnot_circuits(orc):
    """Sec. 5.3: the 4-qubit 1-bit full adder is affine equivalent to the
    Toffoli (equal up to CNOTs), so it has the Toffoli's T-count.  Pinned as
    permutations (adder = L2 . Toffoli(u, v -> d) . L1 with L1, L2 linear maps
    of the bits) and in channel form, where L1 and L2 are Cliffords (signed
    permutations, sde 0) and the channel of the composition is the product
    of the channels."""
    n, adder = W.permutation_targets()["adder"]
    assert n == 4 and sorted(adder) == list(range(16))

    def bits(c):
        return [(c >> q) & 1 for q in range(4)]

    def word(b):
        return b[0] | (b[1] << 1) | (b[2] << 2) | (b[3] << 3)

    def l1(c):  # (a, b, c, d) -> (a ^ c, b ^ c, c, d)
        a, b, ci, d = bits(c)
        return word([a ^ ci, b ^ ci, ci, d])

    def tof(c):  # d ^= u v
        u, v, ci, d = bits(c)
        return word([u, v, ci, d ^ (u & v)])

    def l2(c):  # (u, v, c, d) -> (u ^ c, v ^ c, u ^ v ^ c, d ^ c)
        u, v, ci, d = bits(c)
        return word([u ^ ci, v ^ ci, u ^ v ^ ci, d ^ ci])

    assert [l2(tof(l1(c))) for c in range(16)] == adder
    P1, PT, P2 = ([f(c) for c in range(16)] for f in (l1, tof, l2))
    C1, CT, C2, CA = (orc.channel_from_unitary(4, _perm_unitary(p), 0) for p in (P1, PT, P2, adder))
    for Cl in (C1, C2):
        assert orc.sde(Cl) == 0 and orc.is_clifford(Cl)
    assert CA.equals(C2 @ CT @ C1)
    assert orc.sde(CA) == orc.sde(CT)


@pytest.mark.parametrize("name", ["peres", "quantum_or"])
def test_table1_gates_are_toffolis_between_cliffords(orc, name):
    """Table 1: the Peres gate is a Toffoli followed by CNOT(0 -> 1), and the
    OR gate (bit 2 ^= bit 0 OR bit 1) is a Toffoli between X layers, since
    a OR b = 1 ^ (NOT a AND NOT b).  Pinned as permutations and in channel
    form, where the outer layers are Cliffords (signed permutations), so
    each gate has the Toffoli's T-count."""
    n, perm = W.permutation_targets()[name]
    _, tof = W.permutation_targets()["toffoli"]
    assert n == 3 and sorted(perm) == list(range(8))
    if name == "peres":
        l1 = list(range(8))
        l2 = [c ^ ((c & 1) << 1) for c in range(8)]  # CNOT 0 -> 1
    else:
        l1 = [c ^ 3 for c in range(8)]  # X on bits 0, 1
        l2 = [c ^ 7 for c in range(8)]  # X on bits 0, 1, 2
    assert [l2[tof[l1[c]]] for c in range(8)] == perm
    C1, CT, C2, CG = (orc.channel_from_unitary(3, _perm_unitary(p), 0) for p in (l1, tof, l2, perm))
    for Cl in (C1, C2):
        assert orc.is_clifford(Cl)
    assert CG.equals(C2 @ CT @ C1) and orc.sde(CG) == orc.sde(CT)


def test_construction_bound_and_sde_lower_bound(orc):
    for cfg in (1, 2):
        c = W.CONFIGS[cfg]
        gates, _ = W.config_target(cfg)
        C = orc.channel_from_circuit(c["n"], gates)
        assert orc.sde(C) <= c["t"]
    gates, _ = W.config_target(1)
    C = orc.channel_from_circuit(2, gates)
    t, paulis = orc.mitm_tcount(C, 3)
    assert orc.sde(C) <= t <= 3 and orc.verify(C, paulis)


def test_verify_rejects_wrong_decompositions(orc):
    gates, _ = W.config_target(1)
    C = orc.channel_from_circuit(2, gates)
    t, paulis = orc.mitm_tcount(C, 3)
    assert orc.verify(C, paulis)
    assert not orc.verify(C, paulis[::-1]) or paulis == paulis[::-1]
    bad = list(paulis)
    bad[0] = bad[0] % 15 + 1
    assert not orc.verify(C, bad)


# --------------------------------------------------- walk, claws and re-walking (Sec. 3)

def test_claw_halves_hash_equal(orc):
    """A decomposition split as in Eq. mitm gives V and W in one coset, so the
    walk maps both sides to the same next state."""
    for cfg in (1, 2):
        c = W.CONFIGS[cfg]
        gates, _ = W.config_target(cfg)
        C = orc.channel_from_circuit(c["n"], gates)
        if cfg == 1:
            t, p = orc.mitm_tcount(C, 3)
        else:
            t, p = orc.mitm_level(C, 5) and (5, orc.mitm_level(C, 5))
        h = t // 2
        chunk = p[2 * h] if t & 1 else 0
        V = orc.half_product(C, t, chunk, 0, p[:h])
        Wm = orc.half_product(C, t, chunk, 1, p[h:2 * h])
        assert V.E == Wm.E == orc.sde(C) + (t & 1) + h
        assert orc.same_coset(V, Wm)
        assert orc.matrix_hash(V, t, chunk, 3, c["L"]) == orc.matrix_hash(Wm, t, chunk, 3, c["L"])
        # the states that decode to these halves step to the same point
        xv = orc.encode(c["n"], t, c["L"], 0, p[:h])
        xw = orc.encode(c["n"], t, c["L"], 1, p[h:2 * h])
        assert orc.decode(c["n"], t, c["L"], xv) == (0, p[:h])
        assert orc.decode(c["n"], t, c["L"], xw) == (1, p[h:2 * h])
        y = orc.walk_step(C, t, chunk, 3, c["L"], [xv, xw])
        assert y[0] == y[1]
        cls, a, b, paulis = orc.rewalk(C, t, chunk, 3, c["L"], xv, 1, xw, 1)
        assert cls == orc.CLAW and orc.verify(C, paulis)


def test_walk_step_is_a_function_of_the_decoded_point(orc):
    gates, _ = W.config_target(1)
    C = orc.channel_from_circuit(2, gates)
    ell = orc.field_bits(2, 2, 32)
    assert ell == 16
    # bits above the side bit and the rotation field do not matter
    x = np.asarray([7, 7 + (1 << (1 + ell)), 7 + (12345 << (1 + ell))], np.uint64)
    y = orc.walk_step(C, 2, 0, 1, 32, x)
    assert y[0] == y[1] == y[2]
    assert orc.classify(C, 2, 0, 32, int(x[0]), int(x[1]))[0] == orc.TRIVIAL
    y = orc.walk_step(C, 2, 0, 1, 32, np.asarray([6, 7], np.uint64))
    assert y[0] != y[1]


@pytest.mark.parametrize("n,k,L", [(1, 15, 32), (2, 2, 32), (2, 7, 32), (3, 5, 48), (3, 15, 48), (4, 7, 64),
                                   (4, 15, 64)])
def test_decode_fields_cover_every_rotation_evenly(orc, n, k, L):
    """Each rotation reads its own l-bit field (Sec. 2 concatenation of
    codes); the multiply-shift map of a field onto the 4^n - 1 Paulis is onto,
    and every Pauli gets floor or ceil of 2^l / xi field values."""
    xi, h = 4 ** n - 1, k // 2
    ell = orc.field_bits(n, k, L)
    assert 1 + ell * h <= L and (1 << ell) >= xi
    counts = np.bincount([(v * xi) >> ell for v in range(1 << ell)], minlength=xi)
    assert counts.min() >= (1 << ell) // xi and counts.max() <= -(-(1 << ell) // xi)
    rng = np.random.default_rng(n * 100 + k)
    for _ in range(50):
        q = [int(v) for v in rng.integers(1, xi + 1, size=h)]
        side = int(rng.integers(2))
        x = orc.encode(n, k, L, side, q)
        assert x < (1 << L) and orc.decode(n, k, L, x) == (side, q)


def test_serial_walk_search_finds_the_optimal_tcount(orc):
    rng = np.random.default_rng(12)
    for trial in range(3):
        gates, _ = W.seeded_target(2, 3, 500 + trial)
        C = orc.channel_from_circuit(2, gates)
        t_exact, _ = orc.mitm_tcount(C, 3)
        t, paulis, st = orc.vow_search(C, 3, dtheta=2, L=32, max_len=400, per_version=4000,
                                       per_level=2_000_000, table_log2=14, seed=int(rng.integers(1 << 40)))
        assert t == t_exact and orc.verify(C, paulis)
        assert st["claws"] >= 1 and st["no_merge"] == 0


def test_dp_predicate(orc):
    y = np.asarray([0, 1 << 20, (1 << 26) - 1, 1 << 26, (1 << 31) | 5], np.uint64)
    assert orc.is_dp(y, 32, 6).tolist() == [True, True, True, False, False]


def _noncommuting_chain(orc, rng, n, t):
    """t Pauli codes with every neighbour pair anticommuting."""
    ps = [int(rng.integers(1, 4 ** n))]
    while len(ps) < t:
        q = int(rng.integers(1, 4 ** n))
        if orc.pauli_phase(n, ps[-1], q) != orc.pauli_phase(n, q, ps[-1]):
            ps.append(q)
    return ps


@pytest.mark.parametrize("n,t", [(2, 4), (2, 5), (3, 4), (3, 5)])
def test_known_normal_form_is_a_claw(orc, n, t):
    """Build C = R(P_t)...R(P_1) D directly (Eq. tcount_synthesis) with
    non-commuting neighbours; then V_(P_1..P_h) and W_(P_h+1..P_2h) (chunk P_t
    for odd t) are one coset (Eq. mitm), and the half products equal the
    explicit products of the (trace-pinned) R^ matrices."""
    rng = np.random.default_rng(100 * n + t)
    ps = _noncommuting_chain(orc, rng, n, t)
    rows = [tuple(r) for r in W.clifford_word(rng, n, 40)] + [(W.OP_RP, p, 0) for p in ps]
    C = orc.channel_from_circuit(n, np.asarray(rows, np.int32))
    h = t // 2
    chunk = ps[2 * h] if t & 1 else 0
    V = orc.half_product(C, t, chunk, 0, ps[:h])
    Wm = orc.half_product(C, t, chunk, 1, ps[h:2 * h])
    # explicit products
    Vx = orc.identity(n)
    for p in ps[:h]:
        Vx = orc.rhat(n, p) @ Vx
    Wx = C
    if t & 1:
        Wx = orc.rhat(n, chunk, transpose=True) @ Wx
    for p in reversed(ps[h:2 * h]):
        Wx = orc.rhat(n, p, transpose=True) @ Wx
    assert V.equals(Vx) and Wm.equals(Wx)
    assert orc.same_coset(V, Wm)
    assert orc.verify(C, ps)
    # swapping the two W-side factors breaks the claw (they do not commute)
    Wswap = orc.half_product(C, t, chunk, 1, ps[h:2 * h][::-1])
    assert not orc.same_coset(V, Wswap)
    L = {2: 32, 3: 48}[n]
    xv = orc.encode(n, t, L, 0, ps[:h])
    xw = orc.encode(n, t, L, 1, ps[h:2 * h])
    y = orc.walk_step(C, t, chunk, 9, L, [xv, xw])
    assert y[0] == y[1]
    cls, paulis = orc.classify(C, t, chunk, L, xv, xw)
    assert cls == orc.CLAW and paulis == ps


@pytest.mark.parametrize("n,t", [(2, 3), (2, 5), (3, 5)])
def test_moving_a_rotation_across_the_split_keeps_the_claw(orc, n, t):
    """Eq. mitm with the odd level's extra rotation on the other side, as
    the exhaustive pass splits it when C^ has a denominator: for a
    decomposition C = R(P_t)...R(P_1) D, V' = R(P_(h+1))...R(P_1) and
    W' = R(P_(h+2))^T...R(P_t)^T C lie in one Clifford coset, and a wrong
    order of W' factors (or another rotation) breaks it (exact products,
    checked by the oracle's exact coset test)."""
    rng = np.random.default_rng(300 + 10 * n + t)
    ps = _noncommuting_chain(orc, rng, n, t)
    rows = [tuple(r) for r in W.clifford_word(rng, n, 40)] + [(W.OP_RP, p, 0) for p in ps]
    C = orc.channel_from_circuit(n, np.asarray(rows, np.int32))
    assert orc.sde(C) >= 1
    h = t // 2
    Vp = orc.identity(n)
    for p in ps[:h + 1]:
        Vp = orc.rhat(n, p) @ Vp
    Wp = C
    for p in reversed(ps[h + 1:]):
        Wp = orc.rhat(n, p, transpose=True) @ Wp
    assert orc.same_coset(Vp, Wp)
    wrong = list(ps[h + 1:])
    if len(wrong) >= 2:
        wrong[0], wrong[1] = wrong[1], wrong[0]  # non-commuting neighbours in the wrong order
    else:
        wrong[0] = wrong[0] % (4 ** n - 1) + 1  # another rotation
    Ws = C
    for p in reversed(wrong):
        Ws = orc.rhat(n, p, transpose=True) @ Ws
    assert not orc.same_coset(Vp, Ws)
    assert orc.verify(C, ps)


def _is_signed_permutation_product(V, Wm):
    """V^T W in exact (a, b) arithmetic: value (a + b sqrt2) / sqrt2^E with
    E = E_V + E_W; a signed permutation has one entry of value +-1 in every
    row and column and zeros elsewhere."""
    Va, Vb, Wa, Wb = (np.asarray(x, dtype=object) for x in (V.a, V.b, Wm.a, Wm.b))
    Pa = Va.T.dot(Wa) + 2 * Vb.T.dot(Wb)
    Pb = Va.T.dot(Wb) + Vb.T.dot(Wa)
    E = V.E + Wm.E

    def unit(a, b):
        if E % 2 == 0:
            return b == 0 and abs(a) == 2 ** (E // 2)
        return a == 0 and abs(b) == 2 ** ((E - 1) // 2)

    D = Pa.shape[0]
    for i in range(D):
        units = 0
        for j in range(D):
            a, b = int(Pa[i, j]), int(Pb[i, j])
            if unit(a, b):
                units += 1
            elif a != 0 or b != 0:
                return False
        if units != 1:
            return False
    return True


@pytest.mark.parametrize("n,t,seed", [(1, 2, 21), (1, 3, 22), (2, 2, 23), (2, 3, 24)])
def test_same_coset_is_the_signed_permutation_test_by_brute_force(orc, n, t, seed):
    """Sec. 4.1: two channel matrices lie in one Clifford coset exactly when
    V^T W is a signed permutation (both are orthogonal, and a Clifford's
    channel is a signed permutation).  Over every V and W point of the
    level (every chunk for odd t), the oracle's canonical-form equality
    agrees with that test done here in exact integer arithmetic, and the
    construction's level has at least one such pair."""
    import itertools

    gates, _ = W.seeded_target(n, t, seed)
    C = orc.channel_from_circuit(n, gates)
    k, h, xi = t, t // 2, 4 ** n - 1
    found = 0
    for chunk in (range(1, xi + 1) if k & 1 else [0]):
        tuples = [list(q) for q in itertools.product(range(1, xi + 1), repeat=h)]
        Vs = [orc.half_product(C, k, chunk, 0, q) for q in tuples]
        Ws = [orc.half_product(C, k, chunk, 1, q) for q in tuples]
        for V in Vs:
            for Wm in Ws:
                want = _is_signed_permutation_product(V, Wm)
                assert orc.same_coset(V, Wm) == want
                found += want
    assert found >= 1


@pytest.mark.parametrize("n,t,seed,chunk", [(1, 3, 31, 2), (2, 2, 32, 0), (2, 3, 33, 5)])
def test_rewalk_matches_brute_force_trail_enumeration(orc, n, t, seed, chunk):
    """Sec. 3, Fig. 2 on a walk small enough to tabulate (2^6 states): for
    trails that end at a common point, the re-walk must report the first
    point where they meet, found here by enumerating both trails.  A start
    that lies on the other trail is Robin Hood; otherwise the two distinct
    predecessors of the meeting point are classified by their decoded sides
    and rotations and, across sides, by exact coset equality.  Trails that
    never meet within their lengths are no merge.  Six-bit states make hash
    collisions between distinct points common, so every class occurs."""
    gates, _ = W.seeded_target(n, t, seed)
    C = orc.channel_from_circuit(n, gates)
    k, L, version = t, 6, 3
    F = orc.walk_step(C, k, chunk, version, L, np.arange(1 << L, dtype=np.uint64)).astype(np.int64)

    def trail(x, m):
        out = [x]
        for _ in range(m):
            out.append(int(F[out[-1]]))
        return out

    def expected_class(a, b):
        sa, qa = orc.decode(n, k, L, a)
        sb, qb = orc.decode(n, k, L, b)
        if sa == sb:
            return orc.TRIVIAL if qa == qb else orc.SAME_SIDE
        qv, qw = (qa, qb) if sa == 0 else (qb, qa)
        V = orc.half_product(C, k, chunk, 0, qv)
        Wm = orc.half_product(C, k, chunk, 1, qw)
        return orc.CLAW if orc.same_coset(V, Wm) else orc.FALSE_HASH

    rng = np.random.default_rng(seed)
    seen = {}
    for _ in range(400):
        a, b = (int(v) for v in rng.integers(0, 1 << L, size=2))
        A, B = trail(a, 60), trail(b, 60)
        pos_a = {}
        for i, x in enumerate(A):
            pos_a.setdefault(x, i)
        meet = next(((pos_a[y], j) for j, y in enumerate(B) if y in pos_a), None)
        if meet is None or a == b:
            continue
        i0, j0 = meet
        tail = 3  # both trails go on to a common end point
        la, lb = i0 + tail, j0 + tail
        cls, x, y, paulis = orc.rewalk(C, k, chunk, version, L, a, la, b, lb)
        if j0 == 0 or i0 == 0:
            want = orc.ROBIN_HOOD
            assert (x, y) == ((b, b) if j0 == 0 else (a, a)) and cls == want
        else:
            want = expected_class(A[i0 - 1], B[j0 - 1])
            assert cls == want and {x, y} == {A[i0 - 1], B[j0 - 1]}
            if want == orc.CLAW:
                assert orc.verify(C, paulis)
        seen[want] = seen.get(want, 0) + 1
    # two trails that do not meet within their lengths
    for _ in range(200):
        a, b = (int(v) for v in rng.integers(0, 1 << L, size=2))
        A, B = trail(a, 1), trail(b, 1)
        if not set(A) & set(B):
            assert orc.rewalk(C, k, chunk, version, L, a, 1, b, 1)[0] == orc.NO_MERGE
            seen[orc.NO_MERGE] = seen.get(orc.NO_MERGE, 0) + 1
            break
    assert seen.get(orc.ROBIN_HOOD, 0) >= 1 and seen.get(orc.NO_MERGE, 0) == 1
    assert sum(seen.get(c, 0) for c in (orc.TRIVIAL, orc.SAME_SIDE, orc.CLAW, orc.FALSE_HASH)) >= 10


def test_fingerprint_weights_are_the_splitmix64_stream(orc):
    """The fingerprint weights (Ua, Ub) of row i >= 1 are outputs 2i and 2i + 1
    of the SplitMix64 stream (Steele, Lea & Flood 2014) seeded with
    0x6A09E667F3BCC908, and row 0 has weight 0.  The generator is written
    here from its published definition and checked against its published
    first output for seed 0."""
    M64 = (1 << 64) - 1
    gamma = 0x9E3779B97F4A7C15

    def output(seed, j):  # j-th output (0-based) of the stream seeded with seed
        z = (seed + (j + 1) * gamma) & M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    assert output(0, 0) == 0xE220A8397B1DCDAF
    for n in (1, 2, 3):
        ua, ub = orc.fp_weights(n)
        assert ua[0] == 0 and ub[0] == 0
        for i in range(1, 4 ** n):
            assert int(ua[i]) == output(0x6A09E667F3BCC908, 2 * i) & 0xFFFFFFFF
            assert int(ub[i]) == output(0x6A09E667F3BCC908, 2 * i + 1) & 0xFFFFFFFF


@pytest.mark.parametrize("n,t,seed,kmax", [(1, 3, 41, 7), (1, 5, 42, 7), (2, 3, 43, 5), (2, 5, 44, 5),
                                            (2, 7, 45, 5), (2, 7, 46, 5)])
def test_the_other_odd_split_finds_the_same_levels(orc, n, t, seed, kmax):
    """The exhaustive pass of an odd level k = 2h + 1 may put the extra
    rotation on V: V' = R(r_(h+1))..R(r_1) against W' = R(s_1)^T..R(s_h)^T C
    (Eq. mitm with the split moved by one).  Both splits enumerate every
    product of k rotations, so a level has a claw under one exactly when it
    has one under the other: brute force over every V' and W' (canonical
    forms joined in a dictionary) against the oracle's meet in the middle."""
    import itertools

    gates, _ = W.seeded_target(n, t, seed)
    C = orc.channel_from_circuit(n, gates)
    xi = 4 ** n - 1

    def key(M):
        f, sde = orc.canon(M)
        return sde, f.tobytes()

    for k in range(3, kmax + 1, 2):
        h = k // 2
        stored = set()
        for s_ in itertools.product(range(1, xi + 1), repeat=h):
            Wp = C
            for p in reversed(s_):
                Wp = orc.rhat(n, p, transpose=True) @ Wp
            stored.add(key(Wp))
        claw = False
        for r in itertools.product(range(1, xi + 1), repeat=h + 1):
            Vp = orc.identity(n)
            for p in r:
                Vp = orc.rhat(n, p) @ Vp
            if key(Vp) in stored:
                claw = True
                break
        assert claw == (orc.mitm_level(C, k) is not None), (n, t, k)

