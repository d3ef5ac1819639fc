"""Seeded synthetic inputs for the deterministic-walk T-count search.

This module draws random choices (Pauli codes, Clifford gate words and walk
states) and lists the named circuits the paper's text fixes, as basis-state
permutations.  It holds none of the method's arithmetic (no unitary or channel
products, no rotation matrices, no canonical form, no hash); both the CUDA path
and the CPU oracle receive these choices and build every matrix themselves.

Workload recipe (the paper's workloads are specific 3- and 4-qubit T-count-7
circuits, Table 1 and Sec. 5.3; none is a public dataset, so seeded stand-ins of
the same shape are drawn here):

* a target is ``C0 . R(P_t) ... R(P_1)`` (Eq. tcount_synthesis with the Clifford
  moved to the left), with every ``P_j`` uniform over the ``4^n - 1``
  non-identity Pauli codes and ``C0`` a word of 200 gates drawn uniformly from
  ``{H_q, S_q, CNOT_qr}``;
* a walk state is a uniform ``L``-bit string (Sec. 3: trails start at random
  points of the walk space).

The paper's named circuits that a textbook definition or the text fixes are
given as basis-state permutations (``permutation_targets``): the Toffoli,
Fredkin, Peres and OR gates (Table 1) and a 4-qubit 1-bit full adder
(Sec. 5.3).

Gate lists are ``(m, 3)`` int32 arrays of ``(op, a, b)`` rows in time order
(first row acts first, so the circuit unitary is ``G_m ... G_1``).
"""
from __future__ import annotations

import numpy as np

# Gate op codes of the circuit input format (the same values are declared in
# include/qcs.h; the oracle keeps its own copy of this interface table).
OP_H, OP_S, OP_CNOT, OP_T, OP_RP, OP_X, OP_Z, OP_SDG, OP_TDG = range(9)

BASE_SEED = 1606074130


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def clifford_word(rng: np.random.Generator, n: int, length: int = 200) -> np.ndarray:
    """A uniform word over {H_q, S_q, CNOT_qr} (CNOT only when n >= 2)."""
    rows = []
    kinds = 3 if n >= 2 else 2
    for _ in range(length):
        kind = int(rng.integers(kinds))
        if kind == 0:
            rows.append((OP_H, int(rng.integers(n)), 0))
        elif kind == 1:
            rows.append((OP_S, int(rng.integers(n)), 0))
        else:
            c = int(rng.integers(n))
            t = int(rng.integers(n - 1))
            t = t + 1 if t >= c else t
            rows.append((OP_CNOT, c, t))
    return np.asarray(rows, dtype=np.int32).reshape(-1, 3)


def permutation_targets() -> dict:
    """name -> (n, perm): classical reversible circuits as permutations of the
    computational basis, basis state c mapped to perm[c]; qubit q is bit q.

    * toffoli: bit 2 ^= bit 0 AND bit 1 (Table 1);
    * fredkin: bits 1 and 2 swapped when bit 0 is set (Table 1);
    * peres: (a, b, c) -> (a, a ^ b, c ^ a b), a Toffoli then a CNOT (Table 1);
    * quantum_or: bit 2 ^= bit 0 OR bit 1 (Table 1); since a OR b =
      1 ^ (NOT a AND NOT b), it is a Toffoli between X gates;
    * adder: the 1-bit full adder (Sec. 5.3) on (a, b, c, d) = bits 0..3,
      (a, b, c, d) -> (a, b, a ^ b ^ c, d ^ maj(a, b, c)).  With u = a ^ c
      and v = b ^ c, maj(a, b, c) = u v ^ c, so the adder is a Toffoli on
      (u, v -> d) between two CNOT circuits: the affine equivalence to the
      Toffoli that Sec. 5.3 reports.
    """
    def bit(c, q):
        return (c >> q) & 1

    tof = [c ^ (4 if (c & 3) == 3 else 0) for c in range(8)]
    fred = [(c & 1) | (bit(c, 2) << 1) | (bit(c, 1) << 2) if c & 1 else c for c in range(8)]
    adder = []
    for c in range(16):
        a, b, ci, d = bit(c, 0), bit(c, 1), bit(c, 2), bit(c, 3)
        maj = (a & b) | (a & ci) | (b & ci)
        adder.append(a | (b << 1) | ((a ^ b ^ ci) << 2) | ((d ^ maj) << 3))
    peres = [(c & 1) | ((bit(c, 0) ^ bit(c, 1)) << 1) | ((bit(c, 2) ^ (bit(c, 0) & bit(c, 1))) << 2)
             for c in range(8)]
    qor = [c ^ (4 if (c & 3) else 0) for c in range(8)]
    return {"toffoli": (3, tof), "fredkin": (3, fred), "peres": (3, peres), "quantum_or": (3, qor),
            "adder": (4, adder)}


def random_paulis(rng: np.random.Generator, n: int, t: int) -> np.ndarray:
    """t Pauli codes uniform over the non-identity codes 1 .. 4^n - 1."""
    return rng.integers(1, 4 ** n, size=t).astype(np.int32)


def seeded_target(n: int, t: int, seed: int, clifford_len: int = 200):
    """Gate list of C = C0 . R(P_t) ... R(P_1); returns (gates, paulis).

    ``paulis[j-1]`` is P_j.  The rotations act first in time order, then C0.
    """
    rng = _rng(seed)
    paulis = random_paulis(rng, n, t)
    word = clifford_word(rng, n, clifford_len)
    rot = np.asarray([(OP_RP, int(p), 0) for p in paulis], dtype=np.int32).reshape(-1, 3)
    return np.concatenate([rot, word], axis=0), paulis


def seeded_states(count: int, L: int, seed: int) -> np.ndarray:
    """count uniform L-bit walk states as uint64."""
    rng = _rng(seed)
    x = rng.integers(0, 2 ** 63, size=count, dtype=np.int64).astype(np.uint64)
    x = (x << np.uint64(1)) ^ rng.integers(0, 2, size=count, dtype=np.int64).astype(np.uint64)
    if L < 64:
        x &= np.uint64((1 << L) - 1)
    return x


# The five workloads (n, construction T-count, walks, state bits L,
# distinguished-point exponent d_theta (theta = 2^-d_theta), log2 table slots,
# k_max).  Seeds are BASE_SEED + config number.
CONFIGS = {
    1: dict(name="n2_t3_single", n=2, t=3, walks=4096, L=32, dtheta=6, table_log2=16, k_max=3),
    2: dict(name="n3_t5_single", n=3, t=5, walks=1 << 16, L=48, dtheta=10, table_log2=22, k_max=5),
    3: dict(name="n4_t7_single", n=4, t=7, walks=1 << 20, L=64, dtheta=12, table_log2=26, k_max=7),
}


def config_target(cfg: int):
    c = CONFIGS[cfg]
    return seeded_target(c["n"], c["t"], BASE_SEED + cfg)


def batched_targets(count: int = 256, seed: int = BASE_SEED + 4):
    """Targets with n ~ U{2,3,4} and construction T-count ~ U{3..7}."""
    rng = _rng(seed)
    out = []
    for j in range(count):
        n = int(rng.integers(2, 5))
        t = int(rng.integers(3, 8))
        gates, paulis = seeded_target(n, t, int(rng.integers(0, 2 ** 62)))
        out.append(dict(n=n, t=t, gates=gates, paulis=paulis))
    return out


def poisson_arrivals(count: int = 2000, rate: float = 50.0, seed: int = BASE_SEED + 5):
    """Arrival times (seconds) of a Poisson stream and its targets."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    times = np.cumsum(gaps)
    targets = batched_targets(count, seed=seed + 1)
    return times, targets
