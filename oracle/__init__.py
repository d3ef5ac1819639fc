"""Python access to the CPU oracle (``qcs_oracle.c``).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` leg may import this module.  The product path
(``paper_1606_07413_gb300``) never imports it and fails loudly when its CUDA
library is missing.

The oracle is plain single-threaded C compiled with gcc; this wrapper only
marshals numpy arrays.  Matrices over Z[1/sqrt2] travel as ``(a, b, E)``: two
``(4^n, 4^n)`` int64 arrays and the shared sqrt2 exponent, value
``(a + b sqrt2) / sqrt2^E``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

# merge classes (Sec. 3, Fig. 2)
ROBIN_HOOD, TRIVIAL, SAME_SIDE, CLAW, FALSE_HASH, NO_MERGE = range(6)

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_intp = ctypes.POINTER(ctypes.c_int)
_ci, _cu32, _cu64, _ci64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64


def _declare(L):
    sig = {
        "or_pauli_phase": (_ci, [_ci, _ci, _ci]),
        "or_unitary_from_circuit": (_ci, [_ci, _i32p, _ci, _i64p, _intp]),
        "or_channel_from_unitary": (_ci, [_ci, _i64p, _ci, _i64p, _i64p, _intp]),
        "or_channel_from_circuit": (_ci, [_ci, _i32p, _ci, _i64p, _i64p, _intp]),
        "or_pm_mul": (_ci, [_ci, _i64p, _i64p, _ci, _i64p, _i64p, _ci, _i64p, _i64p, _intp]),
        "or_pm_reduce": (_ci, [_ci, _i64p, _i64p, _intp]),
        "or_rhat_cols": (_ci, [_ci, _ci, _ci, _i64p, _i64p]),
        "or_rhat_trace": (_ci, [_ci, _ci, _i64p, _i64p, _intp]),
        "or_half_product": (_ci, [_ci, _i64p, _i64p, _ci, _ci, _ci, _ci, _i32p, _i64p, _i64p, _intp]),
        "or_fp_weights": (None, [_ci, _u32p, _u32p]),
        "or_matrix_hash": (_cu64, [_ci, _i64p, _i64p, _ci, _ci, _ci, _cu32, _ci]),
        "or_decode": (_ci, [_ci, _ci, _ci, _cu64, _i32p]),
        "or_field_bits": (_ci, [_ci, _ci, _ci]),
        "or_walk_step": (_ci, [_ci, _i64p, _i64p, _ci, _ci, _ci, _cu32, _ci, _u64p, _u64p, _ci]),
        "or_canon": (_ci, [_ci, _i64p, _i64p, _ci, _i64p, _intp]),
        "or_is_clifford": (_ci, [_ci, _i64p, _i64p, _ci]),
        "or_sde": (_ci, [_ci, _i64p, _i64p, _ci]),
        "or_verify": (_ci, [_ci, _i64p, _i64p, _ci, _i32p, _ci]),
        "or_brute_tcount": (_ci, [_ci, _i64p, _i64p, _ci, _ci, _i32p]),
        "or_mitm_level": (_ci, [_ci, _i64p, _i64p, _ci, _ci, _i32p]),
        "or_rewalk": (_ci, [_ci, _i64p, _i64p, _ci, _ci, _ci, _cu32, _ci, _cu64, _ci64, _cu64, _ci64,
                            _u64p, _i32p]),
        "or_classify": (_ci, [_ci, _i64p, _i64p, _ci, _ci, _ci, _ci, _cu64, _cu64, _i32p]),
        "or_vow_search": (_ci, [_ci, _i64p, _i64p, _ci, _ci, _i64p, _i32p, _i64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def dim(n: int) -> int:
    return 1 << (2 * n)


class Chan:
    """An exact matrix over Z[1/sqrt2]: value (a + b sqrt2) / sqrt2^E."""

    __slots__ = ("n", "a", "b", "E")

    def __init__(self, n, a, b, E):
        self.n, self.a, self.b, self.E = n, np.ascontiguousarray(a, np.int64), np.ascontiguousarray(b, np.int64), int(E)

    def reduced(self) -> "Chan":
        a, b = self.a.copy(), self.b.copy()
        E = ctypes.c_int(self.E)
        lib().or_pm_reduce(dim(self.n), a, b, ctypes.byref(E))
        return Chan(self.n, a, b, E.value)

    def __matmul__(self, other: "Chan") -> "Chan":
        D = dim(self.n)
        a = np.zeros((D, D), np.int64)
        b = np.zeros((D, D), np.int64)
        E = ctypes.c_int(0)
        lib().or_pm_mul(D, self.a, self.b, self.E, other.a, other.b, other.E, a, b, ctypes.byref(E))
        return Chan(self.n, a, b, E.value)

    def equals(self, other: "Chan") -> bool:
        x, y = self.reduced(), other.reduced()
        return x.E == y.E and np.array_equal(x.a, y.a) and np.array_equal(x.b, y.b)

    def values(self) -> np.ndarray:
        return (self.a + self.b * np.sqrt(2.0)) / np.sqrt(2.0) ** self.E


def identity(n: int) -> Chan:
    D = dim(n)
    return Chan(n, np.eye(D, dtype=np.int64), np.zeros((D, D), np.int64), 0)


def pauli_phase(n: int, p: int, q: int) -> int:
    return int(lib().or_pauli_phase(n, p, q))


def unitary_from_circuit(n: int, gates) -> tuple[np.ndarray, int]:
    g = np.ascontiguousarray(np.asarray(gates, np.int32).reshape(-1, 3))
    d = 1 << n
    u = np.zeros((d, d, 4), np.int64)
    e = ctypes.c_int(0)
    if lib().or_unitary_from_circuit(n, g, len(g), u, ctypes.byref(e)) != 0:
        raise ValueError("bad n")
    return u, e.value


def channel_from_unitary(n: int, u: np.ndarray, e: int) -> Chan:
    D = dim(n)
    a = np.zeros((D, D), np.int64)
    b = np.zeros((D, D), np.int64)
    E = ctypes.c_int(0)
    lib().or_channel_from_unitary(n, np.ascontiguousarray(u, np.int64), int(e), a, b, ctypes.byref(E))
    return Chan(n, a, b, E.value)


def channel_from_circuit(n: int, gates) -> Chan:
    g = np.ascontiguousarray(np.asarray(gates, np.int32).reshape(-1, 3))
    D = dim(n)
    a = np.zeros((D, D), np.int64)
    b = np.zeros((D, D), np.int64)
    E = ctypes.c_int(0)
    lib().or_channel_from_circuit(n, g, len(g), a, b, ctypes.byref(E))
    return Chan(n, a, b, E.value)


def rhat(n: int, p: int, transpose: bool = False) -> Chan:
    """R^(P) from its columns (sparse rule), at exponent 1."""
    D = dim(n)
    a = np.zeros((D, D), np.int64)
    b = np.zeros((D, D), np.int64)
    lib().or_rhat_cols(n, p, int(transpose), a, b)
    return Chan(n, a, b, 1)


def rhat_trace(n: int, p: int) -> Chan:
    """R^(P) from the trace definition applied to the unitary R(P)."""
    D = dim(n)
    a = np.zeros((D, D), np.int64)
    b = np.zeros((D, D), np.int64)
    E = ctypes.c_int(0)
    lib().or_rhat_trace(n, p, a, b, ctypes.byref(E))
    return Chan(n, a, b, E.value)


def half_product(C: Chan, k: int, chunk: int, side: int, q) -> Chan:
    D = dim(C.n)
    a = np.zeros((D, D), np.int64)
    b = np.zeros((D, D), np.int64)
    K = ctypes.c_int(0)
    qa = np.zeros(16, np.int32)
    qa[: len(q)] = q
    lib().or_half_product(C.n, C.a, C.b, C.E, k, chunk, side, qa, a, b, ctypes.byref(K))
    return Chan(C.n, a, b, K.value)


def fp_weights(n: int) -> tuple[np.ndarray, np.ndarray]:
    D = dim(n)
    ua = np.zeros(D, np.uint32)
    ub = np.zeros(D, np.uint32)
    lib().or_fp_weights(n, ua, ub)
    return ua, ub


def matrix_hash(M: Chan, k: int, chunk: int, version: int, L: int) -> int:
    return int(lib().or_matrix_hash(M.n, M.a, M.b, M.E, k, chunk, version, L))


def decode(n: int, k: int, L: int, x: int) -> tuple[int, list[int]]:
    q = np.zeros(16, np.int32)
    side = lib().or_decode(n, k, L, int(x), q)
    return int(side), [int(v) for v in q[: k // 2]]


def field_bits(n: int, k: int, L: int) -> int:
    return int(lib().or_field_bits(n, k, L))


def encode(n: int, k: int, L: int, side: int, q) -> int:
    """A state that decodes to (side, q): the smallest field value per rotation."""
    xi = 4 ** n - 1
    ell = field_bits(n, k, L)
    x = side & 1
    for j, qj in enumerate(q):
        v = -(-(qj - 1) * (1 << ell) // xi)  # ceil((q_j - 1) 2^l / xi)
        x |= v << (1 + ell * j)
    return x


def walk_step(C: Chan, k: int, chunk: int, version: int, L: int, states) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(states, np.uint64))
    y = np.zeros_like(x)
    lib().or_walk_step(C.n, C.a, C.b, C.E, k, chunk, version, L, x, y, len(x))
    return y


def is_dp(y: np.ndarray, L: int, dtheta: int) -> np.ndarray:
    if dtheta == 0:
        return np.ones(len(y), bool)
    return (np.asarray(y, np.uint64) >> np.uint64(L - dtheta)) == 0


def canon(M: Chan) -> tuple[np.ndarray, int]:
    d = dim(M.n) - 1
    out = np.zeros((d, 2 * d), np.int64)
    sde = ctypes.c_int(0)
    lib().or_canon(M.n, M.a, M.b, M.E, out, ctypes.byref(sde))
    return out, sde.value


def same_coset(A: Chan, B: Chan) -> bool:
    ca, ea = canon(A)
    cb, eb = canon(B)
    return ea == eb and np.array_equal(ca, cb)


def is_clifford(M: Chan) -> bool:
    return bool(lib().or_is_clifford(M.n, M.a, M.b, M.E))


def sde(M: Chan) -> int:
    return int(lib().or_sde(M.n, M.a, M.b, M.E))


def verify(C: Chan, paulis) -> bool:
    p = np.ascontiguousarray(np.asarray(paulis, np.int32))
    if len(p) == 0:
        p = np.zeros(1, np.int32)
        return bool(lib().or_verify(C.n, C.a, C.b, C.E, p, 0))
    return bool(lib().or_verify(C.n, C.a, C.b, C.E, p, len(paulis)))


def brute_tcount(C: Chan, tmax: int):
    p = np.zeros(max(tmax, 1), np.int32)
    t = lib().or_brute_tcount(C.n, C.a, C.b, C.E, tmax, p)
    return (None, None) if t < 0 else (t, [int(v) for v in p[:t]])


def mitm_level(C: Chan, k: int):
    p = np.zeros(max(k, 1), np.int32)
    ok = lib().or_mitm_level(C.n, C.a, C.b, C.E, k, p)
    return [int(v) for v in p[:k]] if ok else None


def mitm_tcount(C: Chan, kmax: int):
    """Exact optimal T-count by exhaustive meet-in-the-middle, levels sde..kmax."""
    for k in range(sde(C), kmax + 1):
        p = mitm_level(C, k)
        if p is not None:
            return k, p
    return None, None


def rewalk(C: Chan, k, chunk, version, L, x0a, la, x0b, lb):
    ab = np.zeros(2, np.uint64)
    p = np.zeros(16, np.int32)
    cls = lib().or_rewalk(C.n, C.a, C.b, C.E, k, chunk, version, L, int(x0a), int(la), int(x0b), int(lb), ab, p)
    return int(cls), int(ab[0]), int(ab[1]), [int(v) for v in p[:k]]


def classify(C: Chan, k, chunk, L, a, b):
    p = np.zeros(16, np.int32)
    cls = lib().or_classify(C.n, C.a, C.b, C.E, k, chunk, L, int(a), int(b), p)
    return int(cls), [int(v) for v in p[:k]]


def vow_search(C: Chan, k_max: int, dtheta: int, L: int, max_len: int, per_version: int,
               per_level: int, table_log2: int, seed: int):
    """Serial walk search with the T-count ladder; returns (t, paulis, stats)."""
    params = np.asarray([dtheta, L, max_len, per_version, per_level, table_log2, seed], np.int64)
    p = np.zeros(16, np.int32)
    stats = np.zeros(11, np.int64)
    t = lib().or_vow_search(C.n, C.a, C.b, C.E, k_max, params, p, stats)
    keys = ["steps", "dps", "merges", "robin_hood", "trivial", "same_side", "claws",
            "false_hash", "no_merge", "dropped", "level"]
    st = {k_: int(v) for k_, v in zip(keys, stats)}
    return (None if t < 0 else int(t)), [int(v) for v in p[: max(t, 0)]], st
