"""Python binding of libqcs (include/qcs.h): GB300-native deterministic-walk
optimal T-count synthesis (Di Matteo & Mosca, "Parallelizing quantum circuit
synthesis", Sec. 2-4).

Argument marshalling only: every step of the search runs in the CUDA kernels
of ``csrc/``; device buffers are PyTorch CUDA tensors passed by pointer.  There
is no CPU fallback: importing the binding fails loudly when ``libqcs.so`` has
not been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

__all__ = ["lib", "Params", "Result", "Problem", "Batch", "BatchParams", "default_params",
           "default_batch_params", "verify_decomposition", "channel_from_unitary", "strerror", "QcsError",
           "plan_level", "launch_shapes", "shard_bin"]

OK = 0
ERR_ARG, ERR_NOT_UNITARY, ERR_NOMEM, ERR_CUDA, ERR_MISMATCH, ERR_OVERFLOW, ERR_BUSY, ERR_TIMEOUT, ERR_DEVICE = \
    -1, -2, -3, -4, -5, -6, -7, -8, -9
IDLE, SEARCHING, FOUND, BUDGET_EXHAUSTED, CANCELLED, ERROR = range(6)
MERGE_ROBIN_HOOD, MERGE_TRIVIAL, MERGE_SAME_SIDE, MERGE_CLAW, MERGE_FALSE_HASH, MERGE_NO_MERGE = range(6)
STATUS_NAMES = {IDLE: "idle", SEARCHING: "searching", FOUND: "found", BUDGET_EXHAUSTED: "budget_exhausted",
                CANCELLED: "cancelled", ERROR: "error"}


class Params(ctypes.Structure):
    _fields_ = [("state_bits", ctypes.c_int32), ("dp_bits", ctypes.c_int32), ("walks", ctypes.c_int32),
                ("table_log2", ctypes.c_int32), ("steps_per_launch", ctypes.c_int32),
                ("max_trail_factor", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("budget_factor", ctypes.c_int32), ("theta_policy", ctypes.c_int32),
                ("version_factor", ctypes.c_int32), ("stop_on_claw", ctypes.c_int32), ("theta_min_bits", ctypes.c_int32),
                ("exhaustive_log2", ctypes.c_int32), ("exhaustive_first", ctypes.c_int32),
                ("launch_shape", ctypes.c_int32), ("c_layout", ctypes.c_int32),
                ("rewalk_budget", ctypes.c_int32), ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("error", ctypes.c_int32), ("k", ctypes.c_int32),
                ("t_count", ctypes.c_int32), ("paulis", ctypes.c_uint32 * 16), ("sde", ctypes.c_int32),
                ("version", ctypes.c_uint32), ("steps", ctypes.c_int64), ("dps", ctypes.c_int64),
                ("merges", ctypes.c_int64), ("robin_hood", ctypes.c_int64), ("trivial", ctypes.c_int64),
                ("same_side", ctypes.c_int64), ("claws", ctypes.c_int64), ("false_hash", ctypes.c_int64),
                ("no_merge", ctypes.c_int64), ("abandoned", ctypes.c_int64), ("dropped", ctypes.c_int64),
                ("queue_overflow", ctypes.c_int64), ("launches", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("w_steps", ctypes.c_int64), ("rewalk_steps", ctypes.c_int64),
                ("certified_levels", ctypes.c_int64), ("cert_points", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64), ("rewalk_carried", ctypes.c_int64)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["paulis"] = [int(v) for v in self.paulis[: max(self.t_count, 0)]]
        d["status_name"] = STATUS_NAMES.get(self.status, "?")
        return d


class Plan(ctypes.Structure):
    _fields_ = [("dp_bits", ctypes.c_int32), ("walks", ctypes.c_uint32), ("steps", ctypes.c_uint32),
                ("launches_per_version", ctypes.c_uint64), ("min_launches", ctypes.c_uint64),
                ("points", ctypes.c_uint64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class BatchParams(ctypes.Structure):
    _fields_ = [("max_jobs", ctypes.c_int32), ("walks_per_job", ctypes.c_int32),
                ("steps_per_round", ctypes.c_int32), ("table_log2", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("rewalk_budget", ctypes.c_int32), ("launch_shape", ctypes.c_int32 * 4),
                ("cert_points_log2", ctypes.c_int32)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["launch_shape"] = list(self.launch_shape)
        return d


class QcsError(RuntimeError):
    def __init__(self, code, where=""):
        msg = strerror(code)
        if code == ERR_CUDA:
            msg += ": " + lib().qcs_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({code})" if where else f"{msg} ({code})")
        self.code = code


_lib = None
_vp, _sz = ctypes.c_void_p, ctypes.c_size_t
_i32, _u32, _u64, _i64 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64


def lib():
    """The loaded libqcs.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _build_mod.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libqcs.so is missing at {path}; build it with __graft_entry__.build() "
                               "(the CUDA library is required, there is no CPU fallback)")
        L = ctypes.CDLL(path)
        sig = {
            "qcs_default_params": (None, [ctypes.c_int, ctypes.POINTER(Params)]),
            "qcs_create_problem": (ctypes.c_int, [ctypes.c_int, _vp, _i32, ctypes.c_int, ctypes.POINTER(Params),
                                                  ctypes.POINTER(_vp)]),
            "qcs_create_problem_channel": (ctypes.c_int, [ctypes.c_int, _vp, _i32, ctypes.c_int,
                                                          ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
            "qcs_create_problem_circuit": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int,
                                                          ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
            "qcs_run_walks": (ctypes.c_int, [_vp, _u64, _vp]),
            "qcs_poll_collisions": (ctypes.c_int, [_vp, ctypes.POINTER(Result)]),
            "qcs_wait": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(Result)]),
            "qcs_cancel": (ctypes.c_int, [_vp]),
            "qcs_get_clifford": (ctypes.c_int, [_vp, _vp, _vp]),
            "qcs_verify_decomposition": (ctypes.c_int, [ctypes.c_int, _vp, _i32, _vp, ctypes.c_int]),
            "qcs_walk_step": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _u32, _vp, _vp, _vp, _sz, _vp]),
            "qcs_rewalk": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _u32, _vp, _vp, _vp, _vp, _sz, _vp,
                                          _vp, _vp]),
            "qcs_level_begin": (ctypes.c_int, [_vp, ctypes.c_int, _u32, ctypes.c_int, _vp]),
            "qcs_level_walk": (ctypes.c_int, [_vp, _u32, _vp]),
            "qcs_level_rewalk": (ctypes.c_int, [_vp, _vp]),
            "qcs_level_collect": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(Result)]),
            "qcs_certify_level": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_int)]),
            "qcs_level_begin_shard": (ctypes.c_int, [_vp, ctypes.c_int, _u32, ctypes.c_int, _u32, _u32, _vp]),
            "qcs_level_walk_out": (ctypes.c_int, [_vp, _u32, _vp, _u32, _vp, _vp]),
            "qcs_shard_bin": (ctypes.c_int, [_vp, _u32, _u32, _vp, _vp, _vp]),
            "qcs_level_insert": (ctypes.c_int, [_vp, _vp, _u32, _vp]),
            "qcs_level_merges": (ctypes.c_int, [_vp, _vp, _u32, ctypes.POINTER(_u32), _vp]),
            "qcs_plan_level": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params), ctypes.POINTER(Plan)]),
            "qcs_level_walk_static": (ctypes.c_int, [_vp, ctypes.c_int, _u32, ctypes.c_int, ctypes.c_int, _vp, _u32,
                                                     _u32, _vp, _u32, _vp, _vp]),
            "qcs_batch_default_params": (None, [ctypes.POINTER(BatchParams)]),
            "qcs_launch_shapes": (ctypes.c_int, [ctypes.c_int, _vp, _vp, ctypes.c_int]),
            "qcs_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchParams), _vp, ctypes.POINTER(_vp)]),
            "qcs_batch_job_bytes": (_u64, [_vp, _vp]),
            "qcs_batch_add": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_int)]),
            "qcs_batch_remove": (ctypes.c_int, [_vp, ctypes.c_int]),
            "qcs_batch_round": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
            "qcs_batch_poll": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(Result)]),
            "qcs_batch_destroy": (None, [_vp]),
            "qcs_problem_sde": (ctypes.c_int, [_vp]),
            "qcs_level_points": (_u64, [_vp, ctypes.c_int]),
            "qcs_get_channel": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(_i32)]),
            "qcs_channel_from_unitary": (ctypes.c_int, [ctypes.c_int, _vp, _i32, _vp, _vp, ctypes.POINTER(_i32)]),
            "qcs_destroy_problem": (None, [_vp]),
            "qcs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "qcs_last_cuda_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().qcs_strerror(int(code)).decode()


def _check(rc, where):
    if rc != OK:
        raise QcsError(rc, where)


def default_params(n: int, **overrides) -> Params:
    p = Params()
    lib().qcs_default_params(int(n), ctypes.byref(p))
    names = {name for name, _ in Params._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError(f"unknown search parameter {k!r}")
        setattr(p, k, v)
    return p


def launch_shapes(n: int) -> list[dict]:
    """qcs_launch_shapes: the walk kernel's launch shapes for n qubits, as
    [{"shape": i, "warps": .., "min_blocks": ..}] (shape 0 is the default)."""
    warps = np.zeros(8, np.int32)
    minb = np.zeros(8, np.int32)
    cnt = lib().qcs_launch_shapes(int(n), warps.ctypes.data_as(_vp), minb.ctypes.data_as(_vp), 8)
    if cnt < 0:
        _check(cnt, "qcs_launch_shapes")
    return [{"shape": i, "warps": int(warps[i]), "min_blocks": int(minb[i])} for i in range(cnt)]


def plan_level(n: int, k: int, params: Params) -> dict:
    """qcs_plan_level: how the search walks level k (host arithmetic only)."""
    out = Plan()
    _check(lib().qcs_plan_level(int(n), int(k), ctypes.byref(params), ctypes.byref(out)), "qcs_plan_level")
    return out.as_dict()


def _ptr(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _device_tensors(**tensors):
    """Every tensor whose pointer and size go to the library: contiguous, on
    the GPU, int64 (point pairs) or int32 (counts)."""
    import torch

    for name, t in tensors.items():
        if t.dtype not in (torch.int64, torch.int32) or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous int64/int32 CUDA tensor")


def shard_bin(points, count, n_owners, out, owner_counts, stream=None):
    """qcs_shard_bin: group `count` points (int64 CUDA tensor, 2 per point) by
    owner rank into `out`; owner_counts (int32 CUDA tensor, 2 n_owners) gets
    the group sizes in its first n_owners entries."""
    _device_tensors(points=points, out=out, owner_counts=owner_counts)
    if owner_counts.numel() < 2 * n_owners or out.numel() < 2 * count or points.numel() < 2 * count:
        raise ValueError("buffers too small for the points and owners")
    _check(lib().qcs_shard_bin(_ptr(points), int(count), int(n_owners), _ptr(out), _ptr(owner_counts),
                               _stream(stream)), "qcs_shard_bin")


def _stream(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class Problem:
    """One target; owns its device memory (freed by close())."""

    def __init__(self, handle, n, k_max):
        self._h = handle
        self.n, self.k_max = n, k_max

    # ---- construction -------------------------------------------------
    @classmethod
    def from_circuit(cls, n, gates, k_max, params: Params | None = None):
        g = np.ascontiguousarray(np.asarray(gates, np.int32).reshape(-1, 3))
        h = _vp()
        rc = lib().qcs_create_problem_circuit(int(n), g.ctypes.data_as(_vp), len(g), int(k_max),
                                              ctypes.byref(params) if params is not None else None, ctypes.byref(h))
        _check(rc, "qcs_create_problem_circuit")
        return cls(h, n, k_max)

    @classmethod
    def from_unitary(cls, n, target, exp, k_max, params: Params | None = None):
        u = np.ascontiguousarray(np.asarray(target, np.int64))
        h = _vp()
        rc = lib().qcs_create_problem(int(n), u.ctypes.data_as(_vp), int(exp), int(k_max),
                                      ctypes.byref(params) if params is not None else None, ctypes.byref(h))
        _check(rc, "qcs_create_problem")
        return cls(h, n, k_max)

    @classmethod
    def from_channel(cls, n, a, b, exp, k_max, params: Params | None = None):
        ab = np.ascontiguousarray(np.stack([np.asarray(a, np.int64), np.asarray(b, np.int64)], axis=-1))
        h = _vp()
        rc = lib().qcs_create_problem_channel(int(n), ab.ctypes.data_as(_vp), int(exp), int(k_max),
                                              ctypes.byref(params) if params is not None else None, ctypes.byref(h))
        _check(rc, "qcs_create_problem_channel")
        return cls(h, n, k_max)

    # ---- facts -----------------------------------------------------------
    @property
    def sde(self) -> int:
        return int(lib().qcs_problem_sde(self._h))

    def level_points(self, k: int) -> int:
        return int(lib().qcs_level_points(self._h, int(k)))

    def channel(self):
        D = 4 ** self.n
        a = np.zeros((D, D), np.int64)
        b = np.zeros((D, D), np.int64)
        e = _i32(0)
        _check(lib().qcs_get_channel(self._h, a.ctypes.data_as(_vp), b.ctypes.data_as(_vp), ctypes.byref(e)),
               "qcs_get_channel")
        return a, b, int(e.value)

    # ---- device entry points --------------------------------------------
    def walk_step(self, k, chunk, version, states, out, is_dp=None, stream=None):
        """out = f(states) on the device; tensors are int64 (bit patterns of uint64)."""
        rc = lib().qcs_walk_step(self._h, int(k), int(chunk), int(version), _ptr(states), _ptr(out),
                                 _ptr(is_dp), states.numel(), _stream(stream))
        _check(rc, "qcs_walk_step")

    def rewalk(self, k, chunk, version, start_a, len_a, start_b, len_b, cls, ab, stream=None):
        rc = lib().qcs_rewalk(self._h, int(k), int(chunk), int(version), _ptr(start_a), _ptr(len_a),
                              _ptr(start_b), _ptr(len_b), start_a.numel(), _ptr(cls), _ptr(ab), _stream(stream))
        _check(rc, "qcs_rewalk")

    # manual stepping of one level (Sec. 3): begin, walk, re-walk, collect
    def level_begin(self, k, version=0, dp_bits=0, stream=None):
        _check(lib().qcs_level_begin(self._h, int(k), int(version), int(dp_bits), _stream(stream)),
               "qcs_level_begin")

    def level_walk(self, steps, stream=None):
        _check(lib().qcs_level_walk(self._h, int(steps), _stream(stream)), "qcs_level_walk")

    def level_rewalk(self, stream=None):
        _check(lib().qcs_level_rewalk(self._h, _stream(stream)), "qcs_level_rewalk")

    def level_collect(self, stream=None) -> dict:
        r = Result()
        _check(lib().qcs_level_collect(self._h, _stream(stream), ctypes.byref(r)), "qcs_level_collect")
        return r.as_dict()

    # one level sharded across ranks (Sec. 4.2 collectors; see shard.py)
    def level_begin_shard(self, k, version, dp_bits, walk_base, total_walks, stream=None):
        _check(lib().qcs_level_begin_shard(self._h, int(k), int(version), int(dp_bits), int(walk_base),
                                           int(total_walks), _stream(stream)), "qcs_level_begin_shard")

    def level_walk_out(self, steps, outbox, count, stream=None):
        """Walk `steps` steps; distinguished points go to outbox (int64 CUDA
        tensor, 2 per point) and count (int32 CUDA tensor) counts them."""
        _device_tensors(outbox=outbox, count=count)
        _check(lib().qcs_level_walk_out(self._h, int(steps), _ptr(outbox), outbox.numel() // 2, _ptr(count),
                                        _stream(stream)), "qcs_level_walk_out")

    def level_insert(self, points, count=None, stream=None):
        """Store received points (int64 CUDA tensor, 2 per point) in the level's table."""
        _device_tensors(points=points)
        n = points.numel() // 2 if count is None else int(count)
        _check(lib().qcs_level_insert(self._h, _ptr(points) if n else None, n, _stream(stream)),
               "qcs_level_insert")

    def level_merges(self, cap=1 << 20, stream=None) -> np.ndarray:
        """The merges queued by the last walk or insert, as an (m, 3) uint64
        array of {trail ref a, trail ref b, distinguished point}."""
        out = np.zeros((cap, 3), np.uint64)
        n = _u32(0)
        _check(lib().qcs_level_merges(self._h, out.ctypes.data_as(_vp), int(cap), ctypes.byref(n),
                                      _stream(stream)), "qcs_level_merges")
        return out[: n.value]

    def certify_level(self, k, stream=None) -> bool:
        """qcs_certify_level: exhaustive pass over level k; True iff a
        decomposition with k rotations exists (it is then recorded)."""
        has = ctypes.c_int(0)
        _check(lib().qcs_certify_level(self._h, int(k), _stream(stream), ctypes.byref(has)), "qcs_certify_level")
        return bool(has.value)

    def level_walk_static(self, k, version, dp_bits, begin, walk_states, steps, merges, counts, stream=None):
        """qcs_level_walk_static: the level walk without any device allocation.
        walk_states: int64 tensor of 4 * n_walks entries; merges: int64 tensor
        of 3 * cap entries; counts: int64 tensor of 8 entries (the counters of
        include/qcs.h; the high 32 bits of counts[7] are nonzero only if a
        bounded wait of the n = 4 tensor-core walk ran out, and then nothing
        the call wrote is valid).  All three must be contiguous int64 CUDA
        tensors: their sizes become the kernel's bounds."""
        import torch

        for name, t in (("walk_states", walk_states), ("merges", merges), ("counts", counts)):
            if t.dtype != torch.int64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous int64 CUDA tensor")
        if walk_states.numel() % 4 or merges.numel() % 3 or counts.numel() < 8:
            raise ValueError("walk_states needs 4 int64 per walk, merges 3 per triple, counts at least 8")
        n_walks = walk_states.numel() // 4
        rc = lib().qcs_level_walk_static(self._h, int(k), int(version), int(dp_bits), int(begin),
                                         _ptr(walk_states), n_walks, int(steps), _ptr(merges),
                                         merges.numel() // 3, _ptr(counts), _stream(stream))
        _check(rc, "qcs_level_walk_static")

    def run_walks(self, step_budget: int = 0, stream=None):
        _check(lib().qcs_run_walks(self._h, int(step_budget), _stream(stream)), "qcs_run_walks")

    def poll(self) -> dict:
        r = Result()
        _check(lib().qcs_poll_collisions(self._h, ctypes.byref(r)), "qcs_poll_collisions")
        return r.as_dict()

    def wait(self, timeout_ms: int = -1) -> dict:
        r = Result()
        rc = lib().qcs_wait(self._h, int(timeout_ms), ctypes.byref(r))
        if rc not in (OK, ERR_TIMEOUT):
            _check(rc, "qcs_wait")
        d = r.as_dict()
        d["timed_out"] = rc == ERR_TIMEOUT
        return d

    def cancel(self):
        _check(lib().qcs_cancel(self._h), "qcs_cancel")

    def clifford(self):
        D = 4 ** self.n
        perm = np.zeros(D, np.int32)
        sign = np.zeros(D, np.int8)
        _check(lib().qcs_get_clifford(self._h, perm.ctypes.data_as(_vp), sign.ctypes.data_as(_vp)),
               "qcs_get_clifford")
        return perm, sign

    def close(self):
        if self._h:
            lib().qcs_destroy_problem(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_batch_params(**overrides) -> BatchParams:
    """Batch parameters; launch_shape may be given as a list of 4 shapes
    (n = 1..4) or as a dict {n: shape}."""
    p = BatchParams()
    lib().qcs_batch_default_params(ctypes.byref(p))
    names = {name for name, _ in BatchParams._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError(f"unknown batch parameter {k!r}")
        if k == "launch_shape":
            items = v.items() if isinstance(v, dict) else enumerate(v, start=1)
            for n, sh in items:
                p.launch_shape[int(n) - 1] = int(sh)
            continue
        setattr(p, k, v)
    return p


class Batch:
    """Many problems searched together (qcs_batch_*): one round advances every
    active job; jobs join and leave between rounds."""

    def __init__(self, params: BatchParams | None = None, stream=None):
        self._h = _vp()
        s = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        _check(lib().qcs_batch_create(ctypes.byref(params) if params is not None else None, s,
                                      ctypes.byref(self._h)), "qcs_batch_create")
        self._problems = {}

    def job_bytes(self, prob: "Problem") -> int:
        return int(lib().qcs_batch_job_bytes(self._h, prob._h))

    def add(self, prob: "Problem") -> int:
        j = ctypes.c_int(-1)
        _check(lib().qcs_batch_add(self._h, prob._h, ctypes.byref(j)), "qcs_batch_add")
        self._problems[j.value] = prob
        return j.value

    def remove(self, job: int):
        _check(lib().qcs_batch_remove(self._h, int(job)), "qcs_batch_remove")
        self._problems.pop(job, None)

    def round(self) -> int:
        n = ctypes.c_int(0)
        _check(lib().qcs_batch_round(self._h, ctypes.byref(n)), "qcs_batch_round")
        return n.value

    def poll(self, job: int) -> dict:
        r = Result()
        _check(lib().qcs_batch_poll(self._h, int(job), ctypes.byref(r)), "qcs_batch_poll")
        return r.as_dict()

    def close(self):
        if self._h:
            lib().qcs_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def peak_lib():
    """libqcs_peak.so: integer-ALU throughput microbenchmarks (measurement only)."""
    path = _build_mod.PEAK_LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libqcs_peak.so is missing at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name in ("qcs_peak_imad", "qcs_peak_iadd", "qcs_peak_idp4a", "qcs_peak_hmma", "qcs_peak_imma"):
        f = getattr(L, name)
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    return L


def measure_int_peak(kind: str = "imad", blocks_per_sm: int = 8, iters: int = 4096) -> tuple[float, float]:
    """(ops per second, kernel ms) of the IMAD, IADD3 or dp4a microbenchmark,
    or (multiply-adds per second, ms) of the hmma / imma tensor-core ones."""
    ops, ms = ctypes.c_double(0), ctypes.c_double(0)
    rc = getattr(peak_lib(), f"qcs_peak_{kind}")(blocks_per_sm, iters, ctypes.byref(ops), ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError(f"qcs_peak_{kind} failed with CUDA error {-rc}")
    return ops.value, ms.value


def channel_from_unitary(n, target, exp):
    """qcs_channel_from_unitary: the exact channel representation of a target
    unitary, reduced: (a, b, sde) with entries (a + b sqrt2) / sqrt2^sde (no
    GPU needed)."""
    u = np.ascontiguousarray(np.asarray(target, np.int64))
    D = 4 ** int(n)
    a = np.zeros((D, D), np.int64)
    b = np.zeros((D, D), np.int64)
    e = _i32(0)
    _check(lib().qcs_channel_from_unitary(int(n), u.ctypes.data_as(_vp), int(exp), a.ctypes.data_as(_vp),
                                          b.ctypes.data_as(_vp), ctypes.byref(e)), "qcs_channel_from_unitary")
    return a, b, int(e.value)


def verify_decomposition(n, target, exp, paulis) -> bool:
    """Exact host check of C = e^{i phi} R(P_t)..R(P_1) D (no GPU needed)."""
    u = np.ascontiguousarray(np.asarray(target, np.int64))
    p = np.ascontiguousarray(np.asarray(paulis, np.uint32))
    rc = lib().qcs_verify_decomposition(int(n), u.ctypes.data_as(_vp), int(exp),
                                        p.ctypes.data_as(_vp) if len(p) else None, len(p))
    if rc == ERR_MISMATCH:
        return False
    _check(rc, "qcs_verify_decomposition")
    return True
