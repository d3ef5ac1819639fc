/*
 * qcs.h -- C ABI of libqcs, a GB300 (sm_103a) implementation of the
 * deterministic-walk optimal T-count search of Di Matteo & Mosca,
 * "Parallelizing quantum circuit synthesis".
 *
 * The library finds, for a target unitary C over Clifford+T, the smallest t
 * and Paulis P_1..P_t with  C = e^{i phi} R(P_t) ... R(P_1) D,  D Clifford
 * (Sec. 4.1, Eq. tcount_synthesis), by a parallel claw search between the two
 * halves of Eq. mitm (Sec. 3) on one GPU.
 *
 * Conventions shared by every entry point:
 *  - Pauli code j in [0, 4^n): x = j >> n, z = j & (2^n - 1), qubit q is bit q;
 *    P(j) = i^{|x&z|} X^x Z^z.  Basis state c has qubit q in bit q of c.
 *  - Exact targets are 2^n x 2^n row-major matrices of Z[omega] numbers, four
 *    int64 per entry (c0 + c1 w + c2 w^2 + c3 w^3, w = e^{i pi/4}), all divided
 *    by sqrt2^exp.
 *  - Channel matrices (Sec. 4.1, U^_ij = Tr(P_i U P_j U^dag)/2^n) are 4^n x 4^n
 *    row-major, two int64 per entry (a, b) meaning (a + b sqrt2)/sqrt2^exp.
 *  - Walk states are L-bit strings in uint64 (L = params.state_bits).  A state
 *    x names side x & 1 (0: V = R(q_h)..R(q_1), 1: W = R(q_1)^T..R(q_h)^T
 *    [R(c)^T] C^ in channel form; Sec. 3 chunks c for odd k) and rotations
 *    q_1..q_h: rotation j (0-based) reads the l-bit field v at bit 1 + l j,
 *    l = min(16, (L - 1) / h), and q_{j+1} = floor(v xi / 2^l) + 1 with
 *    xi = 4^n - 1 (Sec. 2 mapping mu: one code per rotation, concatenated).
 *  - The next state (Sec. 2 mappings nu and h) hashes the product's Clifford
 *    coset: per column Q >= 1 the 16-bit fingerprint L_Q = sum_i Ua_i a_iQ +
 *    Ub_i b_iQ mod 2^16 (weights: SplitMix64 outputs, row 0 weight 0), folded
 *    to phi_Q = min(L_Q, -L_Q); the multiset of the phi_Q is hashed as the
 *    sum mod 2^64 of the SplitMix64 finaliser of base ^ phi_Q, where the base
 *    mixes the function version, n, k, the chunk and the common exponent K,
 *    and the sum's finaliser is cut to L bits.
 *
 * Ownership: every pointer argument stays owned by the caller; the library
 * copies what it keeps.  The library owns every device allocation it makes and
 * frees it in qcs_destroy_problem.  Errors are returned as status codes, never
 * thrown across the ABI.  A problem handle may be used by one host thread at a
 * time (qcs_poll_collisions and qcs_cancel may be called concurrently with a
 * running search).
 */
#ifndef QCS_H
#define QCS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QCS_API __attribute__((visibility("default")))
#else
#define QCS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define QCS_OK 0
#define QCS_ERR_ARG (-1)         /* argument out of range or inconsistent */
#define QCS_ERR_NOT_UNITARY (-2) /* target is not an exact unitary / channel */
#define QCS_ERR_NOMEM (-3)       /* host or device allocation failed */
#define QCS_ERR_CUDA (-4)        /* a CUDA call failed (see qcs_last_cuda_error) */
#define QCS_ERR_MISMATCH (-5)    /* decomposition does not reproduce the target */
#define QCS_ERR_OVERFLOW (-6)    /* exact arithmetic would overflow int64 */
#define QCS_ERR_BUSY (-7)        /* a search is already running on this problem */
#define QCS_ERR_TIMEOUT (-8)     /* qcs_wait ran out of time */
#define QCS_ERR_DEVICE (-9)      /* a device-side bounded wait gave up */

/* search status reported by qcs_poll_collisions */
#define QCS_IDLE 0
#define QCS_SEARCHING 1
#define QCS_FOUND 2
#define QCS_BUDGET_EXHAUSTED 3
#define QCS_CANCELLED 4
#define QCS_ERROR 5

/* gate ops of the circuit input format: rows (op, a, b) in time order */
#define QCS_GATE_H 0    /* H on qubit a */
#define QCS_GATE_S 1    /* S = diag(1, i) on qubit a */
#define QCS_GATE_CNOT 2 /* control a, target b */
#define QCS_GATE_T 3    /* T = diag(1, w) on qubit a */
#define QCS_GATE_RP 4   /* R(P_a) of Sec. 4.1, a = Pauli code in [1, 4^n) */
#define QCS_GATE_X 5
#define QCS_GATE_Z 6
#define QCS_GATE_SDG 7
#define QCS_GATE_TDG 8

/* merge classes of a re-walked collision (Sec. 3, Fig. 2) */
#define QCS_MERGE_ROBIN_HOOD 0 /* one start lies on the other trail */
#define QCS_MERGE_TRIVIAL 1    /* both states decode to the same point */
#define QCS_MERGE_SAME_SIDE 2  /* both sides V (or both W): no solution */
#define QCS_MERGE_CLAW 3       /* V meets W: a decomposition */
#define QCS_MERGE_FALSE_HASH 4 /* V meets W by hash only, not exactly */
#define QCS_MERGE_NO_MERGE 5   /* trails did not meet (inconsistent input) */

typedef struct qcs_params {
    int32_t state_bits;       /* L, 32..64 */
    int32_t dp_bits;          /* d_theta, theta = 2^-d_theta (Sec. 3), 1 .. L-1 */
    int32_t walks;            /* concurrent walks (one lane group each: min(32, 4^n) lanes) */
    int32_t table_log2;       /* distinguished-point table holds 2^table_log2 slots (16 B each) */
    int32_t steps_per_launch; /* walk steps each walk advances per kernel launch */
    int32_t max_trail_factor; /* a trail is abandoned after max_trail_factor * 2^d_theta steps */
    int32_t queue_capacity;   /* collision pairs kept per launch */
    int32_t budget_factor;    /* a level gives up after budget_factor * (points at that level) steps */
    int32_t theta_policy;     /* 0: d_theta fixed; 1: theta from the level size N and the table size w
                                 (qcs_plan_level) */
    int32_t version_factor;   /* new function version every version_factor * points steps (0: never) */
    int32_t stop_on_claw;     /* 1: stop at the first verified claw; 0: keep walking to the step budget
                                 (the first decomposition is still reported) */
    int32_t theta_min_bits;   /* theta_policy 1 never raises theta above 2^-theta_min_bits (>= 1) */
    int32_t exhaustive_log2;  /* a level whose V and W points number at most 2^exhaustive_log2, and
                                 whose key table fits in half the free device memory, is settled
                                 exactly by qcs_certify_level when its walk budget ends without a
                                 claw (0: never; at most 40) */
    int32_t exhaustive_first; /* 1: qcs_run_walks settles such levels by qcs_certify_level alone,
                                 without walking them (0: walk first) */
    int32_t launch_shape;     /* launch shape of the level-walk kernel, 0 .. qcs_launch_shapes(n) - 1
                                 (default 3 at n = 4, else 0); the walks and results do not depend on
                                 it.  n = 4, shape 3: the W side's contraction on the tensor cores
                                 (f16 byte planes, exact f32 sums) in warps of its own, beside the
                                 warps that evaluate the stages, when C^ is held in int8 (c_layout
                                 0); otherwise, and in a batch, it runs shape 0 */
    int32_t c_layout;         /* device layout of C^ for the W side's contraction (n >= 3): 0 = signed
                                 byte quads when every entry fits in int8 (dp4a), else 32-bit words;
                                 1 = 32-bit words always (IMAD).  Results do not depend on it */
    int32_t rewalk_budget;    /* evaluations of f one re-walk of a merge (Sec. 3, Fig. 2) may take per
                                 launch; an unfinished re-walk is carried to the next launch of the same
                                 level and function version (up to queue_capacity of them; more are
                                 dropped and counted in queue_overflow).  0: no bound, every merge is
                                 re-walked to its end in its own launch */
    int32_t reserved;
    uint64_t seed;            /* seed of trail starting points */
} qcs_params;

typedef struct qcs_result {
    int32_t status;      /* QCS_IDLE .. QCS_ERROR */
    int32_t error;       /* status code when status == QCS_ERROR */
    int32_t k;           /* level (T-count candidate) being searched or found */
    int32_t t_count;     /* optimal T-count when FOUND, else -1 */
    uint32_t paulis[16]; /* P_1 .. P_t when FOUND */
    int32_t sde;         /* smallest denominator exponent of C^ (lower bound on t) */
    uint32_t version;    /* current function version */
    int64_t steps;       /* walk steps taken (all levels) */
    int64_t dps;         /* distinguished points reached */
    int64_t merges;      /* trail pairs re-walked */
    int64_t robin_hood, trivial, same_side, claws, false_hash, no_merge;
    int64_t abandoned;   /* trails cut at the maximum length */
    int64_t dropped;     /* distinguished points lost to a full table neighbourhood */
    int64_t queue_overflow;
    int64_t launches;    /* walk-kernel launches */
    double seconds;      /* wall time since qcs_run_walks */
    int64_t w_steps;     /* walk steps taken on the W side (the 4^n x 4^n contraction) */
    int64_t rewalk_steps; /* evaluations of f made by the re-walk (Fig. 2 trace-back) */
    int64_t certified_levels; /* levels proved claw-free by the exhaustive pass */
    int64_t cert_points;      /* points (V and W) evaluated by the exhaustive pass */
    int64_t h2d_bytes;        /* since the problem's creation (searches do not reset these two):
                                 bytes this problem copied host to device: the upload of C^, its
                                 weights and rotation tables at creation (and the shared stage tables
                                 when this creation uploaded them); device-side resets not counted */
    int64_t d2h_bytes;        /* bytes copied device to host for this problem: per launch the
                                 counters and queue heads, plus the claw candidates and exhaustive-pass
                                 matches actually queued (batch jobs: 0, the batch copies per round) */
    int64_t rewalk_carried;   /* re-walks carried into the next launch (params.rewalk_budget > 0):
                                 merges queued so far = the re-walk classes + this + queue_overflow */
} qcs_result;

typedef struct qcs_problem qcs_problem;

/* Launch shapes of the walk kernels for n qubits (the autotuner's space; not
 * a passage of the paper: how walks map onto the GPU).  Returns the number
 * of shapes (>= 1) and fills, for shape i < max_shapes, warps[i] (warps per
 * CTA of the level walk, each warp evaluating 32 / min(32, 4^n) walks; at
 * n = 4, shape 3 is the tensor-core walk: 12 warps evaluating two walks of
 * each of two sets, and 8 warps doing the contraction) and min_blocks[i] (the
 * resident CTAs per SM the kernel is compiled for, capping its registers at
 * 65536 / (32 warps[i] min_blocks[i])).  Either pointer may be NULL.
 * QCS_ERR_ARG if n is not in 1..4. */
QCS_API int qcs_launch_shapes(int n_qubits, int32_t *warps, int32_t *min_blocks, int max_shapes);

/* Fill *p with the defaults for n qubits (L = 32/48/64, d_theta = 6/10/12 ...). */
QCS_API void qcs_default_params(int n_qubits, qcs_params *p);

/* Create a search problem from an exact target unitary (see conventions).
 * Checks exact unitarity, forms C^ (Sec. 4.1) exactly and reduces it to its
 * smallest denominator exponent, then uploads it.  k_max in [0, 15] bounds the
 * T-count ladder.  p may be NULL for defaults.  Errors: QCS_ERR_ARG (n not in
 * 1..4, k_max out of range, bad params), QCS_ERR_NOT_UNITARY, QCS_ERR_OVERFLOW,
 * QCS_ERR_NOMEM, QCS_ERR_CUDA.  On success *out owns device memory. */
QCS_API int qcs_create_problem(int n_qubits, const int64_t *target, int32_t target_exp, int k_max,
                       const qcs_params *p, qcs_problem **out);

/* Same, from a 4^n x 4^n channel matrix given as (a, b) pairs over sqrt2^exp
 * (chan_ab[2*(i*4^n + j)] = a_ij, [.. + 1] = b_ij).  Checks exact
 * orthogonality and that row and column 0 are e_0; it does not check that the
 * matrix is the channel of a unitary. */
QCS_API int qcs_create_problem_channel(int n_qubits, const int64_t *chan_ab, int32_t exp, int k_max,
                               const qcs_params *p, qcs_problem **out);

/* Same, from a gate list of n_gates rows (op, a, b) in time order (QCS_GATE_*);
 * the target is the product of the gates' textbook matrices. */
QCS_API int qcs_create_problem_circuit(int n_qubits, const int32_t *gates, int n_gates, int k_max,
                               const qcs_params *p, qcs_problem **out);

/* Start the T-count ladder on the given CUDA stream (a cudaStream_t; NULL =
 * legacy default stream; a PyTorch stream handle is fine).  Sec. 4.1, Eq.
 * tcount_synthesis: the optimal T-count is the smallest t for which C =
 * R(P_t)..R(P_1) D has a solution, so levels t = sde(C^) .. k_max are
 * searched in increasing order (sde(C^) is a lower bound: every R^(P) adds
 * one power of sqrt2 to the denominator, and D^ is an integer matrix), and
 * the first level with a verified claw between the halves of Eq. mitm
 * (Sec. 3: a V point and a W point in one Clifford coset) is the answer.
 * Levels 0 and 1 are checked directly; each higher level is walked by the
 * parallel collision search of Sec. 3 (distinguished points, trails,
 * re-walks of merges, Fig. 2) with the theta of Sec. 5.1 and the Appendix.
 * Returns at once: a library-owned host thread drives the launches.
 * step_budget bounds the total walk steps (0 = no bound).  The stream must
 * stay valid until the search ends (qcs_wait, or status != SEARCHING).
 * Errors: QCS_ERR_BUSY if a search is running, QCS_ERR_ARG. */
QCS_API int qcs_run_walks(qcs_problem *prob, uint64_t step_budget, void *cuda_stream);

/* Exhaustive meet-in-the-middle pass over level k (Sec. 2 Eq. mitm, the
 * deterministic counterpart of the collision search): the k rotations are
 * split between a product of rotations alone (V side) and a product of
 * transposed rotations applied to C (W side), and every point of both sides
 * is evaluated on the GPU with the walk's own product and fingerprint
 * canonical form.  Even k, or sde(C) = 0: V = R(q_h)..R(q_1) and W =
 * R(q_1)^T..R(q_h)^T [R(c)^T] C (all xi^h tuples, all xi chunks c for odd
 * k).  Odd k with sde(C) >= 1: V = R(r_(h+1))..R(r_1) (xi^(h+1) points) and
 * W = R(s_1)^T..R(s_h)^T C (xi^h points), so the larger side needs no
 * product with C.  The xi^h points of the smaller side go into a device
 * hash table of coset keys, the other side's points probe it, and every key
 * match is checked exactly on the host (its decomposition is verified: D^
 * must be a signed permutation).  Equal cosets always have equal keys, so
 * when no match verifies, level k has no decomposition: *has_claw = 0 is a
 * proof.  With *has_claw = 1 the decomposition is recorded as by a FOUND
 * search.  Runs synchronously on cuda_stream (NULL = legacy default stream);
 * allocates 16 * 2^ceil(log2(2 xi^h)) bytes of table for the call.  k in
 * [2, k_max].  Errors: QCS_ERR_ARG, QCS_ERR_BUSY (a search is running),
 * QCS_ERR_NOMEM, QCS_ERR_OVERFLOW (more than 65536 key matches in one slice
 * of at most 2^24 probing points and none verified: inconclusive),
 * QCS_ERR_CUDA. */
QCS_API int qcs_certify_level(qcs_problem *prob, int k, void *cuda_stream, int *has_claw);

/* Non-blocking snapshot of the search: status, level, the collision
 * counters of Sec. 3 (distinguished points reached, merges re-walked and how
 * Fig. 2's re-walk classified them: Robin Hood, trivial, same side, claw,
 * false hash), and once FOUND the decomposition of Eq. tcount_synthesis
 * (P_1 .. P_t in out->paulis; D via qcs_get_clifford), which the library has
 * verified exactly before reporting it. */
QCS_API int qcs_poll_collisions(qcs_problem *prob, qcs_result *out);

/* Block until the running search ends or timeout_ms passes (< 0: forever);
 * fills *out like qcs_poll_collisions.  QCS_ERR_TIMEOUT on time-out. */
QCS_API int qcs_wait(qcs_problem *prob, int64_t timeout_ms, qcs_result *out);

/* Ask a running search to stop before its next launch; qcs_wait then reports
 * QCS_CANCELLED. */
QCS_API int qcs_cancel(qcs_problem *prob);

/* Once FOUND: the Clifford D of Eq. tcount_synthesis as a signed permutation of
 * Pauli codes, D P_j D^dag = sign[j] P_perm[j] (arrays of 4^n entries). */
QCS_API int qcs_get_clifford(qcs_problem *prob, int32_t *perm, int8_t *sign);

/* Manual stepping of one level of the search (qcs_run_walks drives these
 * from its own thread; do not mix the two on one problem while a search runs:
 * QCS_ERR_BUSY).  All are asynchronous on `stream` except qcs_level_collect.
 *
 * qcs_level_begin: clear the distinguished-point table and start a fresh
 * trail on every walk at level k (2 <= k <= k_max), function version
 * `version`, distinguished-point exponent dp_bits (0 = params.dp_bits). */
QCS_API int qcs_level_begin(qcs_problem *prob, int k, uint32_t version, int dp_bits, void *stream);

/* Every walk advances `steps` steps (Sec. 3 trails); a trail that reaches a
 * distinguished point is stored in (or merged against) the table and a new
 * trail starts; merges with another start are queued. */
QCS_API int qcs_level_walk(qcs_problem *prob, uint32_t steps, void *stream);

/* Re-walk every queued merge on the device (Fig. 2) and start copying the
 * classified results to pinned host memory. */
QCS_API int qcs_level_rewalk(qcs_problem *prob, void *stream);

/* Wait for `stream`, check every claw candidate exactly on the host, fold the
 * launch's counters into the problem's result and copy it to *out (may be
 * NULL).  out->status becomes QCS_FOUND, with t_count and paulis set, when a
 * claw verified (Eq. tcount_synthesis). */
QCS_API int qcs_level_collect(qcs_problem *prob, void *stream, qcs_result *out);

/* ---- one level sharded across ranks (DP-owner exchange) ---------------
 * Sec. 4.2 and Fig. 4: workers walk and send each distinguished point to a
 * collector, which stores it and hands merged trails to a verifier.  Here
 * every rank (one GPU each) is worker, collector and verifier: rank r walks
 * its own walks and owns the distinguished points whose owner index (a hash
 * of the point, computed on the device by qcs_shard_bin) is r.  One round:
 *   qcs_level_walk_out  - walk; distinguished points go to an outbox;
 *   qcs_shard_bin       - group the outbox by owner rank;
 *   (the caller exchanges the groups, e.g. one all-to-all over NCCL);
 *   qcs_level_insert    - store the received points in the local table,
 *                         queueing merges exactly as qcs_level_walk would;
 *   qcs_level_rewalk, qcs_level_collect - as for an unsharded level.
 * Trail references name walks by their index among all ranks' walks, and
 * every rank uses the same params.seed, so any rank recomputes any trail's
 * start: the owner re-walks merges of trails from every rank.
 *
 * qcs_level_begin_shard: qcs_level_begin for rank-local walks walk_base ..
 * walk_base + params.walks - 1 of total_walks <= 2^24 walks in all.
 * QCS_ERR_ARG if that range does not fit. */
QCS_API int qcs_level_begin_shard(qcs_problem *prob, int k, uint32_t version, int dp_bits, uint32_t walk_base,
                                  uint32_t total_walks, void *stream);

/* qcs_level_walk for a sharded level: the distinguished points reached go to
 * `outbox` (DEVICE, cap pairs {point, trail reference} of uint64) instead of
 * the local table (outbox must not be NULL: QCS_ERR_ARG); *count (DEVICE
 * uint32, zeroed by the call) counts every
 * point reached, also those past cap (which are lost: size the outbox for
 * walks x steps x theta with room to spare).  Resets the launch counters and
 * the merge queue like qcs_level_walk.  Asynchronous on `stream`. */
QCS_API int qcs_level_walk_out(qcs_problem *prob, uint32_t steps, uint64_t *outbox, uint32_t cap,
                               uint32_t *count, void *stream);

/* Group `count` points (DEVICE pairs {point, trail reference}) by owner rank
 * in 0 .. n_owners - 1 (n_owners <= 1024): `out` (DEVICE, count pairs) gets
 * them owner by owner in rank order, owner_counts (DEVICE, 2 n_owners
 * uint32; the first n_owners hold the counts, the rest is scratch) the size
 * of each group.  The order within a group is arbitrary.  No problem is
 * needed: the owner is a fixed hash of the point.  Asynchronous. */
QCS_API int qcs_shard_bin(const uint64_t *points, uint32_t count, uint32_t n_owners, uint64_t *out,
                          uint32_t *owner_counts, void *stream);

/* Store `count` received points (DEVICE pairs {point, trail reference}) in
 * the level's table (Sec. 3: a point already stored from another trail is a
 * merge, queued for qcs_level_rewalk).  Call after qcs_level_walk_out and
 * before qcs_level_rewalk of the same round.  Asynchronous on `stream`. */
QCS_API int qcs_level_insert(qcs_problem *prob, const uint64_t *points, uint32_t count, void *stream);

/* Copy the merges queued by the last qcs_level_walk / qcs_level_insert
 * (Sec. 3: pairs of trails that reached one distinguished point, each to be
 * re-walked as in Fig. 2) to HOST memory: up to cap triples {trail ref a, trail ref b, distinguished
 * point} into out (3 cap uint64), *n_out = the number copied.  Waits for the
 * problem's queue on `stream` first.  For inspection and tests: the search
 * itself re-walks the queue on the device (qcs_level_rewalk). */
QCS_API int qcs_level_merges(qcs_problem *prob, uint64_t *out, uint32_t cap, uint32_t *n_out, void *stream);

/* qcs_level_walk_static: the walk of qcs_level_walk (begin = 1: preceded by
 * the reset of qcs_level_begin) for callers that must not allocate device
 * memory: code whose device memory belongs to a framework's caching allocator
 * or to a fixed arena (a stray cudaMalloc fragments it, or fails once the
 * arena has reserved the free memory), and loops that cannot take
 * cudaMalloc's implicit device synchronisation.  The paper has no
 * counterpart; this is a property of the library, not of the method.
 *
 * It allocates nothing: the distinguished-point table is a static device
 * array of 2^18 16-byte slots (4 MiB) that every GPU loading libqcs holds
 * until exit, so the problem's params.table_log2 must be <= 18 (QCS_ERR_ARG
 * otherwise).  The problem itself must already exist (its creation does
 * allocate), and its device must be the current device (QCS_ERR_ARG
 * otherwise; the call never switches devices).  The first call on each
 * device is its set-up: with that device current it looks up the array's
 * device address, marks every slot empty and synchronises `stream` once;
 * make that first call before any stream capture.  All calls on a device
 * share the one table and it keeps the last call's contents: begin = 1
 * clears the problem's 2^table_log2 slots, and calls that overlap on the GPU
 * race on it.
 *
 * The caller passes, as DEVICE pointers: walk_states, n_walks records of 32
 * bytes (written when begin = 1, then advanced by `steps` steps each);
 * merges, merge_cap triples {trail ref a, trail ref b, distinguished point};
 * counts, 8 uint64 zeroed by the call: [0] walk steps, [1] W-side steps,
 * [2] distinguished points, [3] abandoned trails, [4] overwritten points,
 * [5] duplicate inserts, [6] merges found, [7] merges pushed (low 32 bits;
 * it counts pushes past merge_cap too, so the valid triples number
 * min(counts[7], merge_cap)); the high 32 bits of [7] are nonzero only if a
 * bounded wait inside the n = 4 tensor-core walk (launch_shape 3) ran out,
 * and then nothing the call wrote is valid.  k, version, dp_bits (0 = params.dp_bits) as
 * in qcs_level_begin; n_walks <= 2^24.  Asynchronous on `stream` after the
 * set-up. */
QCS_API int qcs_level_walk_static(qcs_problem *prob, int k, uint32_t version, int dp_bits, int begin,
                                  void *walk_states, uint32_t n_walks, uint32_t steps, uint64_t *merges,
                                  uint32_t merge_cap, uint64_t *counts, void *stream);

/* ---- many targets at once (the batched search) -------------------------
 * A batch runs many problems together: each job is one target on its own
 * T-count ladder with its own walks, distinguished-point table and merge
 * queue (Sec. 3); one round advances every active job by one launch of its
 * level (walk, re-walk, exact claw checks), with all jobs of one qubit count
 * in one persistent walk kernel and one persistent re-walk kernel.  With
 * use_graph = 1 a round is one replay of a CUDA graph captured at the first
 * round.  Jobs may be added and removed between rounds.  A job's levels are
 * settled by the exhaustive pass (the work of qcs_certify_level, run in
 * shares of cert_points_log2 per round, each job holding its own key table
 * until its pass ends) as its problem's exhaustive_log2 / exhaustive_first
 * ask: before the level's walk (exhaustive_first) or when its walk budget
 * ends. */
typedef struct qcs_batch qcs_batch;

typedef struct qcs_batch_params {
    int32_t max_jobs;        /* job slots, 1..65536 */
    int32_t walks_per_job;   /* concurrent walks of each job (multiple of 16, at least 16) */
    int32_t steps_per_round; /* walk steps per walk per round (upper bound) */
    int32_t table_log2;      /* distinguished-point table of each job: 2^table_log2 slots */
    int32_t queue_capacity;  /* merges kept per job per round */
    int32_t use_graph;       /* 1: each round is one CUDA-graph replay */
    int32_t rewalk_budget;   /* evaluations of f one re-walk may take per round; an unfinished
                                re-walk resumes in the next round (0: no bound) */
    int32_t launch_shape[4];  /* launch shape of the batched walk kernel for n = 1..4 qubits
                                 (index n - 1; 0 = default; see qcs_launch_shapes) */
    int32_t cert_points_log2; /* a round runs at most 2^cert_points_log2 points' worth of exhaustive-pass
                                 work (a point with the contraction against C^ counts four), the job
                                 with the least pass work left first (ties: the oldest); a job whose
                                 pass is unfinished keeps it and is not walked that round.  0: every
                                 pass a round starts runs to its end in that round */
} qcs_batch_params;

QCS_API void qcs_batch_default_params(qcs_batch_params *p);

/* Allocates the pooled per-job arrays for max_jobs jobs.  stream: the CUDA
 * stream of every round (a non-default stream is needed for graph capture;
 * NULL makes the batch create its own). */
QCS_API int qcs_batch_create(const qcs_batch_params *p, void *stream, qcs_batch **out);

/* Device bytes one job of this problem's size needs in this batch (its walks,
 * table and queue plus the problem's matrices): the basis of admission. */
QCS_API uint64_t qcs_batch_job_bytes(const qcs_batch *batch, const qcs_problem *prob);

/* Add a created problem as a job (its ladder starts at sde(C^)); the batch
 * borrows prob until the job is removed or the batch destroyed.  Allocates the
 * job's walks, table and queue.  *job gets the job's slot.  QCS_ERR_BUSY when
 * every slot is used or the problem is running qcs_run_walks. */
QCS_API int qcs_batch_add(qcs_batch *batch, qcs_problem *prob, int *job);

/* Remove a job (finished or not) and free its buffers. */
QCS_API int qcs_batch_remove(qcs_batch *batch, int job);

/* One round for every active job; blocks until the round's results are in.
 * *n_active (may be NULL) gets the number of jobs still searching. */
QCS_API int qcs_batch_round(qcs_batch *batch, int *n_active);

/* A job's result (as qcs_poll_collisions reports it for the problem). */
QCS_API int qcs_batch_poll(qcs_batch *batch, int job, qcs_result *out);

/* Frees the batch and every job's buffers (not the problems). */
QCS_API void qcs_batch_destroy(qcs_batch *batch);

/* Exact host check that C = e^{i phi} R(P_t)..R(P_1) D for a Clifford D
 * (Sec. 4.1): forms D^ = R^(P_1)^T..R^(P_t)^T C^ and tests that it is a signed
 * permutation.  target as in qcs_create_problem; paulis[0] is P_1.  Pure host,
 * no GPU.  QCS_OK or QCS_ERR_MISMATCH (or QCS_ERR_ARG / QCS_ERR_NOT_UNITARY /
 * QCS_ERR_OVERFLOW). */
QCS_API int qcs_verify_decomposition(int n_qubits, const int64_t *target, int32_t target_exp,
                             const uint32_t *paulis, int t);

/* One walk step f = h o nu o mu (Sec. 2, Fig. 1; Sec. 3 z_b) for count states
 * at level k (chunk c in 1..4^n-1 for odd k, 0 for even k) and function
 * version `version`: out[i] = f(in[i]), is_dp[i] = 1 when out[i] is
 * distinguished (its top d_theta of L bits are zero).  in, out, is_dp are
 * DEVICE pointers (is_dp may be NULL); asynchronous on `stream`.  count = 0 is
 * a no-op.  Errors: QCS_ERR_ARG (k > k_max or chunk out of range), QCS_ERR_CUDA. */
QCS_API int qcs_walk_step(qcs_problem *prob, int k, int chunk, uint32_t version, const uint64_t *in,
                  uint64_t *out, uint8_t *is_dp, size_t count, void *stream);

/* Re-walk count trail pairs on the device (Sec. 3, Fig. 2): pair i is
 * (start_a[i], len_a[i]) and (start_b[i], len_b[i]) ending at one
 * distinguished point, at level k, chunk, version.  cls[i] gets a
 * QCS_MERGE_* class (claw candidates are reported as QCS_MERGE_CLAW before the
 * exact check), ab[2i], ab[2i+1] the two distinct states whose images
 * coincide.  Lengths above 2^20 are reported as QCS_MERGE_NO_MERGE without
 * walking.  All pointers are DEVICE pointers; asynchronous on `stream`. */
QCS_API int qcs_rewalk(qcs_problem *prob, int k, int chunk, uint32_t version, const uint64_t *start_a,
               const uint32_t *len_a, const uint64_t *start_b, const uint32_t *len_b,
               size_t count, int32_t *cls, uint64_t *ab, void *stream);

/* How the search walks level k of an n-qubit problem with parameters p (pure
 * host arithmetic, no device).  N = 2 xi^h (xi chunks for odd k) points,
 * w = 2^table_log2 slots.  theta_policy 1 takes theta = 2^-d_theta with
 * d_theta the larger of theta_min_bits and the rounded log2 of sqrt(N / 2w),
 * the minimum over theta of the steps per collision N theta / w + 2 / theta
 * (Appendix, after van Oorschot and Wiener); when w >= N that is
 * 2^-theta_min_bits, the large theta the paper found fastest for small
 * spaces (Sec. 5.1).  d_theta never exceeds p->dp_bits.  A launch covers at
 * most one function version (version_factor * N steps), its expected merges
 * (distinguished points times the stored fraction min(1, w / (theta N))) fit
 * half the merge queue, and a level ends after budget_factor * N steps and at
 * least four versions.  Errors: QCS_ERR_ARG. */
typedef struct qcs_plan {
    int32_t dp_bits;               /* d_theta used at this level */
    uint32_t walks;                /* concurrent walks */
    uint32_t steps;                /* steps per walk per launch */
    uint64_t launches_per_version; /* ~0: one version for the level */
    uint64_t min_launches;         /* launches before the level is given up */
    uint64_t points;               /* N */
} qcs_plan;

QCS_API int qcs_plan_level(int n_qubits, int k, const qcs_params *p, qcs_plan *out);

/* Facts about a created problem: sde of C^ (smallest denominator exponent),
 * and the number of walk points 2 xi^h at level k (per chunk). */
QCS_API int qcs_problem_sde(const qcs_problem *prob);
QCS_API uint64_t qcs_level_points(const qcs_problem *prob, int k);

/* Copy C^ (reduced) to host arrays a, b (4^n x 4^n) and its exponent. */
QCS_API int qcs_get_channel(const qcs_problem *prob, int64_t *a, int64_t *b, int32_t *exp);

/* The channel representation C^ of a target unitary (Sec. 4.1: entry
 * (i, j) = Tr(P_i U P_j U^dagger) / 2^n over the Pauli codes), exactly and
 * reduced to its smallest exponent: entry (i, j) = (a + b sqrt2) / sqrt2^exp
 * at a[i 4^n + j], b[i 4^n + j] (row-major, 4^n x 4^n, caller-owned), and
 * *exp = sde(C^).  target as in qcs_create_problem.  Pure host, no GPU; the
 * same arithmetic that qcs_create_problem uses.  QCS_OK, or QCS_ERR_ARG /
 * QCS_ERR_NOT_UNITARY / QCS_ERR_OVERFLOW. */
QCS_API int qcs_channel_from_unitary(int n_qubits, const int64_t *target, int32_t target_exp, int64_t *a,
                                     int64_t *b, int32_t *exp);

/* Synchronises and frees everything the problem owns.  NULL is a no-op. */
QCS_API void qcs_destroy_problem(qcs_problem *prob);

/* Text for a status code; never NULL. */
QCS_API const char *qcs_strerror(int code);

/* Last CUDA error string seen by this thread's calls into the library. */
QCS_API const char *qcs_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QCS_H */
