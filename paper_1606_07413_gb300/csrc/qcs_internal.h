// qcs_internal.h -- structures shared by the host library (qcs_api.cpp,
// qcs_exact.cpp) and the CUDA kernels (qcs_walk.cu).  Not part of the ABI.
#pragma once

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "qcs.h"

namespace qcs {

constexpr int kMaxH = 8;              // h = floor(k/2) <= 7 for k <= 15
constexpr uint64_t kEmptyKey = ~0ull; // empty table slot / unwritten meta

// Hash constants of the walk function (written specification, Sec. 2 "h"):
// SplitMix64 output function (Steele, Lea & Flood 2014), its stream increment,
// and two seeds taken from the fractional parts of sqrt2 and sqrt3.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kSeedU = 0x6A09E667F3BCC908ull;
constexpr uint64_t kSeedH = 0xBB67AE8584CAA73Bull;

// Everything a warp needs to evaluate one step f of the walk at one level.
struct LevelCtx {
    // C^ numerators mod 2^32 as (a, b), 4^n x 4^n.  With W = lanes_per_walk(n)
    // and R = 4^n / W, row i, column Q = sub + W t sits at i * 4^n + sub * R +
    // t, so one lane's R columns of a row are contiguous.
    const uint2 *C32;
    // n >= 3: C^ as signed byte quads when every entry fits in int8, else
    // null.  Quad q holds rows 4q .. 4q+3 of a column as the bytes 0 .. 3 of
    // one word.  uint4 number (q R/2 + j) W + sub carries, for the columns
    // Q0 = sub + 2 W j and Q1 = Q0 + W, the words (a-quad Q0, b-quad Q0,
    // a-quad Q1, b-quad Q1) (W, R as above).
    const uint4 *Cq;
    // n = 4, when every entry of C^ fits in int8: C^ for the tensor-core
    // contraction (launch shape 3 of k_walks<4>), else null.  K = 512 rows
    // (the a-parts of the 256 rows, then the b-parts; within a part, K index
    // 8 l + t is row 32 t + l), N = 256 columns, each entry stored as the
    // byte entry + 128.  Column n takes 512 bytes at
    // n * 512: 16-byte chunk c = 4 s + q (s = K-block of 64, q = 0..3),
    // stored at chunk c ^ (4 (n & 1)), holds for the four 16-row K-blocks
    // kb = 4 s .. 4 s + 3 the bytes of rows 16 kb + 2q, 2q + 1, 2q + 8, 2q + 9.
    const uint4 *Cm;
    const uint2 *U;    // fingerprint weights (Ua, Ub) per row, 4^n
    // The weights after the first adjoint stage of a side (index 0: V, 1: W),
    // mod 2^16, for every Pauli: entry e = q_a - 1, where q_a is the side's
    // first stage rotation (V: q_h; W: q_1); word e 4^n + row = Ua | Ub << 16.
    const uint32_t *T1[2];
    // rotation masks: for Pauli p and lane sub, the 16-bit word at index
    // p W + sub has bit t set when row sub + W t anticommutes with p and bit
    // 8 + t when the sign s(p, row) is +1 (t < R <= 8).  4^n x W uint16,
    // read as 4^n W / 2 uint32.
    const uint32_t *coef;
    uint64_t xi_h;     // xi^h, the number of rotation tuples per side
    int32_t ell;       // bits of one rotation's field in the state: min(16, (L - 1) / h)
    uint32_t fmask;    // 2^ell - 1
    uint64_t maskL;    // low L bits
    uint32_t xi;       // 4^n - 1
    int32_t n, k, h, K;
    int32_t ev;        // V side is raised from exponent h to K: ev = K - h
    int32_t dshift;    // distinguished iff (x >> dshift) == 0, dshift = L - d_theta
    uint32_t version;
    int32_t n_chunks;  // xi for odd k (trail chunk drawn from its start), 0 for even k
    uint64_t seed;     // seed of trail starting points
};

// A trail is named by a 64-bit reference: walk index (24 bits), its trail
// sequence number (23 bits) and its length (17 bits).  Its starting state and
// chunk are recomputed from (seed, version, walk, sequence), so a
// distinguished point fits in one 16-byte slot.
constexpr int kRefWalkBits = 24, kRefSeqBits = 23, kRefLenBits = 17;
constexpr uint32_t kMaxWalks = 1u << kRefWalkBits;
constexpr uint32_t kMaxTrailLen = (1u << kRefLenBits) - 1;

// One distinguished point (Sec. 3: the triple start, end, length, with the
// start and length folded into the trail reference).  16 bytes, written with
// one 128-bit atomic exchange: the memory keeps the newest trail per slot.
struct alignas(16) Slot {
    unsigned long long key; // the distinguished state, kEmptyKey when free
    unsigned long long ref; // trail reference
};

// Two trails that reached one distinguished point with different starts.
struct Pair {
    unsigned long long ref_a, ref_b, dp;
};

// A merge of a V point and a W point (before the exact check).
struct Cand {
    unsigned long long a, b;
    uint32_t chunk, pad;
};

// A re-walk carried over to the next round (batched search): the two
// states, the steps each trail still has to its shared point, the chunk.
struct Pending {
    unsigned long long a, b;
    uint32_t la, lb, chunk, pad;
};

struct RewalkOut {
    int32_t cls;    // QCS_MERGE_* (claw = candidate before the exact check)
    uint32_t chunk; // chunk of the pair (odd k)
    unsigned long long a, b;
};

// Per-walk state kept in device memory between launches.  32 bytes.
struct WalkState {
    unsigned long long start, cur;
    uint32_t len, chunk, seq, pad;
};

enum Counter {
    C_STEPS = 0,
    C_WSTEPS,      // steps on the W side (these do the 4^n x 4^n contraction)
    C_DPS,
    C_ABANDONED,
    C_EVICTED,     // distinguished points overwritten by another one
    C_DUPLICATE,
    C_PAIRS,       // merges pushed (including overflowed ones)
    C_CANDS,       // claw candidates found by the re-walk (including overflowed ones)
    C_RSTEPS,      // walk steps taken by the re-walk (evaluations of f)
    C_CLS0,        // re-walk classes QCS_MERGE_ROBIN_HOOD .. QCS_MERGE_NO_MERGE at C_CLS0 + class
    C_STALLED = C_CLS0 + 6, // warps of the tensor-core walk whose bounded wait ran out (low word)
    C_NCOUNTERS
};

struct WalkLaunch {
    LevelCtx lv;
    WalkState *walks;
    int32_t n_walks;    // walks advanced by this launch
    uint32_t steps;     // steps per walk in this launch
    uint32_t max_len;
    Slot *table;
    uint64_t table_mask;
    Pair *queue;
    uint32_t *qhead;
    uint32_t qcap;
    Cand *cands;
    uint32_t *ccount;
    uint32_t ccap;
    unsigned long long *counters;
    // batched search: a re-walk gets rewalk_budget evaluations of f per
    // round (0: no bound); unfinished ones go to pend_out and come back as
    // pend_in in the next round, before that round's new merges
    uint32_t rewalk_budget;
    uint32_t pend_in_n, pend_cap;
    const Pending *pend_in;
    Pending *pend_out;
    uint32_t *pend_out_n;
    int32_t shape;       // launch shape of k_walks (host-side choice; see launch_shapes)
    // DP-owner sharding (Sec. 4.2 collectors): the walks of this launch are
    // walks walk_base .. walk_base + n_walks - 1 of all ranks' walks (trail
    // references and starts use the global index), and with outbox set their
    // distinguished points go to outbox (up to ocap, *ohead counts every one)
    // instead of the local table, for the exchange with their owners
    uint32_t walk_base;
    uint32_t ocap;
    Slot *outbox;
    uint32_t *ohead;
    // single-target re-walk: merges are claimed from this device counter
    // (zeroed before the launch); null: a fixed stride (the batched re-walk)
    uint32_t *rw_next;
    // the tensor-core walk (n = 4, launch shape 3) counts here the warps
    // whose bounded wait ran out (the launch's results are then invalid);
    // it refuses to launch without it
    uint32_t *stall;
};

// Many jobs in one launch: per qubit count, the device list of tasks
// (job index, first walk) with walks_per_task(n) walks each, and of job indices.
struct BatchArgs {
    const WalkLaunch *jobs;   // device array indexed by job
    const uint32_t *tasks;    // 2 * n_tasks entries
    const uint32_t *n_tasks;  // device scalar
    const uint32_t *job_ids;  // jobs of this qubit count
    const uint32_t *n_jobs;   // device scalar
};
// Exhaustive meet-in-the-middle pass over one level (Sec. 2 Eq. mitm, the
// collision search's exact counterpart): the points of the smaller side are
// hashed into an open-addressing table of coset keys, then every point of
// the other side probes it and each key match is queued for the exact host
// check.  Point index -> rotations: base-xi digits, q_j = digit_j + 1 (q_1
// the lowest digit); a W index of a level context with odd k is chunk-major,
// chunk = index / xi^h + 1.
struct alignas(16) CertSlot {
    uint64_t key; // ~0: empty
    uint64_t idx; // stored point index
};

struct CertArgs {
    LevelCtx lv;       // the side's level context (lv.h rotations per point)
    int32_t side;      // which product a point is: 0 V, 1 W
    int32_t insert;    // 1: insert the points' keys, 0: probe the table with them
    uint64_t first;    // point indices [first, first + count)
    uint64_t count;
    uint64_t xi_h;     // rotation tuples of the h-rotation W side (chunk stride)
    uint64_t base;     // hash base of the keys, the same for every chunk
    CertSlot *table;
    uint64_t mask;     // table slots - 1 (a power of two, at least twice the stored points)
    uint64_t *pairs;   // key matches (stored index, probing index)
    uint32_t *n_pairs; // matches found (may exceed cap; only cap are stored)
    uint32_t cap;
};
cudaError_t launch_certify(const CertArgs &a, cudaStream_t s);
// Host driver of the exhaustive pass (qcs_certify_level); *got = verified claw.
int certify_level(::qcs_problem *P, int k, cudaStream_t s, bool *got);

// The exhaustive pass as a resumable job (the batch engine runs a bounded
// share of it per round): cert_begin allocates and clears the key table,
// cert_advance evaluates points (stored side first, then probing slices,
// each slice's key matches checked exactly) until the pass is done or
// `budget` streamed-point equivalents are spent (*used), and cert_end frees
// the table and folds the pass into the problem's result (QCS_ERR_OVERFLOW:
// done without a claw but inconclusive).  certify_level is the three in a row.
struct CertPass {
    static constexpr uint32_t kCap = 1u << 16;          // key matches read back per slice
    static constexpr uint64_t kSliceMin = 1ull << 20;   // probing points of the first slice
    static constexpr uint64_t kSliceMax = 1ull << 24;   // slices double up to this
    int k = 0, h = 0;
    bool v_heavy = false, done = false, got = false, overflow = false;
    uint64_t xi = 0, xi_h = 0, n_probe = 0, stored = 0, probed = 0, slice = 0;
    uint64_t table_bytes = 0;
    int64_t d2h = 0;
    LevelCtx lv_store{}, lv_probe{};
    CertArgs a{};
    uint32_t *hN = nullptr;
    uint64_t *hPairs = nullptr;
};
int cert_begin(::qcs_problem *P, int k, cudaStream_t s, CertPass *c);
int cert_advance(::qcs_problem *P, CertPass *c, cudaStream_t s, uint64_t budget, uint64_t *used);
int cert_end(::qcs_problem *P, CertPass *c, cudaStream_t s);
uint64_t exhaustive_points(const ::qcs_problem *P, int k); // V + W points of level k
bool exhaustive_eligible(const ::qcs_problem *P, int k);   // within exhaustive_log2 and device memory

int walks_per_task(int n, int shape); // walks (lane groups) per CTA of the walk kernels of that launch shape
int lanes_per_walk(int n); // lanes of a warp that evaluate one walk (the device layouts follow it)
int launch_shapes(int n);                    // launch shapes of the walk kernels for n qubits
int shape_warps_of(int n, int shape);        // warps per CTA of a launch shape
int shape_min_blocks_of(int n, int shape);   // minimum resident CTAs per SM (the register cap) of a shape

// ---- kernel launchers (qcs_walk.cu); all return cudaError_t of the launch ----
cudaError_t launch_walks_batch(int n, int shape, const BatchArgs &a, cudaStream_t s);
cudaError_t launch_rewalk_batch(int n, const BatchArgs &a, cudaStream_t s);
cudaError_t launch_walk_step(const LevelCtx &lv, int chunk, const uint64_t *in, uint64_t *out,
                             uint8_t *is_dp, size_t count, cudaStream_t s);
cudaError_t launch_init_walks(const WalkLaunch &w, cudaStream_t s);
cudaError_t launch_walks(const WalkLaunch &w, cudaStream_t s);
// DP-owner sharding: insert `count` distinguished points {dp, trail ref}
// into w's table (merges queued as by the walk), and bin points by owner
// rank (owner_of in qcs_walk.cu): out gets the points grouped by owner in
// rank order, counts[r] the number for rank r (device arrays; counts has
// 2 n_owners entries, the first n_owners zeroed by the caller, the rest are
// the scatter's cursors)
cudaError_t launch_insert_points(const WalkLaunch &w, const Slot *pts, uint32_t count, cudaStream_t s);
cudaError_t launch_bin_owners(const Slot *in, uint32_t count, uint32_t n_owners, Slot *out, uint32_t *counts,
                              cudaStream_t s);
cudaError_t launch_rewalk_pairs(const WalkLaunch &w, cudaStream_t s);
cudaError_t launch_rewalk_arrays(const LevelCtx &lv, int chunk, const uint64_t *sa, const uint32_t *la,
                                 const uint64_t *sb, const uint32_t *lb, size_t count, int32_t *cls,
                                 uint64_t *ab, cudaStream_t s);
// For the allocation-free walk entry point (qcs_noalloc.cu): the level
// context and trail cut-off that qcs_level_begin would use, and the problem's
// table size; QCS_ERR_ARG when k or dp_bits are out of range.
int noalloc_level(const ::qcs_problem *P, int k, uint32_t version, int dp_bits, LevelCtx *lv,
                  uint32_t *max_len, int *table_log2);
int record_cuda_error(cudaError_t e); // stores the text for qcs_last_cuda_error, returns QCS_ERR_CUDA

// number of resident CTAs of the walk kernel per SM for n qubits (occupancy)
int walk_blocks_per_sm(int n);
int num_sms();

// ---- exact host arithmetic (qcs_exact.cpp) ----
// A matrix over Z[1/sqrt2]: (a + b sqrt2) / sqrt2^E, D x D row-major.
struct PMat {
    int D = 0, E = 0;
    std::vector<int64_t> a, b;
};

// status codes mirror qcs.h; overflow is reported, never wraps
int exact_channel_from_unitary(int n, const int64_t *u, int e, PMat *out);
int exact_unitary_from_circuit(int n, const int32_t *gates, int n_gates, std::vector<int64_t> *u, int *e);
int exact_check_channel(int n, const PMat &C);
void exact_reduce(PMat *M);
bool exact_is_clifford(const PMat &M);
// left-multiply by R^(p) (transpose = false) or R^(p)^T (true); exponent + 1
int exact_rhat_left(int n, uint32_t p, bool transpose, const PMat &M, PMat *out);
// D^ = R^(P_1)^T .. R^(P_t)^T C^; QCS_OK if a signed permutation, else QCS_ERR_MISMATCH
int exact_verify(int n, const PMat &C, const uint32_t *paulis, int t, PMat *Dout);
int pauli_phase(int n, uint32_t p, uint32_t q); // P(p)P(q) = i^lambda P(p^q)
// device tables of the first adjoint stage (LevelCtx::T1), built once per
// device and qubit count and kept for the life of the process
// (*uploaded, when given, grows by the bytes this call copied to the device)
int stage_tables(int n, const uint32_t *t1[2], int64_t *uploaded = nullptr);

// How a level is walked (Sec. 3 and Appendix): theta, the launch shape, the
// function-version period and the level's step budget.
struct LevelPlan {
    int dp_bits;
    uint32_t walks, steps;
    uint64_t launches_per_version, min_launches;
    uint64_t points;
};

// helpers of the host library shared by qcs_api.cpp and qcs_batch.cpp
uint64_t upow(uint64_t b, int e);
int field_bits(int L, int h);
void decode_state(uint64_t x, int n, int L, int h, uint32_t *q);
LevelCtx make_level(const ::qcs_problem *P, int k, uint32_t version, int dp_bits);
LevelPlan plan_level(const ::qcs_problem *P, int k, const qcs_params &p);
LevelPlan plan_level_n(int D, int k, const qcs_params &p); // D = 4^n
void found(::qcs_problem *P, int k, const uint32_t *paulis, PMat &&Dh); // keeps the first decomposition
void found(::qcs_problem *P, int k, const uint32_t *paulis);              // forms D^ itself
// Exact check of a claw candidate (Eq. tcount_synthesis): paulis gets
// (q_1..q_h, q'_1..q'_h [, c]) from the V rotations qv, the W rotations qw and
// the chunk, and the candidate is a claw iff D^ = R^(P_1)^T..R^(P_k)^T C^ is a
// signed permutation; *Dh gets D^ then.
bool verify_claw(const ::qcs_problem *P, int k, int chunk, const uint32_t *qv, const uint32_t *qw,
                 uint32_t *paulis, PMat *Dh);

} // namespace qcs

// A search problem (include/qcs.h): the exact target and its device copies.
struct qcs_problem {
    int n = 0, D = 0, k_max = 0, device = 0;
    qcs_params p{};
    qcs::PMat C; // reduced, exponent = sde
    // device data
    uint2 *dC32 = nullptr, *dU = nullptr;
    uint32_t *dCq = nullptr; // n >= 3, when every entry of C^ fits in int8
    uint32_t *dCm = nullptr; // n = 4, when every entry fits in int8: the tensor-core layout (LevelCtx::Cm)
    const uint32_t *dT1[2] = {nullptr, nullptr}; // shared stage tables
    uint32_t *dCoef = nullptr;
    qcs::Slot *dTable = nullptr;
    qcs::Pair *dQueue = nullptr;
    uint32_t *dQhead = nullptr; // [0] queued merges, [1] claw candidates, [2] carried re-walks, [3] re-walk cursor
    qcs::Pending *dPend[2] = {nullptr, nullptr}; // carried re-walks (params.rewalk_budget > 0)
    qcs::Cand *dCands = nullptr;
    qcs::WalkState *dWalks = nullptr;
    unsigned long long *dCounters = nullptr;
    // pinned host mirrors
    unsigned long long *hCounters = nullptr;
    qcs::Cand *hCands = nullptr;
    uint32_t *hQhead = nullptr; // mirrors dQhead
    // search state
    std::thread driver;
    std::mutex mu;
    std::condition_variable cv;
    std::atomic<bool> cancel{false};
    bool running = false;
    qcs_result res{};
    std::chrono::steady_clock::time_point t0;
    qcs::PMat Dhat;
    bool have_D = false;
    // the level being stepped (qcs_level_* and the driver)
    struct {
        bool active = false;
        int k = 0, h = 0, dp_bits = 0;
        qcs::WalkLaunch w{};
        int pp = 0;          // dPend[pp] holds the re-walks carried into the next launch
        uint32_t pend_n = 0; // how many
    } lvl;
};
