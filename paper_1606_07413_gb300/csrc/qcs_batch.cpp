// qcs_batch.cpp -- many targets searched together (include/qcs.h, qcs_batch_*).
//
// Every job is one target on its own T-count ladder (Sec. 4.1) with its own
// walks, distinguished-point table and merge queue (Sec. 3).  A round runs
// every active job's walks in one persistent walk kernel per qubit count and
// re-walks every job's merges in one persistent re-walk kernel per qubit
// count: the CTAs take (job, walk range) tasks from a device task list.  The
// launch records, task lists, counters and claw candidates of all jobs live
// in pooled arrays, so a whole round is one CUDA-graph replay (captured once:
// the grid is persistent and every size is read from device memory), and the
// host then advances each job's ladder exactly as qcs_run_walks does.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "qcs.h"
#include "qcs_internal.h"

using namespace qcs;

namespace {

constexpr uint32_t kBatchCandCap = 1024; // claw candidates kept per job per round
constexpr int kClasses = 5;              // qubit counts 1..4 (index 0 unused)
constexpr int kHeads = 4;                // per slot: merge queue, candidates, carried re-walks, unused

struct Job {
    qcs_problem *P = nullptr;
    bool used = false, active = false, need_begin = true;
    int status = QCS_IDLE;
    int k = 0;
    uint32_t version = 0;
    uint64_t launches = 0, in_version = 0;
    qcs_params jp{};
    LevelPlan pl{};
    WalkLaunch w{};
    WalkState *walks = nullptr;
    Slot *table = nullptr;
    Pair *queue = nullptr;
    Pending *pend[2] = {nullptr, nullptr}; // re-walks carried between rounds (double-buffered)
    int pp = 0;                            // pend[pp] feeds the next round
    uint32_t pend_n = 0;
    std::chrono::steady_clock::time_point t0;
    // the exhaustive pass of the job's level, run a share per round
    CertPass *cert = nullptr;
    bool cert_after_walk = false; // the level's walk budget ended: settle it exactly next
    int cert_skip_k = -1;         // a level whose pass was inconclusive is walked instead
    bool parked = false;          // busy with its pass this round: not walked
    uint64_t seq = 0;             // order of arrival (the passes' share goes to the oldest first)
};

int fail(cudaError_t e) { return record_cuda_error(e); }

} // namespace

struct qcs_batch {
    qcs_batch_params bp{};
    cudaStream_t s = nullptr;
    bool own_stream = false;
    std::vector<Job> jobs;
    // pooled device arrays and their pinned host mirrors
    WalkLaunch *dJobs = nullptr, *hJobs = nullptr;
    unsigned long long *dCounters = nullptr, *hCounters = nullptr; // [slot][C_NCOUNTERS]
    uint32_t *dHeads = nullptr, *hHeads = nullptr;                 // [slot][kHeads]
    Cand *dCands = nullptr, *hCands = nullptr;                     // [slot][kBatchCandCap]
    uint32_t *dTasks = nullptr, *hTasks = nullptr;                 // [class][2 * max_tasks]
    uint32_t *dIds = nullptr, *hIds = nullptr;                     // [class][max_jobs]
    uint32_t *dCounts = nullptr, *hCounts = nullptr;               // [class][2]: tasks, jobs
    uint32_t max_tasks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t rounds = 0;
    // one branch per qubit count: its walk and re-walk kernels run on their
    // own stream, forked from and joined back into s, so the classes' kernels
    // (and the long tail of one class's re-walks) overlap
    cudaStream_t cs[kClasses] = {};
    cudaEvent_t fork = nullptr, join[kClasses] = {};
    uint64_t next_seq = 0;
};

namespace {

size_t job_bytes(const qcs_batch_params &bp)
{
    return sizeof(WalkState) * (size_t)bp.walks_per_job + (sizeof(Slot) << bp.table_log2) +
           (sizeof(Pair) + 2 * sizeof(Pending)) * (size_t)bp.queue_capacity;
}

void free_job(Job &j, cudaStream_t s)
{
    if (j.cert) {
        cert_end(j.P, j.cert, s);
        delete j.cert;
    }
    cudaFree(j.walks);
    cudaFree(j.table);
    cudaFree(j.queue);
    cudaFree(j.pend[0]);
    cudaFree(j.pend[1]);
    j = Job();
}

// the ladder below level 2 needs no walks (as in qcs_run_walks)
void settle_small_levels(Job &j)
{
    qcs_problem *P = j.P;
    while (j.k <= 1 && j.k <= P->k_max) {
        uint32_t paulis[16] = {0};
        bool ok = false;
        if (j.k == 0) {
            ok = exact_is_clifford(P->C);
        } else {
            for (uint32_t c = 1; c < (uint32_t)P->D && !ok; c++) {
                paulis[0] = c;
                ok = exact_verify(P->n, P->C, paulis, 1, nullptr) == QCS_OK;
            }
        }
        if (ok) {
            found(P, j.k, paulis);
            j.status = QCS_FOUND;
            j.active = false;
            return;
        }
        j.k++;
    }
    if (j.k > P->k_max) {
        j.status = QCS_BUDGET_EXHAUSTED;
        j.active = false;
    }
}

void job_error(Job &j, int rc)
{
    std::lock_guard<std::mutex> g(j.P->mu);
    j.P->res.error = rc;
    j.status = QCS_ERROR;
    j.active = false;
}

void next_level(Job &j)
{
    j.k++;
    j.version++;
    j.launches = 0;
    j.in_version = 0;
    j.need_begin = true;
    if (j.k > j.P->k_max) {
        j.status = QCS_BUDGET_EXHAUSTED;
        j.active = false;
    }
}

// Exhaustive-pass work the job still has at its current level, in the
// streamed-point units of cert_advance (a point with the contraction against
// C^ counts four); 0 when it runs no pass.
uint64_t pass_work_left(const Job &j)
{
    const qcs_problem *P = j.P;
    const int k = j.cert ? j.cert->k : j.k;
    const uint64_t xi = (uint64_t)(P->D - 1), xi_h = upow(xi, k / 2);
    const bool v_heavy = (k & 1) && P->C.E >= 1;
    const uint64_t cs = v_heavy ? 4 : 1, cp = v_heavy ? 1 : 4;
    if (j.cert) return (xi_h - j.cert->stored) * cs + (j.cert->n_probe - j.cert->probed) * cp;
    const bool first =
        P->p.exhaustive_first && j.need_begin && j.launches == 0 && j.k != j.cert_skip_k && exhaustive_eligible(P, k);
    if (!first && !j.cert_after_walk) return 0;
    return xi_h * cs + xi_h * ((k & 1) ? xi : 1) * cp;
}

// The job's exhaustive passes: exhaustive_first settles each qualifying level
// by the pass alone, before any walk of it; a level whose walk budget ended
// without a claw is settled by the pass before the next level.  A pass runs
// for as much of *budget (streamed-point equivalents, see cert_advance) as
// it needs; if the budget runs out first the job is parked: it keeps its
// pass and is not walked this round.
int cert_work(qcs_batch *B, Job &j, uint64_t *budget)
{
    qcs_problem *P = j.P;
    j.parked = false;
    while (j.active) {
        if (!j.cert) {
            const bool first = P->p.exhaustive_first && j.need_begin && j.launches == 0 && j.k != j.cert_skip_k &&
                               exhaustive_eligible(P, j.k);
            if (!first && !j.cert_after_walk) return QCS_OK;
            if (*budget == 0) {
                j.parked = true;
                return QCS_OK;
            }
            j.cert = new (std::nothrow) CertPass();
            if (!j.cert) return QCS_ERR_NOMEM;
            const int rc = cert_begin(P, j.k, B->s, j.cert);
            if (rc != QCS_OK) {
                delete j.cert;
                j.cert = nullptr;
                if (rc == QCS_ERR_NOMEM && !j.cert_after_walk) { // no room for the table now: walk the level
                    j.cert_skip_k = j.k;
                    return QCS_OK;
                }
                j.cert_after_walk = false;
                if (rc == QCS_ERR_NOMEM) {
                    next_level(j);
                    continue;
                }
                job_error(j, rc);
                return QCS_OK;
            }
        }
        uint64_t used = 0;
        int rc = cert_advance(P, j.cert, B->s, *budget, &used);
        *budget -= std::min(used, *budget);
        if (rc != QCS_OK) {
            cert_end(P, j.cert, B->s);
            delete j.cert;
            j.cert = nullptr;
            job_error(j, rc);
            return QCS_OK;
        }
        if (!j.cert->done) {
            j.parked = true;
            return QCS_OK;
        }
        const bool claw = j.cert->got;
        rc = cert_end(P, j.cert, B->s);
        delete j.cert;
        j.cert = nullptr;
        const bool after_walk = j.cert_after_walk;
        j.cert_after_walk = false;
        if (claw) {
            j.status = QCS_FOUND;
            j.active = false;
            return QCS_OK;
        }
        if (rc == QCS_ERR_OVERFLOW && !after_walk) { // inconclusive: walk the level
            j.cert_skip_k = j.k;
            return QCS_OK;
        }
        if (rc != QCS_OK && rc != QCS_ERR_OVERFLOW) {
            job_error(j, rc);
            return QCS_OK;
        }
        next_level(j); // proved empty (or walked and inconclusive): the next level
    }
    return QCS_OK;
}

// start level j.k (or a new function version of it): plan, clear, seed walks
int begin_level(qcs_batch *B, Job &j, int slot)
{
    qcs_problem *P = j.P;
    if (j.launches == 0) j.pl = plan_level(P, j.k, j.jp);
    WalkLaunch &w = j.w;
    w = WalkLaunch{};
    w.lv = make_level(P, j.k, j.version, j.pl.dp_bits);
    w.walks = j.walks;
    w.n_walks = (int32_t)j.pl.walks;
    w.steps = j.pl.steps;
    w.max_len = (uint32_t)std::min<uint64_t>((uint64_t)j.jp.max_trail_factor << j.pl.dp_bits, kMaxTrailLen);
    w.table = j.table;
    w.table_mask = ((uint64_t)1 << j.jp.table_log2) - 1;
    w.queue = j.queue;
    w.qhead = B->dHeads + kHeads * slot;
    w.qcap = (uint32_t)j.jp.queue_capacity;
    w.cands = B->dCands + (size_t)slot * kBatchCandCap;
    w.ccount = B->dHeads + kHeads * slot + 1;
    w.ccap = kBatchCandCap;
    w.counters = B->dCounters + (size_t)slot * C_NCOUNTERS;
    cudaError_t e = cudaMemsetAsync(j.table, 0xFF, sizeof(Slot) << j.jp.table_log2, B->s);
    if (e == cudaSuccess) e = launch_init_walks(w, B->s);
    if (e != cudaSuccess) return fail(e);
    B->hJobs[slot] = w;
    j.in_version = 0;
    j.need_begin = false;
    j.pend_n = 0; // re-walks of the previous function version do not carry over
    std::lock_guard<std::mutex> g(P->mu);
    P->res.k = j.k;
    P->res.version = j.version;
    return QCS_OK;
}

// rebuild the per-class task and job lists of the active jobs
void build_tasks(qcs_batch *B)
{
    uint32_t nt[kClasses] = {0}, nj[kClasses] = {0};
    for (size_t slot = 0; slot < B->jobs.size(); slot++) {
        const Job &j = B->jobs[slot];
        if (!j.active || j.parked) continue;
        const int c = j.P->n;
        B->hIds[(size_t)c * B->bp.max_jobs + nj[c]++] = (uint32_t)slot;
        const int per = walks_per_task(c, B->bp.launch_shape[c - 1]);
        for (int first = 0; first < j.w.n_walks; first += per) {
            uint32_t *t = B->hTasks + (size_t)c * 2 * B->max_tasks + 2 * nt[c]++;
            t[0] = (uint32_t)slot;
            t[1] = (uint32_t)first;
        }
    }
    for (int c = 0; c < kClasses; c++) {
        B->hCounts[2 * c] = nt[c];
        B->hCounts[2 * c + 1] = nj[c];
    }
}

// the device work of one round, in stream order (captured into the graph)
int enqueue_round(qcs_batch *B)
{
    cudaStream_t s = B->s;
    const size_t J = (size_t)B->bp.max_jobs;
    cudaError_t e = cudaMemcpyAsync(B->dJobs, B->hJobs, sizeof(WalkLaunch) * J, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(B->dTasks, B->hTasks, sizeof(uint32_t) * kClasses * 2 * B->max_tasks,
                                cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(B->dIds, B->hIds, sizeof(uint32_t) * kClasses * J, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(B->dCounts, B->hCounts, sizeof(uint32_t) * kClasses * 2, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemsetAsync(B->dHeads, 0, sizeof(uint32_t) * kHeads * J, s);
    if (!e) e = cudaMemsetAsync(B->dCounters, 0, sizeof(unsigned long long) * C_NCOUNTERS * J, s);
    if (!e) e = cudaEventRecord(B->fork, s);
    for (int c = 1; c < kClasses && !e; c++) {
        BatchArgs a{B->dJobs, B->dTasks + (size_t)c * 2 * B->max_tasks, B->dCounts + 2 * c, B->dIds + (size_t)c * J,
                    B->dCounts + 2 * c + 1};
        e = cudaStreamWaitEvent(B->cs[c], B->fork, 0);
        if (!e) e = launch_walks_batch(c, B->bp.launch_shape[c - 1], a, B->cs[c]);
        if (!e) e = launch_rewalk_batch(c, a, B->cs[c]);
        if (!e) e = cudaEventRecord(B->join[c], B->cs[c]);
        if (!e) e = cudaStreamWaitEvent(s, B->join[c], 0);
    }
    if (!e) e = cudaMemcpyAsync(B->hCounters, B->dCounters, sizeof(unsigned long long) * C_NCOUNTERS * J,
                                cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(B->hHeads, B->dHeads, sizeof(uint32_t) * kHeads * J, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(B->hCands, B->dCands, sizeof(Cand) * kBatchCandCap * J, cudaMemcpyDeviceToHost, s);
    return e ? fail(e) : QCS_OK;
}

// fold one job's round into its result and advance its ladder
void collect_job(Job &j, const unsigned long long *c, const uint32_t *heads, const Cand *cands)
{
    qcs_problem *P = j.P;
    const int k = j.k, h = k / 2;
    const uint32_t npairs = std::min(heads[0], (uint32_t)j.jp.queue_capacity);
    // re-walks that ran out of budget resume from the other buffer next round
    const uint32_t carried = heads[2];
    j.pend_n = std::min(carried, (uint32_t)j.jp.queue_capacity);
    j.pp ^= 1;
    const uint32_t ncand = std::min(heads[1], kBatchCandCap);
    uint32_t paulis[16] = {0};
    PMat Dh;
    int64_t claws = 0, false_hash = 0;
    bool got = false;
    for (uint32_t i = 0; i < ncand && !got; i++) {
        const Cand &r = cands[i];
        const uint64_t xv = (r.a & 1) ? r.b : r.a, xw = (r.a & 1) ? r.a : r.b;
        uint32_t qv[kMaxH], qw[kMaxH];
        decode_state(xv, P->n, P->p.state_bits, h, qv);
        decode_state(xw, P->n, P->p.state_bits, h, qw);
        const int chunk = (k & 1) ? (int)r.chunk : 0;
        if (verify_claw(P, k, chunk, qv, qw, paulis, &Dh)) {
            claws++;
            got = true;
            continue;
        }
        false_hash++;
    }
    {
        std::lock_guard<std::mutex> g(P->mu);
        qcs_result &R = P->res;
        R.steps += (int64_t)c[C_STEPS];
        R.w_steps += (int64_t)c[C_WSTEPS];
        R.rewalk_steps += (int64_t)c[C_RSTEPS];
        R.dps += (int64_t)c[C_DPS];
        R.abandoned += (int64_t)c[C_ABANDONED];
        R.dropped += (int64_t)c[C_EVICTED];
        R.merges += (int64_t)npairs;
        R.queue_overflow += (int64_t)(c[C_PAIRS] - npairs) + (int64_t)(carried - j.pend_n);
        R.robin_hood += (int64_t)c[C_CLS0 + QCS_MERGE_ROBIN_HOOD];
        R.trivial += (int64_t)c[C_CLS0 + QCS_MERGE_TRIVIAL];
        R.same_side += (int64_t)c[C_CLS0 + QCS_MERGE_SAME_SIDE];
        R.no_merge += (int64_t)c[C_CLS0 + QCS_MERGE_NO_MERGE];
        R.claws += claws;
        R.false_hash += false_hash;
        R.launches += 1;
        R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - j.t0).count();
    }
    j.launches++;
    j.in_version++;
    if (got) {
        found(P, k, paulis, std::move(Dh));
        j.status = QCS_FOUND;
        j.active = false;
        return;
    }
    if (j.launches >= j.pl.min_launches) { // level exhausted: the next one
        if (exhaustive_eligible(P, k)) {
            // settle the level exactly before moving on (a claw the walk
            // missed): the pass runs from the next round on (cert_work)
            j.cert_after_walk = true;
            return;
        }
        next_level(j);
    } else if (j.in_version >= j.pl.launches_per_version) {
        j.version++;
        j.need_begin = true;
    }
}

void publish_status(Job &j)
{
    std::lock_guard<std::mutex> g(j.P->mu);
    j.P->res.status = j.status;
    j.P->res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - j.t0).count();
}

} // namespace

extern "C" {

void qcs_batch_default_params(qcs_batch_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->max_jobs = 512;
    p->walks_per_job = 2048;
    p->steps_per_round = 64;
    p->table_log2 = 18;
    p->queue_capacity = 1 << 16;
    p->use_graph = 1;
    p->rewalk_budget = 64;
}

int qcs_batch_create(const qcs_batch_params *pin, void *stream, qcs_batch **out)
{
    if (!out) return QCS_ERR_ARG;
    *out = nullptr;
    qcs_batch_params bp;
    if (pin) bp = *pin; else qcs_batch_default_params(&bp);
    if (bp.max_jobs < 1 || bp.max_jobs > 65536 || bp.walks_per_job < 16 ||
        (uint32_t)bp.walks_per_job > kMaxWalks || bp.walks_per_job % 16 || bp.steps_per_round < 1 ||
        bp.table_log2 < 4 || bp.table_log2 > 30 || bp.queue_capacity < 16 || bp.rewalk_budget < 0)
        return QCS_ERR_ARG;
    for (int n = 1; n <= 4; n++)
        if (bp.launch_shape[n - 1] < 0 || bp.launch_shape[n - 1] >= launch_shapes(n)) return QCS_ERR_ARG;
    if (bp.cert_points_log2 < 0 || bp.cert_points_log2 > 40) return QCS_ERR_ARG;
    qcs_batch *B = new (std::nothrow) qcs_batch();
    if (!B) return QCS_ERR_NOMEM;
    B->bp = bp;
    B->s = (cudaStream_t)stream;
    if (!B->s) {
        if (cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking) != cudaSuccess) {
            delete B;
            return QCS_ERR_CUDA;
        }
        B->own_stream = true;
    }
    cudaError_t es = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    for (int c = 1; c < kClasses && es == cudaSuccess; c++) {
        es = cudaStreamCreateWithFlags(&B->cs[c], cudaStreamNonBlocking);
        if (es == cudaSuccess) es = cudaEventCreateWithFlags(&B->join[c], cudaEventDisableTiming);
    }
    if (es != cudaSuccess) {
        qcs_batch_destroy(B);
        return QCS_ERR_CUDA;
    }
    B->jobs.resize((size_t)bp.max_jobs);
    B->max_tasks = (uint32_t)bp.max_jobs * ((uint32_t)bp.walks_per_job / 8); // at least 8 walks per task
    const size_t J = (size_t)bp.max_jobs;
    cudaError_t e = cudaSuccess;
    auto dev = [&](void **p, size_t bytes) { if (!e) e = cudaMalloc(p, bytes); };
    auto pin_ = [&](void **p, size_t bytes) {
        if (!e) e = cudaMallocHost(p, bytes);
        if (!e) memset(*p, 0, bytes);
    };
    dev((void **)&B->dJobs, sizeof(WalkLaunch) * J);
    pin_((void **)&B->hJobs, sizeof(WalkLaunch) * J);
    dev((void **)&B->dCounters, sizeof(unsigned long long) * C_NCOUNTERS * J);
    pin_((void **)&B->hCounters, sizeof(unsigned long long) * C_NCOUNTERS * J);
    dev((void **)&B->dHeads, sizeof(uint32_t) * kHeads * J);
    pin_((void **)&B->hHeads, sizeof(uint32_t) * kHeads * J);
    dev((void **)&B->dCands, sizeof(Cand) * kBatchCandCap * J);
    pin_((void **)&B->hCands, sizeof(Cand) * kBatchCandCap * J);
    dev((void **)&B->dTasks, sizeof(uint32_t) * kClasses * 2 * B->max_tasks);
    pin_((void **)&B->hTasks, sizeof(uint32_t) * kClasses * 2 * B->max_tasks);
    dev((void **)&B->dIds, sizeof(uint32_t) * kClasses * J);
    pin_((void **)&B->hIds, sizeof(uint32_t) * kClasses * J);
    dev((void **)&B->dCounts, sizeof(uint32_t) * kClasses * 2);
    pin_((void **)&B->hCounts, sizeof(uint32_t) * kClasses * 2);
    if (e) {
        qcs_batch_destroy(B);
        return e == cudaErrorMemoryAllocation ? QCS_ERR_NOMEM : fail(e);
    }
    *out = B;
    return QCS_OK;
}

uint64_t qcs_batch_job_bytes(const qcs_batch *B, const qcs_problem *P)
{
    if (!B || !P) return 0;
    const size_t D = (size_t)P->D;
    return job_bytes(B->bp) + D * D * sizeof(uint2) + D * sizeof(uint2) + D * 2 * 8 * sizeof(uint32_t);
}

int qcs_batch_add(qcs_batch *B, qcs_problem *P, int *job)
{
    if (!B || !P || !job) return QCS_ERR_ARG;
    int slot = -1;
    for (size_t i = 0; i < B->jobs.size(); i++)
        if (!B->jobs[i].used) {
            slot = (int)i;
            break;
        }
    if (slot < 0) return QCS_ERR_BUSY;
    {
        std::lock_guard<std::mutex> g(P->mu);
        if (P->running) return QCS_ERR_BUSY;
        const int sde = P->res.sde;
        const int64_t h2d = P->res.h2d_bytes, d2h = P->res.d2h_bytes; // kept for the problem's lifetime
        memset(&P->res, 0, sizeof P->res);
        P->res.h2d_bytes = h2d;
        P->res.d2h_bytes = d2h;
        P->res.sde = sde;
        P->res.t_count = -1;
        P->res.status = QCS_SEARCHING;
        P->have_D = false;
        P->t0 = std::chrono::steady_clock::now();
    }
    Job &j = B->jobs[(size_t)slot];
    j = Job();
    j.P = P;
    j.used = true;
    j.jp = P->p;
    j.jp.walks = B->bp.walks_per_job;
    j.jp.steps_per_launch = B->bp.steps_per_round;
    j.jp.table_log2 = B->bp.table_log2;
    j.jp.queue_capacity = B->bp.queue_capacity;
    j.t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaMalloc(&j.walks, sizeof(WalkState) * (size_t)j.jp.walks);
    if (!e) e = cudaMalloc(&j.table, sizeof(Slot) << j.jp.table_log2);
    if (!e) e = cudaMalloc(&j.queue, sizeof(Pair) * (size_t)j.jp.queue_capacity);
    if (!e) e = cudaMalloc(&j.pend[0], sizeof(Pending) * (size_t)j.jp.queue_capacity);
    if (!e) e = cudaMalloc(&j.pend[1], sizeof(Pending) * (size_t)j.jp.queue_capacity);
    if (e) {
        free_job(j, B->s);
        return e == cudaErrorMemoryAllocation ? QCS_ERR_NOMEM : fail(e);
    }
    j.seq = B->next_seq++;
    j.k = P->C.E;
    j.active = true;
    j.status = QCS_SEARCHING;
    settle_small_levels(j);
    if (!j.active) publish_status(j);
    *job = slot;
    return QCS_OK;
}

int qcs_batch_remove(qcs_batch *B, int job)
{
    if (!B || job < 0 || job >= (int)B->jobs.size() || !B->jobs[(size_t)job].used) return QCS_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(B->s);
    Job &j = B->jobs[(size_t)job];
    if (j.active) {
        j.status = QCS_CANCELLED;
        publish_status(j);
    }
    memset(&B->hJobs[job], 0, sizeof(WalkLaunch));
    free_job(j, B->s);
    return e ? fail(e) : QCS_OK;
}

int qcs_batch_round(qcs_batch *B, int *n_active)
{
    if (!B) return QCS_ERR_ARG;
    int rc;
    int active = 0, parked = 0;
    // 1. exhaustive passes within the round's share, the job with the least
    //    pass work left first (ties: the oldest), so that a long pass does
    //    not hold back the short passes of jobs that arrived after it
    {
        std::vector<std::pair<uint64_t, size_t>> order;
        for (size_t slot = 0; slot < B->jobs.size(); slot++)
            if (B->jobs[slot].active) order.push_back({pass_work_left(B->jobs[slot]), slot});
        std::sort(order.begin(), order.end(), [B](const std::pair<uint64_t, size_t> &x,
                                                 const std::pair<uint64_t, size_t> &y) {
            return x.first != y.first ? x.first < y.first : B->jobs[x.second].seq < B->jobs[y.second].seq;
        });
        uint64_t budget = B->bp.cert_points_log2 > 0 ? (1ull << B->bp.cert_points_log2) : ~0ull;
        for (const auto &o : order) {
            const size_t slot = o.second;
            Job &j = B->jobs[slot];
            if ((rc = cert_work(B, j, &budget))) return rc;
            if (!j.active) { // settled by its pass
                publish_status(j);
                memset(&B->hJobs[slot], 0, sizeof(WalkLaunch));
            }
        }
    }
    // 2. the walkers
    for (size_t slot = 0; slot < B->jobs.size(); slot++) {
        Job &j = B->jobs[slot];
        if (!j.active) continue;
        if (j.parked) {
            parked++;
            memset(&B->hJobs[slot], 0, sizeof(WalkLaunch));
            continue;
        }
        if (j.need_begin && (rc = begin_level(B, j, (int)slot))) return rc;
        // this round's re-walk budget and the carried re-walks it resumes
        WalkLaunch &w = B->hJobs[slot];
        w.rewalk_budget = (uint32_t)B->bp.rewalk_budget;
        w.pend_cap = (uint32_t)j.jp.queue_capacity;
        w.pend_in = j.pend[j.pp];
        w.pend_in_n = j.pend_n;
        w.pend_out = j.pend[j.pp ^ 1];
        w.pend_out_n = B->dHeads + kHeads * slot + 2;
        active++;
    }
    if (n_active) *n_active = active + parked;
    if (!active) return QCS_OK;
    build_tasks(B);
    if (B->bp.use_graph) {
        if (!B->exec) {
            cudaError_t e = cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal);
            if (e) return fail(e);
            rc = enqueue_round(B);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(B->s, &g);
            if (rc) return rc;
            if (e) return fail(e);
            B->graph = g;
            e = cudaGraphInstantiate(&B->exec, g, 0);
            if (e) return fail(e);
        }
        cudaError_t e = cudaGraphLaunch(B->exec, B->s);
        if (e) return fail(e);
    } else if ((rc = enqueue_round(B))) {
        return rc;
    }
    cudaError_t e = cudaStreamSynchronize(B->s);
    if (e) return fail(e);
    B->rounds++;
    active = 0;
    for (size_t slot = 0; slot < B->jobs.size(); slot++) {
        Job &j = B->jobs[slot];
        if (!j.active || j.parked) continue;
        collect_job(j, B->hCounters + slot * C_NCOUNTERS, B->hHeads + kHeads * slot,
                    B->hCands + slot * kBatchCandCap);
        if (!j.active) {
            publish_status(j);
            memset(&B->hJobs[slot], 0, sizeof(WalkLaunch));
        } else {
            active++;
        }
    }
    if (n_active) *n_active = active + parked;
    return QCS_OK;
}

int qcs_batch_poll(qcs_batch *B, int job, qcs_result *out)
{
    if (!B || !out || job < 0 || job >= (int)B->jobs.size() || !B->jobs[(size_t)job].used) return QCS_ERR_ARG;
    Job &j = B->jobs[(size_t)job];
    std::lock_guard<std::mutex> g(j.P->mu);
    *out = j.P->res;
    out->status = j.status;
    return QCS_OK;
}

void qcs_batch_destroy(qcs_batch *B)
{
    if (!B) return;
    if (B->s) cudaStreamSynchronize(B->s);
    for (Job &j : B->jobs)
        if (j.used) free_job(j, B->s);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    cudaFree(B->dJobs); cudaFreeHost(B->hJobs);
    cudaFree(B->dCounters); cudaFreeHost(B->hCounters);
    cudaFree(B->dHeads); cudaFreeHost(B->hHeads);
    cudaFree(B->dCands); cudaFreeHost(B->hCands);
    cudaFree(B->dTasks); cudaFreeHost(B->hTasks);
    cudaFree(B->dIds); cudaFreeHost(B->hIds);
    cudaFree(B->dCounts); cudaFreeHost(B->hCounts);
    for (int c = 1; c < kClasses; c++) {
        if (B->cs[c]) cudaStreamDestroy(B->cs[c]);
        if (B->join[c]) cudaEventDestroy(B->join[c]);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->own_stream) cudaStreamDestroy(B->s);
    delete B;
}

} // extern "C"
