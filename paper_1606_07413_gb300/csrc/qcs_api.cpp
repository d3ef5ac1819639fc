// qcs_api.cpp -- the C ABI of libqcs (include/qcs.h): problem set-up, the
// T-count ladder driver, polling, exact verification and the raw step entry.
//
// Host-side roles (Fig. 4 of the paper, mapped onto one GPU): the workers and
// collectors are device warps (walk kernel + distinguished-point table), the
// verifiers are the re-walk kernel plus the exact claw check here.  One
// library-owned host thread per running search drives the launches on the
// caller's stream so that qcs_run_walks never blocks.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>

#include "qcs.h"
#include "qcs_internal.h"

using namespace qcs;

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e)
{
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s", cudaGetErrorString(e));
    return QCS_ERR_CUDA;
}
#define CK(call)                                                                                                     \
    do {                                                                                                             \
        cudaError_t _e = (call);                                                                                     \
        if (_e != cudaSuccess) return cuda_fail(_e);                                                                 \
    } while (0)

uint64_t smix_host(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t upow(uint64_t b, int e)
{
    uint64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

bool params_ok(int n, int k_max, const qcs_params &p)
{
    if (n < 1 || n > 4 || k_max < 0 || k_max > 15) return false;
    if (p.state_bits < 16 || p.state_bits > 64) return false;
    if (p.dp_bits < 1 || p.dp_bits >= p.state_bits) return false;
    if (p.walks < 1 || p.table_log2 < 4 || p.table_log2 > 32) return false;
    if (p.steps_per_launch < 1 || p.max_trail_factor < 1 || p.queue_capacity < 1) return false;
    if (p.budget_factor < 0 || p.version_factor < 0) return false;
    // the rotation index needs room below the state's top bits
    const uint64_t xi = (1u << (2 * n)) - 1;
    const int h = k_max / 2;
    long double span = 1;
    for (int j = 0; j < h; j++) span *= (long double)xi;
    long double room = 1;
    for (int j = 0; j < p.state_bits - 1; j++) room *= 2;
    return span * 16 <= room;
}

} // namespace

struct qcs_problem {
    int n = 0, D = 0, k_max = 0, device = 0;
    qcs_params p{};
    PMat C; // reduced, exponent = sde
    // device data
    uint2 *dC32 = nullptr, *dU = nullptr;
    Slot *dTable = nullptr;
    Pair *dQueue = nullptr;
    uint32_t *dQhead = nullptr;
    WalkState *dWalks = nullptr;
    unsigned long long *dCounters = nullptr;
    RewalkOut *dOut = nullptr;
    // pinned host mirrors
    unsigned long long *hCounters = nullptr;
    RewalkOut *hOut = nullptr;
    uint32_t *hQhead = nullptr;
    // search state
    std::thread driver;
    std::mutex mu;
    std::condition_variable cv;
    std::atomic<bool> cancel{false};
    bool running = false;
    qcs_result res{};
    std::chrono::steady_clock::time_point t0;
    PMat Dhat;
    bool have_D = false;
};

namespace {

LevelCtx make_level(const qcs_problem *P, int k, uint32_t version, int dp_bits)
{
    LevelCtx lv{};
    lv.C32 = P->dC32;
    lv.U = P->dU;
    lv.n = P->n;
    lv.k = k;
    lv.h = k / 2;
    lv.xi = (uint32_t)(P->D - 1);
    lv.xi_h = upow(lv.xi, lv.h);
    lv.K = P->C.E + (k & 1) + lv.h;
    lv.ev = lv.K - lv.h;
    lv.maskL = P->p.state_bits >= 64 ? ~0ull : ((1ull << P->p.state_bits) - 1);
    lv.dshift = P->p.state_bits - dp_bits;
    lv.version = version;
    return lv;
}

int upload_problem(qcs_problem *P)
{
    const int D = P->D;
    std::vector<uint2> c32((size_t)D * D), u(D);
    for (size_t i = 0; i < c32.size(); i++)
        c32[i] = make_uint2((uint32_t)(uint64_t)P->C.a[i], (uint32_t)(uint64_t)P->C.b[i]);
    // fingerprint weights: the SplitMix64 stream seeded with kSeedU, outputs
    // 2i and 2i+1 give (Ua[i], Ub[i]); row 0 (the identity) gets zero weight
    u[0] = make_uint2(0, 0);
    for (int i = 1; i < D; i++) {
        uint64_t wa = smix_host(kSeedU + (2ull * i + 1) * kGamma);
        uint64_t wb = smix_host(kSeedU + (2ull * i + 2) * kGamma);
        u[i] = make_uint2((uint32_t)wa, (uint32_t)wb);
    }
    CK(cudaGetDevice(&P->device));
    CK(cudaMalloc(&P->dC32, sizeof(uint2) * c32.size()));
    CK(cudaMalloc(&P->dU, sizeof(uint2) * D));
    CK(cudaMemcpy(P->dC32, c32.data(), sizeof(uint2) * c32.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->dU, u.data(), sizeof(uint2) * D, cudaMemcpyHostToDevice));
    return QCS_OK;
}

int ensure_search_buffers(qcs_problem *P)
{
    if (P->dTable) return QCS_OK;
    const size_t slots = (size_t)1 << P->p.table_log2;
    CK(cudaMalloc(&P->dTable, sizeof(Slot) * slots));
    CK(cudaMalloc(&P->dQueue, sizeof(Pair) * (size_t)P->p.queue_capacity));
    CK(cudaMalloc(&P->dQhead, sizeof(uint32_t)));
    CK(cudaMalloc(&P->dWalks, sizeof(WalkState) * (size_t)P->p.walks));
    CK(cudaMalloc(&P->dCounters, sizeof(unsigned long long) * C_NCOUNTERS));
    CK(cudaMalloc(&P->dOut, sizeof(RewalkOut) * (size_t)P->p.queue_capacity));
    CK(cudaMallocHost(&P->hCounters, sizeof(unsigned long long) * C_NCOUNTERS));
    CK(cudaMallocHost(&P->hOut, sizeof(RewalkOut) * (size_t)P->p.queue_capacity));
    CK(cudaMallocHost(&P->hQhead, sizeof(uint32_t)));
    return QCS_OK;
}

void free_problem_memory(qcs_problem *P)
{
    cudaFree(P->dC32); cudaFree(P->dU); cudaFree(P->dTable); cudaFree(P->dQueue); cudaFree(P->dQhead);
    cudaFree(P->dWalks); cudaFree(P->dCounters); cudaFree(P->dOut);
    cudaFreeHost(P->hCounters); cudaFreeHost(P->hOut); cudaFreeHost(P->hQhead);
}

int finish_create(int n, int k_max, const qcs_params *pin, PMat &&C, qcs_problem **out)
{
    qcs_params p;
    if (pin) p = *pin; else qcs_default_params(n, &p);
    if (!params_ok(n, k_max, p)) return QCS_ERR_ARG;
    qcs_problem *P = new (std::nothrow) qcs_problem();
    if (!P) return QCS_ERR_NOMEM;
    P->n = n;
    P->D = 1 << (2 * n);
    P->k_max = k_max;
    P->p = p;
    P->C = std::move(C);
    exact_reduce(&P->C);
    P->res.t_count = -1;
    P->res.sde = P->C.E;
    int rc = upload_problem(P);
    if (rc != QCS_OK) {
        free_problem_memory(P);
        delete P;
        return rc;
    }
    *out = P;
    return QCS_OK;
}

// levels 0 and 1 need no walk: C^ itself, or R^(c)^T C^ for one c, is Clifford
bool small_level(qcs_problem *P, int k, uint32_t *paulis)
{
    if (k == 0) return exact_is_clifford(P->C);
    for (uint32_t c = 1; c < (uint32_t)P->D; c++) {
        paulis[0] = c;
        if (exact_verify(P->n, P->C, paulis, 1, nullptr) == QCS_OK) return true;
    }
    return false;
}

void set_status(qcs_problem *P, int status, int error)
{
    std::lock_guard<std::mutex> g(P->mu);
    P->res.status = status;
    P->res.error = error;
    P->res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - P->t0).count();
}

void found(qcs_problem *P, int k, const uint32_t *paulis)
{
    PMat Dh;
    exact_verify(P->n, P->C, paulis, k, &Dh);
    std::lock_guard<std::mutex> g(P->mu);
    P->res.t_count = k;
    P->res.k = k;
    for (int j = 0; j < 16; j++) P->res.paulis[j] = j < k ? paulis[j] : 0;
    P->Dhat = std::move(Dh);
    P->have_D = true;
}

// the search driver: levels sde .. k_max, walks until a verified claw
int drive(qcs_problem *P, uint64_t budget, cudaStream_t s)
{
    CK(cudaSetDevice(P->device));
    int rc = ensure_search_buffers(P);
    if (rc) return rc;
    uint64_t total_steps = 0;
    uint32_t version = 0;
    for (int k = P->C.E; k <= P->k_max; k++) {
        {
            std::lock_guard<std::mutex> g(P->mu);
            P->res.k = k;
        }
        uint32_t paulis[16] = {0};
        if (k <= 1) {
            if (small_level(P, k, paulis)) {
                found(P, k, paulis);
                return QCS_OK;
            }
            continue;
        }
        const int h = k / 2;
        const uint64_t xi = (uint64_t)(P->D - 1);
        const uint64_t n_chunks = (k & 1) ? xi : 1;
        const long double points = 2.0L * (long double)upow(xi, h) * (long double)n_chunks;
        int dp_bits = P->p.dp_bits;
        if (P->p.theta_policy == 1) {
            // keep theta * points within half the table, theta as large as 1/2
            const long double slots = (long double)((uint64_t)1 << P->p.table_log2);
            int d = 1;
            while (d < P->p.dp_bits && points / (long double)((uint64_t)1 << d) > slots / 2) d++;
            dp_bits = d;
        }
        const uint64_t max_len = (uint64_t)P->p.max_trail_factor << dp_bits;
        const long double level_budget_ld = (long double)P->p.budget_factor * points;
        const uint64_t level_budget = level_budget_ld > 1.8e19L ? ~0ull : (uint64_t)level_budget_ld;
        const long double vp = (long double)P->p.version_factor * points;
        const uint64_t version_period = P->p.version_factor == 0 ? ~0ull : (vp > 1.8e19L ? ~0ull : (uint64_t)vp);

        WalkLaunch w{};
        w.walks = P->dWalks;
        w.n_walks = P->p.walks;
        w.n_chunks = (int32_t)((k & 1) ? xi : 0);
        w.steps = (uint32_t)P->p.steps_per_launch;
        w.max_len = (uint32_t)std::min<uint64_t>(max_len, 0xFFFFFFF0ull);
        w.seed = P->p.seed;
        w.table = P->dTable;
        w.table_mask = ((uint64_t)1 << P->p.table_log2) - 1;
        w.queue = P->dQueue;
        w.qhead = P->dQhead;
        w.qcap = (uint32_t)P->p.queue_capacity;
        w.counters = P->dCounters;

        uint64_t level_steps = 0, version_steps = 0;
        bool fresh = true;
        while (true) {
            if (P->cancel.load()) return QCS_ERR_BUSY; // reported as CANCELLED
            if (fresh) {
                w.lv = make_level(P, k, version, dp_bits);
                CK(cudaMemsetAsync(P->dTable, 0xFF, sizeof(Slot) << P->p.table_log2, s));
                CK(launch_init_walks(w, s));
                fresh = false;
                std::lock_guard<std::mutex> g(P->mu);
                P->res.version = version;
            }
            CK(cudaMemsetAsync(P->dQhead, 0, sizeof(uint32_t), s));
            CK(cudaMemsetAsync(P->dCounters, 0, sizeof(unsigned long long) * C_NCOUNTERS, s));
            CK(launch_walks(w, s));
            CK(launch_rewalk_pairs(w.lv, P->dQueue, P->dQhead, w.qcap, P->dOut, s));
            CK(cudaMemcpyAsync(P->hCounters, P->dCounters, sizeof(unsigned long long) * C_NCOUNTERS,
                               cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(P->hQhead, P->dQhead, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(P->hOut, P->dOut, sizeof(RewalkOut) * w.qcap, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const uint32_t npairs = std::min(*P->hQhead, w.qcap);
            int64_t cls_count[6] = {0, 0, 0, 0, 0, 0};
            bool got = false;
            for (uint32_t i = 0; i < npairs && !got; i++) {
                const RewalkOut &r = P->hOut[i];
                int cls = r.cls;
                if (cls == QCS_MERGE_CLAW) {
                    // exact check of the candidate: the V point and the W point
                    const uint64_t xv = (r.a & 1) ? r.b : r.a, xw = (r.a & 1) ? r.a : r.b;
                    uint64_t rv = (xv >> 1) % w.lv.xi_h, rw = (xw >> 1) % w.lv.xi_h;
                    uint32_t qv[kMaxH], qw[kMaxH];
                    for (int j = 0; j < h; j++) {
                        qv[j] = (uint32_t)(rv % xi) + 1; rv /= xi;
                        qw[j] = (uint32_t)(rw % xi) + 1; rw /= xi;
                    }
                    const int chunk = (k & 1) ? (int)r.chunk : 0;
                    bool equal = false;
                    if (exact_same_coset(P->n, P->C, k, chunk, qv, qw, &equal) != QCS_OK) equal = false;
                    if (equal) {
                        for (int j = 0; j < h; j++) { paulis[j] = qv[j]; paulis[h + j] = qw[j]; }
                        if (k & 1) paulis[2 * h] = (uint32_t)chunk;
                        if (exact_verify(P->n, P->C, paulis, k, nullptr) == QCS_OK) got = true;
                        else cls = QCS_MERGE_FALSE_HASH;
                    } else {
                        cls = QCS_MERGE_FALSE_HASH;
                    }
                }
                if (cls >= 0 && cls < 6) cls_count[cls]++;
            }
            const unsigned long long *c = P->hCounters;
            total_steps += c[C_STEPS];
            level_steps += c[C_STEPS];
            version_steps += c[C_STEPS];
            {
                std::lock_guard<std::mutex> g(P->mu);
                qcs_result &R = P->res;
                R.steps += (int64_t)c[C_STEPS];
                R.dps += (int64_t)c[C_DPS];
                R.abandoned += (int64_t)c[C_ABANDONED];
                R.dropped += (int64_t)c[C_DROPPED];
                R.merges += (int64_t)npairs;
                R.queue_overflow += (int64_t)(c[C_PAIRS] - npairs);
                R.robin_hood += cls_count[0];
                R.trivial += cls_count[1];
                R.same_side += cls_count[2];
                R.claws += cls_count[3];
                R.false_hash += cls_count[4];
                R.no_merge += cls_count[5];
                R.launches += 1;
                R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - P->t0).count();
            }
            if (c[C_WAIT_TIMEOUT]) return QCS_ERR_DEVICE;
            if (got) {
                found(P, k, paulis);
                return QCS_OK;
            }
            if (budget && total_steps >= budget) return QCS_ERR_TIMEOUT; // reported as BUDGET_EXHAUSTED
            if (level_steps >= level_budget) break;
            if (version_steps >= version_period) {
                version++;
                version_steps = 0;
                fresh = true;
            }
        }
    }
    return QCS_ERR_TIMEOUT;
}

void driver_main(qcs_problem *P, uint64_t budget, cudaStream_t s)
{
    int rc = drive(P, budget, s);
    int status;
    if (rc == QCS_OK) status = QCS_FOUND;
    else if (rc == QCS_ERR_TIMEOUT) status = QCS_BUDGET_EXHAUSTED;
    else if (rc == QCS_ERR_BUSY && P->cancel.load()) status = QCS_CANCELLED;
    else status = QCS_ERROR;
    set_status(P, status, status == QCS_ERROR ? rc : 0);
    std::lock_guard<std::mutex> g(P->mu);
    P->running = false;
    P->cv.notify_all();
}

} // namespace

extern "C" {

void qcs_default_params(int n_qubits, qcs_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    switch (n_qubits) {
    case 1:
    case 2: p->state_bits = 32; p->dp_bits = 6; p->walks = 4096; p->table_log2 = 16; break;
    case 3: p->state_bits = 48; p->dp_bits = 10; p->walks = 1 << 16; p->table_log2 = 22; break;
    default: p->state_bits = 64; p->dp_bits = 12; p->walks = 1 << 20; p->table_log2 = 26; break;
    }
    p->steps_per_launch = 64;
    p->max_trail_factor = 20;
    p->queue_capacity = 4096;
    p->budget_factor = 8;
    p->theta_policy = 1;
    p->version_factor = 2;
    p->seed = 0x2545F4914F6CDD1Dull;
}

int qcs_create_problem(int n, const int64_t *target, int32_t target_exp, int k_max, const qcs_params *p,
                       qcs_problem **out)
{
    if (!out || !target || n < 1 || n > 4) return QCS_ERR_ARG;
    *out = nullptr;
    PMat C;
    int rc = exact_channel_from_unitary(n, target, target_exp, &C);
    if (rc) return rc;
    return finish_create(n, k_max, p, std::move(C), out);
}

int qcs_create_problem_channel(int n, const int64_t *chan_ab, int32_t exp, int k_max, const qcs_params *p,
                               qcs_problem **out)
{
    if (!out || !chan_ab || n < 1 || n > 4 || exp < 0) return QCS_ERR_ARG;
    *out = nullptr;
    const int D = 1 << (2 * n);
    PMat C;
    C.D = D;
    C.E = exp;
    C.a.resize((size_t)D * D);
    C.b.resize((size_t)D * D);
    for (size_t i = 0; i < (size_t)D * D; i++) {
        C.a[i] = chan_ab[2 * i];
        C.b[i] = chan_ab[2 * i + 1];
    }
    exact_reduce(&C);
    int rc = exact_check_channel(n, C);
    if (rc) return rc;
    // row and column 0 must be e_0 (the identity Pauli is fixed)
    for (int i = 1; i < D; i++)
        if (C.a[i] || C.b[i] || C.a[(size_t)i * D] || C.b[(size_t)i * D]) return QCS_ERR_NOT_UNITARY;
    return finish_create(n, k_max, p, std::move(C), out);
}

int qcs_create_problem_circuit(int n, const int32_t *gates, int n_gates, int k_max, const qcs_params *p,
                               qcs_problem **out)
{
    if (!out || n < 1 || n > 4) return QCS_ERR_ARG;
    *out = nullptr;
    std::vector<int64_t> u;
    int e = 0;
    int rc = exact_unitary_from_circuit(n, gates, n_gates, &u, &e);
    if (rc) return rc;
    return qcs_create_problem(n, u.data(), e, k_max, p, out);
}

int qcs_run_walks(qcs_problem *P, uint64_t step_budget, void *stream)
{
    if (!P) return QCS_ERR_ARG;
    std::unique_lock<std::mutex> g(P->mu);
    if (P->running) return QCS_ERR_BUSY;
    if (P->driver.joinable()) {
        g.unlock();
        P->driver.join();
        g.lock();
    }
    P->running = true;
    P->cancel = false;
    const int sde = P->res.sde;
    memset(&P->res, 0, sizeof P->res);
    P->res.status = QCS_SEARCHING;
    P->res.t_count = -1;
    P->res.sde = sde;
    P->have_D = false;
    P->t0 = std::chrono::steady_clock::now();
    try {
        P->driver = std::thread(driver_main, P, step_budget, (cudaStream_t)stream);
    } catch (...) {
        P->running = false;
        P->res.status = QCS_ERROR;
        return QCS_ERR_NOMEM;
    }
    return QCS_OK;
}

int qcs_poll_collisions(qcs_problem *P, qcs_result *out)
{
    if (!P || !out) return QCS_ERR_ARG;
    std::lock_guard<std::mutex> g(P->mu);
    *out = P->res;
    if (P->running)
        out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - P->t0).count();
    return QCS_OK;
}

int qcs_wait(qcs_problem *P, int64_t timeout_ms, qcs_result *out)
{
    if (!P) return QCS_ERR_ARG;
    std::unique_lock<std::mutex> g(P->mu);
    auto done = [&] { return !P->running; };
    if (timeout_ms < 0) P->cv.wait(g, done);
    else if (!P->cv.wait_for(g, std::chrono::milliseconds(timeout_ms), done)) {
        if (out) *out = P->res;
        return QCS_ERR_TIMEOUT;
    }
    if (out) *out = P->res;
    return QCS_OK;
}

int qcs_cancel(qcs_problem *P)
{
    if (!P) return QCS_ERR_ARG;
    P->cancel = true;
    return QCS_OK;
}

int qcs_get_clifford(qcs_problem *P, int32_t *perm, int8_t *sign)
{
    if (!P || !perm || !sign) return QCS_ERR_ARG;
    std::lock_guard<std::mutex> g(P->mu);
    if (!P->have_D) return QCS_ERR_ARG;
    const int D = P->D;
    for (int c = 0; c < D; c++)
        for (int r = 0; r < D; r++) {
            int64_t a = P->Dhat.a[(size_t)r * D + c];
            if (a) {
                perm[c] = r;
                sign[c] = (int8_t)(a > 0 ? 1 : -1);
            }
        }
    return QCS_OK;
}

int qcs_verify_decomposition(int n, const int64_t *target, int32_t target_exp, const uint32_t *paulis, int t)
{
    if (n < 1 || n > 4 || !target || t < 0 || (t > 0 && !paulis)) return QCS_ERR_ARG;
    for (int j = 0; j < t; j++)
        if (paulis[j] == 0 || paulis[j] >= (1u << (2 * n))) return QCS_ERR_ARG;
    PMat C;
    int rc = exact_channel_from_unitary(n, target, target_exp, &C);
    if (rc) return rc;
    return exact_verify(n, C, paulis, t, nullptr);
}

int qcs_walk_step(qcs_problem *P, int k, int chunk, uint32_t version, const uint64_t *in, uint64_t *out,
                  uint8_t *is_dp, size_t count, void *stream)
{
    if (!P || k < 0 || k > P->k_max) return QCS_ERR_ARG;
    if ((k & 1) ? (chunk < 1 || chunk >= P->D) : (chunk != 0)) return QCS_ERR_ARG;
    if (count && (!in || !out)) return QCS_ERR_ARG;
    LevelCtx lv = make_level(P, k, version, P->p.dp_bits);
    cudaError_t e = launch_walk_step(lv, chunk, in, out, is_dp, count, (cudaStream_t)stream);
    return e == cudaSuccess ? QCS_OK : cuda_fail(e);
}

int qcs_rewalk(qcs_problem *P, int k, int chunk, uint32_t version, const uint64_t *start_a, const uint32_t *len_a,
               const uint64_t *start_b, const uint32_t *len_b, size_t count, int32_t *cls, uint64_t *ab,
               void *stream)
{
    if (!P || k < 0 || k > P->k_max) return QCS_ERR_ARG;
    if ((k & 1) ? (chunk < 1 || chunk >= P->D) : (chunk != 0)) return QCS_ERR_ARG;
    if (count && (!start_a || !len_a || !start_b || !len_b || !cls || !ab)) return QCS_ERR_ARG;
    LevelCtx lv = make_level(P, k, version, P->p.dp_bits);
    cudaError_t e = launch_rewalk_arrays(lv, chunk, start_a, len_a, start_b, len_b, count, cls, ab,
                                         (cudaStream_t)stream);
    return e == cudaSuccess ? QCS_OK : cuda_fail(e);
}

int qcs_problem_sde(const qcs_problem *P) { return P ? P->C.E : -1; }

uint64_t qcs_level_points(const qcs_problem *P, int k)
{
    if (!P || k < 0) return 0;
    return 2 * upow((uint64_t)(P->D - 1), k / 2);
}

int qcs_get_channel(const qcs_problem *P, int64_t *a, int64_t *b, int32_t *exp)
{
    if (!P || !a || !b || !exp) return QCS_ERR_ARG;
    memcpy(a, P->C.a.data(), sizeof(int64_t) * P->C.a.size());
    memcpy(b, P->C.b.data(), sizeof(int64_t) * P->C.b.size());
    *exp = P->C.E;
    return QCS_OK;
}

void qcs_destroy_problem(qcs_problem *P)
{
    if (!P) return;
    P->cancel = true;
    if (P->driver.joinable()) P->driver.join();
    cudaDeviceSynchronize();
    free_problem_memory(P);
    delete P;
}

const char *qcs_strerror(int code)
{
    switch (code) {
    case QCS_OK: return "ok";
    case QCS_ERR_ARG: return "invalid argument";
    case QCS_ERR_NOT_UNITARY: return "target is not an exact unitary";
    case QCS_ERR_NOMEM: return "out of memory";
    case QCS_ERR_CUDA: return "CUDA error";
    case QCS_ERR_MISMATCH: return "decomposition does not reproduce the target";
    case QCS_ERR_OVERFLOW: return "exact arithmetic overflow";
    case QCS_ERR_BUSY: return "a search is already running";
    case QCS_ERR_TIMEOUT: return "timed out";
    case QCS_ERR_DEVICE: return "a device-side bounded wait gave up";
    default: return "unknown status";
    }
}

const char *qcs_last_cuda_error(void) { return g_cuda_err; }

} // extern "C"
