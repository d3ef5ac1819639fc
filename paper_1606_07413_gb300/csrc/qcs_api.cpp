// qcs_api.cpp -- the C ABI of libqcs (include/qcs.h): problem set-up, the
// T-count ladder driver, polling, exact verification and the raw step entry.
//
// Host-side roles (Fig. 4 of the paper, mapped onto one GPU): the workers and
// collectors are device warps (walk kernel + distinguished-point table), the
// verifiers are the re-walk kernel plus the exact claw check here.  One
// library-owned host thread per running search drives the launches on the
// caller's stream so that qcs_run_walks never blocks.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include "qcs.h"
#include "qcs_internal.h"

using namespace qcs;

namespace {

thread_local char g_cuda_err[256] = "";
constexpr uint32_t kCandCap = 4096; // claw candidates kept per launch

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

} // namespace

uint64_t qcs::upow(uint64_t b, int e)
{
    uint64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

// bits of one rotation's field in an L-bit state at h rotations per side
int qcs::field_bits(int L, int h)
{
    if (h == 0) return 0;
    const int l = (L - 1) / h;
    return l > 16 ? 16 : l;
}

// the rotations of state x at h rotations per side (see decode in qcs_walk.cu)
void qcs::decode_state(uint64_t x, int n, int L, int h, uint32_t *q)
{
    const int l = field_bits(L, h);
    const uint64_t xi = (1u << (2 * n)) - 1;
    for (int j = 0; j < h; j++) {
        const uint64_t v = (x >> (1 + l * j)) & ((1ull << l) - 1);
        q[j] = (uint32_t)((v * xi) >> l) + 1;
    }
}

namespace {

bool params_ok(int n, int k_max, const qcs_params &p)
{
    if (n < 1 || n > 4 || k_max < 0 || k_max > 15) return false;
    if (p.state_bits < 16 || p.state_bits > 64) return false;
    if (p.dp_bits < 1 || p.dp_bits >= p.state_bits) return false;
    if (p.walks < 1 || (uint32_t)p.walks > kMaxWalks || p.table_log2 < 4 || p.table_log2 > 34) return false;
    if (p.steps_per_launch < 1 || p.max_trail_factor < 1 || p.queue_capacity < 1) return false;
    if (p.budget_factor < 0 || p.version_factor < 0 || p.theta_min_bits < 0) return false;
    if (p.exhaustive_log2 < 0 || p.exhaustive_log2 > 40) return false;
    if (p.launch_shape < 0 || p.launch_shape >= launch_shapes(n) || p.c_layout < 0 || p.c_layout > 1) return false;
    // every rotation field must reach all 4^n - 1 Paulis: 2^ell > xi
    const int h = k_max / 2;
    return h == 0 || field_bits(p.state_bits, h) >= 2 * n;
}

} // namespace


LevelCtx qcs::make_level(const qcs_problem *P, int k, uint32_t version, int dp_bits)
{
    LevelCtx lv{};
    lv.C32 = P->dC32;
    lv.Cq = reinterpret_cast<const uint4 *>(P->dCq);
    lv.Cm = reinterpret_cast<const uint4 *>(P->dCm);
    lv.U = P->dU;
    for (int side = 0; side < 2; side++) lv.T1[side] = P->dT1[side];
    lv.coef = P->dCoef;
    lv.n = P->n;
    lv.k = k;
    lv.h = k / 2;
    lv.xi = (uint32_t)(P->D - 1);
    lv.xi_h = upow(lv.xi, lv.h);
    lv.ell = field_bits(P->p.state_bits, lv.h);
    lv.fmask = lv.ell ? (uint32_t)((1ull << lv.ell) - 1) : 0u;
    lv.K = P->C.E + (k & 1) + lv.h;
    lv.ev = lv.K - lv.h;
    lv.maskL = P->p.state_bits >= 64 ? ~0ull : ((1ull << P->p.state_bits) - 1);
    lv.dshift = P->p.state_bits - dp_bits;
    lv.version = version;
    lv.n_chunks = (k & 1) ? (int32_t)(P->D - 1) : 0;
    lv.seed = P->p.seed;
    return lv;
}

namespace {

// one adjoint butterfly stage of the weights mod 2^16 (the host twin of
// adj_stage in qcs_walk.cu): rows that commute with p map (ua, ub) to
// (ub, 2 ua); an anticommuting row j adds (adjoint of R^) or subtracts
// (adjoint of R^T) s(p, j) times row j ^ p
void host_adj_stage(int n, uint32_t p, bool adj_of_transpose, std::vector<uint32_t> &ua, std::vector<uint32_t> &ub)
{
    const uint32_t D = 1u << (2 * n), m = (1u << n) - 1;
    std::vector<uint32_t> na(D), nb(D);
    for (uint32_t j = 0; j < D; j++) {
        const bool anti = (__builtin_popcount(((p >> n) & (j & m)) ^ ((p & m) & (j >> n))) & 1) != 0;
        if (anti) {
            const bool add = (pauli_phase(n, p, j) == 1) != adj_of_transpose;
            na[j] = add ? ua[j] + ua[j ^ p] : ua[j] - ua[j ^ p];
            nb[j] = add ? ub[j] + ub[j ^ p] : ub[j] - ub[j ^ p];
        } else {
            na[j] = ub[j];
            nb[j] = ua[j] << 1;
        }
    }
    for (uint32_t j = 0; j < D; j++) {
        ua[j] = na[j] & 0xFFFFu;
        ub[j] = nb[j] & 0xFFFFu;
    }
}

std::mutex g_tab_mu;
std::map<std::pair<int, int>, std::array<uint32_t *, 2>> g_tabs; // (device, n) -> T1v, T1w

} // namespace

int qcs::stage_tables(int n, const uint32_t *t1[2], int64_t *uploaded)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(g_tab_mu);
    auto it = g_tabs.find({dev, n});
    if (it == g_tabs.end()) {
        const uint32_t D = 1u << (2 * n), xi = D - 1;
        std::vector<uint32_t> u0a(D), u0b(D);
        for (uint32_t i = 1; i < D; i++) {
            u0a[i] = (uint32_t)smix_host(kSeedU + (2ull * i + 1) * kGamma) & 0xFFFFu;
            u0b[i] = (uint32_t)smix_host(kSeedU + (2ull * i + 2) * kGamma) & 0xFFFFu;
        }
        std::array<uint32_t *, 2> tabs{nullptr, nullptr};
        for (int side = 0; side < 2; side++) {
            std::vector<uint32_t> t1((size_t)xi * D);
            for (uint32_t qa = 1; qa <= xi; qa++) {
                std::vector<uint32_t> ua = u0a, ub = u0b;
                host_adj_stage(n, qa, side == 1, ua, ub);
                for (uint32_t j = 0; j < D; j++) t1[(size_t)(qa - 1) * D + j] = ua[j] | (ub[j] << 16);
            }
            CK(cudaMalloc(&tabs[side], sizeof(uint32_t) * t1.size()));
            CK(cudaMemcpy(tabs[side], t1.data(), sizeof(uint32_t) * t1.size(), cudaMemcpyHostToDevice));
            if (uploaded) *uploaded += (int64_t)(sizeof(uint32_t) * t1.size());
        }
        it = g_tabs.emplace(std::make_pair(dev, n), tabs).first;
    }
    t1[0] = it->second[0];
    t1[1] = it->second[1];
    return QCS_OK;
}

namespace {

int upload_problem(qcs_problem *P)
{
    const int D = P->D, n = P->n;
    const int Wl = lanes_per_walk(n), R = D / Wl; // lanes per walk and columns per lane in the walk kernel
    // C^ low words; row i keeps lane l's columns l + Wl t (t < R) next to
    // each other at i * D + l * R + t
    std::vector<uint2> c32((size_t)D * D), u(D);
    for (int i = 0; i < D; i++)
        for (int Q = 0; Q < D; Q++) {
            const size_t src = (size_t)i * D + Q;
            const size_t dst = (size_t)i * D + (size_t)(Q % Wl) * R + (size_t)(Q / Wl);
            c32[dst] = make_uint2((uint32_t)(uint64_t)P->C.a[src], (uint32_t)(uint64_t)P->C.b[src]);
        }
    // fingerprint weights: the SplitMix64 stream seeded with kSeedU, outputs
    // 2i and 2i+1 give (Ua[i], Ub[i]); row 0 (the identity) gets zero weight
    u[0] = make_uint2(0, 0);
    for (int i = 1; i < D; i++) {
        uint64_t wa = smix_host(kSeedU + (2ull * i + 1) * kGamma);
        uint64_t wb = smix_host(kSeedU + (2ull * i + 2) * kGamma);
        u[i] = make_uint2((uint32_t)wa, (uint32_t)wb);
    }
    // rotation masks per Pauli p and lane l (LevelCtx::coef): a 16-bit word
    // whose bit t says that row l + Wl t anticommutes with p and bit 8 + t
    // that s(p, row) = +1 (lambda = 1); two words to a uint32
    std::vector<uint16_t> coef16((size_t)D * Wl, 0);
    const uint32_t m = (1u << n) - 1;
    for (uint32_t p = 0; p < (uint32_t)D; p++)
        for (uint32_t j = 0; j < (uint32_t)D; j++) {
            const uint32_t t = j / (uint32_t)Wl, l = j % (uint32_t)Wl;
            const bool anti = (__builtin_popcount(((p >> n) & (j & m)) ^ ((p & m) & (j >> n))) & 1) != 0;
            const bool plus = pauli_phase(n, p, j) == 1;
            if (anti) coef16[(size_t)p * Wl + l] |= (uint16_t)(1u << t);
            if (plus) coef16[(size_t)p * Wl + l] |= (uint16_t)(1u << (8 + t));
        }
    std::vector<uint32_t> coef(coef16.size() / 2);
    memcpy(coef.data(), coef16.data(), sizeof(uint32_t) * coef.size());
    // n >= 3: also C^ as signed byte quads (rows 4q .. 4q+3 of a column in
    // one word) when every entry fits in int8, laid out for the walk
    // kernel's byte-plane contraction (LevelCtx::Cq)
    std::vector<uint32_t> cq, cm;
    if (n >= 3 && P->p.c_layout == 0) {
        bool fits = true;
        for (size_t i = 0; i < P->C.a.size() && fits; i++)
            fits = P->C.a[i] >= -128 && P->C.a[i] <= 127 && P->C.b[i] >= -128 && P->C.b[i] <= 127;
        if (fits) {
            const int quads = D / 4, half = R / 2;
            cq.assign((size_t)D * D / 2, 0);
            for (int q = 0; q < quads; q++)
                for (int j = 0; j < half; j++)
                    for (int lane = 0; lane < Wl; lane++)
                        for (int c = 0; c < 2; c++) {
                            const int Q = lane + 2 * Wl * j + Wl * c;
                            uint32_t wa = 0, wb = 0;
                            for (int r = 0; r < 4; r++) {
                                const size_t src = (size_t)(4 * q + r) * D + Q;
                                wa |= (uint32_t)(uint8_t)(int8_t)P->C.a[src] << (8 * r);
                                wb |= (uint32_t)(uint8_t)(int8_t)P->C.b[src] << (8 * r);
                            }
                            const size_t o = (((size_t)q * half + j) * Wl + lane) * 4 + 2 * c;
                            cq[o] = wa;
                            cq[o + 1] = wb;
                        }
            if (n == 4) {
                // the tensor-core layout (LevelCtx::Cm): biased bytes, K-blocks of 16 rows
                cm.assign((size_t)D * 2 * D / 4, 0);
                // K index k = part * 256 + 8 l + t holds row 32 t + l of the a-part
                // (part 0) or b-part (part 1): the eight rows one lane of the
                // walk kernel holds form one K chunk of eight
                auto entry = [&](int k, int col) -> uint32_t {
                    const int kk = k & (D - 1), row = (kk % 8) * 32 + kk / 8;
                    const size_t src = (size_t)row * D + col;
                    return (uint32_t)(uint8_t)((k < D ? P->C.a[src] : P->C.b[src]) + 128);
                };
                for (int col = 0; col < D; col++)
                    for (int kb = 0; kb < 2 * D / 16; kb++)
                        for (int q = 0; q < 4; q++) {
                            const int k0 = 16 * kb + 2 * q;
                            const uint32_t w = entry(k0, col) | entry(k0 + 1, col) << 8 | entry(k0 + 8, col) << 16 |
                                               entry(k0 + 9, col) << 24;
                            const int chunk = (4 * (kb / 4) + q) ^ (4 * (col & 1));
                            cm[(size_t)col * 128 + (size_t)chunk * 4 + (kb % 4)] = w;
                        }
            }
        }
    }
    CK(cudaGetDevice(&P->device));
    int64_t h2d = 0;
    if (int rc = stage_tables(n, P->dT1, &h2d)) return rc;
    if (!cq.empty()) {
        CK(cudaMalloc(&P->dCq, sizeof(uint32_t) * cq.size()));
        CK(cudaMemcpy(P->dCq, cq.data(), sizeof(uint32_t) * cq.size(), cudaMemcpyHostToDevice));
        h2d += (int64_t)(sizeof(uint32_t) * cq.size());
    }
    if (!cm.empty()) {
        CK(cudaMalloc(&P->dCm, sizeof(uint32_t) * cm.size()));
        CK(cudaMemcpy(P->dCm, cm.data(), sizeof(uint32_t) * cm.size(), cudaMemcpyHostToDevice));
        h2d += (int64_t)(sizeof(uint32_t) * cm.size());
    }
    CK(cudaMalloc(&P->dC32, sizeof(uint2) * c32.size()));
    CK(cudaMalloc(&P->dU, sizeof(uint2) * D));
    CK(cudaMalloc(&P->dCoef, sizeof(uint32_t) * coef.size()));
    CK(cudaMemcpy(P->dC32, c32.data(), sizeof(uint2) * c32.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->dU, u.data(), sizeof(uint2) * D, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->dCoef, coef.data(), sizeof(uint32_t) * coef.size(), cudaMemcpyHostToDevice));
    h2d += (int64_t)(sizeof(uint2) * c32.size() + sizeof(uint2) * D + sizeof(uint32_t) * coef.size());
    P->res.h2d_bytes += h2d;
    return QCS_OK;
}

int ensure_search_buffers(qcs_problem *P)
{
    if (P->dTable) return QCS_OK;
    const size_t slots = (size_t)1 << P->p.table_log2;
    CK(cudaMalloc(&P->dTable, sizeof(Slot) * slots));
    CK(cudaMalloc(&P->dQueue, sizeof(Pair) * (size_t)P->p.queue_capacity));
    CK(cudaMalloc(&P->dQhead, 4 * sizeof(uint32_t))); // merges, candidates, carried re-walks, re-walk cursor
    if (P->p.rewalk_budget > 0)
        for (int i = 0; i < 2; i++) CK(cudaMalloc(&P->dPend[i], sizeof(Pending) * (size_t)P->p.queue_capacity));
    CK(cudaMalloc(&P->dCands, sizeof(Cand) * kCandCap));
    CK(cudaMalloc(&P->dWalks, sizeof(WalkState) * (size_t)P->p.walks));
    CK(cudaMalloc(&P->dCounters, sizeof(unsigned long long) * C_NCOUNTERS));
    CK(cudaMallocHost(&P->hCounters, sizeof(unsigned long long) * C_NCOUNTERS));
    CK(cudaMallocHost(&P->hCands, sizeof(Cand) * kCandCap));
    CK(cudaMallocHost(&P->hQhead, 3 * sizeof(uint32_t)));
    return QCS_OK;
}

void free_problem_memory(qcs_problem *P)
{
    cudaFree(P->dC32); cudaFree(P->dCq); cudaFree(P->dCm); cudaFree(P->dU); cudaFree(P->dCoef); cudaFree(P->dTable); cudaFree(P->dQueue); cudaFree(P->dQhead);
    cudaFree(P->dCands); cudaFree(P->dWalks); cudaFree(P->dCounters); cudaFree(P->dPend[0]); cudaFree(P->dPend[1]);
    cudaFreeHost(P->hCounters); cudaFreeHost(P->hCands); cudaFreeHost(P->hQhead);
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

} // namespace

bool qcs::verify_claw(const qcs_problem *P, int k, int chunk, const uint32_t *qv, const uint32_t *qw,
                      uint32_t *paulis, PMat *Dh)
{
    const int h = k / 2;
    for (int j = 0; j < 16; j++) paulis[j] = 0;
    for (int j = 0; j < h; j++) {
        paulis[j] = qv[j];
        paulis[h + j] = qw[j];
    }
    if (k & 1) paulis[2 * h] = (uint32_t)chunk;
    return exact_verify(P->n, P->C, paulis, k, Dh) == QCS_OK;
}

void qcs::found(qcs_problem *P, int k, const uint32_t *paulis)
{
    PMat Dh;
    exact_verify(P->n, P->C, paulis, k, &Dh);
    found(P, k, paulis, std::move(Dh));
}

void qcs::found(qcs_problem *P, int k, const uint32_t *paulis, PMat &&Dh)
{
    std::lock_guard<std::mutex> g(P->mu);
    if (P->have_D) return; // keep the first decomposition
    P->res.t_count = k;
    P->res.k = k;
    for (int j = 0; j < 16; j++) P->res.paulis[j] = j < k ? paulis[j] : 0;
    P->Dhat = std::move(Dh);
    P->have_D = true;
}

namespace {

int level_begin(qcs_problem *P, int k, uint32_t version, int dp_bits, uint32_t n_walks, cudaStream_t s,
                uint32_t walk_base = 0)
{
    if (k < 2 || k > P->k_max) return QCS_ERR_ARG;
    if (dp_bits == 0) dp_bits = P->p.dp_bits;
    if (dp_bits < 1 || dp_bits >= P->p.state_bits) return QCS_ERR_ARG;
    int rc = ensure_search_buffers(P);
    if (rc) return rc;
    auto &L = P->lvl;
    L.k = k;
    L.h = k / 2;
    L.dp_bits = dp_bits;
    WalkLaunch &w = L.w;
    w = WalkLaunch{};
    w.lv = make_level(P, k, version, dp_bits);
    w.walks = P->dWalks;
    w.n_walks = (int32_t)std::min<uint32_t>(n_walks ? n_walks : (uint32_t)P->p.walks, (uint32_t)P->p.walks);
    w.steps = (uint32_t)P->p.steps_per_launch;
    w.max_len = (uint32_t)std::min<uint64_t>((uint64_t)P->p.max_trail_factor << dp_bits, kMaxTrailLen);
    w.table = P->dTable;
    w.table_mask = ((uint64_t)1 << P->p.table_log2) - 1;
    w.queue = P->dQueue;
    w.qhead = P->dQhead;
    w.qcap = (uint32_t)P->p.queue_capacity;
    w.cands = P->dCands;
    w.ccount = P->dQhead + 1;
    w.ccap = kCandCap;
    w.counters = P->dCounters;
    w.stall = reinterpret_cast<uint32_t *>(P->dCounters + C_STALLED); // its low word
    w.shape = P->p.launch_shape;
    w.walk_base = walk_base;
    L.pp = 0;
    L.pend_n = 0; // a new level or function version drops carried re-walks
    CK(cudaMemsetAsync(P->dTable, 0xFF, sizeof(Slot) << P->p.table_log2, s));
    CK(cudaMemsetAsync(P->dQhead, 0, 2 * sizeof(uint32_t), s));
    CK(launch_init_walks(w, s));
    L.active = true;
    std::lock_guard<std::mutex> g(P->mu);
    P->res.k = k;
    P->res.version = version;
    return QCS_OK;
}

int level_walk(qcs_problem *P, uint32_t steps, cudaStream_t s)
{
    if (!P->lvl.active || steps == 0) return QCS_ERR_ARG;
    P->lvl.w.steps = steps;
    CK(cudaMemsetAsync(P->dQhead, 0, 2 * sizeof(uint32_t), s));
    CK(cudaMemsetAsync(P->dCounters, 0, sizeof(unsigned long long) * C_NCOUNTERS, s));
    CK(launch_walks(P->lvl.w, s));
    return QCS_OK;
}

int level_rewalk(qcs_problem *P, cudaStream_t s)
{
    if (!P->lvl.active) return QCS_ERR_ARG;
    auto &L = P->lvl;
    WalkLaunch w = L.w;
    if (P->p.rewalk_budget > 0) {
        // the re-walks carried from the previous launch first, then this
        // launch's merges; unfinished ones go to the other buffer
        w.rewalk_budget = (uint32_t)P->p.rewalk_budget;
        w.pend_in = P->dPend[L.pp];
        w.pend_in_n = L.pend_n;
        w.pend_out = P->dPend[L.pp ^ 1];
        w.pend_out_n = P->dQhead + 2;
        w.pend_cap = (uint32_t)P->p.queue_capacity;
        CK(cudaMemsetAsync(P->dQhead + 2, 0, sizeof(uint32_t), s));
    }
    w.rw_next = P->dQhead + 3;
    CK(cudaMemsetAsync(P->dQhead + 3, 0, sizeof(uint32_t), s));
    CK(launch_rewalk_pairs(w, s));
    CK(cudaMemcpyAsync(P->hCounters, P->dCounters, sizeof(unsigned long long) * C_NCOUNTERS,
                       cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(P->hQhead, P->dQhead, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    return QCS_OK;
}

// Wait, check claw candidates exactly, fold counters into res.  *steps gets
// the launch's walk steps.
int level_collect(qcs_problem *P, cudaStream_t s, bool *got, uint64_t *steps)
{
    if (!P->lvl.active) return QCS_ERR_ARG;
    CK(cudaStreamSynchronize(s));
    const auto &L = P->lvl;
    const int k = L.k, h = L.h;
    const unsigned long long *c = P->hCounters;
    if (c[C_STALLED]) return QCS_ERR_DEVICE; // a bounded wait of the walk kernel ran out: nothing here is valid
    const uint32_t npairs = std::min(P->hQhead[0], L.w.qcap);
    const uint32_t ncand = std::min(P->hQhead[1], kCandCap);
    int64_t d2h = (int64_t)(sizeof(unsigned long long) * C_NCOUNTERS + 3 * sizeof(uint32_t));
    int64_t carried_lost = 0;
    if (P->p.rewalk_budget > 0) {
        // re-walks carried into the next launch (those past the buffer are lost)
        auto &Lm = P->lvl;
        const uint32_t cap = (uint32_t)P->p.queue_capacity;
        carried_lost = P->hQhead[2] > cap ? (int64_t)(P->hQhead[2] - cap) : 0;
        Lm.pend_n = std::min(P->hQhead[2], cap);
        Lm.pp ^= 1;
    }
    if (ncand > 0) {
        // read back only the candidates the re-walk queued
        CK(cudaMemcpyAsync(P->hCands, P->dCands, sizeof(Cand) * ncand, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        d2h += (int64_t)(sizeof(Cand) * ncand);
    }
    uint32_t paulis[16] = {0};
    PMat Dh;
    int64_t claws = 0, false_hash = 0;
    *got = false;
    for (uint32_t i = 0; i < ncand && !*got; i++) {
        // exact check of the candidate: decode the V point and the W point
        const Cand &r = P->hCands[i];
        const uint64_t xv = (r.a & 1) ? r.b : r.a, xw = (r.a & 1) ? r.a : r.b;
        uint32_t qv[kMaxH], qw[kMaxH];
        decode_state(xv, P->n, P->p.state_bits, h, qv);
        decode_state(xw, P->n, P->p.state_bits, h, qw);
        const int chunk = (k & 1) ? (int)r.chunk : 0;
        if (verify_claw(P, k, chunk, qv, qw, paulis, &Dh)) {
            claws++;
            *got = true;
            continue;
        }
        false_hash++;
    }
    *steps = c[C_STEPS];
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
        R.queue_overflow += (int64_t)(c[C_PAIRS] - npairs) + carried_lost;
        R.rewalk_carried = (int64_t)P->lvl.pend_n;
        R.robin_hood += (int64_t)c[C_CLS0 + QCS_MERGE_ROBIN_HOOD];
        R.trivial += (int64_t)c[C_CLS0 + QCS_MERGE_TRIVIAL];
        R.same_side += (int64_t)c[C_CLS0 + QCS_MERGE_SAME_SIDE];
        R.no_merge += (int64_t)c[C_CLS0 + QCS_MERGE_NO_MERGE];
        R.claws += claws;
        R.false_hash += false_hash;
        R.launches += 1;
        R.d2h_bytes += d2h;
        R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - P->t0).count();
    }
    if (*got) found(P, k, paulis, std::move(Dh));
    return QCS_OK;
}



} // namespace

LevelPlan qcs::plan_level_n(int D, int k, const qcs_params &p)
{
    LevelPlan pl{};
    const uint64_t xi = (uint64_t)(D - 1);
    const long double points = 2.0L * (long double)upow(xi, k / 2) * (long double)((k & 1) ? xi : 1);
    pl.points = points > 1.8e19L ? ~0ull : (uint64_t)points;
    pl.dp_bits = p.dp_bits;
    const long double slots = (long double)((uint64_t)1 << p.table_log2);
    if (p.theta_policy == 1) {
        // minimise N theta / w + 2 / theta: theta = sqrt(2 w / N), i.e.
        // d = log2(sqrt(N / 2w)), at least theta_min_bits
        const long double ratio = points / (2.0L * slots);
        const int d_opt = ratio > 1.0L ? (int)std::lround(0.5L * std::log2(ratio)) : 0;
        pl.dp_bits = std::min(p.dp_bits, std::max(std::max(1, p.theta_min_bits), d_opt));
    }
    const long double theta = 1.0L / (long double)((uint64_t)1 << pl.dp_bits);
    const long double vf = p.version_factor > 0 ? (long double)p.version_factor : 1e30L;
    const long double version_steps = vf * points;
    // a launch covers at most one version; trails of a few 1/theta must fit
    long double steps = (long double)p.steps_per_launch, walks = (long double)p.walks;
    const long double s_min = std::min<long double>(steps, 4.0L / theta);
    if (walks * steps > version_steps) steps = std::max(s_min, std::floor(version_steps / walks));
    if (walks * steps > version_steps) walks = std::max(32.0L, std::floor(version_steps / steps));
    // expected merges per launch (distinguished points that meet a stored
    // one, about the stored fraction of all distinguished points) fit half
    // the queue
    // half the queue; fewer walks first (down to a few per resident warp),
    // then fewer steps, so that launches stay long
    const long double stored = std::min(1.0L, slots / (theta * points));
    const long double qroom = (long double)p.queue_capacity / 2, per_step = theta * stored;
    if (walks * steps * per_step > qroom) {
        const long double keep = std::max(1.0L, std::min(steps, s_min));
        walks = std::min(walks, std::max(std::min(walks, 8192.0L), std::floor(qroom / (keep * per_step))));
        steps = std::max(1.0L, std::min(steps, std::floor(qroom / (walks * per_step))));
        if (walks * steps * per_step > qroom) walks = std::max(32.0L, std::floor(qroom / (steps * per_step)));
    }
    pl.walks = (uint32_t)walks;
    pl.steps = (uint32_t)std::max(1.0L, steps);
    const long double per_launch = (long double)pl.walks * pl.steps;
    pl.launches_per_version = p.version_factor > 0
                                  ? (uint64_t)std::max(1.0L, std::floor(version_steps / per_launch))
                                  : ~0ull;
    const long double budget = (long double)p.budget_factor * points;
    const long double lmin = std::ceil(budget / per_launch);
    pl.min_launches = lmin > 1.8e19L ? ~0ull : (uint64_t)std::max(1.0L, lmin);
    if (p.version_factor > 0 && pl.min_launches < 4 * pl.launches_per_version)
        pl.min_launches = 4 * pl.launches_per_version; // at least four function versions
    return pl;
}

LevelPlan qcs::plan_level(const qcs_problem *P, int k, const qcs_params &p) { return plan_level_n(P->D, k, p); }

uint64_t qcs::exhaustive_points(const qcs_problem *P, int k)
{
    const uint64_t xi = (uint64_t)(P->D - 1);
    const long double v = (long double)upow(xi, k / 2), w = v * (long double)((k & 1) ? xi : 1);
    return v + w > 1.8e19L ? ~0ull : (uint64_t)(v + w);
}

bool qcs::exhaustive_eligible(const qcs_problem *P, int k)
{
    if (P->p.exhaustive_log2 <= 0 || k < 2 || exhaustive_points(P, k) > (1ull << P->p.exhaustive_log2)) return false;
    uint64_t slots = 1024;
    const uint64_t xi_h = upow((uint64_t)(P->D - 1), k / 2);
    while (slots < 2 * xi_h) slots <<= 1;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return false;
    return sizeof(CertSlot) * slots <= free_b / 2;
}

int qcs::cert_begin(qcs_problem *P, int k, cudaStream_t s, CertPass *c)
{
    *c = CertPass();
    c->k = k;
    c->h = k / 2;
    c->xi = (uint64_t)(P->D - 1);
    c->xi_h = upow(c->xi, c->h);
    // Odd k puts 2h + 1 rotations into two products, so one side gets h + 1
    // and has xi times the points of the other.  With a denominator in C^
    // (E >= 1) the extra rotation goes on V: the xi^(h+1) streamed points are
    // products V' = R(r_(h+1))..R(r_1) with no contraction against C^, and
    // the stored xi^h points are W' = R(s_1)^T..R(s_h)^T C^, both at exponent
    // E + h (V' raised from h + 1 by sqrt2^(E-1)).  A claw V' ~ W' is
    // C^ ~ R(s_h)..R(s_1) R(r_(h+1))..R(r_1).  Otherwise (even k, or E = 0)
    // V = h rotations is stored and W (with the chunk rotation) streamed.
    c->v_heavy = (k & 1) && P->C.E >= 1;
    c->n_probe = c->xi_h * ((k & 1) ? c->xi : 1);
    uint64_t slots = 1024;
    while (slots < 2 * c->xi_h) slots <<= 1;
    {
        // the key table must fit: refuse before allocating
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        if (sizeof(CertSlot) * slots > free_b) return QCS_ERR_NOMEM;
    }
    c->lv_store = make_level(P, c->v_heavy ? 2 * c->h : k, 0, P->p.dp_bits);
    c->lv_probe = make_level(P, c->v_heavy ? 2 * c->h + 2 : k, 0, P->p.dp_bits);
    if (c->v_heavy) {
        c->lv_probe.K = c->lv_store.K; // E + h
        c->lv_probe.ev = P->C.E - 1;
    }
    CertArgs &a = c->a;
    a.xi_h = c->xi_h;
    a.mask = slots - 1;
    a.cap = CertPass::kCap;
    // one hash base for every chunk, so the keys of a coset agree on both sides
    const uint64_t tag =
        (uint64_t)P->n | ((uint64_t)k << 8) | (0xFFFFull << 16) | ((uint64_t)(uint32_t)c->lv_store.K << 32);
    a.base = smix_host(smix_host(kSeedH ^ 0xCE27u) ^ tag);
    c->slice = CertPass::kSliceMin;
    cudaError_t e = cudaMalloc(&a.table, sizeof(CertSlot) * slots);
    if (e == cudaSuccess) e = cudaMalloc(&a.pairs, sizeof(uint64_t) * 2 * CertPass::kCap);
    if (e == cudaSuccess) e = cudaMalloc(&a.n_pairs, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&c->hN, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&c->hPairs, sizeof(uint64_t) * 2 * CertPass::kCap);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.table, 0xFF, sizeof(CertSlot) * slots, s);
    if (e != cudaSuccess) {
        cert_end(P, c, s);
        return e == cudaErrorMemoryAllocation ? QCS_ERR_NOMEM : cuda_fail(e);
    }
    c->table_bytes = sizeof(CertSlot) * slots;
    return QCS_OK;
}

int qcs::cert_advance(qcs_problem *P, CertPass *c, cudaStream_t s, uint64_t budget, uint64_t *used)
{
    // A stored point with the contraction against C^ costs about four
    // streamed ones without it; `budget` and *used count in streamed points.
    constexpr uint64_t kStoreCost = 4;
    *used = 0;
    CertArgs &a = c->a;
    cudaError_t e = cudaSuccess;
    while (!c->done && *used < budget) {
        if (P->cancel.load()) return QCS_ERR_BUSY;
        if (c->stored < c->xi_h) {
            // the smaller side into the key table, in slices (W' carries the
            // contraction with C^ when the extra rotation went on V)
            const uint64_t cost = c->v_heavy ? kStoreCost : 1;
            uint64_t n = std::min<uint64_t>(c->xi_h - c->stored, CertPass::kSliceMax);
            n = std::max<uint64_t>(1, std::min<uint64_t>(n, (budget - *used + cost - 1) / cost));
            a.lv = c->lv_store;
            a.side = c->v_heavy ? 1 : 0;
            a.insert = 1;
            a.first = c->stored;
            a.count = n;
            if ((e = launch_certify(a, s)) != cudaSuccess) break;
            c->stored += n;
            *used += n * cost;
            continue;
        }
        if (c->probed >= c->n_probe) {
            c->done = true;
            break;
        }
        // the other side probes the table, one slice at a time; the key
        // matches of each slice are checked exactly on the host
        const uint64_t cost = c->v_heavy ? 1 : kStoreCost;
        uint64_t n = std::min(c->slice, c->n_probe - c->probed);
        n = std::max<uint64_t>(1, std::min<uint64_t>(n, (budget - *used + cost - 1) / cost));
        a.lv = c->lv_probe;
        a.side = c->v_heavy ? 0 : 1;
        a.insert = 0;
        a.first = c->probed;
        a.count = n;
        if ((e = cudaMemsetAsync(a.n_pairs, 0, sizeof(uint32_t), s)) != cudaSuccess) break;
        if ((e = launch_certify(a, s)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(c->hN, a.n_pairs, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        c->d2h += (int64_t)sizeof(uint32_t);
        c->probed += n;
        *used += n * cost;
        if (n == c->slice) c->slice = std::min(2 * c->slice, CertPass::kSliceMax);
        const uint32_t m = std::min(*c->hN, CertPass::kCap);
        if (*c->hN > CertPass::kCap) c->overflow = true;
        if (m > 0) {
            // read back only the matches the slice queued
            if ((e = cudaMemcpyAsync(c->hPairs, a.pairs, sizeof(uint64_t) * 2 * m, cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess)
                break;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
            c->d2h += (int64_t)(sizeof(uint64_t) * 2 * m);
        }
        const int k = c->k, h = c->h;
        const uint64_t xi = c->xi;
        for (uint32_t i = 0; i < m && !c->got; i++) {
            // exact check of the key match: rotations from the point indices
            uint32_t paulis[16] = {0};
            uint64_t st = c->hPairs[2 * i], pr = c->hPairs[2 * i + 1];
            PMat Dh;
            bool ok;
            if (c->v_heavy) {
                // P_1..P_(h+1) = r_1..r_(h+1) (probing V'), P_(h+2)..P_k = s_1..s_h (stored W')
                for (int j = 0; j <= h; j++, pr /= xi) paulis[j] = (uint32_t)(pr % xi) + 1;
                for (int j = 0; j < h; j++, st /= xi) paulis[h + 1 + j] = (uint32_t)(st % xi) + 1;
                ok = exact_verify(P->n, P->C, paulis, k, &Dh) == QCS_OK;
            } else {
                uint32_t qv[kMaxH], qw[kMaxH];
                const int chunk = (k & 1) ? (int)(pr / c->xi_h) + 1 : 0;
                pr %= c->xi_h;
                for (int j = 0; j < h; j++) {
                    qv[j] = (uint32_t)(st % xi) + 1;
                    qw[j] = (uint32_t)(pr % xi) + 1;
                    st /= xi;
                    pr /= xi;
                }
                ok = verify_claw(P, k, chunk, qv, qw, paulis, &Dh);
            }
            if (ok) {
                found(P, k, paulis, std::move(Dh));
                c->got = true;
            }
        }
        if (c->got) c->done = true;
    }
    return e == cudaSuccess ? QCS_OK : cuda_fail(e);
}

int qcs::cert_end(qcs_problem *P, CertPass *c, cudaStream_t s)
{
    cudaStreamSynchronize(s);
    cudaFree(c->a.table);
    cudaFree(c->a.pairs);
    cudaFree(c->a.n_pairs);
    cudaFreeHost(c->hN);
    cudaFreeHost(c->hPairs);
    c->a.table = nullptr;
    c->a.pairs = nullptr;
    c->a.n_pairs = nullptr;
    c->hN = nullptr;
    c->hPairs = nullptr;
    {
        std::lock_guard<std::mutex> g(P->mu);
        P->res.cert_points += (int64_t)(c->stored + c->probed);
        P->res.d2h_bytes += c->d2h;
        if (c->done && !c->got && !c->overflow) P->res.certified_levels += 1;
    }
    c->d2h = 0;
    return (c->done && !c->got && c->overflow) ? QCS_ERR_OVERFLOW : QCS_OK;
}

int qcs::certify_level(qcs_problem *P, int k, cudaStream_t s, bool *got)
{
    *got = false;
    CertPass c;
    int rc = cert_begin(P, k, s, &c);
    if (rc != QCS_OK) return rc;
    uint64_t used = 0;
    while (rc == QCS_OK && !c.done) rc = cert_advance(P, &c, s, ~0ull, &used);
    const int rc_end = cert_end(P, &c, s);
    *got = c.got;
    return rc != QCS_OK ? rc : rc_end;
}

namespace {

bool have_decomposition(qcs_problem *P)
{
    std::lock_guard<std::mutex> g(P->mu);
    return P->have_D;
}

// the search driver: levels sde .. k_max, walks until a verified claw
int drive(qcs_problem *P, uint64_t budget, cudaStream_t s)
{
    CK(cudaSetDevice(P->device));
    uint64_t total_steps = 0;
    uint32_t version = 0;
    for (int k = P->C.E; k <= P->k_max; k++) {
        {
            std::lock_guard<std::mutex> g(P->mu);
            P->res.k = k;
        }
        if (k <= 1) {
            uint32_t paulis[16] = {0};
            if (small_level(P, k, paulis)) {
                found(P, k, paulis);
                return QCS_OK;
            }
            continue;
        }
        if (P->p.exhaustive_first && exhaustive_eligible(P, k)) {
            bool got = false;
            const int rc = certify_level(P, k, s, &got);
            if (rc == QCS_OK) {
                if (got) return QCS_OK;
                continue; // proved empty: the next level
            }
            if (rc != QCS_ERR_OVERFLOW) return rc;
            // inconclusive: walk the level
        }
        const LevelPlan pl = plan_level(P, k, P->p);
        uint64_t launches = 0, in_version = 0;
        bool fresh = true;
        while (true) {
            if (P->cancel.load()) return QCS_ERR_BUSY; // reported as CANCELLED
            int rc;
            if (fresh) {
                rc = level_begin(P, k, version, pl.dp_bits, pl.walks, s);
                if (rc) return rc;
                fresh = false;
                in_version = 0;
            }
            if ((rc = level_walk(P, pl.steps, s))) return rc;
            if ((rc = level_rewalk(P, s))) return rc;
            bool got = false;
            uint64_t steps = 0;
            if ((rc = level_collect(P, s, &got, &steps))) return rc;
            if (got && P->p.stop_on_claw) return QCS_OK;
            total_steps += steps;
            launches++;
            in_version++;
            if (budget && total_steps >= budget) return have_decomposition(P) ? QCS_OK : QCS_ERR_TIMEOUT;
            if (launches >= pl.min_launches) break;
            if (in_version >= pl.launches_per_version) {
                version++;
                fresh = true;
            }
        }
        version++;
        if (have_decomposition(P)) return QCS_OK; // the optimal level is the first with a claw
        if (exhaustive_eligible(P, k)) {
            // the walk budget ended without a claw: settle the level exactly
            bool got = false;
            const int rc = certify_level(P, k, s, &got);
            if (rc != QCS_OK && rc != QCS_ERR_OVERFLOW) return rc;
            if (got) return QCS_OK;
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

int qcs::noalloc_level(const qcs_problem *P, int k, uint32_t version, int dp_bits, LevelCtx *lv, uint32_t *max_len,
                       int *table_log2)
{
    if (!P || !lv || !max_len || !table_log2 || k < 2 || k > P->k_max) return QCS_ERR_ARG;
    if (dp_bits == 0) dp_bits = P->p.dp_bits;
    if (dp_bits < 1 || dp_bits >= P->p.state_bits) return QCS_ERR_ARG;
    *lv = make_level(P, k, version, dp_bits);
    *max_len = (uint32_t)std::min<uint64_t>((uint64_t)P->p.max_trail_factor << dp_bits, kMaxTrailLen);
    *table_log2 = P->p.table_log2;
    return QCS_OK;
}

int qcs::record_cuda_error(cudaError_t e) { return cuda_fail(e); }

extern "C" {

int qcs_launch_shapes(int n_qubits, int32_t *warps, int32_t *min_blocks, int max_shapes)
{
    if (n_qubits < 1 || n_qubits > 4) return QCS_ERR_ARG;
    const int cnt = launch_shapes(n_qubits);
    for (int i = 0; i < cnt && i < max_shapes; i++) {
        if (warps) warps[i] = shape_warps_of(n_qubits, i);
        if (min_blocks) min_blocks[i] = shape_min_blocks_of(n_qubits, i);
    }
    return cnt;
}

void qcs_default_params(int n_qubits, qcs_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    switch (n_qubits) {
    case 1:
    case 2: p->state_bits = 32; p->dp_bits = 6; p->walks = 4096; p->table_log2 = 16; break;
    case 3: p->state_bits = 48; p->dp_bits = 10; p->walks = 1 << 16; p->table_log2 = 22; break;
    default:
        p->state_bits = 64; p->dp_bits = 12; p->walks = 1 << 20; p->table_log2 = 26;
        p->launch_shape = 3; // the tensor-core walk (shape 0 where C^ does not fit int8)
        break;
    }
    p->steps_per_launch = 64;
    p->max_trail_factor = 20;
    p->queue_capacity = 1 << 20;
    p->budget_factor = 16;
    p->theta_policy = 1;
    p->version_factor = 2;
    p->stop_on_claw = 1;
    p->theta_min_bits = 1;
    p->exhaustive_log2 = 24;
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
    const int64_t h2d = P->res.h2d_bytes, d2h = P->res.d2h_bytes; // kept for the problem's lifetime
    memset(&P->res, 0, sizeof P->res);
    P->res.h2d_bytes = h2d;
    P->res.d2h_bytes = d2h;
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

static bool busy(qcs_problem *P)
{
    std::lock_guard<std::mutex> g(P->mu);
    return P->running;
}

static int begin_levels(qcs_problem *P, int k, uint32_t version, int dp_bits, void *stream, uint32_t walk_base)
{
    if (!P) return QCS_ERR_ARG;
    if (busy(P)) return QCS_ERR_BUSY;
    {
        std::lock_guard<std::mutex> g(P->mu);
        if (P->res.status != QCS_SEARCHING) {
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
    }
    return level_begin(P, k, version, dp_bits, 0, (cudaStream_t)stream, walk_base);
}

int qcs_level_begin(qcs_problem *P, int k, uint32_t version, int dp_bits, void *stream)
{
    return begin_levels(P, k, version, dp_bits, stream, 0);
}

int qcs_level_walk(qcs_problem *P, uint32_t steps, void *stream)
{
    if (!P) return QCS_ERR_ARG;
    if (busy(P)) return QCS_ERR_BUSY;
    return level_walk(P, steps, (cudaStream_t)stream);
}

int qcs_level_begin_shard(qcs_problem *P, int k, uint32_t version, int dp_bits, uint32_t walk_base,
                          uint32_t total_walks, void *stream)
{
    if (!P) return QCS_ERR_ARG;
    if (total_walks > kMaxWalks || walk_base > total_walks || (uint64_t)P->p.walks > total_walks - walk_base)
        return QCS_ERR_ARG;
    return begin_levels(P, k, version, dp_bits, stream, walk_base);
}

int qcs_level_walk_out(qcs_problem *P, uint32_t steps, uint64_t *outbox, uint32_t cap, uint32_t *count,
                       void *stream)
{
    if (!P || !count || !outbox) return QCS_ERR_ARG; // a null outbox would send the points to the local table
    if (busy(P)) return QCS_ERR_BUSY;
    if (!P->lvl.active || steps == 0) return QCS_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    WalkLaunch w = P->lvl.w;
    w.steps = steps;
    w.outbox = reinterpret_cast<Slot *>(outbox);
    w.ocap = cap;
    w.ohead = count;
    CK(cudaMemsetAsync(count, 0, sizeof(uint32_t), s));
    CK(cudaMemsetAsync(P->dQhead, 0, 2 * sizeof(uint32_t), s));
    CK(cudaMemsetAsync(P->dCounters, 0, sizeof(unsigned long long) * C_NCOUNTERS, s));
    CK(launch_walks(w, s));
    return QCS_OK;
}

int qcs_shard_bin(const uint64_t *points, uint32_t count, uint32_t n_owners, uint64_t *out, uint32_t *owner_counts,
                  void *stream)
{
    if (n_owners == 0 || n_owners > 1024 || !owner_counts || (count && (!points || !out))) return QCS_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(owner_counts, 0, sizeof(uint32_t) * n_owners, s));
    CK(launch_bin_owners(reinterpret_cast<const Slot *>(points), count, n_owners, reinterpret_cast<Slot *>(out),
                         owner_counts, s));
    return QCS_OK;
}

int qcs_level_insert(qcs_problem *P, const uint64_t *points, uint32_t count, void *stream)
{
    if (!P || (count && !points)) return QCS_ERR_ARG;
    if (busy(P)) return QCS_ERR_BUSY;
    if (!P->lvl.active) return QCS_ERR_ARG;
    CK(launch_insert_points(P->lvl.w, reinterpret_cast<const Slot *>(points), count, (cudaStream_t)stream));
    return QCS_OK;
}

int qcs_level_merges(qcs_problem *P, uint64_t *out, uint32_t cap, uint32_t *n_out, void *stream)
{
    if (!P || !n_out || (cap && !out)) return QCS_ERR_ARG;
    if (!P->lvl.active) return QCS_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    uint32_t head = 0;
    CK(cudaMemcpyAsync(&head, P->dQhead, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint32_t n = std::min(std::min(head, P->lvl.w.qcap), cap);
    if (n) CK(cudaMemcpy(out, P->dQueue, sizeof(Pair) * n, cudaMemcpyDeviceToHost));
    *n_out = n;
    return QCS_OK;
}

int qcs_level_rewalk(qcs_problem *P, void *stream)
{
    if (!P) return QCS_ERR_ARG;
    if (busy(P)) return QCS_ERR_BUSY;
    return level_rewalk(P, (cudaStream_t)stream);
}

int qcs_level_collect(qcs_problem *P, void *stream, qcs_result *out)
{
    if (!P) return QCS_ERR_ARG;
    if (busy(P)) return QCS_ERR_BUSY;
    bool got = false;
    uint64_t steps = 0;
    int rc = level_collect(P, (cudaStream_t)stream, &got, &steps);
    std::lock_guard<std::mutex> g(P->mu);
    if (got) P->res.status = QCS_FOUND;
    if (out) *out = P->res;
    return rc;
}

int qcs_certify_level(qcs_problem *P, int k, void *stream, int *has_claw)
{
    if (!P || !has_claw || k < 2 || k > P->k_max) return QCS_ERR_ARG;
    if (busy(P)) return QCS_ERR_BUSY;
    bool got = false;
    const int rc = certify_level(P, k, (cudaStream_t)stream, &got);
    *has_claw = got ? 1 : 0;
    if (rc == QCS_OK && got) {
        std::lock_guard<std::mutex> g(P->mu);
        P->res.status = QCS_FOUND;
    }
    return rc;
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

int qcs_channel_from_unitary(int n, const int64_t *target, int32_t target_exp, int64_t *a, int64_t *b,
                             int32_t *exp)
{
    if (n < 1 || n > 4 || !target || !a || !b || !exp) return QCS_ERR_ARG;
    PMat C;
    const int rc = exact_channel_from_unitary(n, target, target_exp, &C);
    if (rc) return rc;
    memcpy(a, C.a.data(), sizeof(int64_t) * C.a.size());
    memcpy(b, C.b.data(), sizeof(int64_t) * C.b.size());
    *exp = C.E;
    return QCS_OK;
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

int qcs_plan_level(int n, int k, const qcs_params *p, qcs_plan *out)
{
    if (!p || !out || n < 1 || n > 4 || k < 2 || k > 15) return QCS_ERR_ARG;
    if (p->table_log2 < 4 || p->table_log2 > 34 || p->dp_bits < 1 || p->walks < 1 || p->steps_per_launch < 1 ||
        p->queue_capacity < 1)
        return QCS_ERR_ARG;
    const LevelPlan pl = plan_level_n(1 << (2 * n), k, *p);
    out->dp_bits = pl.dp_bits;
    out->walks = pl.walks;
    out->steps = pl.steps;
    out->launches_per_version = pl.launches_per_version;
    out->min_launches = pl.min_launches;
    out->points = pl.points;
    return QCS_OK;
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
