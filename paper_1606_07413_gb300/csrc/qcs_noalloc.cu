// qcs_noalloc.cu -- qcs_level_walk_static: the walk of qcs_level_walk for
// callers that must not allocate device memory.
//
// Who cannot allocate: code running where a framework's caching allocator or
// a fixed arena owns the device memory (a stray cudaMalloc fragments it, or
// fails its memory accounting once the arena has reserved what is free), and
// real-time loops that cannot afford cudaMalloc's implicit device
// synchronisation.  qcs_level_begin allocates the distinguished-point table,
// merge queue and walk states on first use; this entry point instead keeps
// the table in a fixed array of static device memory, and the caller passes
// the walk states, the merge list and the counters.
#include <cuda_runtime.h>

#include <mutex>

#include "qcs.h"
#include "qcs_internal.h"

namespace {

constexpr int kStaticTableLog2 = 18; // 2^18 slots x 16 bytes = 4 MiB

// The distinguished-point table used by every call on a device.  Every GPU
// that loads libqcs holds these 4 MiB until the process exits.  In host code
// the name is only a stand-in: the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) qcs::Slot g_static_table[1u << kStaticTableLog2];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
qcs::Slot *g_table_addr[kMaxDevices] = {};

// Device address of g_static_table on device `dev` (which must be current),
// looked up once per device and cached.  The array starts zero-filled, and a
// zero slot would read as point 0 stored by trail reference 0, so the set-up
// also marks every slot empty (all ones) and waits for that on `s`.
int static_table(int dev, cudaStream_t s, qcs::Slot **out)
{
    if (dev < 0 || dev >= kMaxDevices) return QCS_ERR_ARG;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_table_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_table);
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0xFF, sizeof(g_static_table), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return qcs::record_cuda_error(e);
        g_table_addr[dev] = static_cast<qcs::Slot *>(p);
    }
    *out = g_table_addr[dev];
    return QCS_OK;
}

} // namespace

extern "C" int qcs_level_walk_static(qcs_problem *prob, int k, uint32_t version, int dp_bits, int begin,
                                     void *walk_states, uint32_t n_walks, uint32_t steps, uint64_t *merges,
                                     uint32_t merge_cap, uint64_t *counts, void *stream)
{
    qcs::LevelCtx lv;
    uint32_t max_len = 0;
    int table_log2 = 0;
    int rc = qcs::noalloc_level(prob, k, version, dp_bits, &lv, &max_len, &table_log2);
    if (rc != QCS_OK) return rc;
    if (table_log2 > kStaticTableLog2) return QCS_ERR_ARG; // the problem's table is larger than the static one
    if (!walk_states || !counts || n_walks == 0 || n_walks > qcs::kMaxWalks || steps == 0) return QCS_ERR_ARG;
    if (merge_cap && !merges) return QCS_ERR_ARG;
    // the problem's matrices live on its own device: launching elsewhere
    // would hand the kernel another GPU's addresses
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return qcs::record_cuda_error(e);
    if (dev != prob->device) return QCS_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    qcs::Slot *table = nullptr;
    if ((rc = static_table(dev, s, &table)) != QCS_OK) return rc;

    qcs::WalkLaunch w{};
    w.lv = lv;
    w.walks = static_cast<qcs::WalkState *>(walk_states);
    w.n_walks = (int32_t)n_walks;
    w.steps = steps;
    w.max_len = max_len;
    w.table = table;
    w.table_mask = ((uint64_t)1 << table_log2) - 1;
    w.queue = reinterpret_cast<qcs::Pair *>(merges);
    w.qhead = reinterpret_cast<uint32_t *>(counts + 7); // low word of counts[7]
    w.qcap = merge_cap;
    w.counters = reinterpret_cast<unsigned long long *>(counts);
    w.stall = reinterpret_cast<uint32_t *>(counts + 7) + 1; // high word of counts[7]
    w.shape = prob->p.launch_shape;
    e = cudaMemsetAsync(counts, 0, 8 * sizeof(uint64_t), s);
    if (e == cudaSuccess && begin) {
        e = cudaMemsetAsync(table, 0xFF, sizeof(qcs::Slot) << table_log2, s);
        if (e == cudaSuccess) e = qcs::launch_init_walks(w, s);
    }
    if (e == cudaSuccess) e = qcs::launch_walks(w, s);
    return e == cudaSuccess ? QCS_OK : qcs::record_cuda_error(e);
}
