// qcs_walk.cu -- the walk step, distinguished-point table and re-walk kernels
// of the deterministic-walk T-count search (Di Matteo & Mosca, Sec. 2-3),
// hand-written for sm_103a.
//
// A group of lanes (a warp, or 16 / 4^n lanes for n <= 3) evaluates one step
// f = h o nu o mu of one walk (Sec. 2, Fig. 1):
//   mu : decode the state into a side b and rotations q_1..q_h (Sec. 3, z_b);
//   nu : the exact product V = R^(q_h)..R^(q_1) or W = R^(q_1)^T..R^(q_h)^T
//        [R^(c)^T] C^ over Z[1/sqrt2] (Eq. mitm in channel form), taken modulo
//        right multiplication by Cliffords (Eq. tcount_synthesis);
//   h  : a coset-invariant hash back to an L-bit state.
//
// The hash is defined on the exact product M at exponent K: every column Q
// gets the 16-bit linear fingerprint L_Q = sum_i Ua[i] a_iQ + Ub[i] b_iQ mod
// 2^16, folded to phi_Q = min(L_Q, -L_Q) (so a column's sign does not matter),
// and the multiset of the phi_Q (Q >= 1) is hashed by summing
// smix(base ^ phi_Q), so a permutation of the columns does not matter either.
// Because L is linear in M's integer
// numerators and every factor acts linearly on them, L(M e_Q) =
// ((adjoint network) U)^T (M's right factor) e_Q: the kernel pushes the weight
// vector U through the transposed sparse R^ butterflies (4^n entries, h
// stages) instead of pushing all 4^n - 1 columns through them.  The V side is
// then read off directly (its right factor is the identity), and the W side is
// one contraction of the transformed weights with C^, staged in shared memory
// as signed byte quads and contracted by byte-plane dp4a, or, at n = 4 in
// launch shape 3, by f16 tensor-core MMAs in warps of their own, beside the
// warps that run the stages of another set of walks (k_walks_mma4).  The
// result is bit-identical to hashing the explicitly formed product.
//
// Also here: the distinguished-point table insert and the re-walk of merged
// trails (Sec. 3, Fig. 2), the batched forms of both, the exhaustive level
// pass (Eq. mitm), and the owner binning and insertion of distinguished
// points for a level sharded across ranks.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "qcs_internal.h"

namespace qcs {
namespace {

// launch shape of the walk kernels, tuned on GB300 by sweeping warps per CTA,
// lanes per walk, the register cap (minimum resident CTAs) and the
// contraction's unrolling
#ifndef QCS_WARPS
#define QCS_WARPS 8 // warps per CTA, n <= 2
#endif
#ifndef QCS_WARPS3
#define QCS_WARPS3 16 // warps per CTA, n = 3
#endif
#ifndef QCS_LPW3
#define QCS_LPW3 32 // lanes per walk at n = 3 (one walk per warp)
#endif
#ifndef QCS_MIN_BLOCKS3
#define QCS_MIN_BLOCKS3 2 // n = 3: 64 registers, two CTAs of 16 warps (16 walks) per SM
#endif
#ifndef QCS_GEMV_UNROLL
#define QCS_GEMV_UNROLL 2 // 32-bit word contraction (rows per unrolled step / 2)
#endif
#ifndef QCS_QUAD_UNROLL3
#define QCS_QUAD_UNROLL3 16 // byte-quad contraction, n = 3 (16 quads)
#endif
#ifndef QCS_QUAD_UNROLL4
#define QCS_QUAD_UNROLL4 16 // byte-quad contraction, n = 4 (64 quads)
#endif
constexpr int kWarps = QCS_WARPS;
constexpr int kWarps3 = QCS_WARPS3;
constexpr int kGemvUnroll = QCS_GEMV_UNROLL;

// Launch shapes of the walk kernels k_walks and k_walks_batch: warps per CTA
// and the minimum resident CTAs per SM, which caps the registers at 65536 /
// (threads x CTAs).  Shape 0 is the default; the others are chosen at run
// time (qcs_params.launch_shape, qcs_batch_params.launch_shape[n - 1]),
// e.g. by the autotuner.  Every shape evaluates the same walks with the
// same per-walk arithmetic, so the trajectories do not depend on it.
//   n <= 2: 8 warps
//   n = 3 : (16, 2) (8, 4) (32, 1) (16, 1)
//   n = 4 : (16, 1) (24, 1) (32, 1)   (one CTA per SM: C^ takes 128 KB)
//           and shape 3: the W side's contraction on the tensor cores
//           (k_walks_mma4, 12 stage and 8 MMA warps; the level walk only,
//           and only when C^ is held in int8; elsewhere shape 3 runs shape
//           0, whose figures shape_warps gives for it)
__host__ __device__ constexpr int shape_count(int nq) { return nq <= 2 ? 1 : 4; }
__host__ __device__ constexpr int shape_warps(int nq, int s)
{
    return nq <= 2 ? kWarps : nq == 3 ? (s == 1 ? 8 : s == 2 ? 32 : kWarps3) : (s == 1 ? 24 : s == 2 ? 32 : 16);
}
__host__ __device__ constexpr int shape_min_blocks(int nq, int s)
{
    return nq <= 2 ? 1 : nq == 3 ? (s == 1 ? 4 : s >= 2 ? 1 : QCS_MIN_BLOCKS3) : 1;
}
constexpr uint32_t kMaxRewalkLen = 1u << 20; // longer trails are reported as no merge

__device__ __forceinline__ uint64_t smix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// smix(base ^ phi) for phi < 2^30, given pre = base ^ (base >> 30): the
// first xorshift of the finaliser cannot see phi (it shifts by 30), so
// (base ^ phi) ^ ((base ^ phi) >> 30) = pre ^ phi, and the rest follows.
// The same value as smix(base ^ phi), one 64-bit xorshift cheaper per column.
__device__ __forceinline__ uint64_t smix_pre(uint64_t pre, uint32_t phi)
{
    uint64_t z = (pre ^ (uint64_t)phi) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <int NQ>
struct Geo {
    static constexpr int DIM = 1 << (2 * NQ);            // 4^n rows and columns
    // one walk is evaluated by LPW consecutive lanes of a warp (4^n lanes for
    // n <= 2, QCS_LPW3 at n = 3, the whole warp at n = 4), GROUPS walks per warp
    static constexpr int LPW = DIM < 32 ? DIM : (NQ == 3 ? QCS_LPW3 : 32);
    static constexpr int GROUPS = 32 / LPW;
    static constexpr int RPL = DIM / LPW;                // rows (and columns) per lane
    // n <= 3: C^ staged whole, as byte quads (8 KB at n = 3) or else as low
    // words (32 KB); n = 4: byte quads (128 KB) when every entry fits, else
    // the low words are read through L2
    static constexpr bool C_SMEM = NQ <= 3;
    static constexpr bool CQ_SMEM = NQ == 4;
    static constexpr int WARPS = NQ == 4 ? 16 : NQ == 3 ? kWarps3 : kWarps; // warps per CTA
    static constexpr int THREADS = WARPS * 32;
    static constexpr int WALKS = WARPS * GROUPS;         // walks (lane groups) per CTA
    static constexpr int QUAD_UNROLL = NQ == 4 ? QCS_QUAD_UNROLL4 : QCS_QUAD_UNROLL3;
    static constexpr int COEF_WORDS = DIM * LPW / 2; // rotation masks: a 16-bit word per Pauli and lane
    static constexpr int MAX_CHUNKS = 256;               // hash bases, one per chunk
    // shared memory: weights | C^ | coefficients | chunk bases | exchange buffers
    static constexpr size_t off_C = sizeof(uint2) * DIM;
    static constexpr size_t off_coef =
        off_C + (C_SMEM ? sizeof(uint2) * DIM * DIM : 0) + (CQ_SMEM ? 2 * DIM * DIM : 0);
    static constexpr size_t off_base = off_coef + sizeof(uint32_t) * COEF_WORDS;
    static constexpr size_t off_xchg = off_base + sizeof(uint64_t) * MAX_CHUNKS;
    static constexpr size_t smem_bytes = off_xchg + sizeof(uint2) * WALKS * DIM;
    // the same without C^, for kernels that evaluate V products only:
    // weights | coefficients | chunk bases | exchange buffers
    static constexpr size_t off_coef_v = off_C;
    static constexpr size_t off_base_v = off_coef_v + sizeof(uint32_t) * COEF_WORDS;
    static constexpr size_t off_xchg_v = off_base_v + sizeof(uint64_t) * MAX_CHUNKS;
    static constexpr size_t smem_bytes_v = off_xchg_v + sizeof(uint2) * WALKS * DIM;
};

// One launch shape of the walk kernels (see shape_warps): the CTA's warps,
// its lane groups (walks) and its shared memory, whose exchange buffers
// grow with the walks.
template <int NQ, int S>
struct Shape {
    static constexpr int WARPS = shape_warps(NQ, S);
    static constexpr int THREADS = WARPS * 32;
    static constexpr int WALKS = WARPS * Geo<NQ>::GROUPS;
    static constexpr int MIN_BLOCKS = shape_min_blocks(NQ, S);
    static constexpr size_t smem_bytes = Geo<NQ>::off_xchg + sizeof(uint2) * WALKS * Geo<NQ>::DIM;
};

// Shared-memory views of one CTA (C may point to global memory for n = 4).
template <int NQ>
struct Smem {
    uint2 *U;
    const uint2 *C;
    const uint4 *Cq;  // n >= 3: C^ as byte quads (LevelCtx::Cq layout), or null
    uint32_t *coef;
    uint64_t *base;
    uint2 *xchg; // this lane group's exchange buffer
};

__device__ __forceinline__ uint32_t shl32(uint32_t v, int s) { return s >= 32 ? 0u : v << s; }

// The lanes evaluating one walk: sub is the lane's index in its group of
// LPW lanes, mask the group's lanes (every shuffle, reduction and warp
// barrier names only the group, so the groups of a warp run independently).
struct Lanes {
    int sub;
    unsigned mask;
};

template <int NQ>
__device__ __forceinline__ Lanes thread_lanes()
{
    constexpr int L = Geo<NQ>::LPW;
    const int lane = threadIdx.x & 31, sub = lane % L;
    return Lanes{sub, (0xFFFFFFFFu >> (32 - L)) << (lane - sub)};
}

// index of the thread's lane group in its CTA
template <int NQ>
__device__ __forceinline__ int group_in_cta()
{
    return (int)(threadIdx.x >> 5) * Geo<NQ>::GROUPS + (int)(threadIdx.x & 31) / Geo<NQ>::LPW;
}

// One adjoint butterfly stage on the weight vector held by the lane group
// (row j = sub + LPW t in registers ua/ub; the group's exchange buffer carries
// the partner rows).  The forward R^(p) maps a row that commutes with p to sqrt2
// times itself, (a, b) -> (2b, a), and an anticommuting row i to
// M_i + s(p, i^p) M_{i^p}; R^(p)^T uses s(p, i) instead, and
// s(p, i^p) = -s(p, i).  The adjoints are (ua, ub) -> (ub, 2 ua) on commuting
// rows and u_j + s(p, j) u_{j^p} (adjoint of R^) or u_j - s(p, j) u_{j^p}
// (adjoint of R^T) on the others.  Commutation and sign come from the
// per-Pauli bit masks staged in shared memory.
template <int NQ, bool ADJ_OF_TRANSPOSE>
__device__ __forceinline__ void adj_stage(uint32_t p, uint32_t (&ua)[Geo<NQ>::RPL],
                                          uint32_t (&ub)[Geo<NQ>::RPL], const Smem<NQ> &sm, Lanes g)
{
    using G = Geo<NQ>;
    uint2 *su = sm.xchg;
#pragma unroll
    for (int t = 0; t < G::RPL; t++) su[g.sub + G::LPW * t] = make_uint2(ua[t], ub[t]);
    __syncwarp(g.mask);
    // this lane's rows of Pauli p: bit t anticommutes, bit 8 + t sign +1
    const uint32_t bits = reinterpret_cast<const uint16_t *>(sm.coef)[p * G::LPW + g.sub];
#pragma unroll
    for (int t = 0; t < G::RPL; t++) {
        const int j = g.sub + G::LPW * t;
        const bool anti = (bits >> t) & 1u;
        const bool plus = (bits >> (8 + t)) & 1u;
        const uint2 v = su[j ^ (int)p];
        const bool add = (plus != ADJ_OF_TRANSPOSE);
        const uint32_t na = add ? ua[t] + v.x : ua[t] - v.x;
        const uint32_t nb = add ? ub[t] + v.y : ub[t] - v.y;
        const uint32_t ca = ub[t], cb = ua[t] << 1;
        ua[t] = anti ? na : ca;
        ub[t] = anti ? nb : cb;
    }
    __syncwarp(g.mask);
}

// d = c + sum_j a_j b_j over the four bytes, a unsigned and b signed (mod 2^32)
__device__ __forceinline__ uint32_t dp4a_us(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Byte planes of the weights for the byte-quad contraction.  Fingerprints
// live mod 2^16, so a row's weight is u = u_0 + 2^8 u_1 (mod 2^16) with bytes
// u_0, u_1, and sum_i u_i c_i = sum_i u_{i,0} c_i + 2^8 sum_i u_{i,1} c_i
// (mod 2^16): an exact identity whose inner sums are byte dot products.  The
// plane words of quad q (rows 4q .. 4q+3) are written, in place of the rows
// (uint2 per row) in the lane group's exchange buffer, as uint4 number q:
// (a plane 0, a plane 1, b plane 0, b plane 1), each word holding that byte
// of the four rows' weights.
template <int NQ>
__device__ __forceinline__ void weight_planes(uint2 *su, Lanes g)
{
    const int lane = g.sub;
    using G = Geo<NQ>;
    constexpr int JOBS = G::DIM >= 2 * G::LPW ? G::DIM / (2 * G::LPW) : 1; // 2 parts x DIM/4 quads over the lanes
    const uint4 *s4 = reinterpret_cast<const uint4 *>(su);
    uint2 pl[JOBS];
#pragma unroll
    for (int r = 0; r < JOBS; r++) {
        const int job = lane + G::LPW * r, q = job >> 1, part = job & 1;
        const uint4 r01 = s4[2 * q], r23 = s4[2 * q + 1]; // rows 4q, 4q+1 and 4q+2, 4q+3
        const uint32_t u0 = part ? r01.y : r01.x, u1 = part ? r01.w : r01.z;
        const uint32_t u2 = part ? r23.y : r23.x, u3 = part ? r23.w : r23.z;
        const uint32_t lo01 = __byte_perm(u0, u1, 0x5140), lo23 = __byte_perm(u2, u3, 0x5140);
        pl[r] = make_uint2(__byte_perm(lo01, lo23, 0x5410), __byte_perm(lo01, lo23, 0x7632));
    }
    __syncwarp(g.mask);
    uint2 *w2 = su;
#pragma unroll
    for (int r = 0; r < JOBS; r++) w2[lane + G::LPW * r] = pl[r];
    __syncwarp(g.mask);
}

struct Decoded {
    int side;
    uint64_t qpack; // q_1 .. q_h, 8 bits each (q <= 255)
};

// mu (Sec. 2, the state is a concatenation of per-rotation codes): bit 0 is
// the side; rotation j reads the ell-bit field at bit 1 + ell j and maps its
// value v onto the xi non-identity Paulis as q_j = floor(v xi / 2^ell) + 1.
__device__ __forceinline__ Decoded decode(uint64_t x, const LevelCtx &lv)
{
    Decoded d;
    d.side = (int)(x & 1);
    d.qpack = 0;
    uint64_t f = x >> 1;
    for (int j = 0; j < lv.h; j++) {
        const uint32_t v = (uint32_t)f & lv.fmask;
        d.qpack |= (uint64_t)(((v * lv.xi) >> lv.ell) + 1) << (8 * j);
        f >>= lv.ell;
    }
    return d;
}

// The fingerprint weights of one decoded point pushed through its side's
// adjoint stages (row j = sub + LPW t in ua, ub): for V (side 0) the result is
// already the column fingerprints, L(V e_Q) = ua[Q]; for W (side 1) it still
// has to be contracted with C^.  All lanes of the group call it with the
// same point.
template <int NQ>
__device__ __forceinline__ void side_weights(int side, uint64_t qpack, uint32_t chunk, const LevelCtx &lv,
                                             const Smem<NQ> &sm, Lanes g, uint32_t (&ua)[Geo<NQ>::RPL],
                                             uint32_t (&ub)[Geo<NQ>::RPL])
{
    using G = Geo<NQ>;
    const Decoded dx{side, qpack};
    const int lane = g.sub;
    const int h = lv.h;

    // The weights enter the side's first adjoint stage from the stage table
    // (fingerprints live mod 2^16, and so does the table): V takes
    // R^(q_h)^* first, W takes (R^(q_1)^T)^* first.  The V side uses it only
    // when further stages follow, so no product is ever a bare lookup; the W
    // side always goes on to the contraction with C^.
    int s0 = 0;
    const uint32_t *tab = nullptr;
    uint32_t e = 0;
    if (h >= (dx.side == 0 ? 2 : 1) && lv.T1[dx.side]) {
        const uint32_t qa = (uint32_t)(dx.qpack >> (8 * (dx.side == 0 ? h - 1 : 0))) & 0xFFu;
        tab = lv.T1[dx.side];
        e = qa - 1;
        s0 = 1;
    }
#pragma unroll
    for (int t = 0; t < G::RPL; t++) {
        const int j = lane + G::LPW * t;
        if (tab) {
            const uint32_t w = __ldg(tab + (size_t)e * G::DIM + j);
            ua[t] = w & 0xFFFFu;
            ub[t] = w >> 16;
        } else {
            const uint2 u = sm.U[j];
            ua[t] = u.x;
            ub[t] = u.y;
        }
    }

    if (dx.side == 0) {
        // V side at exponent K: S R^(q_h)..R^(q_1) with S = multiply by
        // sqrt2^ev.  Weights go through S^* and R^(q_h)^* .. R^(q_1)^*; S^*
        // multiplies every row by the same power of sqrt2, so it commutes
        // with the stages and is applied after the table's.
        const int ev = lv.ev, sh = ev >> 1;
#pragma unroll
        for (int t = 0; t < G::RPL; t++) {
            const uint32_t a = ua[t], b = ub[t];
            ua[t] = (ev & 1) ? shl32(b, sh) : shl32(a, sh);
            ub[t] = (ev & 1) ? shl32(a, sh + 1) : shl32(b, sh);
        }
        for (int j = h - 1 - s0; j >= 0; j--)
            adj_stage<NQ, false>((uint32_t)(dx.qpack >> (8 * j)) & 0xFFu, ua, ub, sm, g);
    } else {
        // W side: R^(q_1)^T .. R^(q_h)^T [R^(c)^T] C^; weights go through
        // (R^(q_1)^T)^* first, ..., (R^(q_h)^T)^*, then (R^(c)^T)^*.
        for (int j = s0; j < h; j++)
            adj_stage<NQ, true>((uint32_t)(dx.qpack >> (8 * j)) & 0xFFu, ua, ub, sm, g);
        if (lv.k & 1) adj_stage<NQ, true>(chunk, ua, ub, sm, g);
    }
}

// The lane's share of the multiset hash: the sum mod 2^64 of
// smix(base ^ phi_Q) over the lane's columns Q = sub + LPW t >= 1, phi_Q the
// sign-folded 16-bit fingerprint of column Q (column 0, the identity, does
// not enter).
template <int NQ>
__device__ __forceinline__ uint64_t lane_column_sum(const uint32_t (&Lc)[Geo<NQ>::RPL], uint64_t base, int lane)
{
    uint64_t acc = 0;
    const uint64_t pre = base ^ (base >> 30);
#pragma unroll
    for (int t = 0; t < Geo<NQ>::RPL; t++) {
        const int Q = lane + Geo<NQ>::LPW * t;
        const uint32_t l = Lc[t] & 0xFFFFu, nl = (0u - l) & 0xFFFFu;
        const uint64_t e = smix_pre(pre, min(l, nl));
        acc += (Q >= 1) ? e : 0ull;
    }
    return acc;
}

// sum mod 2^64 over the lane group from three 32-bit reductions: the high
// words (mod 2^32) and the two 16-bit halves of the low words (no overflow:
// at most 32 terms)
__device__ __forceinline__ uint64_t group_sum64(uint64_t acc, unsigned mask)
{
    const uint32_t lo = (uint32_t)acc, hi = (uint32_t)(acc >> 32);
    const uint32_t s_hi = __reduce_add_sync(mask, hi);
    const uint32_t s_l0 = __reduce_add_sync(mask, lo & 0xFFFFu);
    const uint32_t s_l1 = __reduce_add_sync(mask, lo >> 16);
    return ((uint64_t)s_hi << 32) + ((uint64_t)s_l1 << 16) + (uint64_t)s_l0;
}

// nu and h of one decoded point: the exact product of side `side` (0: V,
// 1: W) for the rotations in qpack (and the chunk, odd k), its column
// fingerprints and their multiset hash with hash base `base`, as a
// full 64-bit value.  All lanes of the group call it with the same point.
template <int NQ>
__device__ uint64_t coset_hash(int side, uint64_t qpack, uint32_t chunk, uint64_t base, const LevelCtx &lv,
                               const Smem<NQ> &sm, Lanes g)
{
    using G = Geo<NQ>;
    const int lane = g.sub;
    uint32_t ua[G::RPL], ub[G::RPL], Lc[G::RPL];
    side_weights<NQ>(side, qpack, chunk, lv, sm, g, ua, ub);
    if (side == 0) {
#pragma unroll
        for (int t = 0; t < G::RPL; t++) Lc[t] = ua[t]; // L(V e_Q) = (U~)_a[Q]
    } else {
        uint2 *su = sm.xchg;
#pragma unroll
        for (int t = 0; t < G::RPL; t++) {
            su[lane + G::LPW * t] = make_uint2(ua[t], ub[t]);
            Lc[t] = 0;
        }
        __syncwarp(g.mask);
        // L(W e_Q) = sum_i U~_a[i] C_a[i][Q] + U~_b[i] C_b[i][Q]; row 0 has
        // zero weight and C[0][Q] = 0 for Q >= 1, so all rows may be summed.
        if (G::DIM >= 64 && sm.Cq) {
            // byte-plane contraction: acc[t][k] = sum over rows of byte k of
            // the weights times C^ (exact byte products), recombined below
            weight_planes<NQ>(su, g);
            const uint4 *w4 = reinterpret_cast<const uint4 *>(su);
            constexpr int CW = G::RPL / 2;
            uint32_t acc[G::RPL][2];
#pragma unroll
            for (int t = 0; t < G::RPL; t++) acc[t][0] = acc[t][1] = 0;
#pragma unroll G::QUAD_UNROLL
            for (int q = 0; q < G::DIM / 4; q++) {
                const uint4 w = w4[q]; // a plane 0, a plane 1, b plane 0, b plane 1
#pragma unroll
                for (int j = 0; j < CW; j++) {
                    const uint4 c = sm.Cq[(q * CW + j) * G::LPW + lane];
                    acc[2 * j][0] = dp4a_us(w.x, c.x, acc[2 * j][0]);
                    acc[2 * j][0] = dp4a_us(w.z, c.y, acc[2 * j][0]);
                    acc[2 * j][1] = dp4a_us(w.y, c.x, acc[2 * j][1]);
                    acc[2 * j][1] = dp4a_us(w.w, c.y, acc[2 * j][1]);
                    acc[2 * j + 1][0] = dp4a_us(w.x, c.z, acc[2 * j + 1][0]);
                    acc[2 * j + 1][0] = dp4a_us(w.z, c.w, acc[2 * j + 1][0]);
                    acc[2 * j + 1][1] = dp4a_us(w.y, c.z, acc[2 * j + 1][1]);
                    acc[2 * j + 1][1] = dp4a_us(w.w, c.w, acc[2 * j + 1][1]);
                }
            }
#pragma unroll
            for (int t = 0; t < G::RPL; t++) Lc[t] = acc[t][0] + (acc[t][1] << 8);
        } else if (G::DIM >= 32) {
            const uint4 *su4 = reinterpret_cast<const uint4 *>(su);
#pragma unroll kGemvUnroll
            for (int i = 0; i < G::DIM; i += 2) {
                const uint4 uu = su4[i >> 1]; // rows i and i + 1
                const uint2 *c0 = sm.C + i * G::DIM + lane * G::RPL;
                const uint2 *c1 = c0 + G::DIM;
#pragma unroll
                for (int t = 0; t < G::RPL; t += 2) {
                    const uint4 a = *reinterpret_cast<const uint4 *>(c0 + t);
                    const uint4 b = *reinterpret_cast<const uint4 *>(c1 + t);
                    Lc[t] += uu.x * a.x + uu.y * a.y + uu.z * b.x + uu.w * b.y;
                    Lc[t + 1] += uu.x * a.z + uu.y * a.w + uu.z * b.z + uu.w * b.w;
                }
            }
        } else {
            for (int i = 0; i < G::DIM; i++) {
                const uint2 u = su[i], c = sm.C[i * G::DIM + lane];
                Lc[0] += u.x * c.x + u.y * c.y;
            }
        }
        __syncwarp(g.mask);
    }

    // sign-invariant 16-bit column fingerprints phi_Q of the columns Q >= 1,
    // hashed as a multiset: the sum mod 2^64 of smix(base ^ phi_Q), a
    // function of the multiset alone
    return smix(group_sum64(lane_column_sum<NQ>(Lc, base, lane), g.mask));
}

// f(x): all lanes of the group call it with the same x; each gets the result.
template <int NQ>
__device__ __forceinline__ uint64_t warp_step(uint64_t x, uint32_t chunk, const LevelCtx &lv, const Smem<NQ> &sm,
                                              Lanes g)
{
    const Decoded dx = decode(x, lv);
    return coset_hash<NQ>(dx.side, dx.qpack, chunk, sm.base[chunk], lv, sm, g) & lv.maskL;
}

// Stage the weights, the rotation coefficients, the per-chunk hash bases and
// (n <= 3) all of C^ into shared memory; returns this warp's views.  WITH_C
// false: the smaller layout without C^ (smem_bytes_v), whose views of C^ are
// null; only V products may then be evaluated.
template <int NQ, bool WITH_C = true>
__device__ __forceinline__ Smem<NQ> stage(const LevelCtx &lv, unsigned char *raw)
{
    using G = Geo<NQ>;
    Smem<NQ> sm;
    sm.U = reinterpret_cast<uint2 *>(raw);
    uint2 *sC = reinterpret_cast<uint2 *>(raw + G::off_C);
    sm.coef = reinterpret_cast<uint32_t *>(raw + (WITH_C ? G::off_coef : G::off_coef_v));
    sm.base = reinterpret_cast<uint64_t *>(raw + (WITH_C ? G::off_base : G::off_base_v));
    sm.xchg = reinterpret_cast<uint2 *>(raw + (WITH_C ? G::off_xchg : G::off_xchg_v)) + group_in_cta<NQ>() * G::DIM;
    for (int i = threadIdx.x; i < G::DIM; i += blockDim.x) sm.U[i] = lv.U[i];
    for (int i = threadIdx.x; i < G::COEF_WORDS; i += blockDim.x) sm.coef[i] = lv.coef[i];
    // base(chunk) = smix(smix(seed_H ^ version) ^ (n | k << 8 | chunk << 16 | K << 32))
    const uint64_t vmix = smix(kSeedH ^ (uint64_t)lv.version);
    for (int c = threadIdx.x; c < G::MAX_CHUNKS; c += blockDim.x) {
        const uint64_t tag = (uint64_t)lv.n | ((uint64_t)lv.k << 8) | ((uint64_t)c << 16) |
                             ((uint64_t)(uint32_t)lv.K << 32);
        sm.base[c] = smix(vmix ^ tag);
    }
    sm.Cq = nullptr;
    if (!WITH_C) {
        sm.C = nullptr;
    } else if (G::C_SMEM) {
        if (lv.Cq && G::DIM >= 64) {
            uint4 *dst = reinterpret_cast<uint4 *>(sC);
            for (int i = threadIdx.x; i < G::DIM * G::DIM * 2 / 16; i += blockDim.x) dst[i] = lv.Cq[i];
            sm.Cq = dst;
        } else {
            const uint4 *src = reinterpret_cast<const uint4 *>(lv.C32);
            uint4 *dst = reinterpret_cast<uint4 *>(sC);
            for (int i = threadIdx.x; i < G::DIM * G::DIM / 2; i += blockDim.x) dst[i] = src[i];
        }
        sm.C = sC;
    } else {
        sm.C = lv.C32;
        if (G::CQ_SMEM && lv.Cq) {
            uint4 *dst = reinterpret_cast<uint4 *>(sC);
            for (int i = threadIdx.x; i < G::DIM * G::DIM * 2 / 16; i += blockDim.x) dst[i] = lv.Cq[i];
            sm.Cq = dst;
        }
    }
    __syncthreads();
    return sm;
}

template <int NQ>
__global__ void __launch_bounds__(Geo<NQ>::THREADS) k_walk_step(LevelCtx lv, uint32_t chunk, const uint64_t *__restrict__ in,
                                                        uint64_t *__restrict__ out, uint8_t *__restrict__ is_dp,
                                                        size_t count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem<NQ> sm = stage<NQ>(lv, smem_raw);
    const Lanes g = thread_lanes<NQ>();
    for (size_t i = (size_t)blockIdx.x * Geo<NQ>::WALKS + group_in_cta<NQ>(); i < count;
         i += (size_t)gridDim.x * Geo<NQ>::WALKS) {
        const uint64_t y = warp_step<NQ>(in[i], chunk, lv, sm, g);
        if (g.sub == 0) {
            out[i] = y;
            if (is_dp) is_dp[i] = (uint8_t)((y >> lv.dshift) == 0);
        }
    }
}

// starting state and chunk of trail (walk, seq) in the current version
__device__ __forceinline__ uint64_t trail_start(const LevelCtx &lv, uint32_t walk, uint32_t seq)
{
    seq &= (1u << kRefSeqBits) - 1;
    return smix(lv.seed ^ smix(((uint64_t)walk << 32) | seq) ^ ((uint64_t)lv.version << 40)) & lv.maskL;
}
__device__ __forceinline__ uint32_t trail_chunk(const LevelCtx &lv, uint64_t start)
{
    return lv.n_chunks ? 1u + (uint32_t)(smix(start ^ 0x5851F42D4C957F2Dull) % (uint64_t)lv.n_chunks) : 0u;
}
__device__ __forceinline__ uint64_t make_ref(uint32_t walk, uint32_t seq, uint32_t len)
{
    return (uint64_t)walk | ((uint64_t)(seq & ((1u << kRefSeqBits) - 1)) << kRefWalkBits) |
           ((uint64_t)len << (kRefWalkBits + kRefSeqBits));
}
__device__ __forceinline__ void split_ref(uint64_t ref, uint32_t &walk, uint32_t &seq, uint32_t &len)
{
    walk = (uint32_t)(ref & ((1u << kRefWalkBits) - 1));
    seq = (uint32_t)((ref >> kRefWalkBits) & ((1u << kRefSeqBits) - 1));
    len = (uint32_t)(ref >> (kRefWalkBits + kRefSeqBits));
}

__device__ __forceinline__ void new_trail(WalkState &st, uint32_t walk, const LevelCtx &lv)
{
    st.seq++;
    st.start = trail_start(lv, walk, st.seq);
    st.cur = st.start;
    st.len = 0;
    st.chunk = trail_chunk(lv, st.start);
}

// per-walk-group tallies, added to the job's counters by the group's first
// lane (the tensor-core kernel keeps them in 32 bits and flushes them before
// they could overflow)
template <typename T>
struct TallyOf {
    T steps = 0, w = 0, dp = 0, ab = 0, evicted = 0, duplicate = 0, pairs = 0;
};
using Tally = TallyOf<unsigned long long>;

template <typename T>
__device__ __forceinline__ void flush_tally(unsigned long long *counters, TallyOf<T> &t, Lanes g)
{
    if (g.sub == 0) {
        if (t.steps) atomicAdd(&counters[C_STEPS], t.steps);
        if (t.w) atomicAdd(&counters[C_WSTEPS], t.w);
        if (t.dp) atomicAdd(&counters[C_DPS], t.dp);
        if (t.ab) atomicAdd(&counters[C_ABANDONED], t.ab);
        if (t.evicted) atomicAdd(&counters[C_EVICTED], t.evicted);
        if (t.duplicate) atomicAdd(&counters[C_DUPLICATE], t.duplicate);
        if (t.pairs) atomicAdd(&counters[C_PAIRS], t.pairs);
    }
    t = TallyOf<T>();
}

// Store the distinguished point (Sec. 3: the triple start, end, length) in
// the slot its value hashes to, keeping the newest trail there (one 128-bit
// atomic exchange, never a wait).  If the slot held the same point from
// another trail the two trails merged: queue them for the re-walk.
template <typename WL, typename T>
__device__ void dp_insert(const WL &w, uint64_t dp, uint64_t ref, TallyOf<T> &c)
{
    if (w.outbox) {
        // DP-owner sharding: the point goes to its owner's table after the exchange
        const uint32_t idx = atomicAdd(w.ohead, 1u);
        if (idx < w.ocap) {
            Slot o;
            o.key = dp;
            o.ref = ref;
            w.outbox[idx] = o;
        }
        return;
    }
    Slot nv;
    nv.key = dp;
    nv.ref = ref;
    Slot *s = &w.table[smix(dp) & w.table_mask];
    const Slot old = atomicExch(s, nv);
    if (old.key == dp) {
        if (old.ref == ref) {
            c.duplicate++;
            return;
        }
        c.pairs++;
        const uint32_t idx = atomicAdd(w.qhead, 1u);
        if (idx < w.qcap) {
            Pair p;
            p.ref_a = old.ref;
            p.ref_b = ref;
            p.dp = dp;
            w.queue[idx] = p;
        }
    } else if (old.key != kEmptyKey) {
        c.evicted++;
    }
}

// Advance one walk by w.steps steps (Sec. 3 trails): a trail that reaches a
// distinguished point is stored and a new one starts; a trail longer than
// the cut-off is abandoned.  All lanes of the group call it.
template <int NQ, typename WL>
__device__ __forceinline__ void walk_one(const WL &w, const Smem<NQ> &sm, int local, Lanes g, Tally &t)
{
    WalkState st = w.walks[local];
    const uint32_t walk = w.walk_base + (uint32_t)local; // index among all ranks' walks
    const uint32_t steps = w.steps, max_len = w.max_len;
    const int dshift = w.lv.dshift;
    for (uint32_t s = 0; s < steps; s++) {
        const uint64_t y = warp_step<NQ>(st.cur, st.chunk, w.lv, sm, g);
        t.steps++;
        t.w += st.cur & 1;
        st.len++;
        if ((y >> dshift) == 0) {
            t.dp++;
            if (g.sub == 0) dp_insert(w, y, make_ref(walk, st.seq, st.len), t);
            __syncwarp(g.mask);
            new_trail(st, walk, w.lv);
        } else if (st.len >= max_len) {
            t.ab++;
            new_trail(st, walk, w.lv);
        } else {
            st.cur = y;
        }
    }
    if (g.sub == 0) w.walks[local] = st;
}

template <int NQ, int S>
__global__ void __launch_bounds__(Shape<NQ, S>::THREADS, Shape<NQ, S>::MIN_BLOCKS) k_walks(WalkLaunch w)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem<NQ> sm = stage<NQ>(w.lv, smem_raw);
    const Lanes g = thread_lanes<NQ>();
    Tally t;
    for (int walk = blockIdx.x * Shape<NQ, S>::WALKS + group_in_cta<NQ>(); walk < w.n_walks;
         walk += gridDim.x * Shape<NQ, S>::WALKS)
        walk_one<NQ>(w, sm, walk, g, t);
    flush_tally(w.counters, t, g);
}

// Many jobs (targets, each at its own level) in one persistent launch: the
// CTA takes a contiguous range of tasks (job, first walk) of this qubit
// count, restages the job's data when the job changes, and each lane group
// walks one of the task's Shape<NQ, S>::WALKS walks.  The job's launch record is copied to
// shared memory.
template <int NQ, int S>
__global__ void __launch_bounds__(Shape<NQ, S>::THREADS, Shape<NQ, S>::MIN_BLOCKS) k_walks_batch(BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ WalkLaunch sw;
    const Lanes g = thread_lanes<NQ>();
    const uint32_t nt = *a.n_tasks;
    int cur = -1;
    Smem<NQ> sm;
    Tally t;
    // a contiguous range of tasks per CTA, so that job changes (restaging) are rare
    const uint32_t t_begin = (uint32_t)(((uint64_t)nt * blockIdx.x) / gridDim.x);
    const uint32_t t_end = (uint32_t)(((uint64_t)nt * (blockIdx.x + 1)) / gridDim.x);
    for (uint32_t task = t_begin; task < t_end; task++) {
        const int job = (int)a.tasks[2 * task];
        const int first = (int)a.tasks[2 * task + 1];
        if (job != cur) {
            if (cur >= 0) flush_tally(sw.counters, t, g);
            __syncthreads(); // every warp is done with the previous job's data
            if (threadIdx.x == 0) sw = a.jobs[job];
            __syncthreads();
            sm = stage<NQ>(sw.lv, smem_raw);
            cur = job;
        }
        const int walk = first + group_in_cta<NQ>();
        if (walk < sw.n_walks) walk_one<NQ>(sw, sm, walk, g, t);
    }
    if (cur >= 0) flush_tally(sw.counters, t, g);
}

// ---- n = 4, launch shape 3: the W side's contraction on the tensor cores ----
//
// Warp-specialised: 12 stage warps and 8 MMA warps per CTA, one CTA per SM.
// A CTA steps 48 walks as two sets of 24; each stage warp owns two walks of
// each set.  For set X, step s:
//  A. the stage warps evaluate the set's adjoint stages (side_weights).  A V
//     walk's weights are already its column fingerprints: it hashes them into
//     its shared sum at once.  A W walk writes its weights as two byte planes
//     in f16 (bytes 0..255 are exact in f16) into its row buffer and flags
//     its slot; then every stage warp signals "rows of X ready";
//  B. the MMA warps multiply the flagged rows (compacted, up to 24: one M
//     tile, rarely two) by C^ with mma.sync m16n8k16 (f16 x f16, f32
//     accumulation), 32 columns per warp (8 accumulator chains; two MMA
//     warps per scheduler keep the tensor pipe busy), hash those columns of
//     every W walk into the walk's shared sum and signal "sums of X ready";
//  C. the stage warps finish each walk's hash and take its step.
// The stage warps run C and A of one set while the MMA warps run B of the
// other (C_0(s) A_0(s+1) beside B_1(s); C_1(s) A_1(s+1) beside B_0(s+1)), so
// the stages' integer work and the contraction overlap.  The hand-offs are
// four mbarriers; every wait on them is bounded, and a wait that runs out
// stops its warp and is counted in *w.stall (the results are then invalid).
// C^'s entries are small integers, exact in f16.  In f16 C^ is 256 KB: more
// than a CTA's shared memory, and exactly an SM's tensor memory (128 lanes x
// 512 columns of 32 bits).  So at the start each MMA warp converts the MMA
// fragments of its columns once and stores them in tensor memory
// (tcgen05.st); it reloads them with tcgen05.ld, two K-blocks at a time.
// Where theta is large the MMA warps also store the distinguished points the
// stage warps find (the instantiation COLLECT; see Rings below).
// Exactness: every product is an integer of magnitude below 2^15 (a byte
// times an int8 entry), and every partial sum of a 512-term dot product is
// below 512 x 255 x 128 < 2^24, so the f32 accumulation is exact and the
// result converts back to the integer dot product; the fingerprint is then
// L = P0 + 2^8 P1 (mod 2^16) from the two planes, as in the dp4a path.
namespace mma4 {

#ifndef QCS_WS_STAGE
#define QCS_WS_STAGE 12 // stage warps
#endif
#ifndef QCS_WS_MMA
#define QCS_WS_MMA 8 // MMA warps (two per scheduler keep the legacy tensor pipe busy)
#endif
#ifndef QCS_WS_WPW
#define QCS_WS_WPW 2 // walks of each set per stage warp
#endif
constexpr int kStageWarps = QCS_WS_STAGE, kMmaWarps = QCS_WS_MMA, kWPW = QCS_WS_WPW;
constexpr int kCtaWarps = kStageWarps + kMmaWarps, kThreads = kCtaWarps * 32;
static_assert(kStageWarps % 4 == 0, "MMA warp m must be warp m % 4 of its warpgroup (tensor-memory lanes 32 (m % 4) ..)");
static_assert(kMmaWarps == 4 || kMmaWarps == 8, "C^'s 256 columns split over 4 or 8 MMA warps");
constexpr int kSets = 2, kWalks = kWPW * kStageWarps; // walks per set
static_assert(kWalks <= 32, "a set's rows are compacted by one warp ballot");
constexpr int kCT = 32 / kMmaWarps; // column tiles of 8 per MMA warp
constexpr int kDim = 256, kK = 2 * kDim;
// shared memory: weights | rotation masks | chunk bases | 2 x 24 row buffers
// (2 KB each: a W walk's two f16 planes, and its stage exchanges) | per set,
// the bookkeeping | the walks' states | the MMA warps' row lists | mbarriers
// | tensor-memory address
constexpr size_t off_coef = sizeof(uint2) * kDim;
constexpr size_t off_base = off_coef + sizeof(uint32_t) * Geo<4>::COEF_WORDS;
constexpr size_t off_xchg = off_base + sizeof(uint64_t) * Geo<4>::MAX_CHUNKS;
static_assert(off_coef == Geo<4>::off_coef_v && off_base == Geo<4>::off_base_v, "layout of stage<4, false>");
constexpr size_t off_book = off_xchg + (size_t)2048 * kWalks * kSets;
struct Book {
    unsigned long long sum[kWalks]; // per walk slot: the multiset hash's sum
    uint64_t wbase[kWalks];         // per walk slot: the hash base (W walks)
    uint32_t isw[kWalks];           // per walk slot: 1 if it is a W walk with a row this step
};
constexpr size_t off_wst = off_book + kSets * sizeof(Book);              // WalkState [set][slot]
constexpr size_t off_rows = off_wst + sizeof(WalkState) * kSets * kWalks; // per MMA warp: slots of the compacted rows
constexpr size_t off_bar = (off_rows + kMmaWarps * kWalks + 7) & ~(size_t)7;
// The MMA warps are also the CTA's collectors (Sec. 4.2's role): they store
// the distinguished points the stage warps hand them, while they wait for a
// set's rows and after their last product, so that no stage warp waits on
// the table's atomics.  One ring per stage warp (its lane 0 the only
// producer; lane r / 8 of MMA warp r % 8 the only consumer of ring r); a
// full ring makes the producer store the point itself.
constexpr uint32_t kRing = 64;
constexpr int kCollectBits = 8;
struct Rings {
    uint64_t dp[kStageWarps][kRing], ref[kStageWarps][kRing];
    uint32_t tail[kStageWarps]; // points pushed (producer)
    uint32_t head[kStageWarps]; // points stored (collector)
    uint32_t done[kStageWarps]; // the stage warp has pushed its last point
};
constexpr size_t off_rings = off_bar + 4 * sizeof(uint64_t); // after: rows ready [2], sums ready [2]
constexpr size_t off_tmem = off_rings + sizeof(Rings);
constexpr size_t smem_bytes = off_tmem + 16;
static_assert(smem_bytes <= 227 * 1024, "shared memory of the tensor-core walk kernel");
// tensor memory: MMA warp m (the warp m % 4 of its warpgroup, so lanes
// 32 (m % 4) .. + 31 are the ones it may access) holds C^'s columns
// 8 kCT m .. 8 kCT (m + 1) - 1 in columns 64 kCT (m / 4) .. of those lanes;
// column 2 kCT kb + 2 ct + h there is the B fragment register h of K-block
// kb and column tile ct (columns 8 kCT m + 8 ct ..).
constexpr uint32_t kTmemCols = 512;
// a bounded wait gives up after this many SM clock cycles (about two seconds)
constexpr long long kWaitCycles = 1ll << 32;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Two bytes of `word` to an f16 pair, exactly: the byte permute `sel` puts
// them in the low bytes of the two halves under 0x64 (0x64b = 1024 + b in
// f16), then `bias` is subtracted (1024 for an unsigned byte; 1152 for a
// signed byte stored with 128 added).
__device__ __forceinline__ uint32_t bytes_to_f16x2(uint32_t word, uint32_t sel, float bias)
{
    const uint32_t v = __byte_perm(word, 0x64646464u, sel);
    __half2 h = *reinterpret_cast<const __half2 *>(&v);
    h = __hsub2(h, __float2half2_rn(bias));
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&a)[4], uint32_t addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

// Tensor memory (whole-warp instructions).  A load is asynchronous: its
// registers are valid after tmem_wait_ld, which takes them as operands so
// that no use can be scheduled before it.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                 "%15,%16};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
                 "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t (&v)[16], uint32_t taddr)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t (&v)[8], uint32_t taddr)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

[[maybe_unused]] __device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[8])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
                 :
                 : "memory");
}

// (the 16-register forms serve 4 MMA warps, the 8-register ones 8)
[[maybe_unused]] __device__ __forceinline__ void tmem_ld(uint32_t (&v)[16], uint32_t taddr) { tmem_ld16(v, taddr); }
[[maybe_unused]] __device__ __forceinline__ void tmem_ld(uint32_t (&v)[8], uint32_t taddr) { tmem_ld8(v, taddr); }
[[maybe_unused]] __device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t (&v)[16]) { tmem_st16(taddr, v); }
[[maybe_unused]] __device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t (&v)[8]) { tmem_st8(taddr, v); }

[[maybe_unused]] __device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                   "+r"(v[15])
                 :
                 : "memory");
}


// mbarriers (shared memory): arrive has release and try_wait acquire
// semantics at CTA scope.
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
                 : "memory");
}

// Whether the phase of parity `ph` has completed (no waiting).
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t ph)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_u32(b)), "r"(ph)
                 : "memory");
    return done != 0;
}

// One bounded try: whether the phase of parity `ph` has completed, waiting
// (suspended) for at most a system-dependent time.
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t ph)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_u32(b)), "r"(ph)
                 : "memory");
    return done != 0;
}

// Wait until the phase of parity `ph` has completed; false if the wait ran
// out (kWaitCycles).
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t ph)
{
    const uint32_t a = smem_u32(b);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(ph)
                     : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// The bounded wait, made warp-uniform: true only if every lane saw the phase
// complete (lanes that time out at different moments must not leave the warp
// split before its next warp-wide operation).
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *b, uint32_t ph)
{
    return __all_sync(0xFFFFFFFFu, mbar_wait(b, ph));
}

} // namespace mma4

// COLLECT: the MMA warps store the distinguished points (launched where
// theta >= 2^-kCollectBits); otherwise the stage warps store their own and
// the collecting code is not compiled in.
template <bool COLLECT>
__global__ void __launch_bounds__(mma4::kThreads, 1) k_walks_mma4(WalkLaunch w)
{
    using mma4::Book;
    using mma4::kWalks;
    using mma4::kK;
    using G = Geo<4>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // weights, rotation masks and chunk bases as the other walk kernels stage them
    Smem<4> sm = stage<4, false>(w.lv, smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Book *books = reinterpret_cast<Book *>(smem_raw + mma4::off_book);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + mma4::off_bar); // rows ready [2], sums ready [2]
    uint32_t *tmem_addr = reinterpret_cast<uint32_t *>(smem_raw + mma4::off_tmem);
    const Lanes g{lane, 0xFFFFFFFFu};
    const int gq = lane >> 2, q = lane & 3; // MMA fragment coordinates
    for (int i = threadIdx.x; i < mma4::kSets * kWalks; i += blockDim.x) {
        books[i / kWalks].sum[i % kWalks] = 0;
        books[i / kWalks].isw[i % kWalks] = 0;
    }
    mma4::Rings &rings = *reinterpret_cast<mma4::Rings *>(smem_raw + mma4::off_rings);
    if (threadIdx.x < mma4::kStageWarps) {
        rings.tail[threadIdx.x] = 0;
        rings.head[threadIdx.x] = 0;
        rings.done[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
        mma4::mbar_init(&bars[0], mma4::kStageWarps);
        mma4::mbar_init(&bars[1], mma4::kStageWarps);
        mma4::mbar_init(&bars[2], mma4::kMmaWarps);
        mma4::mbar_init(&bars[3], mma4::kMmaWarps);
    }
    if (warp == 0) mma4::tmem_alloc(tmem_addr, mma4::kTmemCols);
    mma4::tmem_fence_before();
    __syncthreads();
    mma4::tmem_fence_after();
    const uint32_t tmem = *tmem_addr;
    if (warp >= mma4::kStageWarps) {
        // MMA warp m: the fragments of its C^ columns, from the biased int8
        // layout: column `col` is 512 bytes, its 16-byte chunk
        // (4 (kb / 4) + q) ^ (4 (col & 1)) holds in word kb % 4 the four
        // entries of K-block kb that lane (., q) of an MMA fragment takes
        using mma4::kCT;
        const int m = warp - mma4::kStageWarps;
        const uint32_t tq = tmem + ((uint32_t)(32 * (m & 3)) << 16) + (uint32_t)(64 * kCT * (m >> 2));
        const uint32_t *cm = reinterpret_cast<const uint32_t *>(w.lv.Cm);
#pragma unroll 1
        for (int kb = 0; kb < kK / 16; kb++) {
            uint32_t v[2 * kCT];
#pragma unroll
            for (int ct = 0; ct < kCT; ct++) {
                const int ncol = 8 * kCT * m + 8 * ct + gq;
                const int chunk = (4 * (kb >> 2) + q) ^ (4 * (ncol & 1));
                const uint32_t wd = cm[((size_t)ncol * 32 + chunk) * 4 + (kb & 3)];
                v[2 * ct] = mma4::bytes_to_f16x2(wd, 0x4140, 1152.f);     // rows 2q, 2q + 1
                v[2 * ct + 1] = mma4::bytes_to_f16x2(wd, 0x4342, 1152.f); // rows 2q + 8, 2q + 9
            }
            mma4::tmem_st(tq + (uint32_t)(2 * kCT * kb), v);
        }
        mma4::tmem_wait_st();
    }
    mma4::tmem_fence_before();
    __syncthreads(); // the fragments are in tensor memory; the barriers are initialised
    mma4::tmem_fence_after();

    const LevelCtx &lv = w.lv;
    const uint32_t steps = w.steps, max_len = w.max_len;
    const int dshift = lv.dshift;
    const int n_groups = (w.n_walks + mma4::kSets * kWalks - 1) / (mma4::kSets * kWalks);
    bool stalled = false;
    constexpr bool collect = COLLECT;
    if (warp < mma4::kStageWarps) {
        // ---- stage warp: walks kWPW warp .. kWPW warp + kWPW - 1 of each set ----
        using mma4::kWPW;
        // The walks' states live in shared memory (lane 0 writes them);
        // a trail's start is only written (at a new trail), never read.
        WalkState *wst = reinterpret_cast<WalkState *>(smem_raw + mma4::off_wst); // [set][slot]
        TallyOf<uint32_t> t; // 32-bit tallies (fewer registers), flushed before they could overflow
        uint32_t ph[2] = {0, 0}; // parity of the next "sums ready" phase of each set
        for (int grp = blockIdx.x; grp < n_groups && !stalled; grp += gridDim.x) {
            const int local0 = grp * mma4::kSets * kWalks + kWPW * warp; // + X kWalks + i
            uint32_t live = 0; // bit kWPW X + i: walk i of set X exists
#pragma unroll
            for (int X = 0; X < 2; X++)
#pragma unroll
                for (int i = 0; i < kWPW; i++) {
                    const int local = local0 + X * kWalks + i;
                    if (local < w.n_walks) {
                        live |= 1u << (kWPW * X + i);
                        if (lane == 0) wst[X * kWalks + kWPW * warp + i] = w.walks[local];
                    }
                }
            __syncwarp();
            // A of set X: stages; V walks hash, W walks become matrix rows
            auto phase_a = [&](int X) {
                Book &bk = books[X];
#pragma unroll
                for (int i = 0; i < kWPW; i++) {
                    const int slot = kWPW * warp + i;
                    unsigned char *region = smem_raw + mma4::off_xchg + (size_t)2048 * (X * kWalks + slot);
                    uint32_t isw = 0;
                    if ((live >> (kWPW * X + i)) & 1u) {
                        const uint64_t cur = wst[X * kWalks + slot].cur;
                        const uint32_t chunk = wst[X * kWalks + slot].chunk;
                        sm.xchg = reinterpret_cast<uint2 *>(region);
                        const Decoded dx = decode(cur, lv);
                        const uint64_t base = sm.base[chunk];
                        uint32_t ua[G::RPL], ub[G::RPL];
                        side_weights<4>(dx.side, dx.qpack, chunk, lv, sm, g, ua, ub);
                        if (dx.side == 0) {
                            const uint64_t sum = group_sum64(lane_column_sum<4>(ua, base, lane), 0xFFFFFFFFu);
                            if (lane == 0) bk.sum[slot] = sum;
                        } else {
                            isw = 1;
                            if (lane == 0) bk.wbase[slot] = base;
                            // The K order of the product (as C^ is stored for it)
                            // makes the lane's own rows j = lane + 32 t, t = 0..7,
                            // the 16-byte chunk `lane` of each part (a: chunk lane,
                            // b: chunk 32 + lane) and plane; chunk c is stored at
                            // c ^ (slot & 7).  The region's stage exchange is done
                            // (side_weights ends with a warp sync).
                            uint4 out[4]; // (plane 0, a), (plane 1, a), (plane 0, b), (plane 1, b)
                            uint32_t *o = reinterpret_cast<uint32_t *>(out);
#pragma unroll
                            for (int e = 0; e < 4; e++) {
                                const uint32_t wa = (ua[2 * e] & 0xFFFFu) | (ua[2 * e + 1] << 16);
                                const uint32_t wb = (ub[2 * e] & 0xFFFFu) | (ub[2 * e + 1] << 16);
                                o[0 * 4 + e] = mma4::bytes_to_f16x2(wa, 0x7240, 1024.f);
                                o[1 * 4 + e] = mma4::bytes_to_f16x2(wa, 0x7341, 1024.f);
                                o[2 * 4 + e] = mma4::bytes_to_f16x2(wb, 0x7240, 1024.f);
                                o[3 * 4 + e] = mma4::bytes_to_f16x2(wb, 0x7341, 1024.f);
                            }
                            const uint32_t swz = (uint32_t)slot & 7;
                            uint4 *d4 = reinterpret_cast<uint4 *>(region);
                            d4[0 * 64 + ((uint32_t)lane ^ swz)] = out[0];
                            d4[1 * 64 + ((uint32_t)lane ^ swz)] = out[1];
                            d4[0 * 64 + ((uint32_t)(32 + lane) ^ swz)] = out[2];
                            d4[1 * 64 + ((uint32_t)(32 + lane) ^ swz)] = out[3];
                        }
                    }
                    if (lane == 0) bk.isw[slot] = isw;
                }
                __syncwarp();
                if (lane == 0) mma4::mbar_arrive(&bars[X]); // rows of X ready (this warp's part)
            };
            // C of set X: each walk's step
            auto phase_c = [&](int X) {
                Book &bk = books[X];
#pragma unroll
                for (int i = 0; i < kWPW; i++) {
                    if (!((live >> (kWPW * X + i)) & 1u)) continue;
                    const int slot = kWPW * warp + i;
                    const uint64_t y = smix(bk.sum[slot]) & lv.maskL;
                    WalkState S = wst[X * kWalks + slot];
                    const int local = local0 + X * kWalks + i;
                    const uint32_t gw = w.walk_base + (uint32_t)local;
                    t.steps++;
                    t.w += (uint32_t)(S.cur & 1);
                    S.len++;
                    if ((y >> dshift) == 0) {
                        t.dp++;
                        if (lane == 0) {
                            // to the collector, or stored here if its ring is full
                            volatile uint32_t *vt = rings.tail, *vh = rings.head;
                            const uint32_t tl = vt[warp];
                            if (collect && tl - vh[warp] < mma4::kRing) {
                                rings.dp[warp][tl % mma4::kRing] = y;
                                rings.ref[warp][tl % mma4::kRing] = make_ref(gw, S.seq, S.len);
                                __threadfence_block();
                                vt[warp] = tl + 1;
                            } else {
                                dp_insert(w, y, make_ref(gw, S.seq, S.len), t);
                            }
                        }
                        __syncwarp();
                        new_trail(S, gw, lv);
                        if (lane == 0) w.walks[local].start = S.start;
                    } else if (S.len >= max_len) {
                        t.ab++;
                        new_trail(S, gw, lv);
                        if (lane == 0) w.walks[local].start = S.start;
                    } else {
                        S.cur = y;
                    }
                    __syncwarp(); // every lane has read the old state
                    if (lane == 0) wst[X * kWalks + slot] = S;
                }
                // the sums start again from zero for the set's next products
                __syncwarp();
                if (lane < kWPW) bk.sum[kWPW * warp + lane] = 0;
                __syncwarp();
            };
            if (steps > 0) {
                phase_a(0);
                phase_a(1);
            }
            for (uint32_t step = 0; step < steps && !stalled; step++) {
#pragma unroll
                for (int X = 0; X < 2; X++) {
                    if (stalled) break;
                    if (!mma4::mbar_wait_warp(&bars[2 + X], ph[X])) {
                        stalled = true;
                        break;
                    }
                    ph[X] ^= 1u;
                    phase_c(X);
                    if (step + 1 < steps) phase_a(X);
                }
                if (t.steps >= 0x40000000u) flush_tally(w.counters, t, g); // every tally is at most t.steps
            }
            // the states back to global memory (every lane has written its last update)
#pragma unroll
            for (int X = 0; X < 2; X++)
#pragma unroll
                for (int i = 0; i < kWPW; i++)
                    if (((live >> (kWPW * X + i)) & 1u) && lane == 0) {
                        const WalkState &S = wst[X * kWalks + kWPW * warp + i];
                        WalkState *d = &w.walks[local0 + X * kWalks + i];
                        d->cur = S.cur;
                        d->len = S.len;
                        d->chunk = S.chunk;
                        d->seq = S.seq;
                    }
            __syncwarp();
        }
        flush_tally(w.counters, t, g);
        // every point this warp pushed is in its ring: the collector may stop once they are stored
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            reinterpret_cast<volatile uint32_t *>(rings.done)[warp] = 1;
        }
    } else {
        // ---- MMA warp m: C^'s columns 8 kCT m .. 8 kCT (m + 1) - 1 ----
        using mma4::kCT;
        const int m = warp - mma4::kStageWarps;
        const uint32_t tq = tmem + ((uint32_t)(32 * (m & 3)) << 16) + (uint32_t)(64 * kCT * (m >> 2));
        uint8_t *rows = smem_raw + mma4::off_rows + kWalks * m; // slots of the compacted rows
        uint32_t ph[2] = {0, 0}; // parity of the next "rows ready" phase of each set
        // collecting: lane c < 2 consumes ring m + kMmaWarps c (if there is one)
        TallyOf<uint32_t> tc;
        volatile uint32_t *vt = rings.tail, *vd = rings.done;
        const int ring = m + mma4::kMmaWarps * lane;
        const bool owner = lane < 2 && ring < mma4::kStageWarps;
        uint32_t rhead = 0;
        // store up to `most` pushed points of the owned ring (one at a time
        // while rows may become ready)
        auto drain = [&](uint32_t most) -> bool {
            bool moved = false;
            if (owner) {
                volatile uint32_t *vh = rings.head;
                const uint32_t tl = vt[ring];
                if (tl != rhead) {
                    __threadfence_block(); // the entries before tail are written
                    const uint32_t stop = tl - rhead > most ? rhead + most : tl;
                    for (; rhead != stop; rhead++)
                        dp_insert(w, rings.dp[ring][rhead % mma4::kRing], rings.ref[ring][rhead % mma4::kRing], tc);
                    __threadfence_block();
                    vh[ring] = rhead; // their slots may be reused
                    moved = true;
                }
            }
            return __any_sync(0xFFFFFFFFu, moved);
        };
        // wait for a set's rows, storing distinguished points meanwhile (with
        // nothing to store, the warp sleeps on the barrier itself)
        auto wait_rows = [&](int X) -> bool {
            const long long t0 = clock64();
            for (;;) {
                if (__all_sync(0xFFFFFFFFu, mma4::mbar_test(&bars[X], ph[X]))) return true;
                if (!drain(1)) {
                    if (__all_sync(0xFFFFFFFFu, mma4::mbar_try(&bars[X], ph[X]))) return true;
                    if (clock64() - t0 > mma4::kWaitCycles) return false;
                }
            }
        };
        const int mrow = (lane & 7) + 8 * ((lane >> 3) & 1), mkof = lane >> 4; // ldmatrix row, K offset
        for (int grp = blockIdx.x; grp < n_groups && !stalled; grp += gridDim.x)
            for (uint32_t step = 0; step < steps && !stalled; step++)
#pragma unroll 1
                for (int X = 0; X < 2; X++) {
                    if (!(collect ? wait_rows(X) : mma4::mbar_wait_warp(&bars[X], ph[X]))) {
                        stalled = true;
                        break;
                    }
                    ph[X] ^= 1u;
                    Book &bk = books[X];
                    // the W rows, compacted in slot order
                    const bool flagged = lane < kWalks && bk.isw[lane < kWalks ? lane : 0] != 0;
                    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, flagged);
                    const uint32_t nrows = (uint32_t)__popc(mask);
                    if (flagged) rows[__popc(mask & ((1u << lane) - 1u))] = (uint8_t)lane;
                    __syncwarp();
#pragma unroll 1
                    for (int tile = 0; tile < (int)(nrows + 15) / 16; tile++) {
                        const uint32_t r0 = (uint32_t)(16 * tile + mrow);
                        const uint32_t sl0 = rows[r0 < nrows ? r0 : 0]; // rows past the W walks read row 0 (unused)
                        const uint32_t arow =
                            mma4::smem_u32(smem_raw + mma4::off_xchg + (size_t)2048 * (X * kWalks + sl0));
                        const uint32_t aswz = sl0 & 7;
                        float acc[2][kCT][4]; // [plane][column tile][fragment]
#pragma unroll
                        for (int b = 0; b < 2; b++)
#pragma unroll
                            for (int c = 0; c < kCT; c++)
#pragma unroll
                                for (int d = 0; d < 4; d++) acc[b][c][d] = 0.f;
                        // one K-block: both planes' A fragments times the 8 column tiles
                        auto kblock = [&](int kb, const uint32_t(&f)[2 * kCT]) {
#pragma unroll
                            for (int p = 0; p < 2; p++) {
                                uint32_t af[4];
                                mma4::ldmatrix_x4(af, arow + 1024 * p + 16 * (((uint32_t)(2 * kb + mkof)) ^ aswz));
#pragma unroll
                                for (int ct = 0; ct < kCT; ct++) mma4::mma16816(acc[p][ct], af, f[2 * ct], f[2 * ct + 1]);
                            }
                        };
                        // C^'s fragments from tensor memory, two K-blocks (16
                        // registers) at a time, the next two loading while these are used
                        static_assert(kCT == 4, "two K-blocks per 16-register load");
                        uint32_t f0[16], f1[16];
                        auto half = [](const uint32_t(&f)[16], int i) -> const uint32_t(&)[8] {
                            return *reinterpret_cast<const uint32_t(*)[8]>(&f[8 * i]);
                        };
                        mma4::tmem_ld16(f0, tq);
#pragma unroll 1
                        for (int kb4 = 0; kb4 < kK / 64; kb4++) {
                            mma4::tmem_wait_ld(f0);
                            mma4::tmem_ld16(f1, tq + 16u * (uint32_t)(2 * kb4 + 1));
                            kblock(4 * kb4, half(f0, 0));
                            kblock(4 * kb4 + 1, half(f0, 1));
                            mma4::tmem_wait_ld(f1);
                            if (kb4 + 1 < kK / 64) mma4::tmem_ld16(f0, tq + 16u * (uint32_t)(2 * kb4 + 2));
                            kblock(4 * kb4 + 2, half(f1, 0));
                            kblock(4 * kb4 + 3, half(f1, 1));
                        }
                        // fingerprints of the warp's columns for the tile's rows gq
                        // and gq + 8, hashed into each row's walk
#pragma unroll
                        for (int hh = 0; hh < 2; hh++) {
                            const uint32_t r = (uint32_t)(16 * tile + gq + 8 * hh);
                            const bool valid = r < nrows;
                            const uint32_t sl = rows[valid ? r : 0];
                            const uint64_t base = valid ? bk.wbase[sl] : 0;
                            const uint64_t pre = base ^ (base >> 30);
                            uint64_t part = 0;
#pragma unroll
                            for (int ct = 0; ct < kCT; ct++)
#pragma unroll
                                for (int c = 0; c < 2; c++) {
                                    const int Q = 8 * kCT * m + 8 * ct + 2 * q + c;
                                    const int p0 = __float2int_rn(acc[0][ct][2 * hh + c]);
                                    const int p1 = __float2int_rn(acc[1][ct][2 * hh + c]);
                                    const uint32_t l = ((uint32_t)p0 + ((uint32_t)p1 << 8)) & 0xFFFFu;
                                    const uint32_t nl = (0u - l) & 0xFFFFu;
                                    const uint64_t e = smix_pre(pre, min(l, nl));
                                    part += (Q >= 1) ? e : 0ull;
                                }
                            part += __shfl_xor_sync(0xFFFFFFFFu, part, 1);
                            part += __shfl_xor_sync(0xFFFFFFFFu, part, 2);
                            if (valid && q == 0) atomicAdd(&bk.sum[sl], part);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mma4::mbar_arrive(&bars[2 + X]); // sums of X ready (this warp's part)
                }
        // the stage warps' last steps come after the last product: store
        // their points until each owned ring's producer is done and drained
        long long last = clock64();
        for (; collect;) {
            const bool moved = drain(mma4::kRing);
            bool fin = true;
            if (owner) {
                const bool d = vd[ring] != 0;
                __threadfence_block(); // the final tail, read after its done flag
                fin = d && vt[ring] == rhead;
            }
            if (__all_sync(0xFFFFFFFFu, fin)) break;
            if (moved) {
                last = clock64();
            } else {
                if (clock64() - last > mma4::kWaitCycles) {
                    stalled = true; // a stage warp neither pushed nor finished for too long
                    break;
                }
                __nanosleep(256);
            }
        }
        tc.evicted = __reduce_add_sync(0xFFFFFFFFu, tc.evicted);
        tc.duplicate = __reduce_add_sync(0xFFFFFFFFu, tc.duplicate);
        tc.pairs = __reduce_add_sync(0xFFFFFFFFu, tc.pairs);
        flush_tally(w.counters, tc, g);
    }
    if (stalled && lane == 0) atomicAdd(w.stall, 1u);
    // every warp's tensor-memory loads have completed (each was waited for)
    mma4::tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
        mma4::tmem_fence_after();
        mma4::tmem_dealloc(tmem, mma4::kTmemCols);
    }
}

__global__ void k_init_walks(WalkLaunch w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.n_walks) return;
    WalkState st;
    st.seq = 0;
    st.pad = 0;
    new_trail(st, w.walk_base + (uint32_t)i, w.lv);
    w.walks[i] = st;
}

// DP-owner sharding: the distinguished points received from every rank go
// into this rank's table exactly as the walk's own inserts would.
__global__ void k_insert_points(WalkLaunch w, const Slot *__restrict__ pts, uint32_t count)
{
    Tally t;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const Slot p = pts[i];
        dp_insert(w, p.key, p.ref, t);
    }
    // per-thread tallies (there are no lane groups here)
    if (t.evicted) atomicAdd(&w.counters[C_EVICTED], t.evicted);
    if (t.duplicate) atomicAdd(&w.counters[C_DUPLICATE], t.duplicate);
    if (t.pairs) atomicAdd(&w.counters[C_PAIRS], t.pairs);
}

// owner rank of a distinguished point among n ranks: the high word of a
// second finaliser (independent of the table slot, which takes smix's low
// bits) scaled to [0, n)
__device__ __forceinline__ uint32_t owner_of(uint64_t dp, uint32_t n)
{
    return (uint32_t)(((smix(dp ^ 0xD1B54A32D192ED03ull) >> 32) * (uint64_t)n) >> 32);
}

// Bin points by owner: one counting pass, a prefix over the n owners in
// every block (n <= 1024), then scatter.  Order within a bin is arbitrary
// (the table does not depend on insertion order beyond which trail a slot
// keeps).
__global__ void k_count_owners(const Slot *__restrict__ in, uint32_t count, uint32_t n, uint32_t *counts)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        atomicAdd(&counts[owner_of(in[i].key, n)], 1u);
}

__global__ void k_scatter_owners(const Slot *__restrict__ in, uint32_t count, uint32_t n,
                                 const uint32_t *__restrict__ counts, uint32_t *fill, Slot *out)
{
    extern __shared__ uint32_t start[]; // exclusive prefix of counts
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (uint32_t r = 0; r < n; r++) {
            start[r] = acc;
            acc += counts[r];
        }
    }
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const Slot p = in[i];
        const uint32_t r = owner_of(p.key, n);
        out[start[r] + atomicAdd(&fill[r], 1u)] = p;
    }
}

// Sec. 3, Fig. 2: align the longer trail, step both until the images agree,
// and classify the two distinct preimages.  At most `budget` evaluations of f
// (0: no bound); returns false with (a, la, b, lb) advanced when the budget
// ends first, so the re-walk can resume from there.  Lengths are bounded by
// the maximum trail length, so the loops end.
template <int NQ>
__device__ bool rewalk_resume(const LevelCtx &lv, uint32_t chunk, uint64_t &a, uint32_t &la, uint64_t &b,
                              uint32_t &lb, uint32_t budget, const Smem<NQ> &sm, Lanes g, unsigned long long &nf,
                              RewalkOut &r)
{
    r.chunk = chunk;
    if (la > kMaxRewalkLen || lb > kMaxRewalkLen) {
        r.cls = 5;
        r.a = a;
        r.b = b;
        return true;
    }
    if (la < lb) {
        uint64_t tx = a; a = b; b = tx;
        uint32_t tl = la; la = lb; lb = tl;
    }
    // one evaluation of f per iteration through a single call site (the step
    // is large at n = 4; inlining it once keeps the kernel's code compact):
    // align the longer trail, then step a and b in turn
    uint32_t used = 0;
    uint64_t fa = 0;
    bool second = false, checked = false;
    for (;;) {
        uint64_t x;
        if (la > lb) {
            if (budget && used >= budget) return false;
            x = a;
        } else if (!second) {
            // aligned: equal states mean one start lies on the other trail
            // (after a lockstep step this cannot first happen: the images
            // are compared there)
            if (!checked) {
                checked = true;
                if (a == b) {
                    r.cls = 0; // Robin Hood
                    r.a = r.b = a;
                    return true;
                }
            }
            if (lb == 0) {
                r.cls = 5; // no merge
                r.a = a;
                r.b = b;
                return true;
            }
            if (budget && used + 2 > budget) return false;
            x = a;
        } else {
            x = b;
        }
        const uint64_t y = warp_step<NQ>(x, chunk, lv, sm, g);
        used++;
        nf++;
        if (la > lb) {
            a = y;
            la--;
        } else if (!second) {
            fa = y;
            second = true;
        } else {
            second = false;
            if (fa == y) {
                const Decoded da = decode(a, lv), db = decode(b, lv);
                r.a = a;
                r.b = b;
                if (da.side == db.side) r.cls = (da.qpack == db.qpack) ? 1 : 2; // trivial / same side
                else r.cls = 3;                                          // claw candidate
                return true;
            }
            a = fa;
            b = y;
            la--;
            lb--;
        }
    }
}

template <int NQ>
__device__ RewalkOut rewalk_one(const LevelCtx &lv, uint32_t chunk, uint64_t sa, uint32_t la, uint64_t sb,
                                uint32_t lb, const Smem<NQ> &sm, Lanes g, unsigned long long *fevals = nullptr)
{
    RewalkOut r;
    unsigned long long nf = 0;
    rewalk_resume<NQ>(lv, chunk, sa, la, sb, lb, 0, sm, g, nf, r);
    if (fevals) *fevals += nf;
    return r;
}

// Re-walk this CTA's share of one job's queued merges; classes are counted
// per lane group and claw candidates appended to the job's candidate list.
// With `cursor` set, the lane groups take merges one at a time from that
// device counter instead of by a fixed stride, so that a few long trail
// pairs do not leave the rest of the grid idle.
template <int NQ, typename WL>
__device__ __forceinline__ void rewalk_job(const WL &w, const Smem<NQ> &sm, uint32_t p_begin, uint32_t p_end,
                                           uint32_t p_stride, Lanes g, uint32_t *cursor = nullptr)
{
    unsigned long long c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0; // per class, in registers
    unsigned long long fev = 0;
    auto claim = [&]() -> uint32_t {
        uint32_t v = 0;
        if (g.sub == 0) v = atomicAdd(cursor, 1u);
        return __shfl_sync(g.mask, v, 0, Geo<NQ>::LPW);
    };
    for (uint32_t p = cursor ? claim() : p_begin; p < p_end; p = cursor ? claim() : p + p_stride) {
        // the job's work list: first the re-walks carried from the previous
        // round (batched search), then this launch's queued merges
        uint64_t xa, xb;
        uint32_t la, lb, ca, cb;
        if (p < w.pend_in_n) {
            const Pending q = w.pend_in[p];
            xa = q.a;
            xb = q.b;
            la = q.la;
            lb = q.lb;
            ca = cb = q.chunk;
        } else {
            const Pair P = w.queue[p - w.pend_in_n];
            uint32_t wa, sa, wb, sb;
            split_ref(P.ref_a, wa, sa, la);
            split_ref(P.ref_b, wb, sb, lb);
            xa = trail_start(w.lv, wa, sa);
            xb = trail_start(w.lv, wb, sb);
            ca = trail_chunk(w.lv, xa);
            cb = trail_chunk(w.lv, xb);
        }
        RewalkOut r;
        if (ca != cb) { // the same value reached in two chunks' functions: no merge
            r.cls = 5;
        } else if (!rewalk_resume<NQ>(w.lv, ca, xa, la, xb, lb, w.rewalk_budget, sm, g, fev, r)) {
            // budget spent: carry the re-walk to the next round (if there is room)
            if (g.sub == 0) {
                const uint32_t idx = atomicAdd(w.pend_out_n, 1u);
                if (idx < w.pend_cap) {
                    Pending q;
                    q.a = xa;
                    q.b = xb;
                    q.la = la;
                    q.lb = lb;
                    q.chunk = ca;
                    q.pad = 0;
                    w.pend_out[idx] = q;
                }
            }
            continue;
        }
        c0 += r.cls == 0;
        c1 += r.cls == 1;
        c2 += r.cls == 2;
        c3 += r.cls == 3;
        c4 += r.cls == 4;
        c5 += r.cls == 5;
        if (r.cls == 3 && g.sub == 0) {
            const uint32_t idx = atomicAdd(w.ccount, 1u);
            if (idx < w.ccap) {
                Cand c;
                c.a = r.a;
                c.b = r.b;
                c.chunk = ca;
                c.pad = 0;
                w.cands[idx] = c;
            }
        }
    }
    if (g.sub == 0) {
        const unsigned long long cc[6] = {c0, c1, c2, c3, c4, c5};
#pragma unroll
        for (int c = 0; c < 6; c++)
            if (cc[c]) atomicAdd(&w.counters[C_CLS0 + c], cc[c]);
        if (c3) atomicAdd(&w.counters[C_CANDS], c3);
        if (fev) atomicAdd(&w.counters[C_RSTEPS], fev);
    }
}

template <int NQ>
__global__ void __launch_bounds__(Geo<NQ>::THREADS) k_rewalk_pairs(WalkLaunch w)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t cnt = w.pend_in_n + min(*w.qhead, w.qcap);
    if (cnt <= blockIdx.x * Geo<NQ>::WALKS) return; // no pair for this CTA (uniform)
    const Smem<NQ> sm = stage<NQ>(w.lv, smem_raw);
    rewalk_job<NQ>(w, sm, blockIdx.x * Geo<NQ>::WALKS + group_in_cta<NQ>(), cnt, gridDim.x * Geo<NQ>::WALKS,
                   thread_lanes<NQ>(), w.rw_next);
}

// The batched re-walk: the queued merges of all jobs of this qubit count
// form one index space; each CTA takes a contiguous range of it, so it
// restages a job's data only where its range enters that job.
template <int NQ>
__global__ void __launch_bounds__(Geo<NQ>::THREADS) k_rewalk_batch(BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ WalkLaunch sw;
    const uint32_t nj = *a.n_jobs;
    uint64_t total = 0;
    for (uint32_t j = 0; j < nj; j++) {
        const WalkLaunch &w = a.jobs[a.job_ids[j]];
        total += w.pend_in_n + min(*w.qhead, w.qcap);
    }
    const uint64_t lo = total * blockIdx.x / gridDim.x, hi = total * (blockIdx.x + 1) / gridDim.x;
    const Lanes g = thread_lanes<NQ>();
    uint64_t base = 0;
    for (uint32_t j = 0; j < nj && base < hi; j++) {
        const int job = (int)a.job_ids[j];
        const uint32_t cnt = a.jobs[job].pend_in_n + min(*a.jobs[job].qhead, a.jobs[job].qcap);
        if (base + cnt <= lo) {
            base += cnt;
            continue;
        }
        const uint32_t p_begin = (uint32_t)(max(lo, base) - base), p_end = (uint32_t)(min(hi, base + cnt) - base);
        base += cnt;
        __syncthreads();
        if (threadIdx.x == 0) sw = a.jobs[job];
        __syncthreads();
        const Smem<NQ> sm = stage<NQ>(sw.lv, smem_raw);
        rewalk_job<NQ>(sw, sm, p_begin + group_in_cta<NQ>(), p_end, Geo<NQ>::WALKS, g);
    }
}

template <int NQ>
__global__ void __launch_bounds__(Geo<NQ>::THREADS) k_rewalk_arrays(LevelCtx lv, uint32_t chunk, const uint64_t *sa,
                                                            const uint32_t *la, const uint64_t *sb,
                                                            const uint32_t *lb, size_t count, int32_t *cls,
                                                            uint64_t *ab)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem<NQ> sm = stage<NQ>(lv, smem_raw);
    const Lanes g = thread_lanes<NQ>();
    for (size_t p = (size_t)blockIdx.x * Geo<NQ>::WALKS + group_in_cta<NQ>(); p < count;
         p += (size_t)gridDim.x * Geo<NQ>::WALKS) {
        const RewalkOut r = rewalk_one<NQ>(lv, chunk, sa[p], la[p], sb[p], lb[p], sm, g);
        if (g.sub == 0) {
            cls[p] = r.cls;
            ab[2 * p] = r.a;
            ab[2 * p + 1] = r.b;
        }
    }
}

// The nd low base-xi digits of v, digit j in byte j (xi <= 255).
__device__ __forceinline__ uint64_t base_xi_digits(uint64_t v, uint32_t xi, int nd)
{
    uint64_t r = 0;
    for (int j = 0; j < nd; j++) {
        r |= (v % xi) << (8 * j);
        v /= xi;
    }
    return r;
}

// (d + s) mod xi^nd on packed base-xi digits (digit j in byte j, nd <= 8).
__device__ __forceinline__ uint64_t add_base_xi(uint64_t d, uint64_t s, uint32_t xi, int nd)
{
    uint64_t r = 0;
    uint32_t carry = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        if (j < nd) {
            uint32_t t = (uint32_t)((d >> (8 * j)) & 0xFFu) + (uint32_t)((s >> (8 * j)) & 0xFFu) + carry;
            carry = t >= xi ? 1u : 0u;
            t -= carry * xi;
            r |= (uint64_t)t << (8 * j);
        }
    }
    return r;
}

// Exhaustive level pass (CertArgs): one lane group per point, grid-stride.
// VONLY: the points are V products (a.side == 0), which never touch C^, so
// the CTA stages the smaller layout without it.  A point index is nd base-xi
// digits: the h rotation digits (q_j = digit + 1), then for a W point of odd
// k the chunk digit (chunk = digit + 1).  Each thread divides only for its
// first index and its stride; every further index adds the stride's digits.
template <int NQ, bool VONLY>
__global__ void __launch_bounds__(Geo<NQ>::THREADS) k_certify(CertArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem<NQ> sm = stage<NQ, !VONLY>(a.lv, smem_raw);
    const int side = VONLY ? 0 : a.side;
    const Lanes g = thread_lanes<NQ>();
    const uint32_t xi = a.lv.xi;
    const int h = a.lv.h;
    const bool has_chunk = side == 1 && (a.lv.k & 1);
    const int nd = h + (has_chunk ? 1 : 0);
    const uint64_t hmask = h >= 8 ? ~0ull : (1ull << (8 * h)) - 1;
    const uint64_t stride = (uint64_t)gridDim.x * Geo<NQ>::WALKS;
    uint64_t i = (uint64_t)blockIdx.x * Geo<NQ>::WALKS + group_in_cta<NQ>();
    // While i + stride < count, the stride is below xi^nd and its nd digits
    // are exact; otherwise the loop ends before the sum is used.
    uint64_t dig = 0, sdig = 0;
    if (i < a.count) {
        dig = base_xi_digits(a.first + i, xi, nd);
        sdig = base_xi_digits(stride, xi, nd);
    }
    for (; i < a.count; i += stride, dig = add_base_xi(dig, sdig, xi, nd)) {
        const uint64_t idx = a.first + i;
        const uint64_t qpack = (dig & hmask) + (0x0101010101010101ull & hmask);
        const uint32_t chunk = has_chunk ? (uint32_t)((dig >> (8 * h)) & 0xFFu) + 1 : 0u;
        uint64_t key = coset_hash<NQ>(side, qpack, chunk, a.base, a.lv, sm, g);
        if (key == ~0ull) key = ~0ull - 1; // ~0 marks an empty slot
        if (g.sub == 0) {
            uint64_t s = smix(key) & a.mask;
            if (a.insert) {
                // the table is at most half full, so an empty slot is always found
                for (uint64_t probe = 0; probe <= a.mask; probe++) {
                    const unsigned long long prev = atomicCAS(
                        reinterpret_cast<unsigned long long *>(&a.table[s].key), ~0ull, (unsigned long long)key);
                    if (prev == ~0ull) {
                        a.table[s].idx = idx;
                        break;
                    }
                    s = (s + 1) & a.mask;
                }
            } else {
                for (uint64_t probe = 0; probe <= a.mask; probe++) {
                    const uint64_t k2 = a.table[s].key;
                    if (k2 == ~0ull) break;
                    if (k2 == key) {
                        const uint32_t n = atomicAdd(a.n_pairs, 1u);
                        if (n < a.cap) {
                            a.pairs[2 * (size_t)n] = a.table[s].idx;
                            a.pairs[2 * (size_t)n + 1] = idx;
                        }
                    }
                    s = (s + 1) & a.mask;
                }
            }
        }
        __syncwarp(g.mask);
    }
}

int g_num_sms = 0;

// resident CTAs per SM of k_walks<NQ, S> (occupancy, cached)
template <int NQ, int S = 0>
int blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        using L = Shape<NQ, S>;
        cudaFuncSetAttribute(k_walks<NQ, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::smem_bytes);
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walks<NQ, S>, L::THREADS, L::smem_bytes);
        cached = b > 0 ? b : 1;
    }
    return cached;
}

template <int NQ, int S = 0>
unsigned grid_for(size_t units)
{
    const size_t cap = (size_t)num_sms() * (size_t)blocks_per_sm<NQ, S>();
    size_t g = (units + Shape<NQ, S>::WALKS - 1) / Shape<NQ, S>::WALKS;
    if (g > cap) g = cap;
    if (g == 0) g = 1;
    return (unsigned)g;
}

template <int NQ>
cudaError_t walk_step_n(const LevelCtx &lv, int chunk, const uint64_t *in, uint64_t *out, uint8_t *is_dp,
                        size_t count, cudaStream_t s)
{
    cudaFuncSetAttribute(k_walk_step<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo<NQ>::smem_bytes);
    k_walk_step<NQ><<<grid_for<NQ>(count), Geo<NQ>::THREADS, Geo<NQ>::smem_bytes, s>>>(lv, (uint32_t)chunk, in, out, is_dp,
                                                                               count);
    return cudaGetLastError();
}

template <int NQ, int S>
cudaError_t walks_ns(const WalkLaunch &w, cudaStream_t s)
{
    using L = Shape<NQ, S>;
    k_walks<NQ, S><<<grid_for<NQ, S>((size_t)w.n_walks), L::THREADS, L::smem_bytes, s>>>(w);
    return cudaGetLastError();
}

// the tensor-core level walk (n = 4, launch shape 3): one CTA per SM
cudaError_t walks_mma4(const WalkLaunch &w, cudaStream_t s)
{
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncSetAttribute(k_walks_mma4<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mma4::smem_bytes);
        cudaFuncSetAttribute(k_walks_mma4<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mma4::smem_bytes);
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walks_mma4<false>, mma4::kThreads, mma4::smem_bytes);
        per_sm = b > 0 ? b : 1;
    }
    if (!w.stall) return cudaErrorInvalidValue; // a stalled wait must have somewhere to be counted
    const size_t groups = ((size_t)w.n_walks + mma4::kSets * mma4::kWalks - 1) / (mma4::kSets * mma4::kWalks);
    size_t grid = (size_t)num_sms() * (size_t)per_sm;
    if (grid > groups) grid = groups;
    if (grid == 0) grid = 1;
    // d_theta = L - dshift: the MMA warps collect where theta >= 2^-kCollectBits
    const int dtheta = __builtin_popcountll(w.lv.maskL) - w.lv.dshift;
    if (dtheta <= mma4::kCollectBits)
        k_walks_mma4<true><<<(unsigned)grid, mma4::kThreads, mma4::smem_bytes, s>>>(w);
    else
        k_walks_mma4<false><<<(unsigned)grid, mma4::kThreads, mma4::smem_bytes, s>>>(w);
    return cudaGetLastError();
}

template <int NQ>
cudaError_t walks_n(const WalkLaunch &w, cudaStream_t s)
{
    switch (w.shape) {
    case 0: return walks_ns<NQ, 0>(w, s);
    case 1: if constexpr (shape_count(NQ) > 1) return walks_ns<NQ, 1>(w, s); break;
    case 2: if constexpr (shape_count(NQ) > 2) return walks_ns<NQ, 2>(w, s); break;
    case 3:
        if constexpr (NQ == 4) return w.lv.Cm ? walks_mma4(w, s) : walks_ns<4, 0>(w, s);
        else if constexpr (shape_count(NQ) > 3) return walks_ns<NQ, 3>(w, s);
        break;
    }
    return cudaErrorInvalidValue;
}

// CTAs of the persistent batch walk kernel: every SM x its resident CTAs
template <int NQ, int S>
int batch_grid()
{
    static int g = 0;
    if (!g) {
        using L = Shape<NQ, S>;
        cudaFuncSetAttribute(k_walks_batch<NQ, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::smem_bytes);
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walks_batch<NQ, S>, L::THREADS, L::smem_bytes);
        g = num_sms() * (b > 0 ? b : 1);
    }
    return g;
}

template <int NQ, int S>
cudaError_t walks_batch_ns(const BatchArgs &a, cudaStream_t s)
{
    using L = Shape<NQ, S>;
    k_walks_batch<NQ, S><<<batch_grid<NQ, S>(), L::THREADS, L::smem_bytes, s>>>(a);
    return cudaGetLastError();
}

template <int NQ>
cudaError_t walks_batch_n(int shape, const BatchArgs &a, cudaStream_t s)
{
    switch (shape) {
    case 0: return walks_batch_ns<NQ, 0>(a, s);
    case 1: if constexpr (shape_count(NQ) > 1) return walks_batch_ns<NQ, 1>(a, s); break;
    case 2: if constexpr (shape_count(NQ) > 2) return walks_batch_ns<NQ, 2>(a, s); break;
    case 3:
        if constexpr (NQ == 4) return walks_batch_ns<4, 0>(a, s); // no batched tensor-core form
        else if constexpr (shape_count(NQ) > 3) return walks_batch_ns<NQ, 3>(a, s);
        break;
    }
    return cudaErrorInvalidValue;
}

template <int NQ>
cudaError_t rewalk_batch_n(const BatchArgs &a, cudaStream_t s)
{
    static int g = 0;
    if (!g) {
        cudaFuncSetAttribute(k_rewalk_batch<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Geo<NQ>::smem_bytes);
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_rewalk_batch<NQ>, Geo<NQ>::THREADS, Geo<NQ>::smem_bytes);
        g = num_sms() * (b > 0 ? b : 1);
    }
    k_rewalk_batch<NQ><<<g, Geo<NQ>::THREADS, Geo<NQ>::smem_bytes, s>>>(a);
    return cudaGetLastError();
}

template <int NQ>
cudaError_t rewalk_pairs_n(const WalkLaunch &w, cudaStream_t s)
{
    cudaFuncSetAttribute(k_rewalk_pairs<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)Geo<NQ>::smem_bytes);
    k_rewalk_pairs<NQ><<<grid_for<NQ>(w.qcap), Geo<NQ>::THREADS, Geo<NQ>::smem_bytes, s>>>(w);
    return cudaGetLastError();
}

template <int NQ>
cudaError_t rewalk_arrays_n(const LevelCtx &lv, int chunk, const uint64_t *sa, const uint32_t *la,
                            const uint64_t *sb, const uint32_t *lb, size_t count, int32_t *cls, uint64_t *ab,
                            cudaStream_t s)
{
    cudaFuncSetAttribute(k_rewalk_arrays<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)Geo<NQ>::smem_bytes);
    k_rewalk_arrays<NQ><<<grid_for<NQ>(count), Geo<NQ>::THREADS, Geo<NQ>::smem_bytes, s>>>(lv, (uint32_t)chunk, sa, la,
                                                                                   sb, lb, count, cls, ab);
    return cudaGetLastError();
}

template <int NQ, bool VONLY>
cudaError_t certify_nv(const CertArgs &a, cudaStream_t s)
{
    constexpr size_t smem = VONLY ? Geo<NQ>::smem_bytes_v : Geo<NQ>::smem_bytes;
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncSetAttribute(k_certify<NQ, VONLY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_certify<NQ, VONLY>, Geo<NQ>::THREADS, smem);
        per_sm = b > 0 ? b : 1;
    }
    const size_t cap = (size_t)num_sms() * (size_t)per_sm;
    size_t grid = (a.count + Geo<NQ>::WALKS - 1) / Geo<NQ>::WALKS;
    if (grid > cap) grid = cap;
    k_certify<NQ, VONLY><<<(unsigned)grid, Geo<NQ>::THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NQ>
cudaError_t certify_n(const CertArgs &a, cudaStream_t s)
{
    return a.side == 0 ? certify_nv<NQ, true>(a, s) : certify_nv<NQ, false>(a, s);
}

} // namespace

cudaError_t launch_certify(const CertArgs &a, cudaStream_t s)
{
    if (a.count == 0) return cudaSuccess;
    switch (a.lv.n) {
    case 1: return certify_n<1>(a, s);
    case 2: return certify_n<2>(a, s);
    case 3: return certify_n<3>(a, s);
    case 4: return certify_n<4>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

int num_sms()
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

int lanes_per_walk(int n) { return n == 4 ? Geo<4>::LPW : n == 3 ? Geo<3>::LPW : n == 2 ? Geo<2>::LPW : Geo<1>::LPW; }

int launch_shapes(int n) { return n == 4 ? shape_count(4) : n == 3 ? shape_count(3) : shape_count(2); }

int shape_warps_of(int n, int shape) { return n == 4 && shape == 3 ? mma4::kCtaWarps : shape_warps(n, shape); }

int shape_min_blocks_of(int n, int shape) { return shape_min_blocks(n, shape); }

int walks_per_task(int n, int shape) { return shape_warps(n, shape) * (32 / lanes_per_walk(n)); }

int walk_blocks_per_sm(int n)
{
    switch (n) {
    case 1: return blocks_per_sm<1>();
    case 2: return blocks_per_sm<2>();
    case 3: return blocks_per_sm<3>();
    default: return blocks_per_sm<4>();
    }
}

cudaError_t launch_walk_step(const LevelCtx &lv, int chunk, const uint64_t *in, uint64_t *out, uint8_t *is_dp,
                             size_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    switch (lv.n) {
    case 1: return walk_step_n<1>(lv, chunk, in, out, is_dp, count, s);
    case 2: return walk_step_n<2>(lv, chunk, in, out, is_dp, count, s);
    case 3: return walk_step_n<3>(lv, chunk, in, out, is_dp, count, s);
    case 4: return walk_step_n<4>(lv, chunk, in, out, is_dp, count, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_init_walks(const WalkLaunch &w, cudaStream_t s)
{
    if (w.n_walks > 0) k_init_walks<<<(w.n_walks + 255) / 256, 256, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_insert_points(const WalkLaunch &w, const Slot *pts, uint32_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<uint64_t>(((uint64_t)count + 255) / 256, (uint64_t)num_sms() * 8);
    k_insert_points<<<grid, 256, 0, s>>>(w, pts, count);
    return cudaGetLastError();
}

cudaError_t launch_bin_owners(const Slot *in, uint32_t count, uint32_t n_owners, Slot *out, uint32_t *counts,
                              cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    if (n_owners == 0 || n_owners > 1024) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)std::min<uint64_t>(((uint64_t)count + 255) / 256, (uint64_t)num_sms() * 8);
    k_count_owners<<<grid, 256, 0, s>>>(in, count, n_owners, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the scatter's fill cursors sit right after the counts
    e = cudaMemsetAsync(counts + n_owners, 0, sizeof(uint32_t) * n_owners, s);
    if (e != cudaSuccess) return e;
    k_scatter_owners<<<grid, 256, sizeof(uint32_t) * n_owners, s>>>(in, count, n_owners, counts,
                                                                   counts + n_owners, out);
    return cudaGetLastError();
}

cudaError_t launch_walks(const WalkLaunch &w, cudaStream_t s)
{
    switch (w.lv.n) {
    case 1: return walks_n<1>(w, s);
    case 2: return walks_n<2>(w, s);
    case 3: return walks_n<3>(w, s);
    case 4: return walks_n<4>(w, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rewalk_pairs(const WalkLaunch &w, cudaStream_t s)
{
    switch (w.lv.n) {
    case 1: return rewalk_pairs_n<1>(w, s);
    case 2: return rewalk_pairs_n<2>(w, s);
    case 3: return rewalk_pairs_n<3>(w, s);
    case 4: return rewalk_pairs_n<4>(w, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_walks_batch(int n, int shape, const BatchArgs &a, cudaStream_t s)
{
    switch (n) {
    case 1: return walks_batch_n<1>(shape, a, s);
    case 2: return walks_batch_n<2>(shape, a, s);
    case 3: return walks_batch_n<3>(shape, a, s);
    case 4: return walks_batch_n<4>(shape, a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rewalk_batch(int n, const BatchArgs &a, cudaStream_t s)
{
    switch (n) {
    case 1: return rewalk_batch_n<1>(a, s);
    case 2: return rewalk_batch_n<2>(a, s);
    case 3: return rewalk_batch_n<3>(a, s);
    case 4: return rewalk_batch_n<4>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rewalk_arrays(const LevelCtx &lv, int chunk, const uint64_t *sa, const uint32_t *la,
                                 const uint64_t *sb, const uint32_t *lb, size_t count, int32_t *cls, uint64_t *ab,
                                 cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    switch (lv.n) {
    case 1: return rewalk_arrays_n<1>(lv, chunk, sa, la, sb, lb, count, cls, ab, s);
    case 2: return rewalk_arrays_n<2>(lv, chunk, sa, la, sb, lb, count, cls, ab, s);
    case 3: return rewalk_arrays_n<3>(lv, chunk, sa, la, sb, lb, count, cls, ab, s);
    case 4: return rewalk_arrays_n<4>(lv, chunk, sa, la, sb, lb, count, cls, ab, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace qcs
