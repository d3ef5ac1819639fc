// qcs_exact.cpp -- exact host arithmetic of libqcs: targets over Z[omega],
// channel representations over Z[1/sqrt2] (Sec. 4.1), sparse R^(P) products
// and verification of decompositions (Eq. tcount_synthesis).  Used at problem set-up and for the rare claw checks;
// the walk itself runs on the GPU (qcs_walk.cu).
#include <algorithm>
#include <cstring>

#include "qcs.h"
#include "qcs_internal.h"

namespace qcs {
namespace {

struct Ovf {
    bool bad = false;
};
inline int64_t add(int64_t x, int64_t y, Ovf &o)
{
    int64_t r;
    o.bad |= __builtin_add_overflow(x, y, &r);
    return r;
}
inline int64_t sub(int64_t x, int64_t y, Ovf &o)
{
    int64_t r;
    o.bad |= __builtin_sub_overflow(x, y, &r);
    return r;
}
inline int64_t mul(int64_t x, int64_t y, Ovf &o)
{
    int64_t r;
    o.bad |= __builtin_mul_overflow(x, y, &r);
    return r;
}

// Z[w], w = e^{i pi/4}, w^4 = -1
struct Zw {
    int64_t c[4] = {0, 0, 0, 0};
};
inline Zw zw_mul(const Zw &x, const Zw &y, Ovf &o)
{
    Zw r;
    for (int i = 0; i < 4; i++) {
        if (!x.c[i]) continue;
        for (int j = 0; j < 4; j++) {
            int64_t p = mul(x.c[i], y.c[j], o);
            int t = i + j;
            if (t < 4) r.c[t] = add(r.c[t], p, o);
            else r.c[t - 4] = sub(r.c[t - 4], p, o);
        }
    }
    return r;
}
inline Zw zw_add(const Zw &x, const Zw &y, Ovf &o)
{
    Zw r;
    for (int i = 0; i < 4; i++) r.c[i] = add(x.c[i], y.c[i], o);
    return r;
}
inline Zw zw_conj(const Zw &x)
{
    Zw r;
    r.c[0] = x.c[0]; r.c[1] = -x.c[3]; r.c[2] = -x.c[2]; r.c[3] = -x.c[1];
    return r;
}
inline Zw zw_unit(int k) // w^k
{
    Zw r;
    k &= 7;
    if (k < 4) r.c[k] = 1; else r.c[k - 4] = -1;
    return r;
}
inline bool zw_zero(const Zw &x) { return !(x.c[0] | x.c[1] | x.c[2] | x.c[3]); }

inline int pc(uint32_t v) { return __builtin_popcount(v); }

// P(j)|c> = i^{m} |c ^ x>,  m = |x&z| + 2 |z&c|
inline int pauli_col_phase(int n, uint32_t j, uint32_t c)
{
    uint32_t x = j >> n, z = j & ((1u << n) - 1);
    return (pc(x & z) + 2 * pc(z & c)) & 3;
}

inline bool anticommute(int n, uint32_t p, uint32_t q)
{
    uint32_t m = (1u << n) - 1;
    return (pc(((p >> n) & (q & m)) ^ ((p & m) & (q >> n))) & 1) != 0;
}

// sign s(p, q) with R(P) P_q R(P)^dag = (P_q + s P_{p^q}) / sqrt2, q anticommuting
inline int rot_sign(int n, uint32_t p, uint32_t q) { return pauli_phase(n, p, q) == 1 ? 1 : -1; }

struct UMat {
    int dim = 0, e = 0;
    std::vector<Zw> m;
};

void reduce_unitary(UMat &U)
{
    // divide by sqrt2 = w - w^3 while every entry allows it
    while (U.e > 0) {
        for (const Zw &z : U.m)
            if (((z.c[1] - z.c[3]) & 1) || ((z.c[0] + z.c[2]) & 1)) return;
        for (Zw &z : U.m) {
            Zw r;
            r.c[0] = (z.c[1] - z.c[3]) / 2; r.c[1] = (z.c[0] + z.c[2]) / 2;
            r.c[2] = (z.c[1] + z.c[3]) / 2; r.c[3] = (z.c[2] - z.c[0]) / 2;
            z = r;
        }
        U.e--;
    }
}

int apply_gate(int n, UMat &U, int op, int a, int b, Ovf &o)
{
    const int d = U.dim;
    auto one_qubit = [&](int q, const Zw g[4], int eg) {
        if (q < 0 || q >= n) return QCS_ERR_ARG;
        const int bit = 1 << q;
        for (int r0 = 0; r0 < d; r0++) {
            if (r0 & bit) continue;
            int r1 = r0 | bit;
            for (int c = 0; c < d; c++) {
                Zw x0 = U.m[r0 * d + c], x1 = U.m[r1 * d + c];
                U.m[r0 * d + c] = zw_add(zw_mul(g[0], x0, o), zw_mul(g[1], x1, o), o);
                U.m[r1 * d + c] = zw_add(zw_mul(g[2], x0, o), zw_mul(g[3], x1, o), o);
            }
        }
        U.e += eg;
        return QCS_OK;
    };
    Zw z0, one = zw_unit(0), mone = zw_unit(4);
    switch (op) {
    case QCS_GATE_H: { Zw g[4] = {one, one, one, mone}; return one_qubit(a, g, 1); }
    case QCS_GATE_S: { Zw g[4] = {one, z0, z0, zw_unit(2)}; return one_qubit(a, g, 0); }
    case QCS_GATE_T: { Zw g[4] = {one, z0, z0, zw_unit(1)}; return one_qubit(a, g, 0); }
    case QCS_GATE_X: { Zw g[4] = {z0, one, one, z0}; return one_qubit(a, g, 0); }
    case QCS_GATE_Z: { Zw g[4] = {one, z0, z0, mone}; return one_qubit(a, g, 0); }
    case QCS_GATE_SDG: { Zw g[4] = {one, z0, z0, zw_unit(6)}; return one_qubit(a, g, 0); }
    case QCS_GATE_TDG: { Zw g[4] = {one, z0, z0, zw_unit(7)}; return one_qubit(a, g, 0); }
    case QCS_GATE_CNOT: {
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) return QCS_ERR_ARG;
        std::vector<Zw> m(U.m.size());
        for (int r = 0; r < d; r++) {
            int r2 = r ^ (((r >> a) & 1) << b);
            for (int c = 0; c < d; c++) m[r2 * d + c] = U.m[r * d + c];
        }
        U.m.swap(m);
        return QCS_OK;
    }
    case QCS_GATE_RP: {
        // R(P) = ((1 + w) I + (1 - w) P) / sqrt2^2 (Sec. 4.1)
        if (a < 1 || a >= (1 << (2 * n))) return QCS_ERR_ARG;
        uint32_t x = (uint32_t)a >> n;
        Zw opw = one, omw = one;
        opw.c[1] = 1;
        omw.c[1] = -1;
        std::vector<Zw> m(U.m.size());
        for (int r = 0; r < d; r++) {
            int src = r ^ (int)x; // P|src> = i^m |r>
            Zw ph = zw_unit(2 * pauli_col_phase(n, (uint32_t)a, (uint32_t)src));
            Zw coef = zw_mul(omw, ph, o);
            for (int c = 0; c < d; c++)
                m[r * d + c] = zw_add(zw_mul(opw, U.m[r * d + c], o), zw_mul(coef, U.m[src * d + c], o), o);
        }
        U.m.swap(m);
        U.e += 2;
        return QCS_OK;
    }
    default:
        return QCS_ERR_ARG;
    }
}

} // namespace

int pauli_phase(int n, uint32_t p, uint32_t q)
{
    uint32_t m = (1u << n) - 1;
    uint32_t px = p >> n, pz = p & m, qx = q >> n, qz = q & m, rx = px ^ qx, rz = pz ^ qz;
    return (pc(px & pz) + pc(qx & qz) + 2 * pc(pz & qx) - pc(rx & rz)) & 3;
}

void exact_reduce(PMat *M)
{
    while (M->E > 0) {
        for (int64_t a : M->a)
            if (a & 1) return;
        for (size_t i = 0; i < M->a.size(); i++) {
            int64_t a = M->a[i];
            M->a[i] = M->b[i];
            M->b[i] = a / 2;
        }
        M->E--;
    }
}

int exact_unitary_from_circuit(int n, const int32_t *gates, int n_gates, std::vector<int64_t> *u, int *e)
{
    if (n < 1 || n > 4 || n_gates < 0 || (n_gates > 0 && !gates)) return QCS_ERR_ARG;
    UMat U;
    U.dim = 1 << n;
    U.m.assign((size_t)U.dim * U.dim, Zw());
    for (int r = 0; r < U.dim; r++) U.m[r * U.dim + r] = zw_unit(0);
    Ovf o;
    for (int g = 0; g < n_gates; g++) {
        int rc = apply_gate(n, U, gates[3 * g], gates[3 * g + 1], gates[3 * g + 2], o);
        if (rc != QCS_OK) return rc;
        if (o.bad) return QCS_ERR_OVERFLOW;
        reduce_unitary(U);
    }
    u->resize(U.m.size() * 4);
    for (size_t i = 0; i < U.m.size(); i++)
        for (int t = 0; t < 4; t++) (*u)[4 * i + t] = U.m[i].c[t];
    *e = U.e;
    return QCS_OK;
}

int exact_channel_from_unitary(int n, const int64_t *uin, int e, PMat *out)
{
    if (n < 1 || n > 4 || e < 0 || !uin) return QCS_ERR_ARG;
    const int d = 1 << n, D = d * d;
    UMat U;
    U.dim = d;
    U.e = e;
    U.m.resize((size_t)d * d);
    for (int i = 0; i < d * d; i++)
        for (int t = 0; t < 4; t++) U.m[i].c[t] = uin[4 * i + t];
    reduce_unitary(U);
    Ovf o;
    // unitarity: u u^dag = 2^e I exactly
    for (int r = 0; r < d; r++)
        for (int s = 0; s < d; s++) {
            Zw acc;
            for (int t = 0; t < d; t++) acc = zw_add(acc, zw_mul(U.m[r * d + t], zw_conj(U.m[s * d + t]), o), o);
            if (o.bad || U.e > 60) return QCS_ERR_OVERFLOW;
            Zw want;
            if (r == s) want.c[0] = (int64_t)1 << U.e;
            if (memcmp(&acc, &want, sizeof(Zw)) != 0) return QCS_ERR_NOT_UNITARY;
        }
    out->D = D;
    out->a.assign((size_t)D * D, 0);
    out->b.assign((size_t)D * D, 0);
    std::vector<Zw> B((size_t)d * d), A((size_t)d * d);
    for (uint32_t j = 0; j < (uint32_t)D; j++) {
        uint32_t xj = j >> n;
        for (int r = 0; r < d; r++) // B = u P_j
            for (int c = 0; c < d; c++)
                B[r * d + c] = zw_mul(U.m[r * d + (c ^ (int)xj)], zw_unit(2 * pauli_col_phase(n, j, (uint32_t)c)), o);
        for (int r = 0; r < d; r++) // A = B u^dag
            for (int s = 0; s < d; s++) {
                Zw acc;
                for (int t = 0; t < d; t++) acc = zw_add(acc, zw_mul(B[r * d + t], zw_conj(U.m[s * d + t]), o), o);
                A[r * d + s] = acc;
            }
        for (uint32_t i = 0; i < (uint32_t)D; i++) { // Tr(P_i A) = sum_t i^{m_i(t)} A[t][t ^ x_i]
            uint32_t xi = i >> n;
            Zw tr;
            for (int t = 0; t < d; t++)
                tr = zw_add(tr, zw_mul(zw_unit(2 * pauli_col_phase(n, i, (uint32_t)t)), A[t * d + (t ^ (int)xi)], o), o);
            if (tr.c[2] != 0 || tr.c[3] != -tr.c[1]) return QCS_ERR_NOT_UNITARY;
            out->a[(size_t)i * D + j] = tr.c[0];
            out->b[(size_t)i * D + j] = tr.c[1];
        }
        if (o.bad) return QCS_ERR_OVERFLOW;
    }
    out->E = 2 * n + 2 * U.e;
    exact_reduce(out);
    return QCS_OK;
}

int exact_check_channel(int n, const PMat &C)
{
    const int D = 1 << (2 * n);
    if (C.D != D || C.E < 0 || C.E > 60) return QCS_ERR_ARG;
    if (C.a[0] == 0 && C.b[0] == 0) return QCS_ERR_NOT_UNITARY;
    Ovf o;
    // C C^T = I: sum_t c_it c_jt = delta_ij; at exponent 2E the identity is 2^E
    for (int i = 0; i < D; i++)
        for (int j = i; j < D; j++) {
            int64_t sa = 0, sb = 0;
            for (int t = 0; t < D; t++) {
                int64_t a1 = C.a[(size_t)i * D + t], b1 = C.b[(size_t)i * D + t];
                int64_t a2 = C.a[(size_t)j * D + t], b2 = C.b[(size_t)j * D + t];
                sa = add(sa, add(mul(a1, a2, o), mul(2, mul(b1, b2, o), o), o), o);
                sb = add(sb, add(mul(a1, b2, o), mul(b1, a2, o), o), o);
            }
            if (o.bad) return QCS_ERR_OVERFLOW;
            // (sa + sb sqrt2) / 2^E must be delta_ij
            if (i != j) {
                if (sa || sb) return QCS_ERR_NOT_UNITARY;
            } else if (sb != 0 || sa != ((int64_t)1 << C.E)) {
                return QCS_ERR_NOT_UNITARY;
            }
        }
    return QCS_OK;
}

bool exact_is_clifford(const PMat &Min)
{
    PMat M = Min;
    exact_reduce(&M);
    if (M.E != 0) return false;
    const int D = M.D;
    for (int c = 0; c < D; c++) {
        int nz = 0;
        for (int r = 0; r < D; r++) {
            int64_t a = M.a[(size_t)r * D + c], b = M.b[(size_t)r * D + c];
            if (!a && !b) continue;
            if (b || (a != 1 && a != -1)) return false;
            nz++;
        }
        if (nz != 1) return false;
    }
    return true;
}

// (R^ M)_i = sqrt2 M_i (i commutes with p) or M_i + s(p, i^p) M_{i^p};
// (R^T M)_i uses s(p, i).  Exponent + 1.
int exact_rhat_left(int n, uint32_t p, bool transpose, const PMat &M, PMat *out)
{
    const int D = M.D;
    if (p == 0 || p >= (uint32_t)D) return QCS_ERR_ARG;
    PMat R;
    R.D = D;
    R.E = M.E + 1;
    R.a.resize(M.a.size());
    R.b.resize(M.b.size());
    Ovf o;
    for (uint32_t i = 0; i < (uint32_t)D; i++) {
        const size_t ri = (size_t)i * D, rp = (size_t)(i ^ p) * D;
        if (!anticommute(n, p, i)) {
            for (int c = 0; c < D; c++) {
                R.a[ri + c] = mul(2, M.b[ri + c], o);
                R.b[ri + c] = M.a[ri + c];
            }
        } else {
            int s = transpose ? rot_sign(n, p, i) : rot_sign(n, p, i ^ p);
            for (int c = 0; c < D; c++) {
                R.a[ri + c] = add(M.a[ri + c], s * M.a[rp + c], o);
                R.b[ri + c] = add(M.b[ri + c], s * M.b[rp + c], o);
            }
        }
    }
    if (o.bad) return QCS_ERR_OVERFLOW;
    *out = std::move(R);
    return QCS_OK;
}

int exact_verify(int n, const PMat &C, const uint32_t *paulis, int t, PMat *Dout)
{
    PMat M = C;
    for (int j = t - 1; j >= 0; j--) {
        PMat T;
        int rc = exact_rhat_left(n, paulis[j], true, M, &T);
        if (rc != QCS_OK) return rc;
        M = std::move(T);
        exact_reduce(&M);
    }
    bool ok = exact_is_clifford(M);
    if (Dout) {
        exact_reduce(&M);
        *Dout = M;
    }
    return ok ? QCS_OK : QCS_ERR_MISMATCH;
}

} // namespace qcs
