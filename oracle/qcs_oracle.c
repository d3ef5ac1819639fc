/*
 * qcs_oracle.c -- CPU oracle for the deterministic-walk optimal T-count search
 * of Di Matteo & Mosca, "Parallelizing quantum circuit synthesis" (Sec. 2-4,
 * Appendix).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg load this library.  It is deliberately plain,
 * slow and single-threaded: every quantity is computed from its definition,
 * with no blocking, fusion or reordering, so that it can be checked against the
 * paper by eye.  It shares no code, header, table or constant generator with
 * the CUDA path; both sides implement the same written specification.
 *
 * Every integer operation that could overflow is checked and aborts loudly.
 *
 * Conventions the paper leaves open (fixed here, and in the same words for the
 * CUDA path):
 *  - Pauli code j in [0, 4^n): x = j >> n, z = j & (2^n - 1), qubit q is bit q,
 *    P(j) = i^{|x & z|} X^x Z^z (Hermitian).  X^x Z^z |c> = (-1)^{|z & c|} |c ^ x>.
 *  - Exact reals in Z[1/sqrt2] are pairs (a, b) meaning (a + b sqrt2) / sqrt2^E
 *    with one exponent E shared by a whole matrix.
 *  - Walk state x (L bits): side = x & 1 (0: V side, 1: W side); rotation j
 *    (0-based) reads the l-bit field at bit 1 + l j, l = min(16, (L-1)/h), and
 *    maps its value v to q_j = floor(v xi / 2^l) + 1.
 *  - V_q = R(q_h) ... R(q_1);  W_q' = R(q'_1)^T ... R(q'_h)^T [R(c)^T] C  (Eq. mitm
 *    in channel form; the bracket is present for odd k, chunk c in 1..xi).
 *    Both are represented at K = sde(C) + (k & 1) + h.
 *  - Walk hash: per column Q >= 1 a 16-bit linear fingerprint
 *    L_Q = sum_{i>=1} Ua[i] a_iQ + Ub[i] b_iQ (mod 2^16), folded to
 *    phi_Q = min(L_Q, -L_Q mod 2^16) (invariant under the column's sign).  The
 *    multiset {phi_Q} is what a Clifford (a signed permutation of the columns
 *    Q >= 1) leaves unchanged; it is hashed as the sum mod 2^64 of the
 *    SplitMix64 finaliser (Steele, Lea & Flood 2014) of base ^ phi_Q over the
 *    columns, finalised once more.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* checked 64-bit integer arithmetic                                   */
/* ------------------------------------------------------------------ */
static void die(const char *msg)
{
    fprintf(stderr, "qcs_oracle: fatal: %s\n", msg);
    abort();
}
static int64_t cadd(int64_t x, int64_t y)
{
    int64_t r;
    if (__builtin_add_overflow(x, y, &r)) die("int64 overflow in add");
    return r;
}
static int64_t csub(int64_t x, int64_t y)
{
    int64_t r;
    if (__builtin_sub_overflow(x, y, &r)) die("int64 overflow in sub");
    return r;
}
static int64_t cmul(int64_t x, int64_t y)
{
    int64_t r;
    if (__builtin_mul_overflow(x, y, &r)) die("int64 overflow in mul");
    return r;
}
static void *xcalloc(size_t n, size_t s)
{
    void *p = calloc(n ? n : 1, s);
    if (!p) die("out of memory");
    return p;
}
static int popc(uint32_t v) { return __builtin_popcount(v); }

/* ------------------------------------------------------------------ */
/* Z[omega], omega = e^{i pi/4}: c0 + c1 w + c2 w^2 + c3 w^3, w^4 = -1  */
/* ------------------------------------------------------------------ */
typedef struct { int64_t c[4]; } zw;

static zw zw_zero(void) { zw r = {{0, 0, 0, 0}}; return r; }
static zw zw_omega_pow(int k)
{
    zw r = zw_zero();
    k = ((k % 8) + 8) % 8;
    if (k < 4) r.c[k] = 1; else r.c[k - 4] = -1;
    return r;
}
static zw zw_add(zw x, zw y)
{
    zw r;
    for (int i = 0; i < 4; i++) r.c[i] = cadd(x.c[i], y.c[i]);
    return r;
}
static zw zw_mul(zw x, zw y)
{
    zw r = zw_zero();
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            int64_t p = cmul(x.c[i], y.c[j]);
            if (i + j < 4) r.c[i + j] = cadd(r.c[i + j], p);
            else r.c[i + j - 4] = csub(r.c[i + j - 4], p);
        }
    return r;
}
/* complex conjugate: conj(w) = w^7 = -w^3, conj(w^2) = -w^2, conj(w^3) = -w */
static zw zw_conj(zw x)
{
    zw r = {{x.c[0], -x.c[3], -x.c[2], -x.c[1]}};
    return r;
}
static int zw_is_zero(zw x) { return !x.c[0] && !x.c[1] && !x.c[2] && !x.c[3]; }
/* x / sqrt2 lies in Z[w] iff c1 = c3 and c0 = c2 (mod 2); sqrt2 = w - w^3 */
static int zw_div_sqrt2_ok(zw x)
{
    return (((x.c[1] - x.c[3]) & 1) == 0) && (((x.c[0] + x.c[2]) & 1) == 0);
}
static zw zw_div_sqrt2(zw x)
{
    zw r = {{(x.c[1] - x.c[3]) / 2, (x.c[0] + x.c[2]) / 2,
             (x.c[1] + x.c[3]) / 2, (x.c[2] - x.c[0]) / 2}};
    return r;
}

/* ------------------------------------------------------------------ */
/* Paulis (Sec. 4.1: binary symplectic codes)                          */
/* ------------------------------------------------------------------ */
/* P(j)|c> = i^m |c ^ x>;  returns m in 0..3 and the image basis index. */
static int pauli_on_basis(int n, int j, int c, int *image)
{
    int x = j >> n, z = j & ((1 << n) - 1);
    *image = c ^ x;
    return (popc((uint32_t)(x & z)) + 2 * popc((uint32_t)(z & c))) & 3;
}

/* lambda with P(p) P(q) = i^lambda P(p ^ q), read off by applying both sides
 * to the basis state |0>. */
OR_API int or_pauli_phase(int n, int p, int q)
{
    int y1, y2, y3;
    int m1 = pauli_on_basis(n, q, 0, &y1);
    int m2 = pauli_on_basis(n, p, y1, &y2);
    int m3 = pauli_on_basis(n, p ^ q, 0, &y3);
    if (y2 != y3) die("pauli product lands on a different basis state");
    return ((m1 + m2 - m3) % 4 + 4) % 4;
}

static int pauli_anticommute(int n, int p, int q)
{
    return or_pauli_phase(n, p, q) != or_pauli_phase(n, q, p);
}

/* ------------------------------------------------------------------ */
/* Unitaries over Z[w] / sqrt2^e (the boundary form of a target)       */
/* ------------------------------------------------------------------ */
enum { G_H = 0, G_S, G_CNOT, G_T, G_RP, G_X, G_Z, G_SDG, G_TDG };

typedef struct { int n, dim, e; zw *m; } umat; /* value m / sqrt2^e */

static umat um_new(int n)
{
    umat u;
    u.n = n; u.dim = 1 << n; u.e = 0;
    u.m = (zw *)xcalloc((size_t)u.dim * u.dim, sizeof(zw));
    return u;
}
static void um_free(umat *u) { free(u->m); u->m = NULL; }

static umat um_mul(const umat *A, const umat *B)
{
    umat R = um_new(A->n);
    int d = A->dim;
    R.e = A->e + B->e;
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) {
            zw s = zw_zero();
            for (int t = 0; t < d; t++)
                s = zw_add(s, zw_mul(A->m[r * d + t], B->m[t * d + c]));
            R.m[r * d + c] = s;
        }
    return R;
}
static umat um_dagger(const umat *A)
{
    umat R = um_new(A->n);
    int d = A->dim;
    R.e = A->e;
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) R.m[r * d + c] = zw_conj(A->m[c * d + r]);
    return R;
}
static void um_reduce(umat *A)
{
    size_t cnt = (size_t)A->dim * A->dim;
    for (;;) {
        if (A->e <= 0) return;
        for (size_t i = 0; i < cnt; i++)
            if (!zw_div_sqrt2_ok(A->m[i])) return;
        for (size_t i = 0; i < cnt; i++) A->m[i] = zw_div_sqrt2(A->m[i]);
        A->e -= 1;
    }
}
static umat um_pauli(int n, int j)
{
    umat P = um_new(n);
    for (int c = 0; c < P.dim; c++) {
        int r;
        int m = pauli_on_basis(n, j, c, &r);
        P.m[r * P.dim + c] = zw_omega_pow(2 * m);
    }
    return P;
}
/* embed a one-qubit gate g (2x2, exponent eg) on qubit q */
static umat um_one_qubit(int n, int q, const zw g[4], int eg)
{
    umat G = um_new(n);
    G.e = eg;
    int bit = 1 << q;
    for (int r = 0; r < G.dim; r++)
        for (int c = 0; c < G.dim; c++)
            if ((r & ~bit) == (c & ~bit))
                G.m[r * G.dim + c] = g[((r >> q) & 1) * 2 + ((c >> q) & 1)];
    return G;
}
/* the textbook gate matrix of one circuit row */
static umat um_gate(int n, int op, int a, int b)
{
    zw one = zw_omega_pow(0), zero = zw_zero(), mone = zw_omega_pow(4);
    if (op == G_CNOT) {
        umat G = um_new(n);
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) die("bad CNOT operands");
        for (int c = 0; c < G.dim; c++) {
            int r = c ^ (((c >> a) & 1) << b);
            G.m[r * G.dim + c] = one;
        }
        return G;
    }
    if (op == G_RP) {
        /* R(P) = 1/2 (1 + w) I + 1/2 (1 - w) P   (Eq. for R(P_j), Sec. 4.1) */
        if (a < 1 || a >= (1 << (2 * n))) die("bad RP code");
        umat P = um_pauli(n, a);
        umat G = um_new(n);
        zw onepw = zw_add(one, zw_omega_pow(1));
        zw onemw = zw_add(one, zw_omega_pow(5));
        G.e = 2;
        for (int i = 0; i < G.dim * G.dim; i++) G.m[i] = zw_mul(onemw, P.m[i]);
        for (int r = 0; r < G.dim; r++) G.m[r * G.dim + r] = zw_add(G.m[r * G.dim + r], onepw);
        um_free(&P);
        return G;
    }
    if (a < 0 || a >= n) die("bad qubit index");
    zw g[4];
    int eg = 0;
    switch (op) {
    case G_H: g[0] = one; g[1] = one; g[2] = one; g[3] = mone; eg = 1; break;
    case G_S: g[0] = one; g[1] = zero; g[2] = zero; g[3] = zw_omega_pow(2); break;
    case G_T: g[0] = one; g[1] = zero; g[2] = zero; g[3] = zw_omega_pow(1); break;
    case G_X: g[0] = zero; g[1] = one; g[2] = one; g[3] = zero; break;
    case G_Z: g[0] = one; g[1] = zero; g[2] = zero; g[3] = mone; break;
    case G_SDG: g[0] = one; g[1] = zero; g[2] = zero; g[3] = zw_omega_pow(6); break;
    case G_TDG: g[0] = one; g[1] = zero; g[2] = zero; g[3] = zw_omega_pow(7); break;
    default: die("unknown gate op");
    }
    return um_one_qubit(n, a, g, eg);
}

static umat um_from_circuit(int n, const int32_t *gates, int ngates)
{
    umat U = um_new(n);
    for (int r = 0; r < U.dim; r++) U.m[r * U.dim + r] = zw_omega_pow(0);
    for (int g = 0; g < ngates; g++) {
        umat G = um_gate(n, gates[3 * g], gates[3 * g + 1], gates[3 * g + 2]);
        umat V = um_mul(&G, &U); /* the later gate acts on the left */
        um_free(&G);
        um_free(&U);
        U = V;
        um_reduce(&U);
    }
    return U;
}

OR_API int or_unitary_from_circuit(int n, const int32_t *gates, int ngates, int64_t *u_out, int *e_out)
{
    if (n < 1 || n > 4) return -1;
    umat U = um_from_circuit(n, gates, ngates);
    for (int i = 0; i < U.dim * U.dim; i++)
        for (int t = 0; t < 4; t++) u_out[4 * i + t] = U.m[i].c[t];
    *e_out = U.e;
    um_free(&U);
    return 0;
}

/* ------------------------------------------------------------------ */
/* matrices over Z[1/sqrt2]: entries (a + b sqrt2) / sqrt2^E           */
/* ------------------------------------------------------------------ */
typedef struct { int dim, E; int64_t *a, *b; } pmat;

static pmat pm_new(int dim)
{
    pmat M;
    M.dim = dim; M.E = 0;
    M.a = (int64_t *)xcalloc((size_t)dim * dim, sizeof(int64_t));
    M.b = (int64_t *)xcalloc((size_t)dim * dim, sizeof(int64_t));
    return M;
}
static void pm_free(pmat *M) { free(M->a); free(M->b); M->a = M->b = NULL; }
static pmat pm_copy(const pmat *A)
{
    pmat M = pm_new(A->dim);
    M.E = A->E;
    memcpy(M.a, A->a, sizeof(int64_t) * A->dim * A->dim);
    memcpy(M.b, A->b, sizeof(int64_t) * A->dim * A->dim);
    return M;
}
static pmat pm_identity(int dim)
{
    pmat M = pm_new(dim);
    for (int i = 0; i < dim; i++) M.a[i * dim + i] = 1;
    return M;
}
static pmat pm_wrap(int dim, const int64_t *a, const int64_t *b, int E)
{
    pmat M = pm_new(dim);
    M.E = E;
    memcpy(M.a, a, sizeof(int64_t) * dim * dim);
    memcpy(M.b, b, sizeof(int64_t) * dim * dim);
    return M;
}
static void pm_out(const pmat *M, int64_t *a, int64_t *b, int *E)
{
    memcpy(a, M->a, sizeof(int64_t) * M->dim * M->dim);
    memcpy(b, M->b, sizeof(int64_t) * M->dim * M->dim);
    *E = M->E;
}
/* (a1 + b1 r2)(a2 + b2 r2) = (a1 a2 + 2 b1 b2) + (a1 b2 + b1 a2) r2 */
static void zs_mul(int64_t a1, int64_t b1, int64_t a2, int64_t b2, int64_t *ra, int64_t *rb)
{
    *ra = cadd(cmul(a1, a2), cmul(2, cmul(b1, b2)));
    *rb = cadd(cmul(a1, b2), cmul(b1, a2));
}
/* same value, numerators times sqrt2^s, exponent E + s */
static void pm_raise(pmat *M, int s)
{
    int cnt = M->dim * M->dim;
    for (int t = 0; t < s; t++)
        for (int i = 0; i < cnt; i++) {
            int64_t a = M->a[i], b = M->b[i];
            M->a[i] = cmul(2, b); /* (a + b r2) r2 = 2b + a r2 */
            M->b[i] = a;
        }
    M->E += s;
}
/* lower E while every numerator is divisible by sqrt2 (a even) */
static void pm_reduce(pmat *M)
{
    int cnt = M->dim * M->dim;
    for (;;) {
        if (M->E <= 0) return;
        for (int i = 0; i < cnt; i++)
            if (M->a[i] & 1) return;
        for (int i = 0; i < cnt; i++) {
            int64_t a = M->a[i], b = M->b[i];
            M->a[i] = b;
            M->b[i] = a / 2;
        }
        M->E -= 1;
    }
}
static pmat pm_mul(const pmat *A, const pmat *B)
{
    int d = A->dim;
    pmat R = pm_new(d);
    R.E = A->E + B->E;
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) {
            int64_t sa = 0, sb = 0;
            for (int t = 0; t < d; t++) {
                int64_t pa, pb;
                zs_mul(A->a[r * d + t], A->b[r * d + t], B->a[t * d + c], B->b[t * d + c], &pa, &pb);
                sa = cadd(sa, pa);
                sb = cadd(sb, pb);
            }
            R.a[r * d + c] = sa;
            R.b[r * d + c] = sb;
        }
    return R;
}
OR_API int or_pm_mul(int dim, const int64_t *a1, const int64_t *b1, int E1,
                     const int64_t *a2, const int64_t *b2, int E2,
                     int64_t *ao, int64_t *bo, int *Eo)
{
    pmat A = pm_wrap(dim, a1, b1, E1), B = pm_wrap(dim, a2, b2, E2);
    pmat R = pm_mul(&A, &B);
    pm_reduce(&R);
    pm_out(&R, ao, bo, Eo);
    pm_free(&A); pm_free(&B); pm_free(&R);
    return 0;
}
OR_API int or_pm_reduce(int dim, int64_t *a, int64_t *b, int *E)
{
    pmat A = pm_wrap(dim, a, b, *E);
    pm_reduce(&A);
    pm_out(&A, a, b, E);
    pm_free(&A);
    return 0;
}

/* ------------------------------------------------------------------ */
/* channel representation (Sec. 4.1): U^_ij = Tr(P_i U P_j U^dag) / 2^n */
/* ------------------------------------------------------------------ */
static pmat channel_of(const umat *U)
{
    int n = U->n, d = U->dim, D = d * d;
    pmat C = pm_new(D);
    umat Ud = um_dagger(U);
    for (int j = 0; j < D; j++) {
        umat Pj = um_pauli(n, j);
        umat T1 = um_mul(U, &Pj);
        umat A = um_mul(&T1, &Ud); /* u P_j u^dag, exponent 2e */
        for (int i = 0; i < D; i++) {
            umat Pi = um_pauli(n, i);
            zw tr = zw_zero();
            for (int r = 0; r < d; r++)
                for (int c = 0; c < d; c++) {
                    zw p = Pi.m[r * d + c];
                    if (zw_is_zero(p)) continue;
                    tr = zw_add(tr, zw_mul(p, A.m[c * d + r]));
                }
            um_free(&Pi);
            /* a real element of Z[w] is c0 + c1 (w - w^3) = c0 + c1 sqrt2 */
            if (tr.c[2] != 0 || tr.c[3] != -tr.c[1]) die("channel entry is not real");
            C.a[i * D + j] = tr.c[0];
            C.b[i * D + j] = tr.c[1];
        }
        um_free(&Pj); um_free(&T1); um_free(&A);
    }
    um_free(&Ud);
    C.E = 2 * n + 2 * U->e; /* 1 / (2^n 2^e) */
    pm_reduce(&C);
    return C;
}

OR_API int or_channel_from_unitary(int n, const int64_t *u, int e, int64_t *a, int64_t *b, int *E)
{
    if (n < 1 || n > 4) return -1;
    umat U = um_new(n);
    U.e = e;
    for (int i = 0; i < U.dim * U.dim; i++)
        for (int t = 0; t < 4; t++) U.m[i].c[t] = u[4 * i + t];
    pmat C = channel_of(&U);
    pm_out(&C, a, b, E);
    pm_free(&C); um_free(&U);
    return 0;
}

OR_API int or_channel_from_circuit(int n, const int32_t *gates, int ngates, int64_t *a, int64_t *b, int *E)
{
    if (n < 1 || n > 4) return -1;
    umat U = um_from_circuit(n, gates, ngates);
    pmat C = channel_of(&U);
    pm_out(&C, a, b, E);
    pm_free(&C); um_free(&U);
    return 0;
}

/* ------------------------------------------------------------------ */
/* R^(P): columns from R(P) Q R(P)^dag = (Q - i P Q) / sqrt2 (anticommuting Q), */
/* Q otherwise; the sparse matrix the paper multiplies by (Sec. 4.1)    */
/* ------------------------------------------------------------------ */
typedef struct { int cnt; int *row, *col; int64_t *va, *vb; } sparse; /* exponent 1 */

static sparse rhat_sparse(int n, int p)
{
    int D = 1 << (2 * n);
    sparse S;
    S.cnt = 0;
    S.row = (int *)xcalloc(2 * D, sizeof(int));
    S.col = (int *)xcalloc(2 * D, sizeof(int));
    S.va = (int64_t *)xcalloc(2 * D, sizeof(int64_t));
    S.vb = (int64_t *)xcalloc(2 * D, sizeof(int64_t));
    for (int q = 0; q < D; q++) {
        if (!pauli_anticommute(n, p, q)) {
            /* column q is e_q: the value 1 is sqrt2 / sqrt2 at exponent 1 */
            S.row[S.cnt] = q; S.col[S.cnt] = q; S.va[S.cnt] = 0; S.vb[S.cnt] = 1; S.cnt++;
        } else {
            /* -i P(p) P(q) = i^(lambda + 3) P(p ^ q) must be a real sign */
            int m = (or_pauli_phase(n, p, q) + 3) & 3;
            if (m & 1) die("rotated Pauli has an imaginary coefficient");
            int s = (m == 0) ? 1 : -1;
            S.row[S.cnt] = q; S.col[S.cnt] = q; S.va[S.cnt] = 1; S.vb[S.cnt] = 0; S.cnt++;
            S.row[S.cnt] = q ^ p; S.col[S.cnt] = q; S.va[S.cnt] = s; S.vb[S.cnt] = 0; S.cnt++;
        }
    }
    return S;
}
static void sp_free(sparse *S) { free(S->row); free(S->col); free(S->va); free(S->vb); }

/* R^(p) M (transpose = 0) or R^(p)^T M (transpose = 1), sparse times dense */
static pmat rhat_left_mul(int n, int p, int transpose, const pmat *M)
{
    int d = M->dim;
    sparse S = rhat_sparse(n, p);
    pmat R = pm_new(d);
    R.E = M->E + 1;
    for (int t = 0; t < S.cnt; t++) {
        int r = transpose ? S.col[t] : S.row[t];
        int c = transpose ? S.row[t] : S.col[t];
        for (int k = 0; k < d; k++) {
            int64_t pa, pb;
            zs_mul(S.va[t], S.vb[t], M->a[c * d + k], M->b[c * d + k], &pa, &pb);
            R.a[r * d + k] = cadd(R.a[r * d + k], pa);
            R.b[r * d + k] = cadd(R.b[r * d + k], pb);
        }
    }
    sp_free(&S);
    return R;
}

OR_API int or_rhat_cols(int n, int p, int transpose, int64_t *a, int64_t *b)
{
    int D = 1 << (2 * n);
    pmat I = pm_identity(D);
    pmat R = rhat_left_mul(n, p, transpose, &I); /* exponent 1 */
    memcpy(a, R.a, sizeof(int64_t) * D * D);
    memcpy(b, R.b, sizeof(int64_t) * D * D);
    pm_free(&I); pm_free(&R);
    return 0;
}

/* R^(P) from the trace definition, via the unitary of Eq. for R(P_j) */
OR_API int or_rhat_trace(int n, int p, int64_t *a, int64_t *b, int *E)
{
    umat G = um_gate(n, G_RP, p, 0);
    pmat C = channel_of(&G);
    pm_out(&C, a, b, E);
    pm_free(&C); um_free(&G);
    return 0;
}

/* ------------------------------------------------------------------ */
/* half products (Eq. mitm, channel form; chunks of Sec. 3 for odd k)  */
/* ------------------------------------------------------------------ */
static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

/* q[0..h-1] = q_1..q_h.  side 0: V_q at K; side 1: W_q at K. */
static pmat half_product(int n, const pmat *C, int k, int chunk, int side, const int32_t *q, int *Kout)
{
    int D = 1 << (2 * n);
    int h = k / 2;
    int K = C->E + (k & 1) + h;
    pmat M;
    if (side == 0) {
        M = pm_identity(D);
        for (int j = 0; j < h; j++) { /* R(q_1) first, R(q_h) last */
            pmat T = rhat_left_mul(n, q[j], 0, &M);
            pm_free(&M);
            M = T;
        }
        pm_raise(&M, K - h);
    } else {
        M = pm_copy(C);
        if (k & 1) {
            pmat T = rhat_left_mul(n, chunk, 1, &M);
            pm_free(&M);
            M = T;
        }
        for (int j = h - 1; j >= 0; j--) { /* R(q_h)^T first, R(q_1)^T last */
            pmat T = rhat_left_mul(n, q[j], 1, &M);
            pm_free(&M);
            M = T;
        }
    }
    if (M.E != K) die("exponent bookkeeping");
    *Kout = K;
    return M;
}

OR_API int or_half_product(int n, const int64_t *Ca, const int64_t *Cb, int e, int k, int chunk,
                           int side, const int32_t *q, int64_t *a, int64_t *b, int *K)
{
    int D = 1 << (2 * n);
    pmat C = pm_wrap(D, Ca, Cb, e);
    pmat M = half_product(n, &C, k, chunk, side, q, K);
    memcpy(a, M.a, sizeof(int64_t) * D * D);
    memcpy(b, M.b, sizeof(int64_t) * D * D);
    pm_free(&C); pm_free(&M);
    return 0;
}

/* ------------------------------------------------------------------ */
/* walk hash h (Sec. 2, Fig. 1) and reduction nu                       */
/* ------------------------------------------------------------------ */
static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ull;
static const uint64_t SEED_U = 0x6A09E667F3BCC908ull;
static const uint64_t SEED_H = 0xBB67AE8584CAA73Bull;

/* SplitMix64 output function (Steele, Lea & Flood 2014) */
static uint64_t smix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* j-th output (0-based) of the SplitMix64 stream seeded with s */
static uint64_t splitmix_at(uint64_t s, uint64_t j) { return smix(s + (j + 1) * SM_GAMMA); }

OR_API void or_fp_weights(int n, uint32_t *ua, uint32_t *ub)
{
    int D = 1 << (2 * n);
    ua[0] = ub[0] = 0;
    for (int i = 1; i < D; i++) {
        ua[i] = (uint32_t)splitmix_at(SEED_U, 2 * (uint64_t)i);
        ub[i] = (uint32_t)splitmix_at(SEED_U, 2 * (uint64_t)i + 1);
    }
}

static uint64_t mask_bits(int L) { return L >= 64 ? ~0ull : ((1ull << L) - 1); }

/* hash of the Clifford coset of M (given at exponent K) into an L-bit state:
 * the d = 4^n - 1 folded 16-bit column fingerprints phi_Q (Q = 1..d) as a
 * multiset, hashed as smix(sum_Q smix(base ^ phi_Q) mod 2^64), where base
 * mixes the version and the tag (n, k, chunk, K). */
static uint64_t coset_hash(int n, const pmat *M, int k, int chunk, uint32_t version, int L)
{
    int D = 1 << (2 * n), d = D - 1;
    uint32_t *ua = (uint32_t *)xcalloc(D, 4), *ub = (uint32_t *)xcalloc(D, 4);
    or_fp_weights(n, ua, ub);
    uint64_t tag = (uint64_t)n | ((uint64_t)k << 8) | ((uint64_t)chunk << 16) | ((uint64_t)M->E << 32);
    uint64_t base = smix(smix(SEED_H ^ (uint64_t)version) ^ tag);
    uint64_t acc = 0;
    for (int Q = 1; Q <= d; Q++) {
        uint32_t Lq = 0;
        for (int i = 1; i <= d; i++)
            Lq += ua[i] * (uint32_t)M->a[i * D + Q] + ub[i] * (uint32_t)M->b[i * D + Q];
        uint16_t l16 = (uint16_t)(Lq & 0xFFFFu), neg = (uint16_t)((0x10000u - l16) & 0xFFFFu);
        uint16_t phi = l16 < neg ? l16 : neg;
        acc += smix(base ^ (uint64_t)phi);
    }
    free(ua); free(ub);
    return smix(acc) & mask_bits(L);
}

OR_API uint64_t or_matrix_hash(int n, const int64_t *a, const int64_t *b, int K, int k, int chunk,
                               uint32_t version, int L)
{
    int D = 1 << (2 * n);
    pmat M = pm_wrap(D, a, b, K);
    uint64_t r = coset_hash(n, &M, k, chunk, version, L);
    pm_free(&M);
    return r;
}

/* mu (Sec. 2: the string is the concatenation of one l-bit code per
 * rotation): bit 0 is the side; rotation j (0-based) reads its own field of
 * l = min(16, (L - 1) / h) bits starting at bit 1 + l j, and the field value v
 * names the Pauli code q_j = floor(v xi / 2^l) + 1 (multiply-shift reduction
 * of the l-bit code onto the xi = 4^n - 1 non-identity Paulis). */
OR_API int or_field_bits(int n, int k, int L)
{
    (void)n;
    int h = k / 2;
    if (h == 0) return 0;
    int l = (L - 1) / h;
    return l > 16 ? 16 : l;
}

OR_API int or_decode(int n, int k, int L, uint64_t x, int32_t *q)
{
    int h = k / 2;
    uint64_t xi = (uint64_t)((1 << (2 * n)) - 1);
    int l = or_field_bits(n, k, L);
    for (int j = 0; j < h; j++) {
        uint64_t v = (x >> (1 + l * j)) & ((1ull << l) - 1);
        q[j] = (int32_t)((v * xi) >> l) + 1;
    }
    return (int)(x & 1);
}

static uint64_t walk_f(int n, const pmat *C, int k, int chunk, uint32_t version, int L, uint64_t x)
{
    int32_t q[16];
    int side = or_decode(n, k, L, x, q);
    int K;
    pmat M = half_product(n, C, k, chunk, side, q, &K);
    uint64_t y = coset_hash(n, &M, k, chunk, version, L);
    pm_free(&M);
    return y;
}

OR_API int or_walk_step(int n, const int64_t *Ca, const int64_t *Cb, int e, int k, int chunk,
                        uint32_t version, int L, const uint64_t *x, uint64_t *y, int count)
{
    int D = 1 << (2 * n);
    pmat C = pm_wrap(D, Ca, Cb, e);
    for (int t = 0; t < count; t++) y[t] = walk_f(n, &C, k, chunk, version, L, x[t]);
    pm_free(&C);
    return 0;
}

/* ------------------------------------------------------------------ */
/* exact canonical form modulo Clifford (right multiplication by D^)    */
/* ------------------------------------------------------------------ */
/* exact sign of a + b sqrt2 */
static int zs_sign(int64_t a, int64_t b)
{
    if (a == 0 && b == 0) return 0;
    if (a >= 0 && b >= 0) return 1;
    if (a <= 0 && b <= 0) return -1;
    __int128 a2 = (__int128)a * a, b2 = (__int128)2 * b * b;
    if (a > 0) return a2 > b2 ? 1 : -1;
    return b2 > a2 ? 1 : -1;
}

typedef struct { int d; const int64_t *col; } colref; /* 2d numbers: a_1 b_1 ... a_d b_d */
static int cmp_col(const void *x, const void *y)
{
    const colref *p = (const colref *)x, *q = (const colref *)y;
    for (int t = 0; t < 2 * p->d; t++) {
        if (p->col[t] < q->col[t]) return -1;
        if (p->col[t] > q->col[t]) return 1;
    }
    return 0;
}

/* canonical form: minimal sde, every column 1..d negated when its first
 * nonzero row is negative, columns sorted lexicographically; out is d x d
 * (row-major, rows/cols 1..d), as (a,b) interleaved per column: out[Q][2i+{0,1}] */
static void canon_form(int n, const pmat *Min, int64_t *out, int *sde)
{
    int D = 1 << (2 * n), d = D - 1;
    pmat M = pm_copy(Min);
    pm_reduce(&M);
    int64_t *cols = (int64_t *)xcalloc((size_t)d * 2 * d, sizeof(int64_t));
    colref *refs = (colref *)xcalloc(d, sizeof(colref));
    for (int Q = 1; Q <= d; Q++) {
        int sgn = 0;
        for (int i = 1; i <= d && !sgn; i++) sgn = zs_sign(M.a[i * D + Q], M.b[i * D + Q]);
        if (sgn == 0) die("zero column in a channel matrix");
        int64_t *c = cols + (size_t)(Q - 1) * 2 * d;
        for (int i = 1; i <= d; i++) {
            c[2 * (i - 1)] = sgn * M.a[i * D + Q];
            c[2 * (i - 1) + 1] = sgn * M.b[i * D + Q];
        }
        refs[Q - 1].d = d;
        refs[Q - 1].col = c;
    }
    qsort(refs, d, sizeof(colref), cmp_col);
    for (int Q = 0; Q < d; Q++) memcpy(out + (size_t)Q * 2 * d, refs[Q].col, sizeof(int64_t) * 2 * d);
    *sde = M.E;
    free(cols); free(refs); pm_free(&M);
}

OR_API int or_canon(int n, const int64_t *a, const int64_t *b, int E, int64_t *out, int *sde)
{
    int D = 1 << (2 * n);
    pmat M = pm_wrap(D, a, b, E);
    canon_form(n, &M, out, sde);
    pm_free(&M);
    return 0;
}

static int same_coset(int n, const pmat *A, const pmat *B)
{
    int D = 1 << (2 * n), d = D - 1;
    int64_t *ca = (int64_t *)xcalloc((size_t)d * 2 * d, sizeof(int64_t));
    int64_t *cb = (int64_t *)xcalloc((size_t)d * 2 * d, sizeof(int64_t));
    int ea, eb;
    canon_form(n, A, ca, &ea);
    canon_form(n, B, cb, &eb);
    int eq = (ea == eb) && !memcmp(ca, cb, sizeof(int64_t) * d * 2 * d);
    free(ca); free(cb);
    return eq;
}

/* channel matrix of a Clifford: after reduction every entry is 0 or +-1 and
 * every column holds exactly one nonzero (a signed permutation) */
static int is_clifford(const pmat *Min)
{
    pmat M = pm_copy(Min);
    pm_reduce(&M);
    int D = M.dim, ok = (M.E == 0);
    for (int c = 0; c < D && ok; c++) {
        int nz = 0;
        for (int r = 0; r < D; r++) {
            int64_t a = M.a[r * D + c], b = M.b[r * D + c];
            if (a == 0 && b == 0) continue;
            if (b != 0 || (a != 1 && a != -1)) ok = 0;
            nz++;
        }
        if (nz != 1) ok = 0;
    }
    pm_free(&M);
    return ok;
}

OR_API int or_is_clifford(int n, const int64_t *a, const int64_t *b, int E)
{
    int D = 1 << (2 * n);
    pmat M = pm_wrap(D, a, b, E);
    int r = is_clifford(&M);
    pm_free(&M);
    return r;
}

OR_API int or_sde(int n, const int64_t *a, const int64_t *b, int E)
{
    int D = 1 << (2 * n);
    pmat M = pm_wrap(D, a, b, E);
    pm_reduce(&M);
    int r = M.E;
    pm_free(&M);
    return r;
}

/* D^ = R(P_1)^T ... R(P_t)^T C^ must be a Clifford (Eq. tcount_synthesis) */
static int verify(int n, const pmat *C, const int32_t *paulis, int t)
{
    pmat M = pm_copy(C);
    for (int j = t - 1; j >= 0; j--) {
        pmat T = rhat_left_mul(n, paulis[j], 1, &M);
        pm_free(&M);
        M = T;
    }
    int ok = is_clifford(&M);
    pm_free(&M);
    return ok;
}

OR_API int or_verify(int n, const int64_t *Ca, const int64_t *Cb, int e, const int32_t *paulis, int t)
{
    int D = 1 << (2 * n);
    pmat C = pm_wrap(D, Ca, Cb, e);
    int r = verify(n, &C, paulis, t);
    pm_free(&C);
    return r;
}

/* ------------------------------------------------------------------ */
/* brute force (Sec. 3: all depth-t products) and exhaustive MITM       */
/* ------------------------------------------------------------------ */
OR_API int or_brute_tcount(int n, const int64_t *Ca, const int64_t *Cb, int e, int tmax, int32_t *paulis)
{
    int D = 1 << (2 * n), xi = D - 1;
    pmat C = pm_wrap(D, Ca, Cb, e);
    for (int t = 0; t <= tmax; t++) {
        int total = ipow(xi, t);
        for (int idx = 0; idx < total; idx++) {
            int r = idx;
            for (int j = 0; j < t; j++) { paulis[j] = r % xi + 1; r /= xi; }
            if (verify(n, &C, paulis, t)) { pm_free(&C); return t; }
        }
    }
    pm_free(&C);
    return -1;
}

typedef struct { uint64_t key; int32_t idx; } keyed;
static int cmp_keyed(const void *x, const void *y)
{
    uint64_t a = ((const keyed *)x)->key, b = ((const keyed *)y)->key;
    return (a > b) - (a < b);
}
/* a 64-bit digest of the exact canonical form (used only to sort and search) */
static uint64_t canon_digest(int n, const pmat *M)
{
    int D = 1 << (2 * n), d = D - 1, sde;
    int64_t *c = (int64_t *)xcalloc((size_t)d * 2 * d, sizeof(int64_t));
    canon_form(n, M, c, &sde);
    uint64_t hsh = smix((uint64_t)sde + 1);
    for (int t = 0; t < d * 2 * d; t++) hsh = smix(hsh ^ (uint64_t)c[t]) + (uint64_t)t;
    free(c);
    return hsh;
}
static void index_to_q(int idx, int h, int xi, int32_t *q)
{
    for (int j = 0; j < h; j++) { q[j] = idx % xi + 1; idx /= xi; }
}

/* Is there a decomposition with exactly t = k rotations?  Builds the sorted
 * V database and searches it with every W (Sec. 3, Eq. mitm).  paulis gets
 * P_1..P_k on success. */
OR_API int or_mitm_level(int n, const int64_t *Ca, const int64_t *Cb, int e, int k, int32_t *paulis)
{
    int D = 1 << (2 * n), xi = D - 1;
    pmat C = pm_wrap(D, Ca, Cb, e);
    int found = 0;
    if (k == 0) {
        found = is_clifford(&C);
    } else if (k == 1) {
        for (int c = 1; c <= xi && !found; c++) {
            paulis[0] = c;
            found = verify(n, &C, paulis, 1);
        }
    } else {
        int h = k / 2, span = ipow(xi, h);
        keyed *db = (keyed *)xcalloc(span, sizeof(keyed));
        int32_t q[16], qw[16];
        for (int idx = 0; idx < span; idx++) {
            int K;
            index_to_q(idx, h, xi, q);
            pmat V = half_product(n, &C, k, 0, 0, q, &K);
            db[idx].key = canon_digest(n, &V);
            db[idx].idx = idx;
            pm_free(&V);
        }
        qsort(db, span, sizeof(keyed), cmp_keyed);
        int c_lo = (k & 1) ? 1 : 0, c_hi = (k & 1) ? xi : 0;
        for (int c = c_lo; c <= c_hi && !found; c++) {
            for (int idx = 0; idx < span && !found; idx++) {
                int K;
                index_to_q(idx, h, xi, qw);
                pmat W = half_product(n, &C, k, c, 1, qw, &K);
                keyed probe = {canon_digest(n, &W), 0};
                keyed *hit = (keyed *)bsearch(&probe, db, span, sizeof(keyed), cmp_keyed);
                if (hit) {
                    while (hit > db && hit[-1].key == probe.key) hit--;
                    for (; hit < db + span && hit->key == probe.key && !found; hit++) {
                        index_to_q(hit->idx, h, xi, q);
                        pmat V = half_product(n, &C, k, c, 0, q, &K);
                        if (same_coset(n, &V, &W)) {
                            for (int j = 0; j < h; j++) { paulis[j] = q[j]; paulis[h + j] = qw[j]; }
                            if (k & 1) paulis[2 * h] = c;
                            if (!verify(n, &C, paulis, k)) die("claw does not verify");
                            found = 1;
                        }
                        pm_free(&V);
                    }
                }
                pm_free(&W);
            }
        }
        free(db);
    }
    pm_free(&C);
    return found;
}

/* ------------------------------------------------------------------ */
/* merge classification by re-walking (Sec. 3, Fig. 2)                 */
/* ------------------------------------------------------------------ */
enum { M_ROBIN_HOOD = 0, M_TRIVIAL = 1, M_SAME_SIDE = 2, M_CLAW = 3, M_FALSE_HASH = 4, M_NO_MERGE = 5 };

/* decide what kind of merge f(a) = f(b) with a != b is */
static int classify_merge(int n, const pmat *C, int k, int chunk, int L, uint64_t a, uint64_t b,
                          int32_t *paulis)
{
    int32_t qa[16], qb[16];
    int h = k / 2;
    int sa = or_decode(n, k, L, a, qa), sb = or_decode(n, k, L, b, qb);
    if (sa == sb) {
        int same = 1;
        for (int j = 0; j < h; j++) same &= (qa[j] == qb[j]);
        return same ? M_TRIVIAL : M_SAME_SIDE;
    }
    const int32_t *qv = sa == 0 ? qa : qb, *qw = sa == 0 ? qb : qa;
    int K1, K2;
    pmat V = half_product(n, C, k, chunk, 0, qv, &K1);
    pmat W = half_product(n, C, k, chunk, 1, qw, &K2);
    int eq = same_coset(n, &V, &W);
    pm_free(&V); pm_free(&W);
    if (!eq) return M_FALSE_HASH;
    for (int j = 0; j < h; j++) { paulis[j] = qv[j]; paulis[h + j] = qw[j]; }
    if (k & 1) paulis[2 * h] = chunk;
    return M_CLAW;
}

/* Two trails (start, length) that end at the same distinguished point: align
 * the longer one, then step both until their images agree.  ab[0], ab[1] get
 * the two distinct states whose images coincide (for Robin Hood the shared
 * state). */
static int rewalk(int n, const pmat *C, int k, int chunk, uint32_t version, int L,
                  uint64_t x0a, int64_t la, uint64_t x0b, int64_t lb, uint64_t *ab, int32_t *paulis)
{
    if (la < lb) {
        uint64_t tx = x0a; x0a = x0b; x0b = tx;
        int64_t tl = la; la = lb; lb = tl;
    }
    uint64_t a = x0a, b = x0b;
    for (int64_t s = 0; s < la - lb; s++) a = walk_f(n, C, k, chunk, version, L, a);
    if (a == b) { ab[0] = ab[1] = a; return M_ROBIN_HOOD; }
    for (int64_t s = 0; s < lb; s++) {
        uint64_t fa = walk_f(n, C, k, chunk, version, L, a);
        uint64_t fb = walk_f(n, C, k, chunk, version, L, b);
        if (fa == fb) {
            ab[0] = a; ab[1] = b;
            return classify_merge(n, C, k, chunk, L, a, b, paulis);
        }
        a = fa; b = fb;
    }
    ab[0] = a; ab[1] = b;
    return M_NO_MERGE;
}

OR_API int or_rewalk(int n, const int64_t *Ca, const int64_t *Cb, int e, int k, int chunk,
                     uint32_t version, int L, uint64_t x0a, int64_t la, uint64_t x0b, int64_t lb,
                     uint64_t *ab, int32_t *paulis)
{
    int D = 1 << (2 * n);
    pmat C = pm_wrap(D, Ca, Cb, e);
    int r = rewalk(n, &C, k, chunk, version, L, x0a, la, x0b, lb, ab, paulis);
    pm_free(&C);
    return r;
}

OR_API int or_classify(int n, const int64_t *Ca, const int64_t *Cb, int e, int k, int chunk, int L,
                       uint64_t a, uint64_t b, int32_t *paulis)
{
    int D = 1 << (2 * n);
    pmat C = pm_wrap(D, Ca, Cb, e);
    int r = classify_merge(n, &C, k, chunk, L, a, b, paulis);
    pm_free(&C);
    return r;
}

/* ------------------------------------------------------------------ */
/* serial parallel-collision search (Sec. 3) with the T-count ladder    */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t key; uint64_t start; int64_t len; int32_t chunk; int32_t used; } dp_slot;

/* params: [0] dtheta, [1] L, [2] max trail length, [3] steps per version,
 *         [4] steps per level, [5] log2 table slots, [6] seed
 * stats:  [0] steps, [1] distinguished points, [2] merges, [3] robin hood,
 *         [4] trivial, [5] same side, [6] claws, [7] false hash, [8] no merge,
 *         [9] dropped points, [10] level of the answer */
OR_API int or_vow_search(int n, const int64_t *Ca, const int64_t *Cb, int e, int k_max,
                         const int64_t *params, int32_t *paulis, int64_t *stats)
{
    int D = 1 << (2 * n), xi = D - 1;
    int dth = (int)params[0], L = (int)params[1];
    int64_t max_len = params[2], per_version = params[3], per_level = params[4];
    int tlog = (int)params[5];
    uint64_t rng = (uint64_t)params[6];
    uint64_t mask = mask_bits(L);
    uint64_t tmask = (1ull << tlog) - 1;
    pmat C = pm_wrap(D, Ca, Cb, e);
    for (int s = 0; s < 11; s++) stats[s] = 0;
    int answer = -1;
    pm_reduce(&C);
    for (int k = C.E; k <= k_max && answer < 0; k++) {
        if (k <= 1) {
            if (or_mitm_level(n, C.a, C.b, C.E, k, paulis)) answer = k;
            continue;
        }
        dp_slot *tab = (dp_slot *)xcalloc((size_t)1 << tlog, sizeof(dp_slot));
        uint32_t version = 0;
        int64_t level_steps = 0, version_steps = 0;
        while (level_steps < per_level && answer < 0) {
            if (version_steps >= per_version) {
                memset(tab, 0, sizeof(dp_slot) << tlog);
                version++;
                version_steps = 0;
            }
            rng += SM_GAMMA;
            uint64_t x0 = smix(rng) & mask;
            int chunk = (k & 1) ? (int)(smix(rng ^ 0x5555555555555555ull) % (uint64_t)xi) + 1 : 0;
            uint64_t x = x0;
            int64_t len = 0;
            int dp = 0;
            while (len < max_len) {
                x = walk_f(n, &C, k, chunk, version, L, x);
                len++;
                if ((x >> (L - dth)) == 0 || dth == 0) { dp = 1; break; }
            }
            level_steps += len;
            version_steps += len;
            stats[0] += len;
            if (!dp) continue;
            stats[1]++;
            uint64_t slot = smix(x ^ ((uint64_t)chunk << 48)) & tmask;
            for (int probe = 0;; probe++) {
                if (probe == 64) { stats[9]++; break; }
                dp_slot *s = &tab[slot];
                if (!s->used) {
                    s->used = 1; s->key = x; s->start = x0; s->len = len; s->chunk = chunk;
                    break;
                }
                if (s->key == x && s->chunk == chunk) {
                    if (s->start != x0) {
                        uint64_t ab[2];
                        stats[2]++;
                        int cls = rewalk(n, &C, k, chunk, version, L, s->start, s->len, x0, len, ab, paulis);
                        stats[3 + cls]++;
                        if (cls == M_CLAW) {
                            if (!verify(n, &C, paulis, k)) die("claw does not verify");
                            answer = k;
                        }
                    }
                    break;
                }
                slot = (slot + 1) & tmask;
            }
        }
        free(tab);
    }
    stats[10] = answer;
    pm_free(&C);
    return answer;
}
