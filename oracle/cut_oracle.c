/*
 * cut_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, deliberately slow CPU evaluation of operator products and
 * commutators by direct string multiplication.  It is the reference that the
 * CUDA graph path is checked against; only tests/, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the graph
 * builder or the GPU kernels.
 *
 * What it computes (paper Sec. 2.1-2.2, Eqs. coflow, block-generator,
 * projected-flow): exact products of operator strings, evaluated in the full
 * algebra and normal ordered before anything is projected.
 *
 *  - Pauli strings: product qubit by qubit from the single-qubit table
 *    sigma_a sigma_b = delta_ab I + i eps_abc sigma_c.
 *  - Fermion monomials: the concatenated ladder string is brought to normal
 *    order (creators ascending to the left, annihilators descending to the
 *    right) by repeatedly rewriting the first adjacent out-of-order pair with
 *    the canonical anticommutation relations
 *        a_p a+_q = delta_pq - a+_q a_p,   a+_p a+_q = -a+_q a+_p,
 *        a_p a_q = -a_q a_p,               a+_p a+_p = a_p a_p = 0.
 *
 * Operators are sums of (label, complex coefficient); the label encoding is
 * the one of the cut_inputs package (Pauli: x mask | z mask << 32; fermion:
 * creator mask | annihilator mask << 32; Pauli-boson: see pb_product).
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

#define ALG_PAULI 0
#define ALG_FERMION 1
#define MAXOPS 40

/* ------------------------------------------------------------------ */
/* label -> coefficient accumulator (open addressing)                 */
/* ------------------------------------------------------------------ */
typedef struct {
    uint64_t *keys;
    cplx *vals;
    unsigned char *used;
    size_t cap, n;
} oracle_op;

static uint64_t mix(uint64_t k) {
    k ^= k >> 33; k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

static oracle_op *op_new(size_t cap) {
    oracle_op *m = (oracle_op *)calloc(1, sizeof(oracle_op));
    size_t c = 64;
    while (c < 2 * cap) c <<= 1;
    m->cap = c;
    m->keys = (uint64_t *)calloc(c, sizeof(uint64_t));
    m->vals = (cplx *)calloc(c, sizeof(cplx));
    m->used = (unsigned char *)calloc(c, 1);
    return m;
}

static void op_add(oracle_op *m, uint64_t key, cplx v);

static void op_grow(oracle_op *m) {
    oracle_op old = *m;
    m->cap = old.cap * 2;
    m->n = 0;
    m->keys = (uint64_t *)calloc(m->cap, sizeof(uint64_t));
    m->vals = (cplx *)calloc(m->cap, sizeof(cplx));
    m->used = (unsigned char *)calloc(m->cap, 1);
    for (size_t i = 0; i < old.cap; i++)
        if (old.used[i]) op_add(m, old.keys[i], old.vals[i]);
    free(old.keys); free(old.vals); free(old.used);
}

static void op_add(oracle_op *m, uint64_t key, cplx v) {
    if (2 * (m->n + 1) > m->cap) op_grow(m);
    size_t i = mix(key) & (m->cap - 1);
    while (m->used[i] && m->keys[i] != key) i = (i + 1) & (m->cap - 1);
    if (!m->used[i]) { m->used[i] = 1; m->keys[i] = key; m->vals[i] = 0; m->n++; }
    m->vals[i] += v;
}

void oracle_op_free(oracle_op *m) {
    if (!m) return;
    free(m->keys); free(m->vals); free(m->used); free(m);
}

int64_t oracle_op_size(const oracle_op *m) { return (int64_t)m->n; }

/* Export all entries (coefficients interleaved re, im). */
void oracle_op_export(const oracle_op *m, uint64_t *labels, double *coefs) {
    size_t o = 0;
    for (size_t i = 0; i < m->cap; i++) {
        if (!m->used[i]) continue;
        labels[o] = m->keys[i];
        coefs[2 * o] = creal(m->vals[i]);
        coefs[2 * o + 1] = cimag(m->vals[i]);
        o++;
    }
}

/* ------------------------------------------------------------------ */
/* Pauli strings                                                      */
/* ------------------------------------------------------------------ */
/* single-qubit letters: 0=I 1=X 2=Y 3=Z */
static int letter(uint64_t label, int q) {
    int x = (int)((label >> q) & 1), z = (int)((label >> (32 + q)) & 1);
    if (x && z) return 2;
    if (x) return 1;
    if (z) return 3;
    return 0;
}

/* sigma_a sigma_b = i^PH[a][b] sigma_RES[a][b] */
static const int RES[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 3, 0, 1}, {3, 2, 1, 0}};
static const int PH[4][4] = {{0, 0, 0, 0},   /* I*. */
                             {0, 0, 1, 3},   /* X*I=X, X*X=I, X*Y=iZ, X*Z=-iY */
                             {0, 3, 0, 1},   /* Y*X=-iZ, Y*Y=I, Y*Z=iX */
                             {0, 1, 3, 0}};  /* Z*X=iY, Z*Y=-iX, Z*Z=I */

static const cplx IPOW[4] = {1.0, I, -1.0, -I};

static void pauli_product(int nq, uint64_t a, uint64_t b, cplx coef, oracle_op *out) {
    int phase = 0;
    uint64_t x = 0, z = 0;
    for (int q = 0; q < nq; q++) {
        int la = letter(a, q), lb = letter(b, q);
        int r = RES[la][lb];
        phase += PH[la][lb];
        if (r == 1 || r == 2) x |= 1ULL << q;
        if (r == 2 || r == 3) z |= 1ULL << q;
    }
    op_add(out, x | (z << 32), coef * IPOW[phase & 3]);
}

/* ------------------------------------------------------------------ */
/* Fermion ladder strings                                             */
/* ------------------------------------------------------------------ */
/* op code: +(p+1) = a+_p, -(p+1) = a_p */
static int to_ops(uint64_t label, signed char *ops) {
    uint32_t c = (uint32_t)label, a = (uint32_t)(label >> 32);
    int n = 0;
    for (int p = 0; p < 32; p++)
        if (c >> p & 1) ops[n++] = (signed char)(p + 1);
    for (int p = 31; p >= 0; p--)
        if (a >> p & 1) ops[n++] = (signed char)(-(p + 1));
    return n;
}

static void normal_order(const signed char *ops, int len, cplx coef, oracle_op *out) {
    signed char buf[MAXOPS];
    for (int k = 0; k + 1 < len; k++) {
        int u = ops[k], v = ops[k + 1];
        if (u < 0 && v > 0) {
            /* a_p a+_q = delta_pq - a+_q a_p */
            if (-u == v) {
                int m = 0;
                for (int t = 0; t < len; t++)
                    if (t != k && t != k + 1) buf[m++] = ops[t];
                normal_order(buf, m, coef, out);
            }
            memcpy(buf, ops, (size_t)len);
            buf[k] = (signed char)v;
            buf[k + 1] = (signed char)u;
            normal_order(buf, len, -coef, out);
            return;
        }
        if (u > 0 && v > 0) {
            if (u == v) return;                 /* a+_p a+_p = 0 */
            if (u > v) {                        /* creators ascending */
                memcpy(buf, ops, (size_t)len);
                buf[k] = (signed char)v;
                buf[k + 1] = (signed char)u;
                normal_order(buf, len, -coef, out);
                return;
            }
        }
        if (u < 0 && v < 0) {
            if (u == v) return;                 /* a_p a_p = 0 */
            if (-u < -v) {                      /* annihilators descending */
                memcpy(buf, ops, (size_t)len);
                buf[k] = (signed char)v;
                buf[k + 1] = (signed char)u;
                normal_order(buf, len, -coef, out);
                return;
            }
        }
    }
    uint64_t c = 0, a = 0;
    for (int t = 0; t < len; t++) {
        if (ops[t] > 0) c |= 1ULL << (ops[t] - 1);
        else a |= 1ULL << (-ops[t] - 1);
    }
    op_add(out, c | (a << 32), coef);
}

static void fermion_product(uint64_t a, uint64_t b, cplx coef, oracle_op *out) {
    signed char ops[MAXOPS];
    int n = to_ops(a, ops);
    n += to_ops(b, ops + n);
    normal_order(ops, n, coef, out);
}

/* ------------------------------------------------------------------ */
/* Pauli-boson monomials sigma_tau prod_m (b_m+)^c_m b_m^a_m            */
/* ------------------------------------------------------------------ */
/* The Pauli factor lives in the real basis I, X, iY, Z (2x2 real matrices);
 * a product of two basis matrices is decomposed back onto the basis with
 * the trace inner product (the four matrices are orthogonal, norm^2 = 2).
 * Each boson mode is handled on its own (modes commute): the normal-ordered
 * factor of A is multiplied on the right by the ladder operators of B one at
 * a time, using
 *   (b+)^c b^a . b  = (b+)^c b^(a+1)
 *   (b+)^c b^a . b+ = (b+)^(c+1) b^a + a (b+)^c b^(a-1)     ([b^a, b+] = a b^(a-1)).
 * Label: bits 0-1 tau, mode m: c at bits 2+10m (5 bits), a at bits 7+10m. */
#define ALG_PAULI_BOSON 2
#define PB_MAXDEG 64

static const double RMAT[4][2][2] = {{{1, 0}, {0, 1}}, {{0, 1}, {1, 0}}, {{0, 1}, {-1, 0}}, {{1, 0}, {0, -1}}};

static int pb_get(uint64_t l, int shift) { return (int)((l >> shift) & 31); }

/* one mode: coefficients of (b+)^C b^A, returned in poly[C][A] for
 * C <= c1 + c2, A <= a1 + a2 (the only entries that can be nonzero) */
static void boson_mode_product(int c1, int a1, int c2, int a2, double poly[PB_MAXDEG][PB_MAXDEG]) {
    static double cur[PB_MAXDEG][PB_MAXDEG], nxt[PB_MAXDEG][PB_MAXDEG];
    const int cm = c1 + c2 + 1, am = a1 + a2 + 1;
    for (int c = 0; c < cm; c++)
        for (int a = 0; a < am; a++) cur[c][a] = 0.0;
    cur[c1][a1] = 1.0;
    for (int step = 0; step < c2 + a2; step++) {
        const int create = step < c2;   /* B = (b+)^c2 b^a2: the b+ factors first */
        for (int c = 0; c < cm; c++)
            for (int a = 0; a < am; a++) nxt[c][a] = 0.0;
        for (int c = 0; c < cm; c++)
            for (int a = 0; a < am; a++) {
                double v = cur[c][a];
                if (v == 0.0) continue;
                if (!create) {
                    nxt[c][a + 1] += v;
                } else {
                    nxt[c + 1][a] += v;
                    if (a > 0) nxt[c][a - 1] += a * v;
                }
            }
        for (int c = 0; c < cm; c++)
            for (int a = 0; a < am; a++) cur[c][a] = nxt[c][a];
    }
    for (int c = 0; c < cm; c++)
        for (int a = 0; a < am; a++) poly[c][a] = cur[c][a];
}

static void pb_product(int nmodes, uint64_t x, uint64_t y, cplx coef, oracle_op *out) {
    /* Pauli part */
    double P[2][2] = {{0, 0}, {0, 0}};
    const int t1 = (int)(x & 3), t2 = (int)(y & 3);
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            for (int k = 0; k < 2; k++) P[i][j] += RMAT[t1][i][k] * RMAT[t2][k][j];
    /* boson part: list of (label bits, coefficient), mode by mode */
    static uint64_t lab[2][65536];
    static double val[2][65536];
    static double poly[PB_MAXDEG][PB_MAXDEG];
    int n = 1, cur = 0;
    lab[0][0] = 0;
    val[0][0] = 1.0;
    for (int m = 0; m < nmodes; m++) {
        const int sc = 2 + 10 * m, sa = 7 + 10 * m;
        const int cx = pb_get(x, sc), ax = pb_get(x, sa), cy = pb_get(y, sc), ay = pb_get(y, sa);
        boson_mode_product(cx, ax, cy, ay, poly);
        int nn = 0;
        for (int c = 0; c <= cx + cy; c++)
            for (int a = 0; a <= ax + ay; a++) {
                if (poly[c][a] == 0.0) continue;
                if (c > 31 || a > 31) abort();   /* beyond the 5-bit label fields */
                for (int i = 0; i < n; i++) {
                    lab[1 - cur][nn] = lab[cur][i] | ((uint64_t)c << sc) | ((uint64_t)a << sa);
                    val[1 - cur][nn] = val[cur][i] * poly[c][a];
                    nn++;
                }
            }
        cur = 1 - cur;
        n = nn;
    }
    for (int t = 0; t < 4; t++) {
        double tr = 0.0;   /* Tr(R_t^T P) / 2 */
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) tr += RMAT[t][i][j] * P[i][j];
        tr *= 0.5;
        if (tr == 0.0) continue;
        for (int i = 0; i < n; i++) op_add(out, lab[cur][i] | (uint64_t)t, coef * tr * val[cur][i]);
    }
}

static void product_into(int alg, int nmodes, uint64_t a, uint64_t b, cplx coef, oracle_op *out) {
    if (alg == ALG_PAULI) pauli_product(nmodes, a, b, coef, out);
    else if (alg == ALG_PAULI_BOSON) pb_product(nmodes, a, b, coef, out);
    else fermion_product(a, b, coef, out);
}

/* ------------------------------------------------------------------ */
/* Public entry points                                                */
/* ------------------------------------------------------------------ */

/* A*B for two operators given as term lists (coefficients interleaved). */
oracle_op *oracle_product(int alg, int nmodes, int64_t na, const uint64_t *la, const double *ca,
                          int64_t nb, const uint64_t *lb, const double *cb) {
    oracle_op *out = op_new((size_t)(na + nb + 16));
    for (int64_t i = 0; i < na; i++) {
        cplx x = ca[2 * i] + I * ca[2 * i + 1];
        for (int64_t j = 0; j < nb; j++) {
            cplx y = cb[2 * j] + I * cb[2 * j + 1];
            product_into(alg, nmodes, la[i], lb[j], x * y, out);
        }
    }
    return out;
}

/* [A, B] = sum_ij a_i b_j (A_i B_j - B_j A_i), every product exact, nothing projected. */
oracle_op *oracle_commutator(int alg, int nmodes, int64_t na, const uint64_t *la, const double *ca,
                             int64_t nb, const uint64_t *lb, const double *cb) {
    oracle_op *out = op_new((size_t)(na + nb + 16));
    for (int64_t i = 0; i < na; i++) {
        cplx x = ca[2 * i] + I * ca[2 * i + 1];
        if (x == 0) continue;
        for (int64_t j = 0; j < nb; j++) {
            cplx y = cb[2 * j] + I * cb[2 * j + 1];
            if (y == 0) continue;
            product_into(alg, nmodes, la[i], lb[j], x * y, out);
            product_into(alg, nmodes, lb[j], la[i], -(x * y), out);
        }
    }
    return out;
}
