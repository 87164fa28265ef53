// algebra.h -- exact products of registry labels for the graph compiler.
//
// Products are evaluated in the full algebra and normal ordered before the
// registry is consulted (paper Sec. 2.1); coefficients are exact Gaussian
// integers.  The bitmask formulas here are the compiler's own; the test
// oracle multiplies strings by a different route.
#pragma once
#include <cstdint>

namespace cut {

struct Term {
    uint64_t label;
    int32_t re, im;  // exact coefficient re + i*im
};

static inline uint32_t lo32(uint64_t l) { return (uint32_t)l; }
static inline uint32_t hi32(uint64_t l) { return (uint32_t)(l >> 32); }
static inline int popc(uint32_t v) { return __builtin_popcount(v); }

// Pauli string with X-mask x and Z-mask z is P(x,z) = i^{|x&z|} X^x Z^z, so
// P1 P2 = i^{|x1&z1| + |x2&z2| - |x3&z3| + 2|z1&x2|} P(x1^x2, z1^z2).
static inline int pauli_mul(uint64_t a, uint64_t b, uint64_t *c) {
    uint32_t x1 = lo32(a), z1 = hi32(a), x2 = lo32(b), z2 = hi32(b);
    uint32_t x3 = x1 ^ x2, z3 = z1 ^ z2;
    int k = popc(x1 & z1) + popc(x2 & z2) - popc(x3 & z3) + 2 * popc(z1 & x2);
    *c = (uint64_t)x3 | ((uint64_t)z3 << 32);
    return k & 3;
}

// number of pairs (u in X, v in Y) with u > v
static inline int inversions(uint32_t X, uint32_t Y) {
    int s = 0;
    while (X) {
        int u = __builtin_ctz(X);
        X &= X - 1;
        s += popc(Y & ((1u << u) - 1u));
    }
    return s;
}

// Fermion monomial M(C, A) = Cr(C) An(A): creators ascending, annihilators
// descending (An(S) = Cr(S)^dagger).  The product M(C1,A1) M(C2,A2) needs
// An(A1) Cr(C2) in normal order; moving the annihilators of A1 through
// Cr(C2) smallest first uses
//   a_y Cr(C) = [y in C] (-1)^{|C below y|} Cr(C\y) + (-1)^{|C|} Cr(C) a_y,
// then Cr(C1) Cr(C') = (-1)^{inv(C1,C')} Cr(C1|C') and
// An(A') An(A2) = (-1)^{inv(A2,A')} An(A'|A2) (zero on overlaps).
// Writes at most 2^|A1 & C2| terms; returns their count.
static inline int fermion_mul(uint64_t a, uint64_t b, uint64_t *out, int *sgn) {
    uint32_t C1 = lo32(a), A1 = hi32(a), C2 = lo32(b), A2 = hi32(b);
    struct T { uint32_t C, A; int s; };
    T t[32], nt[32];
    int m = 1;
    t[0] = {C2, 0u, 1};
    uint32_t rem = A1;
    while (rem) {
        int y = __builtin_ctz(rem);
        rem &= rem - 1;
        uint32_t yb = 1u << y;
        int k = 0;
        for (int i = 0; i < m; i++) {
            const T &u = t[i];
            if (u.C & yb) nt[k++] = {u.C & ~yb, u.A, (popc(u.C & (yb - 1u)) & 1) ? -u.s : u.s};
            nt[k++] = {u.C, u.A | yb, (popc(u.C) & 1) ? -u.s : u.s};
        }
        for (int i = 0; i < k; i++) t[i] = nt[i];
        m = k;
    }
    int cnt = 0;
    for (int i = 0; i < m; i++) {
        if ((C1 & t[i].C) || (t[i].A & A2)) continue;
        int par = (inversions(C1, t[i].C) + inversions(A2, t[i].A)) & 1;
        out[cnt] = (uint64_t)(C1 | t[i].C) | ((uint64_t)(t[i].A | A2) << 32);
        sgn[cnt] = par ? -t[i].s : t[i].s;
        cnt++;
    }
    return cnt;
}

// Pauli-boson label: bits 0-1 tau (real Pauli basis I, X, iY, Z), mode m:
// c_m = bits 2+10m..6+10m, a_m = bits 7+10m..11+10m.
constexpr int kPBModes = 6;
static inline int pb_tau(uint64_t l) { return (int)(l & 3); }
static inline int pb_c(uint64_t l, int m) { return (int)((l >> (2 + 10 * m)) & 31); }
static inline int pb_a(uint64_t l, int m) { return (int)((l >> (7 + 10 * m)) & 31); }
static inline int pb_degree(uint64_t l) {
    int d = 0;
    for (int m = 0; m < kPBModes; m++) d += pb_c(l, m) + pb_a(l, m);
    return d;
}

// Real Pauli basis R = {I, X, iY, Z}: R_a R_b = PB_SGN[a][b] R_{a^b}.
static const int PB_SGN[4][4] = {{1, 1, 1, 1}, {1, 1, -1, -1}, {1, 1, -1, -1}, {1, 1, 1, 1}};

static inline int64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

// sigma_t1 B(c1,a1) sigma_t2 B(c2,a2): the Pauli factors multiply in the real
// basis; per mode (b+)^{c1} b^{a1} (b+)^{c2} b^{a2} =
//   sum_k k! C(a1,k) C(c2,k) (b+)^{c1+c2-k} b^{a1+a2-k}  (normal ordering).
// Writes the terms (at most prod_m (min(a1_m, c2_m) + 1)); returns the count,
// or -1 when an exponent would exceed 31 or a factor would not stay an exact
// 32-bit integer.
static inline int pb_mul(uint64_t x, uint64_t y, uint64_t *out, int64_t *coef, int cap) {
    const int t1 = pb_tau(x), t2 = pb_tau(y);
    int n = 1;
    out[0] = (uint64_t)(t1 ^ t2);
    coef[0] = PB_SGN[t1][t2];
    for (int m = 0; m < kPBModes; m++) {
        const int c1 = pb_c(x, m), a1 = pb_a(x, m), c2 = pb_c(y, m), a2 = pb_a(y, m);
        if (!(c1 | a1 | c2 | a2)) continue;
        const int kmax = a1 < c2 ? a1 : c2;
        if (c1 + c2 > 31 || a1 + a2 > 31) return -1;
        const int n0 = n;
        if (n0 * (kmax + 1) > cap) return -1;
        for (int k = kmax; k >= 0; k--) {
            int64_t f = binom(a1, k) * binom(c2, k);
            for (int t = 2; t <= k; t++) f *= t;
            const uint64_t bits = ((uint64_t)(c1 + c2 - k) << (2 + 10 * m)) | ((uint64_t)(a1 + a2 - k) << (7 + 10 * m));
            for (int i = 0; i < n0; i++) {
                const int dst = k == 0 ? i : n + i;
                out[dst] = out[i] | bits;
                coef[dst] = coef[i] * f;
                if (coef[dst] > 0x3FFFFFFFll || coef[dst] < -0x3FFFFFFFll) return -1;  // keep factors exact in int32
            }
            if (k > 0) n += n0;
        }
    }
    return n;
}

static inline void add_term(Term *buf, int &n, uint64_t label, int re, int im) {
    for (int i = 0; i < n; i++)
        if (buf[i].label == label) { buf[i].re += re; buf[i].im += im; return; }
    buf[n++] = {label, re, im};
}

// [A, B] = AB - BA with like terms combined and zeros dropped.  buf >= 512
// for Pauli-boson labels (returns -1 if the product leaves the label range).
static inline int commutator(int alg, uint64_t a, uint64_t b, Term *buf) {
    int n = 0;
    if (alg == 2) {
        uint64_t lab[256];
        int64_t cf[256];
        int m = pb_mul(a, b, lab, cf, 256);
        if (m < 0) return -1;
        for (int i = 0; i < m; i++) add_term(buf, n, lab[i], (int)cf[i], 0);
        m = pb_mul(b, a, lab, cf, 256);
        if (m < 0) return -1;
        for (int i = 0; i < m; i++) add_term(buf, n, lab[i], -(int)cf[i], 0);
    } else if (alg == 0) {
        static const int RE[4] = {1, 0, -1, 0}, IM[4] = {0, 1, 0, -1};
        uint64_t c;
        int k = pauli_mul(a, b, &c);
        add_term(buf, n, c, RE[k], IM[k]);
        k = pauli_mul(b, a, &c);
        add_term(buf, n, c, -RE[k], -IM[k]);
    } else {
        uint64_t lab[32];
        int sg[32];
        int m = fermion_mul(a, b, lab, sg);
        for (int i = 0; i < m; i++) add_term(buf, n, lab[i], sg[i], 0);
        m = fermion_mul(b, a, lab, sg);
        for (int i = 0; i < m; i++) add_term(buf, n, lab[i], -sg[i], 0);
    }
    int w = 0;
    for (int i = 0; i < n; i++)
        if (buf[i].re != 0 || buf[i].im != 0) buf[w++] = buf[i];
    return w;
}

static inline bool is_diagonal(int alg, uint64_t l) {
    if (alg == 2) {  // I or Z Pauli factor and c = a in every mode
        if (pb_tau(l) == 1 || pb_tau(l) == 2) return false;
        for (int m = 0; m < kPBModes; m++)
            if (pb_c(l, m) != pb_a(l, m)) return false;
        return true;
    }
    return alg == 0 ? lo32(l) == 0 : lo32(l) == hi32(l);
}

// fermion: particle rank; Pauli: weight; Pauli-boson: total boson degree
static inline int rank_of(int alg, uint64_t l) {
    if (alg == 2) return pb_degree(l);
    return alg == 0 ? popc(lo32(l) | hi32(l)) : popc(lo32(l));
}

}  // namespace cut
