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

static inline void add_term(Term *buf, int &n, uint64_t label, int re, int im) {
    for (int i = 0; i < n; i++)
        if (buf[i].label == label) { buf[i].re += re; buf[i].im += im; return; }
    buf[n++] = {label, re, im};
}

// [A, B] = AB - BA with like terms combined and zeros dropped.  buf >= 64.
static inline int commutator(int alg, uint64_t a, uint64_t b, Term *buf) {
    int n = 0;
    if (alg == 0) {
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
    return alg == 0 ? lo32(l) == 0 : lo32(l) == hi32(l);
}

static inline int rank_of(int alg, uint64_t l) {
    return alg == 0 ? popc(lo32(l) | hi32(l)) : popc(lo32(l));
}

}  // namespace cut
