"""Dense-matrix representations used to pin the oracle (test helper).

Pauli strings become Kronecker products of 2x2 Pauli matrices; fermion
ladder operators become Jordan-Wigner matrices on the 2**norb Fock space.
Nothing here multiplies operator strings symbolically: the products are
plain matrix products, an independent route to the same algebra.
"""
from functools import reduce
from itertools import combinations

import numpy as np

_I = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def pauli_matrix(label, nq):
    label = int(label)
    x, z = label & 0xFFFFFFFF, label >> 32
    mats = []
    for q in range(nq):
        bx, bz = (x >> q) & 1, (z >> q) & 1
        mats.append(_Y if (bx and bz) else _X if bx else _Z if bz else _I)
    return reduce(np.kron, mats[::-1])


def pauli_coefficients(M, labels, nq):
    """c_P = Tr(P M) / 2**nq (the Pauli strings are orthogonal)."""
    d = 2 ** nq
    return np.array([np.trace(pauli_matrix(l, nq) @ M) / d for l in labels])


def creation(p, norb):
    """Jordan-Wigner a+_p on 2**norb states; bit p of the index = occupation of p."""
    d = 2 ** norb
    M = np.zeros((d, d), dtype=np.complex128)
    for s in range(d):
        if not (s >> p) & 1:
            sign = (-1) ** bin(s & ((1 << p) - 1)).count("1")
            M[s | (1 << p), s] = sign
    return M


def fermion_matrix(label, norb):
    """a+_{c1}..a+_{cm} a_{am}..a_{a1}: creators ascending, annihilators descending."""
    label = int(label)
    c, a = label & 0xFFFFFFFF, label >> 32
    d = 2 ** norb
    M = np.eye(d, dtype=np.complex128)
    for p in range(norb):
        if c >> p & 1:
            M = M @ creation(p, norb)
    for p in reversed(range(norb)):
        if a >> p & 1:
            M = M @ creation(p, norb).conj().T
    return M


def op_matrix(op, alg, nmodes):
    f = pauli_matrix if alg == 0 else fermion_matrix
    d = 2 ** nmodes
    M = np.zeros((d, d), dtype=np.complex128)
    for l, c in op.items():
        if c != 0:
            M = M + c * f(l, nmodes)
    return M


def vec_matrix(labels, coefs, alg, nmodes):
    return op_matrix({int(l): c for l, c in zip(labels, coefs)}, alg, nmodes)


def sector_basis(norb, N):
    """Occupation-number states with N particles (bit masks), lexicographic."""
    return [sum(1 << p for p in occ) for occ in combinations(range(norb), N)]


def sector_block(M, norb, N):
    idx = sector_basis(norb, N)
    return M[np.ix_(idx, idx)]


def wegner_rhs(B):
    """Dense Wegner flow dB/ds = [[diag B, B], B] (eta = [B_d, B_od] = [B_d, B])."""
    Bd = np.diag(np.diag(B))
    eta = Bd @ B - B @ Bd
    return eta @ B - B @ eta, eta


def rk4_dense(f, B, ds, nsteps):
    for _ in range(nsteps):
        k1 = f(B)
        k2 = f(B + 0.5 * ds * k1)
        k3 = f(B + 0.5 * ds * k2)
        k4 = f(B + ds * k3)
        B = B + ds * (k1 + 2 * k2 + 2 * k3 + k4) / 6
    return B


def _apply_monomial(label, state):
    """Jordan-Wigner action of a+_{c1}..a+_{cm} a_{am}..a_{a1} on an occupation
    bit mask: returns (sign, new_state) or (0, None)."""
    label = int(label)
    c, a = label & 0xFFFFFFFF, label >> 32
    sign = 1
    s = state
    for p in range(32):                 # a_{a1} acts first (smallest index)
        if a >> p & 1:
            if not (s >> p) & 1:
                return 0, None
            sign *= (-1) ** bin(s & ((1 << p) - 1)).count("1")
            s ^= 1 << p
    for p in reversed(range(32)):       # then a+_{cm} ... a+_{c1}
        if c >> p & 1:
            if (s >> p) & 1:
                return 0, None
            sign *= (-1) ** bin(s & ((1 << p) - 1)).count("1")
            s |= 1 << p
    return sign, s


def sector_matrix(labels, coefs, norb, N):
    """Matrix of sum_k coefs[k] O_k on the N-particle occupation states."""
    basis = sector_basis(norb, N)
    pos = {s: i for i, s in enumerate(basis)}
    M = np.zeros((len(basis), len(basis)))
    for l, c in zip(labels, coefs):
        if c == 0:
            continue
        for col, s in enumerate(basis):
            sg, t = _apply_monomial(l, s)
            if sg:
                M[pos[t], col] += sg * c
    return M


def rk_dense(f, y, ds, A, B):
    """One explicit RK step with tableau (A, B) for any array state."""
    ks = []
    for i in range(len(B)):
        u = y
        for j, a in enumerate(A[i]):
            if a != 0.0:
                u = u + ds * a * ks[j]
        ks.append(f(u))
    out = y
    for b, k in zip(B, ks):
        if b != 0.0:
            out = out + ds * b * k
    return out
