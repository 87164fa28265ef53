"""Operator registries: the finite sets of canonical labels that index a
coefficient vector (the 'finite operator registry' of Sec. 2.1 of the paper;
which labels are retained is a physical input, not a compiler choice).
"""
from itertools import combinations

import numpy as np

ALG_PAULI = 0
ALG_FERMION = 1
ALG_PAULI_BOSON = 2

# Pauli-boson labels sigma_tau prod_m (b_m^+)^{c_m} b_m^{a_m} (Sec. 2.1, Eq.
# monomial), with the Pauli factor taken from the real basis
# {I, X, iY, Z} (tau = 0, 1, 2, 3) so that every coefficient is real:
# bits 0-1 tau, then per mode m: c_m in bits 2+10m .. 6+10m, a_m in bits
# 7+10m .. 11+10m (degrees up to 31, at most 6 modes).
PB_BITS = 5

_PAULI_DIGIT = {"I": (0, 0), "X": (1, 0), "Y": (1, 1), "Z": (0, 1)}


def make_label(lo, hi):
    return (int(hi) << 32) | int(lo)


def label_lo(label):
    return int(label) & 0xFFFFFFFF


def label_hi(label):
    return (int(label) >> 32) & 0xFFFFFFFF


def pauli_registry(nq):
    """All 4**nq Pauli strings; index = sum_q d_q 4**q with I,X,Y,Z = 0,1,2,3."""
    digits = [(0, 0), (1, 0), (1, 1), (0, 1)]
    out = np.empty(4 ** nq, dtype=np.uint64)
    for idx in range(4 ** nq):
        x = z = 0
        r = idx
        for q in range(nq):
            dx, dz = digits[r & 3]
            r >>= 2
            x |= dx << q
            z |= dz << q
        out[idx] = make_label(x, z)
    return out


def pauli_string(label, nq):
    """Human-readable form, qubit 0 first (for messages and fixtures)."""
    x, z = label_lo(label), label_hi(label)
    rev = {v: k for k, v in _PAULI_DIGIT.items()}
    return "".join(rev[((x >> q) & 1, (z >> q) & 1)] for q in range(nq))


def pauli_label(text):
    x = z = 0
    for q, ch in enumerate(text):
        dx, dz = _PAULI_DIGIT[ch]
        x |= dx << q
        z |= dz << q
    return make_label(x, z)


def _mask(idx):
    m = 0
    for i in idx:
        m |= 1 << i
    return m


def fermion_registry(norb, ranks=(1, 2), extra=None):
    """Number-conserving normal-ordered monomials of the given ranks.

    Order: rank, then creator combination (lexicographic), then annihilator
    combination (lexicographic).  `extra` optionally maps rank -> a boolean
    predicate(creators, annihilators) selecting a subset of that rank.
    """
    labels = []
    for r in ranks:
        combos = list(combinations(range(norb), r))
        pred = None if extra is None else extra.get(r)
        for c in combos:
            cm = _mask(c)
            for a in combos:
                if pred is not None and not pred(c, a):
                    continue
                labels.append(make_label(cm, _mask(a)))
    return np.array(labels, dtype=np.uint64)


def fermion_string(label):
    c, a = label_lo(label), label_hi(label)
    cs = [i for i in range(32) if c >> i & 1]
    an = [i for i in range(32) if a >> i & 1][::-1]
    return " ".join([f"a+{i}" for i in cs] + [f"a{i}" for i in an])


def cfg2_registry(norb=16, keep_shared1=0.0, seed=2, keep_shared0=0.0):
    """Stress registry: every one- and two-body label on `norb` orbitals, plus
    three-body labels whose creator and annihilator sets share at least two
    orbitals (spectator-dressed one-body moves), plus seeded fractions
    `keep_shared1` / `keep_shared0` of the three-body labels sharing exactly
    one / no orbital (fraction 1 keeps all of them).
    """
    rng = np.random.default_rng(seed)
    combos3 = list(combinations(range(norb), 3))
    # one uniform draw per unordered {creator set, annihilator set} pair, so
    # that a label and its Hermitian conjugate are kept together (the
    # registry is closed under conjugation) and the selection is reproducible
    draws = rng.random((len(combos3), len(combos3)))
    draws = np.minimum(draws, draws.T)
    sel = []
    for ci, c in enumerate(combos3):
        cs = set(c)
        for ai, a in enumerate(combos3):
            shared = len(cs.intersection(a))
            if (shared >= 2 or (shared == 1 and draws[ci, ai] < keep_shared1)
                    or (shared == 0 and draws[ci, ai] < keep_shared0)):
                sel.append(make_label(_mask(c), _mask(a)))
    base = fermion_registry(norb, ranks=(1, 2))
    return np.concatenate([base, np.array(sel, dtype=np.uint64)])


def pauli_boson_label(tau, c, a):
    lab = int(tau) & 3
    for m, (cm, am) in enumerate(zip(c, a)):
        assert 0 <= cm < 32 and 0 <= am < 32
        lab |= int(cm) << (2 + 10 * m)
        lab |= int(am) << (7 + 10 * m)
    return lab


def pauli_boson_parts(label, M):
    label = int(label)
    tau = label & 3
    c = tuple((label >> (2 + 10 * m)) & 31 for m in range(M))
    a = tuple((label >> (7 + 10 * m)) & 31 for m in range(M))
    return tau, c, a


def _multi_indices(nvar, deg):
    """All tuples of nvar non-negative integers with sum exactly deg."""
    if nvar == 1:
        yield (deg,)
        return
    for first in range(deg, -1, -1):
        for rest in _multi_indices(nvar - 1, deg - first):
            yield (first,) + rest


def pauli_boson_registry(M, p):
    """Complete degree-p registry: every (tau, c, a) with |c| + |a| <= p,
    ordered by total degree, then tau, then the exponents.  Its size is
    N_op(M, p) = 4 C(2M + p, p) (Eq. basis-size)."""
    out = []
    for deg in range(p + 1):
        idx = list(_multi_indices(2 * M, deg))
        for tau in range(4):
            for ca in idx:
                out.append(pauli_boson_label(tau, ca[:M], ca[M:]))
    return np.array(out, dtype=np.uint64)
