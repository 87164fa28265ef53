"""Seeded coefficient vectors for the workloads.

Every vector is aligned with a registry from `registry.py`: entry k is the
real coefficient of label k.  Nothing here evaluates a commutator.

Workload recipes (the readings used where the workload description is
silent are listed beside each draw):
  * closed Pauli algebra, nq=4: diagonal (I/Z-only) strings ~ U(-2, 2),
    off-diagonal strings with an even number of Y ~ N(0, 0.1) (a real
    symmetric H), odd-Y strings exactly 0.  Seed 0.
  * molecular model on `norb` spin-orbitals: one-body energies
    eps_p = linspace(-1.5, 1.0) on n_p; one-body off-diagonal t_pq = t_qp and
    two-body V_{pq,rs} = V_{rs,pq} drawn as s * N(0, 1) with s = 0.05 (the
    one-body off-diagonal draw is a reading); three-body labels, where the
    registry has them, get 0.2 * s * N(0, 1), Hermitian.  Observables: the
    particle number N and a one-body dipole-like D with symmetric
    d_pq ~ N(0, 0.1).
  * parameter batches: eps_p -> eps_p (1 + U(-0.2, 0.2)) per orbital and
    s ~ U(0.02, 0.1) per instance, applied to the same standard-normal pattern.
"""
from dataclasses import dataclass, field
from itertools import combinations

import numpy as np

from .registry import (ALG_PAULI, ALG_FERMION, ALG_PAULI_BOSON, pauli_registry, fermion_registry,
                       cfg2_registry, label_lo, label_hi, make_label, _mask, pauli_boson_label,
                       pauli_boson_parts, pauli_boson_registry)


def _popcount(v):
    return bin(int(v)).count("1")


def pauli_hamiltonian(nq=4, seed=0, sigma_od=0.1):
    labels = pauli_registry(nq)
    rng_d = np.random.default_rng([seed, 0])
    rng_o = np.random.default_rng([seed, 1])
    h = np.zeros(len(labels))
    for k, lab in enumerate(labels):
        x, z = label_lo(lab), label_hi(lab)
        if x == 0:
            h[k] = rng_d.uniform(-2.0, 2.0)
        elif _popcount(x & z) % 2 == 0:
            h[k] = rng_o.normal(0.0, sigma_od)
    return labels, h


def _index(labels):
    return {int(l): i for i, l in enumerate(labels)}


def molecular_parts(labels, norb, seed=1):
    """Return (eps_base, pattern): h = sum_p eps_p n_p + s * pattern."""
    idx = _index(labels)
    rng = np.random.default_rng(seed)
    eps = np.linspace(-1.5, 1.0, norb)
    pattern = np.zeros(len(labels))
    # one-body off-diagonal, symmetric
    for p in range(norb):
        for q in range(p + 1, norb):
            v = rng.normal()
            for (c, a) in ((p, q), (q, p)):
                k = idx.get(make_label(1 << c, 1 << a))
                if k is not None:
                    pattern[k] = v
    # two-body, symmetric over pair indices (diagonal included)
    pairs = list(combinations(range(norb), 2))
    for i, P in enumerate(pairs):
        for Q in pairs[i:]:
            v = rng.normal()
            for (c, a) in ((P, Q), (Q, P)):
                k = idx.get(make_label(_mask(c), _mask(a)))
                if k is not None:
                    pattern[k] = v
    # three-body labels present in the registry, Hermitian
    rng3 = np.random.default_rng([seed, 3])
    for k, lab in enumerate(labels):
        c, a = label_lo(lab), label_hi(lab)
        if _popcount(c) != 3 or c > a:
            continue
        v = 0.2 * rng3.normal()
        pattern[k] = v
        kc = idx.get(make_label(a, c))
        if kc is not None:
            pattern[kc] = v
    return eps, pattern


def _eps_vector(labels, eps):
    idx = _index(labels)
    out = np.zeros(len(labels))
    for p, e in enumerate(eps):
        out[idx[make_label(1 << p, 1 << p)]] = e
    return out


def molecular_hamiltonian(labels, norb, seed=1, scale=0.05):
    eps, pattern = molecular_parts(labels, norb, seed)
    return _eps_vector(labels, eps) + scale * pattern


def number_operator(labels, norb):
    return _eps_vector(labels, np.ones(norb))


def dipole_operator(labels, norb, seed=1, sigma=0.1):
    idx = _index(labels)
    rng = np.random.default_rng([seed, 1000])
    out = np.zeros(len(labels))
    for p in range(norb):
        for q in range(p, norb):
            v = rng.normal(0.0, sigma)
            out[idx[make_label(1 << p, 1 << q)]] = v
            out[idx[make_label(1 << q, 1 << p)]] = v
    return out


def batched_parameters(labels, norb, batch, seed=3, base_seed=1):
    """Parameter-set batch: [batch, n] Hamiltonians sharing one pattern."""
    eps, pattern = molecular_parts(labels, norb, base_seed)
    rng = np.random.default_rng(seed)
    jitter = rng.uniform(-0.2, 0.2, size=(batch, norb))
    scale = rng.uniform(0.02, 0.1, size=batch)
    eps_idx = [_index(labels)[make_label(1 << p, 1 << p)] for p in range(norb)]
    H = np.outer(scale, pattern)
    H[:, eps_idx] += eps[None, :] * (1.0 + jitter)
    return H


def parameter_directions(labels, norb, n_two_body=24, seed=4):
    """[n, 8 + n_two_body] matrix P: h(theta) = h_ref + P theta.

    Columns: the norb orbital-energy directions (unit vectors on n_p) and
    `n_two_body` seeded unit-norm Hermitian two-body directions.
    """
    idx = _index(labels)
    n = len(labels)
    cols = []
    for p in range(norb):
        v = np.zeros(n)
        v[idx[make_label(1 << p, 1 << p)]] = 1.0
        cols.append(v)
    rng = np.random.default_rng(seed)
    pairs = list(combinations(range(norb), 2))
    for _ in range(n_two_body):
        v = np.zeros(n)
        for i, P in enumerate(pairs):
            for Q in pairs[i:]:
                g = rng.normal()
                for (c, a) in ((P, Q), (Q, P)):
                    v[idx[make_label(_mask(c), _mask(a))]] = g
        cols.append(v / np.linalg.norm(v))
    return np.stack(cols, axis=1)


def pauli_boson_hamiltonian(labels, M, seed=5, sigma_od=0.05):
    """Seeded real-symmetric Pauli-boson Hamiltonian on a registry.

    Real basis {I, X, iY, Z} x boson monomials: the transpose of label
    (tau, c, a) is s_tau (tau, a, c) with s = -1 for iY, so a real symmetric
    H has h(tau, a, c) = s_tau h(tau, c, a).  Diagonal labels (tau in {I, Z},
    c = a): U(-1, 1) / (1 + |c|); the others N(0, sigma_od) / (1 + |c| + |a|).
    (The paper's HBQ parameters are not available; this recipe only fixes the
    structure.)
    """
    idx = _index(labels)
    rng = np.random.default_rng(seed)
    h = np.zeros(len(labels))
    for k, lab in enumerate(labels):
        tau, c, a = pauli_boson_parts(lab, M)
        deg = sum(c) + sum(a)
        if tau in (0, 3) and c == a:
            h[k] = rng.uniform(-1.0, 1.0) / (1 + sum(c))
            continue
        t = idx.get(pauli_boson_label(tau, a, c))
        if t is None or t < k:
            continue
        sgn = -1.0 if tau == 2 else 1.0
        if t == k:
            h[k] = 0.0 if sgn < 0 else rng.normal(0.0, sigma_od) / (1 + deg)
            continue
        v = rng.normal(0.0, sigma_od) / (1 + deg)
        h[k] = v
        h[t] = sgn * v
    return h


@dataclass
class Workload:
    name: str
    alg: int
    nmodes: int
    labels: np.ndarray
    h: np.ndarray
    observables: list = field(default_factory=list)
    method: str = "rk4"
    s_end: float = 10.0
    ds: float = 1e-3
    rtol: float = 1e-10
    atol: float = 0.0
    max_rank: int = 2


def workload(name, **kw):
    """Named workloads with the sizes and distributions described above.

    closed_pauli_4q    : 256 Pauli strings, RK4, ds = 1e-3 to s = 10.
    molecular_8so      : 848 fermion labels, H + N + D, DP45 rtol 1e-10.
    stress_<k>so       : k spin-orbitals + selected three-body labels
                         (stress_16so is the ~3.4e8-record stress graph).
    molecular_<k>so    : the molecular recipe on k spin-orbitals (tests).
    """
    if name == "closed_pauli_4q":
        labels, h = pauli_hamiltonian(4, seed=0)
        return Workload(name, ALG_PAULI, 4, labels, h, [], "rk4", 10.0, 1e-3)
    if name.startswith("molecular_") and name.endswith("so"):
        norb = int(name[len("molecular_"):-2])
        ranks = kw.get("ranks", (1, 2))
        labels = fermion_registry(norb, ranks=ranks)
        h = molecular_hamiltonian(labels, norb, seed=kw.get("seed", 1))
        obs = [number_operator(labels, norb), dipole_operator(labels, norb, seed=kw.get("seed", 1))]
        hmax = np.max(np.abs(h))
        return Workload(name, ALG_FERMION, norb, labels, h, obs, "dp45", 10.0, 1e-2,
                        1e-10, 1e-12 * hmax, max(ranks))
    if name.startswith("pauli_boson_"):
        # pauli_boson_<M>m<p>: M modes, complete degree-p registry
        M, p = name[len("pauli_boson_"):].split("m")
        M, p = int(M), int(p)
        labels = pauli_boson_registry(M, p)
        h = pauli_boson_hamiltonian(labels, M, seed=kw.get("seed", 5))
        return Workload(name, ALG_PAULI_BOSON, M, labels, h, [], "rk4", 1.0, 1e-3, 1e-10, 0.0, p)
    if name.startswith("stress_") and name.endswith("so"):
        norb = int(name[len("stress_"):-2])
        labels = cfg2_registry(norb, keep_shared1=STRESS_KEEP_SHARED1, keep_shared0=STRESS_KEEP_SHARED0,
                               seed=kw.get("seed", 2))
        h = molecular_hamiltonian(labels, norb, seed=kw.get("seed", 2))
        obs = [number_operator(labels, norb), dipole_operator(labels, norb, seed=kw.get("seed", 2))]
        hmax = np.max(np.abs(h))
        return Workload(name, ALG_FERMION, norb, labels, h, obs, "rk4", 10.0, 1e-3,
                        1e-10, 1e-12 * hmax, 3)
    raise KeyError(name)


# Stress registry (16 spin-orbitals, about 3.3e8 records): every three-body
# label sharing >= 1 orbital between its creator and annihilator sets and a
# seeded ~28% of the disjoint ones (a pair is kept when the smaller of its
# two draws is below 0.15).
STRESS_KEEP_SHARED1 = 1.0
STRESS_KEEP_SHARED0 = 0.15
