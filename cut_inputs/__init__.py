"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This package holds no flow arithmetic: it only enumerates operator registries
(which coordinates a coefficient vector has) and draws seeded coefficient
vectors with the distributions of the workloads.  Both the oracle and the
product library take these as plain inputs.

Label encoding (one uint64 per operator):
  * Pauli strings on nq qubits: low 32 bits = X-support mask, high 32 bits =
    Z-support mask (per qubit I=(0,0), X=(1,0), Y=(1,1), Z=(0,1)).
  * Normal-ordered, number-conserving fermion monomials
    a+_{c1}..a+_{cm} a_{am}..a_{a1} (creators ascending, annihilators
    descending): low 32 bits = creator mask, high 32 bits = annihilator mask.
"""
from .registry import (ALG_PAULI, ALG_FERMION, ALG_PAULI_BOSON, pauli_registry, fermion_registry,
                       label_lo, label_hi, make_label, pauli_string, fermion_string,
                       cfg2_registry, pauli_boson_label, pauli_boson_parts, pauli_boson_registry)
from .hamiltonians import (pauli_hamiltonian, molecular_hamiltonian, pauli_boson_hamiltonian,
                           number_operator, dipole_operator, batched_parameters,
                           parameter_directions, Workload, workload)

__all__ = [n for n in dir() if not n.startswith("_")]
