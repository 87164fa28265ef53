"""Pauli-boson algebra (the paper's registry, Sec. 2.1): CPU pins.

- registry sizes against Eq. (basis-size) and the values the paper prints;
- oracle products against truncated Fock-space matrices;
- compiled records against oracle probes, bit-exact;
- the compiled five-mode degree-four graph against the paper's count of
  production contributions (Sec. 3.2).
"""
import json
import os
from itertools import product as iproduct
from math import comb

import numpy as np
import pytest

import oracle
import paper_2609_14831_b300 as cg
from cut_inputs import ALG_PAULI_BOSON, pauli_boson_label, pauli_boson_parts, pauli_boson_registry

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pauli_boson_counts.json")))

RMAT = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, 1], [-1, 0]]), np.diag([1, -1])]


def boson_matrix(c, a, D):
    b = np.diag(np.sqrt(np.arange(1, D)), 1)           # annihilation, truncated at D
    return np.linalg.matrix_power(b.T, c) @ np.linalg.matrix_power(b, a)


def pb_matrix(label, M, D):
    tau, c, a = pauli_boson_parts(label, M)
    mat = RMAT[tau].astype(float)
    for m in range(M):
        mat = np.kron(mat, boson_matrix(c[m], a[m], D))
    return mat


def test_registry_sizes_match_the_closed_form_and_the_paper():
    for M, p, n in GOLD["registry_sizes"]:
        assert 4 * comb(2 * M + p, p) == n
        labels = pauli_boson_registry(M, p)
        assert len(labels) == n and len(set(labels.tolist())) == n


def _low_block(M, D, keep):
    """Indices of the tensor states whose occupations are all < keep."""
    idx = []
    for tau_i in range(2):
        for occ in iproduct(range(D), repeat=M):
            if all(o < keep for o in occ):
                flat = tau_i
                for o in occ:
                    flat = flat * D + o
                idx.append(flat)
    return np.array(idx)


@pytest.mark.parametrize("M,p", [(1, 4), (2, 2)])
def test_oracle_products_match_truncated_fock_matrices(M, p):
    labels = pauli_boson_registry(M, p)
    D = 4 * p + 2
    keep = D - 2 * p - 1       # no truncation effect on these states
    blk = _low_block(M, D, keep)
    rng = np.random.default_rng(33)
    pairs = [(x, y) for x in labels for y in labels] if len(labels) < 80 else \
        [tuple(rng.choice(labels, 2)) for _ in range(400)]
    for x, y in pairs:
        got = oracle.product(ALG_PAULI_BOSON, M, {int(x): 1.0}, {int(y): 1.0})
        want = pb_matrix(x, M, D) @ pb_matrix(y, M, D)
        mat = sum(v.real * pb_matrix(l, M, D) for l, v in got.items() if v != 0)
        np.testing.assert_allclose(np.asarray(mat)[np.ix_(blk, blk)], want[np.ix_(blk, blk)], atol=1e-9)


@pytest.mark.parametrize("M,p", [(1, 4), (2, 2)])
def test_records_match_oracle_probes(tmp_path, M, p):
    labels = pauli_boson_registry(M, p)
    path = str(tmp_path / "pb.cutg")
    cg.build_graph(ALG_PAULI_BOSON, M, labels, path)
    G = cg.Graph(path, device=-1)
    _, gen, diag = G.labels()
    assert list(diag) == [oracle.is_diagonal(ALG_PAULI_BOSON, l) for l in labels]
    num, den = G.weights()
    gidx = {int(l): a for a, l in enumerate(gen)}
    kidx = {int(l): k for k, l in enumerate(labels)}
    want0, want1 = {}, {}
    for i, li in enumerate(labels):
        if not diag[i]:
            continue
        for j, lj in enumerate(labels):
            if diag[j]:
                continue
            for g, v in oracle.commutator(ALG_PAULI_BOSON, M, {int(li): 1.0}, {int(lj): 1.0}).items():
                if v != 0:
                    want0[(gidx[g], i, j)] = int(round(v.real))
    for a, ga in enumerate(gen):
        for j, lj in enumerate(labels):
            for k, v in oracle.commutator(ALG_PAULI_BOSON, M, {int(ga): 1.0}, {int(lj): 1.0}).items():
                if v != 0 and k in kidx:
                    want1[(kidx[k], a, j)] = int(round(v.real))
    for stage, want in ((0, want0), (1, want1)):
        rp, x, y, c = G.records(stage)
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        got = {(int(r), int(u), int(v)): int(num[z]) for r, u, v, z in zip(rows, x, y, c)}
        assert got == want


def test_five_mode_degree_four_graph_has_the_papers_contribution_count(tmp_path):
    g = GOLD["production_contributions"]
    labels = pauli_boson_registry(g["modes"], g["degree"])
    st = cg.build_graph(ALG_PAULI_BOSON, g["modes"], labels, str(tmp_path / "pb5.cutg"))
    assert st["R_g"] + st["R_L"] == g["count"]


def test_five_mode_diagnostic_graph_has_the_papers_outside_count(tmp_path):
    """The diagnostic-enabled build (eta exact, every generated term outside
    the registry recorded) of the five-mode degree-four registry."""
    g = GOLD["outside_contributions"]
    labels = pauli_boson_registry(g["modes"], g["degree"])
    path = str(tmp_path / "pb5d.cutg")
    st = cg.build_graph(ALG_PAULI_BOSON, g["modes"], labels, path, diagnostics=True)
    G = cg.Graph(path, device=-1)
    assert G.R_C == g["count"]
    assert st["R_g"] + st["R_L"] + G.R_C == g["total"]
    G.close()
    os.remove(path)
