"""The compiled graph against the oracle, record by record (CPU only).

Every stored record is an exact integer factor: bit-exact equality is
required.  The expected records come from oracle unit-vector probes:
  generator stage: alpha(g; i, j) = coefficient of G_g in [O_i, O_j]
                   (divided by i for Pauli strings, eta = i sum xi G);
  commutator stage: beta(k; a, j) = coefficient of O_k in P[G_a, O_j]
                   (times i for Pauli strings).
Also: deterministic rebuilds, thread-count independence, validated reload.
"""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2609_14831_b300 as cg
from cut_inputs import (ALG_FERMION, ALG_PAULI, fermion_registry, pauli_registry, workload,
                        cfg2_registry)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_14831_b300 import build
    build.build()


def _graph(tmp_path, alg, nmodes, labels, name, **kw):
    path = str(tmp_path / f"{name}.cutg")
    stats = cg.build_graph(alg, nmodes, labels, path, **kw)
    return path, stats, cg.Graph(path, device=-1)


def _graph_records(G, stage):
    rp, a, b, c = G.records(stage)
    num, den = G.weights()
    assert np.all(den == 1)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return {(int(r), int(x), int(y)): int(num[z]) for r, x, y, z in zip(rows, a, b, c)}


def _expected_gen(alg, nmodes, labels, gen_labels):
    gidx = {int(l): a for a, l in enumerate(gen_labels)}
    diag = [oracle.is_diagonal(alg, l) for l in labels]
    out, dropped = {}, set()
    for i, li in enumerate(labels):
        if not diag[i]:
            continue
        for j, lj in enumerate(labels):
            if diag[j]:
                continue
            for g, v in oracle.commutator(alg, nmodes, {int(li): 1.0}, {int(lj): 1.0}).items():
                if v == 0:
                    continue
                val = v / 1j if alg == ALG_PAULI else v
                assert val.imag == 0 and val.real == round(val.real)
                if g in gidx:
                    out[(gidx[g], i, j)] = int(val.real)
                else:
                    dropped.add(g)
    return out, dropped


def _expected_comm(alg, nmodes, labels, gen_labels, a_subset=None):
    kidx = {int(l): k for k, l in enumerate(labels)}
    out = {}
    for a, ga in enumerate(gen_labels):
        if a_subset is not None and a not in a_subset:
            continue
        for j, lj in enumerate(labels):
            for k, v in oracle.commutator(alg, nmodes, {int(ga): 1.0}, {int(lj): 1.0}).items():
                if v == 0 or k not in kidx:
                    continue
                val = v * 1j if alg == ALG_PAULI else v
                assert val.imag == 0 and val.real == round(val.real)
                out[(kidx[k], a, j)] = int(val.real)
    return out


def _check_dropped_generators_are_inert(alg, nmodes, labels, dropped, max_rank):
    """Generator terms the graph leaves out must not reach the registry."""
    reg = {int(l) for l in labels}
    for g in list(dropped)[:60]:
        for lj in labels:
            F = oracle.commutator(alg, nmodes, {g: 1.0}, {int(lj): 1.0})
            assert all(v == 0 or k not in reg for k, v in F.items()), (hex(g), hex(int(lj)))


@pytest.mark.parametrize("case", ["pauli3", "pauli4", "fermion5", "fermion5_3body"])
def test_records_match_oracle_probes_exactly(tmp_path, case):
    if case.startswith("pauli"):
        nq = int(case[-1])
        alg, nmodes, labels = ALG_PAULI, nq, pauli_registry(nq)
    elif case == "fermion5":
        alg, nmodes, labels = ALG_FERMION, 5, fermion_registry(5)
    else:
        alg, nmodes = ALG_FERMION, 5
        labels = cfg2_registry(5, keep_shared1=0.3, seed=3)
    path, stats, G = _graph(tmp_path, alg, nmodes, labels, case)
    lab, gen_labels, diag = G.labels()
    np.testing.assert_array_equal(lab, labels)
    assert list(diag) == [oracle.is_diagonal(alg, l) for l in labels]
    want_gen, dropped = _expected_gen(alg, nmodes, labels, gen_labels)
    assert _graph_records(G, 0) == want_gen
    assert _graph_records(G, 1) == _expected_comm(alg, nmodes, labels, gen_labels)
    max_rank = max(bin(int(l) & 0xFFFFFFFF).count("1") for l in labels)
    _check_dropped_generators_are_inert(alg, nmodes, labels, dropped, max_rank)
    if case == "pauli4":
        assert (stats["R_g"], stats["R_L"]) == (15 * 128, 240 * 128)   # closed-form counts


def test_molecular_8so_records_sampled(tmp_path):
    w = workload("molecular_8so")
    path, stats, G = _graph(tmp_path, w.alg, w.nmodes, w.labels, "mol8")
    _, gen_labels, _ = G.labels()
    assert stats["n"] == 848
    rng = np.random.default_rng(0)
    subset = set(int(a) for a in rng.choice(len(gen_labels), 24, replace=False))
    want = _expected_comm(w.alg, w.nmodes, w.labels, gen_labels, subset)
    got = {key: v for key, v in _graph_records(G, 1).items() if key[1] in subset}
    assert got == want
    want_gen, _ = _expected_gen(w.alg, w.nmodes, w.labels, gen_labels)
    assert _graph_records(G, 0) == want_gen


def test_rebuild_is_bitwise_identical_for_any_thread_count(tmp_path):
    labels = cfg2_registry(6, keep_shared1=0.2, seed=4)
    paths = []
    for t, threads in enumerate((1, 3, 0)):
        p = str(tmp_path / f"g{t}.cutg")
        cg.build_graph(ALG_FERMION, 6, labels, p, threads=threads)
        paths.append(p)
    blobs = [open(p, "rb").read() for p in paths]
    assert blobs[0] == blobs[1] == blobs[2]
    G = cg.Graph(paths[0], device=-1)
    assert len(G.desc["sha256"]) == 64


def test_validated_reload_rejects_damaged_bundles(tmp_path):
    labels = fermion_registry(4)
    p = str(tmp_path / "g.cutg")
    cg.build_graph(ALG_FERMION, 4, labels, p)
    blob = bytearray(open(p, "rb").read())
    # flipped payload byte -> checksum error
    bad = bytearray(blob)
    bad[len(bad) // 2] ^= 0x40
    q = str(tmp_path / "flip.cutg")
    open(q, "wb").write(bad)
    with pytest.raises(cg.CutError) as e:
        cg.Graph(q, device=-1)
    assert e.value.name == "CHECKSUM"
    # truncated -> format error
    q = str(tmp_path / "trunc.cutg")
    open(q, "wb").write(blob[: len(blob) - 100])
    with pytest.raises(cg.CutError) as e:
        cg.Graph(q, device=-1)
    assert e.value.name == "FORMAT"
    # wrong magic -> format error
    bad = bytearray(blob)
    bad[0:8] = b"NOTAGRPH"
    q = str(tmp_path / "magic.cutg")
    open(q, "wb").write(bad)
    with pytest.raises(cg.CutError) as e:
        cg.Graph(q, device=-1)
    assert e.value.name == "FORMAT"
    # missing -> IO
    with pytest.raises(cg.CutError) as e:
        cg.Graph(str(tmp_path / "absent.cutg"), device=-1)
    assert e.value.name == "IO"


def test_builder_rejects_bad_registries(tmp_path):
    p = str(tmp_path / "x.cutg")
    labels = fermion_registry(3)
    with pytest.raises(cg.CutError) as e:
        cg.build_graph(ALG_FERMION, 3, np.concatenate([labels, labels[:1]]), p)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(cg.CutError):
        cg.build_graph(ALG_FERMION, 2, labels, p)         # label beyond nmodes
    with pytest.raises(cg.CutError):
        cg.build_graph(ALG_FERMION, 3, np.array([1 | (3 << 32)], dtype=np.uint64), p)  # not number conserving


def test_library_exports_every_declared_symbol():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(cut_[a-z0-9_]+)\s*\(", text))
    assert "cut_rhs" in names and "cut_flow_batched" in names
    L = cg.lib()
    for n in sorted(names):
        assert hasattr(L, n), n


def test_traversals_refuse_host_only_handles(tmp_path):
    p = str(tmp_path / "h.cutg")
    cg.build_graph(ALG_PAULI, 2, pauli_registry(2), p)
    G = cg.Graph(p, device=-1)
    rc = cg.lib().cut_rhs(G._h, None, 0, None, None, None, None, None)
    assert rc == 1


def _expected_outside(alg, nmodes, labels, gen_labels, out_labels):
    reg = {int(l) for l in labels}
    qidx = {int(l): q for q, l in enumerate(out_labels)}
    out = {}
    for a, ga in enumerate(gen_labels):
        for j, lj in enumerate(labels):
            for k, v in oracle.commutator(alg, nmodes, {int(ga): 1.0}, {int(lj): 1.0}).items():
                if v == 0 or k in reg:
                    continue
                val = v * 1j if alg == ALG_PAULI else v
                assert val.imag == 0 and val.real == round(val.real)
                out[(qidx[k], a, j)] = int(val.real)
    return out


@pytest.mark.parametrize("case", ["fermion4", "pauli3_sub"])
def test_outside_space_records_match_oracle_probes(tmp_path, case):
    if case == "fermion4":
        alg, nmodes, labels = ALG_FERMION, 4, fermion_registry(4)
    else:
        alg, nmodes, labels = ALG_PAULI, 3, pauli_registry(3)[::3]   # not closed under products
    path = str(tmp_path / f"{case}_d.cutg")
    cg.build_graph(alg, nmodes, labels, path, diagnostics=True)
    G = cg.Graph(path, device=-1)
    _, gen_labels, _ = G.labels()
    out_labels = G.outside_labels()
    assert G.n_out > 0 and G.R_C > 0
    reg = {int(l) for l in labels}
    assert not (set(int(l) for l in out_labels) & reg)
    assert _graph_records(G, 2) == _expected_outside(alg, nmodes, labels, gen_labels, out_labels)
    assert _graph_records(G, 1) == _expected_comm(alg, nmodes, labels, gen_labels)
    # the generator now holds every term of [H_d, H_od] (eta exact)
    want_gen, dropped = _expected_gen(alg, nmodes, labels, gen_labels)
    assert not dropped
    assert _graph_records(G, 0) == want_gen


def test_diagnostics_leave_the_retained_records_unchanged(tmp_path):
    labels = fermion_registry(5)
    p0, p1 = str(tmp_path / "a.cutg"), str(tmp_path / "b.cutg")
    cg.build_graph(ALG_FERMION, 5, labels, p0)
    cg.build_graph(ALG_FERMION, 5, labels, p1, diagnostics=True)
    G0, G1 = cg.Graph(p0, device=-1), cg.Graph(p1, device=-1)
    _, g0, _ = G0.labels()
    _, g1, _ = G1.labels()

    def by_label(G, gl):
        rp, a, b, c = G.records(1)
        num, _ = G.weights()
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        return {(int(r), int(gl[x]), int(y)): int(num[z]) for r, x, y, z in zip(rows, a, b, c)}
    assert by_label(G0, g0) == by_label(G1, g1)


def test_reload_range_checks_every_record_index(tmp_path):
    """A bundle whose checksum matches but one of whose records points past
    the registry is refused (FORMAT) before anything reaches the GPU: the
    kernels index with the stored values unchecked, so the reload checks
    every input index and factor code once.  Layout: 160-byte header (SHA-256
    of the payload at byte 72), then the sections labels, generator labels,
    diagonal mask, factor numerators and denominators, generator row
    pointers and records, commutator row pointers and records, ... each
    padded to 64 bytes."""
    import hashlib
    import struct
    labels = fermion_registry(4)
    p = str(tmp_path / "g.cutg")
    cg.build_graph(ALG_FERMION, 4, labels, p)
    blob = bytearray(open(p, "rb").read())
    n, n_g, R0, R1 = struct.unpack_from("<4Q", blob, 24)
    n_codes = struct.unpack_from("<I", blob, 56)[0]
    pad = lambda b: (b + 63) // 64 * 64
    sizes = [8 * n, 8 * n_g, n, 4 * n_codes, 4 * n_codes, 8 * (n_g + 1), 8 * R0, 8 * (n + 1)]
    rec1 = 160 + sum(pad(b) for b in sizes)
    for field, value in ((4, n), (0, n_g)):          # second input past n; first input past n_g
        bad = bytearray(blob)
        w = struct.unpack_from("<I", bad, rec1 + field)[0]
        new = value if field == 4 else (w & ~0xFFFFFF) | value
        struct.pack_into("<I", bad, rec1 + field, new)
        bad[72:104] = hashlib.sha256(bytes(bad[160:])).digest()
        q = str(tmp_path / f"range{field}.cutg")
        open(q, "wb").write(bad)
        with pytest.raises(cg.CutError) as e:
            cg.Graph(q, device=-1)
        assert e.value.name == "FORMAT" and "out of range" in str(e.value)
    # the unmodified bytes, re-signed the same way, still load
    ok = bytearray(blob)
    ok[72:104] = hashlib.sha256(bytes(ok[160:])).digest()
    assert ok == blob
