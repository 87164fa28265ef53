"""The graph compiler's command line: build a bundle from a named workload
or a label file, reload it on the host (no GPU), refuse damaged files."""
import json
import os
import subprocess
import sys

import numpy as np

from cut_inputs import ALG_FERMION, fermion_registry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, "-m", "paper_2609_14831_b300", *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_build_and_info_of_a_named_workload(tmp_path):
    out = str(tmp_path / "p4.cutg")
    r = _run("build", "--workload", "closed_pauli_4q", "--out", out)
    assert r.returncode == 0, r.stderr
    st = json.loads(r.stdout)
    # 4 qubits: every non-identity Z-string anticommutes with 128 of the 256
    # strings (15 x 128 generator records); 240 x 128 commutator records
    assert (st["n"], st["R_g"], st["R_L"]) == (256, 15 * 128, 240 * 128)
    r = _run("info", out)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout)
    assert (d["n"], d["n_g"], d["R_g"], d["R_L"]) == (st["n"], st["n_g"], st["R_g"], st["R_L"])
    assert len(d["sha256"]) == 64


def test_build_from_a_label_file_matches_the_python_call(tmp_path):
    import paper_2609_14831_b300 as cg
    labels = fermion_registry(4)
    np.save(tmp_path / "reg.npy", labels)
    out = str(tmp_path / "f4.cutg")
    r = _run("build", "--labels", str(tmp_path / "reg.npy"), "--algebra", "fermion", "--nmodes", "4", "--out", out)
    assert r.returncode == 0, r.stderr
    st = json.loads(r.stdout)
    ref = cg.build_graph(ALG_FERMION, 4, labels, str(tmp_path / "ref.cutg"))
    assert (st["R_g"], st["R_L"], st["n_codes"]) == (ref["R_g"], ref["R_L"], ref["n_codes"])
    # the same registry compiles to the same bytes
    assert open(out, "rb").read() == open(tmp_path / "ref.cutg", "rb").read()


def test_info_refuses_a_damaged_bundle(tmp_path):
    out = str(tmp_path / "p4.cutg")
    assert _run("build", "--workload", "closed_pauli_4q", "--out", out).returncode == 0
    raw = bytearray(open(out, "rb").read())
    raw[len(raw) // 2] ^= 0xFF
    open(out, "wb").write(bytes(raw))
    r = _run("info", out)
    assert r.returncode == 1
    assert "CHECKSUM" in r.stderr or "FORMAT" in r.stderr


def test_cut_log_reports_the_phases_only_when_asked(tmp_path):
    out = str(tmp_path / "p4.cutg")
    env = dict(os.environ, CUT_LOG="1")
    r = subprocess.run([sys.executable, "-m", "paper_2609_14831_b300", "build", "--workload", "closed_pauli_4q",
                        "--out", out], cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr
    names = [l.split()[1] for l in r.stderr.splitlines() if l.startswith("[cut] ")]
    assert names == ["cut_build/count", "cut_build/write", "cut_build/store", "cut_build"]
    env.pop("CUT_LOG")
    r = subprocess.run([sys.executable, "-m", "paper_2609_14831_b300", "info", out], cwd=ROOT,
                       capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0 and "[cut]" not in r.stderr
