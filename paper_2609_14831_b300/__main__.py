"""Command line of the graph compiler (the compile-once step of the method).

    python -m paper_2609_14831_b300 build --workload molecular_8so --out m8.cutg
    python -m paper_2609_14831_b300 build --labels reg.npy --algebra fermion --nmodes 8 --out g.cutg
    python -m paper_2609_14831_b300 info g.cutg

build: compile a registry into a checksummed bundle.  The registry is
either a named workload (cut_inputs) or a .npy file of uint64 labels with
its algebra and mode count.  Options: --threads, --max-rank,
--diagnostics (outside-space records).  Prints the build statistics as one
JSON line.

info: reload a bundle on the host (format and checksum validated, no GPU)
and print its sizes and digest as one JSON line.

Exit status 0 on success, 1 on a library error (the message on stderr).
"""
import argparse
import json
import sys

import numpy as np

from . import CutError, Graph, build_graph


def _algebras():
    from cut_inputs import ALG_FERMION, ALG_PAULI, ALG_PAULI_BOSON
    return {"pauli": ALG_PAULI, "fermion": ALG_FERMION, "pauli_boson": ALG_PAULI_BOSON}


def _build(a):
    if a.workload:
        from cut_inputs import workload
        w = workload(a.workload)
        alg, nmodes, labels = w.alg, w.nmodes, w.labels
    else:
        if not (a.labels and a.algebra and a.nmodes):
            raise SystemExit("build: give --workload, or --labels with --algebra and --nmodes")
        alg, nmodes = _algebras()[a.algebra], a.nmodes
        labels = np.load(a.labels).astype(np.uint64)
    st = build_graph(alg, nmodes, labels, a.out, max_rank=a.max_rank, threads=a.threads,
                     diagnostics=a.diagnostics)
    print(json.dumps({"out": a.out, "labels": int(len(labels)), **st}))


def _info(a):
    G = Graph(a.path, device=-1)
    try:
        print(json.dumps({"path": a.path, **G.desc}))
    finally:
        G.close()


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2609_14831_b300", description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    b = sub.add_parser("build", help="compile a registry into a bundle")
    b.add_argument("--workload", help="named workload of cut_inputs (e.g. molecular_8so, stress_12so)")
    b.add_argument("--labels", help=".npy file of uint64 labels")
    b.add_argument("--algebra", choices=["pauli", "fermion", "pauli_boson"])
    b.add_argument("--nmodes", type=int)
    b.add_argument("--out", required=True)
    b.add_argument("--max-rank", type=int, default=0, help="0: the registry's top rank")
    b.add_argument("--threads", type=int, default=0, help="0: every host core")
    b.add_argument("--diagnostics", action="store_true", help="also write the outside-space records")
    i = sub.add_parser("info", help="validated host reload of a bundle")
    i.add_argument("path")
    a = ap.parse_args(argv)
    try:
        (_build if a.cmd == "build" else _info)(a)
    except CutError as e:
        print(f"{a.cmd}: {e}", file=sys.stderr)
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
