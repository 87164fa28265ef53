"""Compile libcut.so in-tree for sm_103a (nvcc cross-compiles without a GPU)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libcut.so")
SOURCES = ["cut_lib.cu", "batched.cu", "mlp.cu", "calib.cu", "builder.cpp", "bundle.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "cut.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile every source to an object in parallel, then link libcut.so."""
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    obj_dir = os.path.join(HERE, "_build")
    os.makedirs(obj_dir, exist_ok=True)
    flags = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O3", *ARCH, "-lineinfo",
             "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    jobs = []
    for src in sources():
        obj = os.path.join(obj_dir, os.path.basename(src) + f".{os.getpid()}.o")
        jobs.append((obj, [nvcc, *flags, "-c", src, "-o", obj]))
    procs = []
    for obj, cmd in jobs:
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append(subprocess.Popen(cmd))
    failed = [cmd for (obj, cmd), p in zip(jobs, procs) if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, failed[0])
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, "-shared", *ARCH, "-o", tmp, *[o for o, _ in jobs], "-lpthread"])
    for o, _ in jobs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
