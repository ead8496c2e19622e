"""Build the gbwave CUDA library in-tree with nvcc for sm_103a.

Produces ``paper_2404_04441_gb300/_build/libgbwave.so``. The library links
the CUDA runtime statically and reaches the driver's tensor-map encoder
through the runtime's entry-point query, so it needs no libcuda at link time.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libgbwave.so")
SOURCES = [os.path.join(CSRC, f) for f in ("wave.cu", "serve.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in ("sweep.cuh", "ptx.cuh", "common.cuh", "cpml.cuh")] + [
    os.path.join(ROOT, "include", f) for f in ("wave.h", "wave_serve.h")]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
    "-Xptxas", "-v",
]


def nvcc_path():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS if os.path.exists(p))


def build(force=False, verbose=False):
    """Compile the library if it is missing or older than its sources; return its path."""
    if not force and not stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + ".tmp%d" % os.getpid()
    # Compile the translation units in parallel, then link the shared library.
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc_path()] + NVCC_FLAGS + ["-c", src, "-o", obj]
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    logs = []
    for p in procs:
        out, err = p.communicate()
        logs.append(err)
        if p.returncode != 0:
            sys.stderr.write(out + err)
            raise RuntimeError("nvcc failed building %s" % LIB)
    link = [nvcc_path(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
            "-Xcompiler", "-fPIC"] + objs + ["-o", tmp]
    proc = subprocess.run(link, capture_output=True, text=True)
    if proc.returncode != 0:
        sys.stderr.write(proc.stdout + proc.stderr)
        raise RuntimeError("nvcc failed linking %s" % LIB)
    with open(os.path.join(OUT_DIR, "ptxas.log"), "w") as f:
        f.write("".join(logs))
    if verbose:
        sys.stderr.write(proc.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
