"""Build the CUDA library libqsim.so in-tree for sm_103a (GB300).

Each translation unit is compiled by its own nvcc process, in parallel, then
linked into ``paper_2311_01512_gb300/libqsim.so`` against the shared CUDA
runtime.  No cmake, no torch extension machinery.
"""

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(PKG, "libqsim.so")

SOURCES = ["qs_gates.cu", "qs_gates_df.cu", "qs_gates_fx.cu", "qs_tc.cu", "qs_tc_ozaki.cu", "qs_density.cu", "qs_reduce.cu", "qs_api.cpp", "qs_noalloc.cu", "qs_fuse.cu", "qs_circuit.cpp", "qs_mlp.cu", "qs_costmodel.cpp", "qs_batch_kernels.cu", "qs_batch.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources_digest():
    """SHA-256 over every kernel source and header (sorted by name): the key
    that ties a recorded ncu measurement to the code it measured."""
    import hashlib
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".cpp", ".h")):
            h.update(name.encode())
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if os.path.exists(cand):
        return cand
    found = shutil.which("nvcc")
    if not found:
        raise RuntimeError("nvcc not found: set CUDA_HOME or put nvcc on PATH")
    return found


def _compile(src, nvcc, verbose):
    obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
           "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, " ".join(cmd), res.stderr))
    return obj, res.stderr


def build(verbose=False):
    """Compile every source and link libqsim.so.  Returns the library path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, nvcc, verbose), SOURCES))
    objs = [r[0] for r in results]
    if verbose:
        for _, err in results:
            if err:
                print(err)
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", LIB_PATH, *objs,
           "-Xlinker", "-rpath," + cuda_lib]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), res.stderr))
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose=True))
