"""Compile the CUDA/C++ library in-tree for sm_103a (nvcc, no cmake).

Produces paper_1801_00246_gb300/_lib/libdg_gb300.so from the sources in csrc/,
compiling translation units in parallel and linking with the CUDA runtime.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB_NAME = "libdg_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def lib_path():
    return os.path.join(OUT_DIR, LIB_NAME)


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, jobs=None):
    nvcc = nvcc_path()
    os.makedirs(os.path.join(OUT_DIR, "obj"), exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "dg.h"))
    common = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
    objs, cmds = [], []
    for src in sources():
        obj = os.path.join(OUT_DIR, "obj", os.path.basename(src) + ".o")
        objs.append(obj)
        if _stale(obj, [src] + headers):
            lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
            cmds.append([nvcc] + common + lang + ["-c", src, "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r

    with ThreadPoolExecutor(max_workers=jobs or min(8, os.cpu_count() or 4)) as ex:
        list(ex.map(run, cmds))
    out = lib_path()
    if cmds or not os.path.exists(out):
        tmp = out + ".tmp"
        run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs)
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
