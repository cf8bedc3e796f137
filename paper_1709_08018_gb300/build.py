"""Compile the CUDA library (sm_103a) in-tree: ``_build/libkl.so`` next to this file.

Each translation unit is compiled in parallel, then linked into one shared
library.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libkl.so")
SOURCES = ["kl_render.cu", "kl_batch.cu", "kl_mlp.cu", "kl_lod.cu", "kl_fsa.cu", "kl_host.cpp"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(p) > t for p in deps)


def _flags():
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "-Xcompiler", "-fvisibility=hidden", "-I", os.path.join(ROOT, "include")]


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libkl.so if any source is newer; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tag = f".tmp{os.getpid()}"
    objs = [os.path.join(OUT_DIR, os.path.splitext(f)[0] + tag + ".o") for f in SOURCES]

    def compile_one(args):
        src, obj = args
        cmd = [_nvcc()] + _flags() + (["-Xptxas", "-v"] if verbose else [])
        cmd += ["-c", os.path.join(CSRC, src), "-o", obj]
        return subprocess.run(cmd, capture_output=True, text=True)

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, zip(SOURCES, objs)))
    for src, r in zip(SOURCES, results):
        if verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError(f"nvcc failed on {src}")
    tmp = LIB + tag
    subprocess.run([_nvcc(), ARCH, "-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB)
    for o in objs:
        os.unlink(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
