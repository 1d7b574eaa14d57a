"""Builds libcufz.so from csrc/ with nvcc for sm_103a (in-tree).

    python -m paper_2601_01048_gb300.build_ext [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcufz.so")
SOURCES = ["engine.cu", "runtime.cu", "loader.cpp", "prex.cpp", "mutate.cpp", "noalloc.cu", "campaign.cu"]
# device headers handed to the runtime compiler for the compiled path, under
# the names the sources include them by
JIT_HEADERS = [("jit_kernel.cuh", "jit_kernel.cuh"), ("jit_launch.cuh", "jit_launch.cuh"),
               ("device_common.cuh", "device_common.cuh"), ("layout.h", "layout.h"),
               ("../../include/cufz.h", os.path.join("..", "..", "include", "cufz.h"))]
HEADERS = ["engine.h", "ir.h", "interp_kernel.cuh", "checked_ops.h", "input_build.h", "mutate.h"] + [h[1] for h in JIT_HEADERS]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the cufz engine needs the CUDA toolkit to build")


def write_jit_embed() -> None:
    """Writes _build/jit_embed.h: the device headers as raw string literals."""
    texts = []
    for name, rel in JIT_HEADERS:
        with open(os.path.join(CSRC, rel)) as f:
            t = f.read()
        if ")CUFZ_EMBED" in t:
            raise RuntimeError(f"{rel} contains the embed delimiter")
        texts.append((name, t))
    out = ["// generated by build_ext.py from the device headers; do not edit", "#pragma once",
           f"static const int kJitHeaderCount = {len(texts)};",
           "static const char* const kJitHeaderName[] = {"]
    out += [f'  "{n}",' for n, _ in texts]
    out += ["};", "static const char* const kJitHeaderText[] = {"]
    out += [f'  R"CUFZ_EMBED({t})CUFZ_EMBED",' for _, t in texts]
    out += ["};", ""]
    path = os.path.join(OUT_DIR, "jit_embed.h")
    data = "\n".join(out)
    if not os.path.exists(path) or open(path).read() != data:
        with open(path, "w") as f:
            f.write(data)


def _stale(force: bool) -> bool:
    if force or not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not _stale(force):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nv = nvcc()
    objs = []
    write_jit_embed()

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src + ".o")
        cmd = [nv, *ARCH, *FLAGS, "-I", OUT_DIR, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nv)), "lib64")
    cmd = [nv, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-lnvrtc",
           "-Xlinker", f"-rpath={cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
