"""Builds the gwhe CUDA library (libgwhe.so) in-tree for sm_103a.

Translation units compile in parallel with nvcc; the result lands in
paper_1902_04303_gb300/_build/libgwhe.so.
"""
import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgwhe.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["ntt.cu", "kernels.cu", "ckks.cu", "gwas.cu", "capi.cu", "noalloc.cu", "probe.cu", "server.cu", "params.cpp"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(SRC, u) for u in UNITS]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(INCLUDE, "gwhe.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def _compile(src):
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    cmd = [nvcc(), "-c", src, "-o", obj, "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
           "-I", SRC, "-I", INCLUDE] + ARCH
    if src.endswith(".cpp"):
        cmd += ["-Xcompiler", "-ffp-contract=off"]
    else:
        cmd += ["--expt-relaxed-constexpr"]
    subprocess.run(cmd, check=True)
    return obj


def build(force: bool = False) -> str:
    """Compile every translation unit and link libgwhe.so (if stale)."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(_compile, _sources()))
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.run([nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
