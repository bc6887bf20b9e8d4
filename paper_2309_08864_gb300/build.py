"""Builds libso2dr.so (the C-ABI library of include/so2dr.h) in-tree.

nvcc for sm_103a only (-gencode arch=compute_103a,code=sm_103a), one object per
translation unit compiled in parallel, static CUDA runtime so the library loads
on machines without a GPU (planning and introspection need none).
"""
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libso2dr.so")
BUILD_DIR = os.path.join(HERE, "_build")

CU_SOURCES = ["run.cu", "kernels.cu", "tma_map.cu", "adjoint.cu", "noalloc.cu", "tune.cu", "stencil_f64.cu", "stencil_f32.cu",
              "stencil_bf16.cu", "stencil_f16.cu"]
CXX_SOURCES = ["plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libso2dr.so")


def _digest():
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            p = os.path.join(d, f)
            if os.path.isfile(p) and f.endswith((".cu", ".cuh", ".cpp", ".hpp", ".h", ".inc")):
                h.update(f.encode())
                with open(p, "rb") as fh:
                    h.update(fh.read())
    h.update(" ".join(ARCH).encode())
    h.update(os.environ.get("SO2DR_NVCC_FLAGS", "").encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False) -> str:
    stamp = os.path.join(BUILD_DIR, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
    # extra nvcc flags from SO2DR_NVCC_FLAGS (part of the build stamp)
    common += os.environ.get("SO2DR_NVCC_FLAGS", "").split()
    cu_flags = common + ARCH + ["-lineinfo", "-fmad=true", "--expt-relaxed-constexpr"]
    jobs = []
    for s in CU_SOURCES:
        jobs.append([nvcc] + cu_flags + ["-c", os.path.join(CSRC, s), "-o",
                                         os.path.join(BUILD_DIR, s + ".o")])
    for s in CXX_SOURCES:
        jobs.append([nvcc] + common + ["-x", "c++", "-c", os.path.join(CSRC, s), "-o",
                                       os.path.join(BUILD_DIR, s + ".o")])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError("compile failed: " + " ".join(cmd))
    objs = [os.path.join(BUILD_DIR, s + ".o") for s in CU_SOURCES + CXX_SOURCES]
    tmp = LIB + ".tmp%d" % os.getpid()
    link = [nvcc, "-shared"] + ARCH + ["-cudart", "static", "-o", tmp] + objs + ["-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
