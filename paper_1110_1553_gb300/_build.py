"""In-tree build of the native library ``libhqr.so`` (sm_103a).

Compiles the host C++ sources with g++ and the CUDA sources with nvcc
(``-gencode arch=compute_103a,code=sm_103a``) in parallel, then links one
shared library next to this file. No cmake; a few translation units.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libhqr.so")
BUILD = os.path.join(HERE, "_build")

GENCODE = "-gencode=arch=compute_103a,code=sm_103a"
CXX_SRCS = ["elim_list.cpp", "dag.cpp"]
CU_SRCS = ["hqr_api.cu", "peaks.cu"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhqr.so")


def _sources_newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Build ``libhqr.so`` if a source is newer than it. Returns its path."""
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "hqr.h"))
    deps.append(os.path.abspath(__file__))
    if not force and not _sources_newer(OUT, deps):
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for f in CXX_SRCS:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-c", os.path.join(CSRC, f), "-o", o])
    for f in CU_SRCS:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([nvcc, GENCODE, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                     "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, f), "-o", o])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for j in jobs]
    failed = []
    for j, pr in zip(jobs, procs):
        out, _ = pr.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if pr.returncode != 0:
            failed.append((" ".join(j), out))
    if failed:
        msg = "\n\n".join("%s\n%s" % f for f in failed)
        raise RuntimeError("libhqr build failed:\n" + msg)
    tmp = OUT + ".tmp"
    link = [nvcc, GENCODE, "-shared", "-o", tmp] + objs
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("libhqr link failed:\n" + r.stdout)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
