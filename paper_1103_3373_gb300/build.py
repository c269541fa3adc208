"""Build libhydro.so (sm_103a) in-tree from paper_1103_3373_gb300/csrc.

Every translation unit is compiled by nvcc in parallel, then linked into one
shared library with a plain C ABI (include/hydro.h).  Flags per unit:
  * FP64 kernels and the auxiliary kernels: -fmad=false, so every addition and
    multiplication is rounded separately, in source order;
  * FP32 / mixed kernels: fast single-precision division and square root with
    flush-to-zero (-prec-div=false -prec-sqrt=false -ftz=true).
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libhydro.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]
EXACT = ["-fmad=false"]
FAST = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]


def units():
    out = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith(".cu"):
            continue
        flags = FAST if (f.endswith("_fp32.cu") or f.endswith("_mixed.cu")) else EXACT
        out.append((f, flags))
    return out


def deps():
    inc = os.path.join(ROOT, "include")
    return ([os.path.join(CSRC, f) for f in os.listdir(CSRC)] +
            [os.path.join(inc, f) for f in os.listdir(inc)] + [os.path.abspath(__file__)])


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in deps())


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.exists(c) or c == "nvcc"):
            return c
    return "nvcc"


def _compile(args):
    src, flags = args
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [nvcc()] + COMMON + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    log = os.path.join(BUILD, src.replace(".cu", ".ptxas.log"))
    with open(log, "w") as fh:
        fh.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr[-4000:]))
    return obj


def build(force=False, jobs=None):
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    us = units()
    jobs = jobs or min(len(us), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(_compile, us))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
