"""Build libgsp.so in-tree for sm_103a with nvcc (no cmake).

Each .cu under csrc/ is compiled in parallel to an object; the objects are
linked into paper_2110_12749_gb300/libgsp.so.  Host code is compiled with
-ffp-contract=off so that the FP64 delay table is evaluated in source order.
"""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libgsp.so")
BUILD = os.path.join(HERE, "_build")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-O3",
         "-I", INC, "-I", CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INC, "gsp.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force=False, verbose=False, extra=()):
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def cc(pair):
        src, obj = pair
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r

    with ThreadPoolExecutor(len(srcs)) as ex:
        results = list(ex.map(cc, zip(srcs, objs)))
    for src, r in results:
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
    tmp = LIB + ".tmp%d" % os.getpid()
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


def run_pipe_probe():
    """Build and run the pipe throughput probe (csrc/probe/pipe_probe.cu), which
    measures the integer, FP32 and shared-load throughput behind the
    dedispersion kernel's roofline; returns its report."""
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "pipe_probe")
    src = os.path.join(CSRC, "probe", "pipe_probe.cu")
    subprocess.run([NVCC, *ARCH, "-O3", "-o", exe, src], check=True)
    return subprocess.run([exe], check=True, capture_output=True, text=True).stdout


if __name__ == "__main__":
    if "--probe" in sys.argv:
        print(run_pipe_probe())
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
