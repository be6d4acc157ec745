"""Build ``libask.so`` (the C-ABI library of ``include/ask.h``) in-tree.

Every CUDA translation unit is compiled for sm_103a only, in parallel:

* ``ask_api.cu`` (host driver), ``ask_kernels.cu`` (exhaustive and ASK
  kernels), ``ask_queue.cu`` (the persistent batch kernel over a device work
  queue), ``ask_schemes.cu`` (the paper's SBR / MBR mappings),
  ``ask_fp64.cu`` (double-precision kernels for deep zooms) and
  ``ask_noalloc.cu`` (the allocation-free ASK entry point) as ordinary
  whole-program device code;
* ``ask_cdp2.cu`` with relocatable device code, device-linked against the
  CUDA device runtime (``cudadevrt``) for the tail-launch variant.

Floating point: ``--fmad=false`` and the ``_rn`` intrinsics keep every
product and sum rounded on its own, denormals are kept (``-ftz=false``),
and host code is compiled without contraction.  The CUDA runtime is linked
statically so the library only needs the driver at run time.
"""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libask.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                      "-Xcompiler", "-ffp-contract=off", "--fmad=false", "-ftz=false",
                      "-prec-div=true", "-prec-sqrt=true", "-I", INCLUDE]
PLAIN_UNITS = ["ask_api.cu", "ask_kernels.cu", "ask_queue.cu", "ask_schemes.cu", "ask_noalloc.cu",
               "ask_fp64.cu"]
RDC_UNITS = ["ask_cdp2.cu"]


def cuda_home():
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "ask.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale():
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(p) > t for p in _inputs())


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed (%d): %s\n%s" % (r.returncode, " ".join(cmd), r.stdout))
    if verbose and r.stdout.strip():
        print(r.stdout, flush=True)
    return r.stdout


def build(force=False, verbose=False, ptxas_verbose=False):
    """Compile libask.so if missing or older than its sources; return its path."""
    if not force and not _stale():
        return LIB_PATH
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    os.makedirs(BUILD_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []
    jobs = []
    for u in PLAIN_UNITS:
        obj = os.path.join(BUILD_DIR, u.replace(".cu", ".o"))
        jobs.append([nvcc] + NVCC_COMMON + extra + ["-c", os.path.join(CSRC, u), "-o", obj])
    for u in RDC_UNITS:
        obj = os.path.join(BUILD_DIR, u.replace(".cu", ".o"))
        jobs.append([nvcc] + NVCC_COMMON + extra + ["-rdc=true", "-c", os.path.join(CSRC, u), "-o", obj])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(lambda c: _run(c, verbose), jobs))
    if ptxas_verbose:
        for o in outs:
            print(o)
    rdc_objs = [os.path.join(BUILD_DIR, u.replace(".cu", ".o")) for u in RDC_UNITS]
    dlink = os.path.join(BUILD_DIR, "ask_dlink.o")
    _run([nvcc] + ARCH + ["-Xcompiler", "-fPIC", "-dlink"] + rdc_objs +
         ["-o", dlink, "-lcudadevrt"], verbose)
    objs = [os.path.join(BUILD_DIR, u.replace(".cu", ".o")) for u in PLAIN_UNITS] + rdc_objs + [dlink]
    libdir = os.path.join(home, "lib64")
    if not os.path.isdir(libdir):
        libdir = os.path.join(home, "lib")
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    _run([os.environ.get("CXX", "g++"), "-shared", "-o", tmp] + objs +
         ["-L" + libdir, "-Wl,-rpath," + libdir, "-lcudadevrt", "-lcudart_static",
          "-lpthread", "-ldl", "-lrt"], verbose)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, ptxas_verbose="-v" in sys.argv))
