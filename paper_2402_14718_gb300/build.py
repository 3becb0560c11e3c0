"""Build the in-tree shared library ``libsbtrack.so`` (CUDA kernels for
sm_103a + host C++) with nvcc and g++; objects go to ``_build/``.
``build(checked=True)`` builds the bounds-checked library
``libsbtrack_checked.so`` instead (every kernel source compiled with
-DSB_CHECKED=1; all its objects in ``_build/checked/``, so the two builds
can run at the same time).

Host C++ is compiled with -ffp-contract=off -fno-builtin: the event generator
and the QUBO builder must evaluate each double expression exactly as written
(no fused multiply-add, libm calls kept as calls) on x86-64 and on aarch64.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libsbtrack.so")
LIB_CHECKED = os.path.join(PKG, "libsbtrack_checked.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU = ["api.cu", "device/kernels.cu", "device/stream.cu", "device/rw.cu", "device/noalloc.cu", "device/build.cu",
      "device/probe.cu", "device/factor.cu"]
# FP64 builder kernels: one IEEE operation per written operation, as on the host
CU_FLAGS = {"device/build.cu": ["-fmad=false"]}
CPP = ["host/events.cpp", "host/qubo.cpp", "host/tracks.cpp"]


def _nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _cuda_home():
    return os.path.dirname(os.path.dirname(os.path.realpath(_nvcc())))


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _stale(obj, srcs):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(s) > t for s in srcs)


def _deps():
    out = [os.path.join(ROOT, "include", "sb.h")]
    for d, _, files in os.walk(CSRC):
        out += [os.path.join(d, f) for f in files if f.endswith((".h", ".cuh"))]
    return out


def build(verbose=False, force=False, ptxas_verbose=False, checked=False):
    """Compile what is stale; SB_EXTRA_NVCC (environment) appends nvcc flags."""
    cu_dir = os.path.join(BUILD, "checked") if checked else BUILD
    lib_path = LIB_CHECKED if checked else LIB
    os.makedirs(cu_dir, exist_ok=True)
    extra = os.environ.get("SB_EXTRA_NVCC", "").split() + (["-DSB_CHECKED=1"] if checked else [])
    deps = _deps()
    nvcc = _nvcc()
    jobs = []
    objs = []
    for f in CU:
        src = os.path.join(CSRC, f)
        obj = os.path.join(cu_dir, f.replace("/", "_") + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + deps):
            cmd = [nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--extended-lambda"] + CU_FLAGS.get(f, []) + extra + ["-c", src, "-o", obj]
            if ptxas_verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    for f in CPP:
        src = os.path.join(CSRC, f)
        obj = os.path.join(cu_dir, f.replace("/", "_") + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + deps):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-builtin",
                         "-Wall", "-c", src, "-o", obj])
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose or ptxas_verbose:
        for o in outs:
            if o.strip():
                print(o)
    if jobs or not os.path.exists(lib_path) or _stale(lib_path, objs):
        lib64 = os.path.join(_cuda_home(), "lib64")
        _run([nvcc, ARCH, "-shared", "-cudart", "shared", "-o", lib_path + ".tmp"] + objs +
             ["-Xlinker", "-rpath," + lib64])
        os.replace(lib_path + ".tmp", lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, ptxas_verbose="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
