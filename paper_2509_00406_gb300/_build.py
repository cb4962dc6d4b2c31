"""In-tree build of libadm.so with nvcc for sm_103a (no cmake, no torch
extension machinery).  Translation units compile in parallel; the result is
``paper_2509_00406_gb300/_build/libadm.so``."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libadm.so")
HOST_LIB = os.path.join(OUT, "libadm_host.so")
HOST_SOURCES = ["host_check.cpp", "mesh.cpp", "tiles.cpp"]
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["atomic_f32.cu", "atomic_f64.cu", "tiled_f32.cu", "tiled_f64.cu", "reduce.cu", "noalloc.cu", "mlp.cu", "dyn.cu", "ring.cu",
           "mesh.cpp", "tiles.cpp", "api.cpp"]
# tiled-kernel variant groups, each tiled_inst.cu compiled with its own defines
# (object name, defines): sets 0-4 = passive+gradient, Hessian, filtered
# Hessian, matrix-free product, filtered matrix-free product
VARIANT_UNITS = [(f"tiled_{t}_{k}", [f"-DADM_INST_T={ty}", f"-DADM_INST_SET={k}"])
                 for t, ty in (("f32", "float"), ("f64", "double")) for k in range(5)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++20", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; libadm needs the CUDA toolkit to build")
    return p


def _digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    h.update(" ".join(ARCH + COMMON).encode())
    h.update(repr((SOURCES, VARIANT_UNITS)).encode())
    return h.hexdigest()


# sources of the tiled FP32 kernel; a change to any of them (or to the flags)
# invalidates ncu counters recorded for that kernel
TILED_KERNEL_SOURCES = ["ad.cuh", "spd.cuh", "terms.cuh", "device_common.cuh", "tiled_impl.cuh", "tiled_inst.cu"]


def kernel_digest(files=None) -> str:
    """Digest of the sources one kernel is compiled from, plus the flags
    (include paths relative to the repository, so that the digest is the
    same on every machine the repository is copied to)."""
    h = hashlib.sha256()
    for name in (files or TILED_KERNEL_SOURCES):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    flags = [os.path.relpath(f, ROOT) if os.path.isabs(f) else f for f in ARCH + COMMON]
    h.update(" ".join(flags).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    stamp = os.path.join(OUT, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    nvcc = _nvcc()

    def compile_one(unit) -> str:
        src, name, defs = (unit, unit, []) if isinstance(unit, str) else ("tiled_inst.cu", unit[0], unit[1])
        obj = os.path.join(OUT, name + ".o")
        cmd = [nvcc, *ARCH, *COMMON, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        with open(os.path.join(OUT, name + ".log"), "w") as f:
            f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-6000:]}")
        if verbose:
            print(r.stderr)
        return obj

    units = SOURCES + VARIANT_UNITS
    with cf.ThreadPoolExecutor(len(units)) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lpthread"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    build_host()
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


def build_host() -> str:
    """libadm_host.so: the creation-time builders (hinges, pattern, tiles)
    compiled with the host C++ compiler alone, for GPU-free tests."""
    os.makedirs(OUT, exist_ok=True)
    h = hashlib.sha256()
    for name in HOST_SOURCES + ["internal.h"]:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    with open(os.path.join(INCLUDE, "adm.h"), "rb") as f:
        h.update(f.read())
    stamp = os.path.join(OUT, "host_stamp")
    if os.path.exists(HOST_LIB) and os.path.exists(stamp) and open(stamp).read() == h.hexdigest():
        return HOST_LIB
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(_nvcc())), "include")
    tmp = HOST_LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++20", "-fPIC", "-shared", "-pthread", "-I", INCLUDE, "-I", CSRC, "-I", cuda_inc,
           *[os.path.join(CSRC, f) for f in HOST_SOURCES], "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"host build failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, HOST_LIB)
    with open(stamp, "w") as f:
        f.write(h.hexdigest())
    return HOST_LIB


if __name__ == "__main__":
    print(build(verbose=True))
