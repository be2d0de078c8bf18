"""Builds libvps.so in-tree for sm_103a (nvcc, parallel, no cmake).

``build()`` compiles every translation unit that is older than its sources
and links ``paper_2405_19004_gb300/_lib/libvps.so``.  The per-(dim, degree)
kernel file is compiled 14 times with -DVPS_DIM / -DVPS_K.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libvps.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                  "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _units():
    headers = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "vps.h"))
    units = []
    for d in (2, 3):
        for k in range(1, 8):
            units.append((os.path.join(CSRC, "kernels_dk.cu"), os.path.join(OBJ, f"kernels_d{d}_k{k}.o"),
                          [f"-DVPS_DIM={d}", f"-DVPS_K={k}"], headers))
    for name in ("ops.cu", "noalloc.cu", "setup.cpp", "api.cpp", "server.cpp"):
        src = os.path.join(CSRC, name)
        units.append((src, os.path.join(OBJ, os.path.splitext(name)[0] + ".o"), [], headers))
    return units


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(nvcc, src, obj, defs, verbose_ptxas):
    cmd = [nvcc] + NVFLAGS + defs + ["-c", src, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc, "-x", "c++", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I" + INCLUDE, "-I" + CSRC, "-c", src, "-o", obj]
    elif verbose_ptxas:
        cmd.insert(1, "-Xptxas=-v")
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    return obj, p.stderr


def build(jobs=None, verbose_ptxas=False, force=False):
    """Compile and link libvps.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    todo = [u for u in _units() if force or _stale(u[1], [u[0]] + u[3])]
    logs = []
    if todo:
        jobs = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = [ex.submit(_compile, nvcc, s, o, d, verbose_ptxas) for s, o, d, _ in todo]
            for f in futs:
                logs.append(f.result())
    objs = [u[1] for u in _units()]
    if force or todo or _stale(LIB, objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
        os.replace(tmp, LIB)
    if verbose_ptxas:
        for obj, err in logs:
            sys.stderr.write(f"== {os.path.basename(obj)}\n{err}")
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force="--force" in sys.argv))
