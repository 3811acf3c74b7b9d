"""Build the C-ABI CUDA library libift.so in-tree for sm_103a.

Every translation unit is compiled in parallel; the element kernels are
instantiated once per (problem, degree, precision) from csrc/asm_inst.cu. A
stamp of the sources and flags skips up-to-date builds.
"""

from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libift.so")
PROBE_SRC = os.path.join(HERE, "probe", "fma_probe.cu")
PROBE_LIB = os.path.join(HERE, "probe", "libfma_probe.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _units():
    units = [("api", "api.cu", []), ("lm", "lm.cu", []), ("refelem", "refelem.cpp", []),
             ("dispatch", "dispatch.cpp", []), ("noalloc", "noalloc.cu", []),
             ("mlp", "mlp.cu", []), ("mlp_tc", "mlp_tc.cu", []),
             ("syrk_tc", "syrk_tc.cu", [])]
    for prob in (1, 2, 3):
        for p in (1, 2, 3):
            for prec in (0, 1):
                units.append((f"asm_{prob}_{p}_{prec}", "asm_inst.cu",
                              [f"-DIFT_PROB={prob}", f"-DIFT_P={p}", f"-DIFT_PREC={prec}"]))
    return units


def _stamp() -> str:
    h = hashlib.sha256()
    with open(PROBE_SRC, "rb") as f:
        h.update(f.read())
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "ift.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile the library (if stale) and return the path of libift.so."""
    stamp = _stamp()
    stamp_file = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read() == stamp:
                return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_unit(u):
        name, src, defs = u
        obj = os.path.join(BUILD, name + ".o")
        cmd = [nvcc] + NVCC_FLAGS + extra + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compiling {name} failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    units = _units()
    workers = max(1, min(len(units), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_unit, units))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "shared", "-Xlinker",
                                                            "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    build_probe(nvcc)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


def build_probe(nvcc=None) -> str:
    """The FMA throughput probe used by the benchmark (a separate small library)."""
    nvcc = nvcc or _nvcc()
    if os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(PROBE_SRC):
        return PROBE_LIB
    tmp = PROBE_LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-O3", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, PROBE_SRC, "-cudart", "shared"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"probe build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv))
