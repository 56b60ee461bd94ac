"""Builds the CUDA library libdns_gb300.so in-tree with nvcc for sm_103a.

One translation unit per (precision, N) instance listed in csrc/instances.h
(and per (precision, Nx, Ny, Nz) grid with other counts per direction),
plus the C-ABI unit, compiled in parallel and linked into a shared library
under paper_1602_03638_gb300/lib/. Object files go to _build/ (git-ignored).
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import re
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIBNAME = "libdns_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-Xptxas", "-O3"]


def library_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def instances():
    """(ctype, tag, N) triples from csrc/instances.h."""
    with open(os.path.join(CSRC, "instances.h")) as f:
        text = f.read()
    return [(t, tag, int(n)) for t, tag, n in re.findall(r"X\((float|double),\s*(f32|f64),\s*(\d+)\)", text)]


def box_instances():
    """(ctype, tag, Nx, Ny, Nz) of the grids with other counts per direction (csrc/instances.h)."""
    with open(os.path.join(CSRC, "instances.h")) as f:
        text = f.read()
    pat = r"B\((float|double),\s*(f32|f64),\s*(\d+),\s*(\d+),\s*(\d+)\)"
    return [(t, tag, int(a), int(b), int(c)) for t, tag, a, b, c in re.findall(pat, text)]


def _sources_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode())
                    h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


KERNEL_SOURCES = ("fft_core.cuh", "solver_kernels.cuh", "dns_internal.h", "solver_inst.cu", "instances.h")


def kernel_digest() -> str:
    """Digest of the files that define the solver kernels (not the C-ABI layer)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    digest = _sources_digest()
    stamp = os.path.join(BUILD, "stamp")
    lib = library_path()
    if not force and os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return lib
    nvcc = _nvcc()
    jobs_list = []
    for ctype, tag, n in instances():
        obj = os.path.join(BUILD, f"inst_{tag}_{n}.o")
        cmd = [nvcc, *ARCH, *FLAGS, f"-DDNS_INST_T={ctype}", f"-DDNS_INST_N={n}",
               f"-DDNS_INST_FN=dns_ops_{tag}_{n}", "-c", os.path.join(CSRC, "solver_inst.cu"), "-o", obj]
        jobs_list.append((obj, cmd))
    for ctype, tag, nx, ny, nz in box_instances():
        shape = f"{nx}x{ny}x{nz}"
        obj = os.path.join(BUILD, f"inst_{tag}_{shape}.o")
        cmd = [nvcc, *ARCH, *FLAGS, f"-DDNS_INST_T={ctype}", f"-DDNS_INST_N={nx}", f"-DDNS_INST_NY={ny}",
               f"-DDNS_INST_NZ={nz}", f"-DDNS_INST_FN=dns_ops_{tag}_{shape}", "-c",
               os.path.join(CSRC, "solver_inst.cu"), "-o", obj]
        jobs_list.append((obj, cmd))
    extra = ["capi.cu", "noalloc.cu", "sgs.cu", "mlp.cu"]
    for name in extra:
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        jobs_list.append((obj, [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, name), "-o", obj]))

    def run(item):
        obj, cmd = item
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr)
        return obj

    workers = jobs or max(1, min(len(jobs_list), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(run, jobs_list))
    tmp = lib + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(digest)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
