"""Builds the CUDA library libasedf.so (sm_103a) in-tree, with nvcc, in parallel.

    python -m paper_2410_05489_gb300.build [--verbose]

Objects and the library go to paper_2410_05489_gb300/_build/.  The sweep kernel file is
compiled once per scheme order (3, 5, 7, 9), and so are the adjoint and gas-kinetic kernel files.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libasedf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _units():
    units = []
    for r in (3, 5, 7, 9):
        units.append(("ase_df_sweep.cu", "sweep_r%d.o" % r, ["-DASE_DF_ORDER=%d" % r]))
        units.append(("ase_df_adjoint.cu", "adjoint_r%d.o" % r, ["-DASE_DF_ORDER=%d" % r]))
        units.append(("ase_df_gks.cu", "gks_r%d.o" % r, ["-DASE_DF_ORDER=%d" % r]))
    for src in ("ase_df_combine.cu", "ase_df_api.cu", "ase_df_fp64_peak.cu", "ase_df_tables.cpp",
                "ase_df_noalloc.cu", "ase_df_batch.cu", "ase_df_gks_combine.cu"):
        if os.path.exists(os.path.join(CSRC, src)):
            units.append((src, os.path.splitext(src)[0] + ".o", []))
    return units


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "ase_df.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile all translation units and link libasedf.so; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC,
                     "--expt-relaxed-constexpr"]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(u):
        src, obj, extra = u
        cmd = [NVCC, *common, *extra, "-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)]
        res = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, res

    units = _units()
    with ThreadPoolExecutor(max_workers=min(8, len(units))) as ex:
        results = list(ex.map(compile_one, units))
    for cmd, res in results:
        if verbose and res.stderr:
            sys.stderr.write(res.stderr)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed: %s\n%s%s" % (" ".join(cmd), res.stdout, res.stderr))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp] + [os.path.join(BUILD, u[1]) for u in units]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), res.stdout, res.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="--verbose" in sys.argv))
