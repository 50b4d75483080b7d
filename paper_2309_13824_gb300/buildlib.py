"""Build the CUDA library in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into ``paper_2309_13824_gb300/_build/libtrime_gb300.so``.  Host code is built
with ``-ffp-contract=off`` (the geometry-grid precomputation follows fixed
floating-point formulas); device code keeps decision-critical arithmetic free
of contractions through explicit round-to-nearest intrinsics.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
OUT_DIR = PKG / "_build"
LIB = OUT_DIR / "libtrime_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["voronoi_f64.cu", "voronoi_f32.cu", "voronoi_f64b.cu", "voronoi_f32b.cu", "bucket.cu", "emit.cu",
         "update.cu", "mesh.cu", "mlp.cu", "peaks.cu", "addition.cu", "sdf.cu", "sizing.cu", "autosize.cu", "init.cu", "adf.cu",
         "quality.cu"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
            "-Xcompiler", "-fPIC,-ffp-contract=off", f"-I{INCLUDE}", f"-I{CSRC}", *extra]


def _stale(obj: Path, src: Path) -> bool:
    if not obj.exists():
        return True
    deps = [src, *CSRC.glob("*.cuh"), *INCLUDE.glob("*.h")]
    return obj.stat().st_mtime < max(d.stat().st_mtime for d in deps)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False) -> Path:
    """Compile every unit (in parallel) and link the shared library."""
    OUT_DIR.mkdir(exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for u in UNITS:
        src = CSRC / u
        obj = OUT_DIR / (u[:-3] + ".o")
        if force or ptxas_info or _stale(obj, src):
            extra = ["-Xptxas", "-v"] if ptxas_info else []
            jobs.append([nvcc, *_flags(extra), "-c", str(src), "-o", str(obj)])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or ptxas_info or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    objs = [str(OUT_DIR / (u[:-3] + ".o")) for u in UNITS]
    if force or jobs or not LIB.exists():
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", str(tmp), *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="--ptxas" in sys.argv, force="--force" in sys.argv)
    print(LIB)
