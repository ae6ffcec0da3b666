"""Compile the package's native libraries in-tree.

libamrgen.so : the seeded octree generator (host C++, OpenMP).
libamr.so    : the ray-casting library (CUDA for sm_103a + host C++ C-ABI).

Both land in ``paper_1210_8014_gb300/lib``.  A library is rebuilt when any of
its sources or headers is newer than it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
LIB = PKG / "lib"
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"

GEN_LIB = LIB / "libamrgen.so"
AMR_LIB = LIB / "libamr.so"

ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libamr")


def _stale(target: Path, deps: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def _run(cmd: list[str], cwd: Path = ROOT) -> None:
    res = subprocess.run(cmd, cwd=cwd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if res.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + res.stdout)


def gen_sources() -> list[Path]:
    return [CSRC / "gen" / "amr_gen.cpp", INCLUDE / "amr_gen.h"]


def amr_sources() -> list[Path]:
    return sorted((CSRC / "amr").glob("*.cu")) + sorted((CSRC / "amr").glob("*.cpp"))


def amr_headers() -> list[Path]:
    return sorted((CSRC / "amr").glob("*.h")) + sorted((CSRC / "amr").glob("*.cuh")) + [INCLUDE / "amr.h"]


def build_gen(force: bool = False) -> Path:
    LIB.mkdir(exist_ok=True)
    if force or _stale(GEN_LIB, gen_sources()):
        tmp = GEN_LIB.with_suffix(".so.tmp")
        _run(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-Wall",
              str(CSRC / "gen" / "amr_gen.cpp"), "-o", str(tmp)])
        tmp.replace(GEN_LIB)
    return GEN_LIB


def _compile_one(src: Path, obj: Path, deps: list[Path]) -> None:
    if not _stale(obj, [src] + deps):
        return
    if src.suffix == ".cu":
        cmd = [_nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
               "-I", str(INCLUDE), "-c", str(src), "-o", str(obj)]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", "-pthread",
               "-I", str(INCLUDE), "-I", "/usr/local/cuda/include", "-c", str(src), "-o", str(obj)]
    _run(cmd)


def build_amr(force: bool = False) -> Path:
    srcs = amr_sources()
    if not srcs:
        raise RuntimeError("no CUDA sources found under " + str(CSRC / "amr"))
    deps = amr_headers()
    objdir = LIB / "obj"
    objdir.mkdir(parents=True, exist_ok=True)
    objs = [objdir / (s.name + ".o") for s in srcs]
    if force:
        for o in objs:
            o.unlink(missing_ok=True)
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        list(ex.map(lambda so: _compile_one(so[0], so[1], deps), zip(srcs, objs)))
    if force or _stale(AMR_LIB, objs):
        tmp = AMR_LIB.with_suffix(".so.tmp")
        _run([_nvcc(), ARCH, "-shared", "-o", str(tmp)] + [str(o) for o in objs] +
             ["-cudart=static", "-lpthread"])
        tmp.replace(AMR_LIB)
    return AMR_LIB


def build_all(force: bool = False) -> None:
    with ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build_gen, force), ex.submit(build_amr, force)]
        for f in futs:
            f.result()


if __name__ == "__main__":
    build_all(force="--force" in sys.argv)
    print("built", GEN_LIB, AMR_LIB)
