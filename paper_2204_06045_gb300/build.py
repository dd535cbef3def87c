"""Build libqtgb.so in-tree: CUDA sources for sm_103a only, the planner with g++.

Translation units compile in parallel into ``_build/``; the shared library is
linked next to this file. Nothing is installed anywhere else.
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
CSRC = HERE / "csrc"
INCLUDE = HERE.parent / "include"
BUILD = HERE.parent / "_build"
LIB = HERE / "libqtgb.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr"] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-pthread"]


def _sources():
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cpp"))


def _deps():
    return (_sources() + sorted(CSRC.glob("*.hpp")) + sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))
            + [Path(__file__)])


def _nvcc() -> str:
    cand = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = Path(cand) / "bin" / "nvcc"
    return str(p) if p.exists() else "nvcc"


def up_to_date() -> bool:
    if not LIB.exists():
        return False
    t = LIB.stat().st_mtime
    return all(d.stat().st_mtime <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, defines=(), out: Path = None) -> Path:
    """Compile and link ``libqtgb.so`` (or a variant with extra -D ``defines``
    at ``out``); returns its path."""
    lib = Path(out) if out else LIB
    if not force and not defines and out is None and up_to_date():
        return LIB
    build_dir = BUILD if out is None else lib.parent / (lib.stem + "_obj")
    build_dir.mkdir(parents=True, exist_ok=True)
    dflags = [f"-D{d}" for d in defines]
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in _sources():
        obj = build_dir / (src.name + ".o")
        objs.append(obj)
        if src.suffix == ".cu":
            cmd = [nvcc, *NVCC_FLAGS, *dflags, "-I", str(INCLUDE), "-c", str(src), "-o", str(obj)]
        else:
            cmd = ["g++", *CXX_FLAGS, *dflags, "-I", str(INCLUDE), "-c", str(src), "-o", str(obj)]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, pr in procs:
        log, _ = pr.communicate()
        if pr.returncode != 0:
            failed.append((cmd, log.decode(errors="replace")))
        elif verbose and log:
            print(log.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError(f"libqtgb build failed:\n{msg}")
    tmp = lib.with_suffix(f".{os.getpid()}.tmp.so")
    link = [nvcc, "-shared", *ARCH, "-o", str(tmp), *map(str, objs), "-lpthread"]
    subprocess.run(link, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
