"""Build the CUDA shared library libsylv_adi.so in-tree (sm_103a only).

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into paper_2312_02891_gb300/_lib/libsylv_adi.so with the CUDA runtime
linked statically, so the library loads without a matching libcudart.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
OUT = PKG / "_lib"
OBJ = PKG / "_lib" / "obj"
LIB = OUT / "libsylv_adi.so"
SOURCES = ["api.cu", "ops.cu", "inst_r64.cu", "inst_r32.cu", "inst_rbf.cu", "inst_c128.cu", "inst_c64.cu",
           "inst_cbf.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libsylv_adi.so")


def flags(debug: bool = False):
    f = ARCH + ["-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", "--expt-relaxed-constexpr",
                "-Xptxas", "-warn-spills", "-I", str(CSRC), "-I", str(PKG.parent / "include")]
    f += ["-O0", "-G"] if debug else ["-O3"]
    return f


def _stale(src: Path, obj: Path) -> bool:
    if not obj.exists():
        return True
    deps = list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h")) + [PKG.parent / "include" / "sylv_adi.h", src]
    t = obj.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps if d.exists())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> Path:
    nvcc = nvcc_path()
    OBJ.mkdir(parents=True, exist_ok=True)
    extra = list(extra or [])

    def compile_one(name: str):
        src = CSRC / name
        obj = OBJ / (Path(name).stem + ".o")
        if not force and not extra and not _stale(src, obj):
            return obj, ""
        cmd = [nvcc, "-c", str(src), "-o", str(obj)] + flags() + extra
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{p.stdout}\n{p.stderr}")
        return obj, p.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            if log:
                print(log)
    objs = [str(o) for o, _ in results]
    tmp = LIB.with_suffix(".so.tmp")
    cmd = [nvcc, "-shared", "-o", str(tmp)] + objs + ARCH + ["-cudart", "static"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
