"""Build libmba.so in-tree with nvcc for sm_103a (GB300).

Each .cu file is compiled in parallel to an object; the objects are linked
into ``_build/libmba.so`` (CUDA runtime linked statically).  No torch headers
are involved: the library's interface is the plain C ABI in include/mba.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmba.so")
HEADER = os.path.join(ROOT, "include", "mba.h")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    inc = os.path.dirname(HEADER)
    deps = (sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")] +
            [os.path.join(inc, f) for f in os.listdir(inc) if f.endswith((".h", ".cuh"))])
    return any(os.path.getmtime(d) > t for d in deps)


def edge_lib(edge_type: str) -> str:
    """Path of the library built with the user edge type edge_type."""
    return os.path.join(BUILD, "edge_" + edge_type, "libmba.so")


def build(force: bool = False, verbose: bool = False, edge: tuple[str, str] | None = None) -> str:
    """Compile and link libmba.so if any source changed; return its path.

    edge = (header path, type name): a library whose dual-number path evaluates
    that user edge type instead of the BAL edge (see csrc/edge_bal.cuh), built
    into its own folder (edge_lib(type name)); the default library is untouched.
    """
    out_dir, lib, defs = BUILD, LIB, []
    if edge is not None:
        header, name = os.path.abspath(edge[0]), edge[1]
        if not name.replace("_", "").replace(":", "").isalnum():
            raise ValueError("edge type must be a C++ identifier")
        out_dir, lib = os.path.dirname(edge_lib(name)), edge_lib(name)
        defs = [f'-DMBA_EDGE_HEADER="{header}"', f"-DMBA_EDGE_TYPE={name}"]
        if not force and os.path.exists(lib) and not _stale() and os.path.getmtime(lib) >= max(
                os.path.getmtime(header), os.path.getmtime(LIB)):
            return lib
    elif not force and not _stale():
        return LIB
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *defs, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def declared_functions() -> list[str]:
    """Names of the functions declared in include/mba.h."""
    import re

    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mba_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))
