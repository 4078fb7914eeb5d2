"""Build the CUDA library in-tree: paper_2510_05392_gb300/_build/libmgpu.so.

Steps: the process compiler writes the tables (_build/gen/mg_tables.inc and
mg_proc_list.h), then nvcc compiles every translation unit for sm_103a in
parallel and links one shared library.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(BUILD, "libmgpu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _newest(paths):
    return max((os.path.getmtime(p) for p in paths if os.path.exists(p)), default=0.0)


def generate_tables(force: bool = False) -> None:
    os.makedirs(GEN, exist_ok=True)
    inc = os.path.join(GEN, "mg_tables.inc")
    srcs = glob.glob(os.path.join(HERE, "compiler", "*.py"))
    if not force and os.path.exists(inc) and os.path.getmtime(inc) >= _newest(srcs):
        return
    from .compiler import emit
    emit.emit(inc + ".tmp", 6, os.path.join(GEN, "mg_proc_list.h.tmp"))
    os.replace(os.path.join(GEN, "mg_proc_list.h.tmp"), os.path.join(GEN, "mg_proc_list.h"))
    os.replace(inc + ".tmp", inc)


def process_tables(ngluon: int, force: bool = False) -> str:
    """Binary table file of a process too large to compile into the library
    (g g > t t~ + 5 g), written by the process compiler on first use (about
    three minutes) and kept in _build/tables until the compiler changes."""
    tdir = os.path.join(BUILD, "tables")
    os.makedirs(tdir, exist_ok=True)
    path = os.path.join(tdir, f"proc_{ngluon}g.bin")
    srcs = glob.glob(os.path.join(HERE, "compiler", "*.py"))
    if force or not os.path.exists(path) or os.path.getmtime(path) < _newest(srcs):
        from .compiler import emit
        emit.emit_blob(ngluon, path)
    return path


def _compile(src: str, obj: str, deps) -> str:
    if os.path.exists(obj) and os.path.getmtime(obj) >= _newest([src] + deps):
        return obj
    inc = ["-I", os.path.join(ROOT, "include"), "-I", GEN, "-I", CSRC]
    if src.endswith(".cu"):
        cmd = [NVCC] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                               "--expt-relaxed-constexpr"] + inc + ["-c", src, "-o", obj]
    else:
        # host-only table data: nvcc drives the host compiler with the CUDA include path
        cmd = [NVCC, "-O1", "-std=c++17", "-Xcompiler", "-fPIC"] + inc + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    generate_tables(force)
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    deps = (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(ROOT, "include", "*.h"))
            + glob.glob(os.path.join(GEN, "*")))
    objs = []
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        futs = []
        for s in srcs:
            o = os.path.join(BUILD, os.path.basename(s) + ".o")
            objs.append(o)
            futs.append(ex.submit(_compile, s, o, deps))
        for f in futs:
            f.result()
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcudart_static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
