"""Build libbcf.so in-tree with nvcc for sm_103a (B300).

Each .cu under csrc/ is compiled to an object in parallel, then linked into
``paper_1507_01391_b300/libbcf.so``.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libbcf.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbcf")


def _deps_mtime(src: str) -> float:
    hdrs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    hdrs += glob.glob(os.path.join(INCLUDE, "*.h"))
    return max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in hdrs])


def _compile(src: str, extra: list[str], out_dir: str = BUILD) -> str:
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= _deps_mtime(src):
        return obj
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), res.stderr))
    os.replace(obj + ".tmp", obj)
    return obj


TRACE_LIB = os.path.join(PKG, "libbcf_trace.so")


def _link(objs: list[str], lib: str) -> None:
    if (not os.path.exists(lib)) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        cmd = [nvcc(), *ARCH, "-shared", "-o", lib + ".tmp", *objs, "-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), res.stderr))
        os.replace(lib + ".tmp", lib)


def build(verbose: bool = False, extra: list[str] | None = None, trace: bool = True) -> str:
    """Compile every CUDA source and link libbcf.so (and the trace build
    libbcf_trace.so, the same sources with -DBCF_TRACE); returns libbcf.so's path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = list(extra or [])
    trace_only = ("trace_abi.cu", "bank_probe.cu")  # entry points of the trace build alone
    jobs = [(s, extra, BUILD) for s in srcs if os.path.basename(s) not in trace_only]
    if trace:
        os.makedirs(os.path.join(BUILD, "trace"), exist_ok=True)
        jobs += [(s, extra + ["-DBCF_TRACE"], os.path.join(BUILD, "trace")) for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    _link([o for o in objs if os.path.dirname(o) == BUILD], LIB)
    if trace:
        _link([o for o in objs if os.path.dirname(o) != BUILD], TRACE_LIB)
    if verbose:
        print("built", LIB, "and", TRACE_LIB if trace else "")
    return LIB


if __name__ == "__main__":
    build(verbose=True)
