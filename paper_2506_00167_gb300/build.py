"""Build the in-tree C-ABI library ``libldpcgb.so`` for sm_103a with nvcc.

Each CUDA translation unit compiles in parallel to an object under
``_build/``, then one link step makes the shared library next to this file.
No CMake; a rebuild is skipped when every object is newer than its sources.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libldpcgb.so")
LIB_CHECKED = os.path.join(HERE, "libldpcgb_checked.so")

SOURCES = ["session.cu", "decode.cu", "decode_cluster.cu", "demap.cu", "crc.cu", "noalloc.cu", "serve.cu",
           "policy.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libldpcgb")


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hdrs + [os.path.join(INCLUDE, "ldpcgb.h"), os.path.abspath(__file__)]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags=None) -> str:
    """Compile (if needed) and return the path of libldpcgb.so.  With LDPCGB_CHECKED=1 in the
    environment the kernels are built with their index checks (-DLDPC_CHECKED, see ldpc_check_log);
    the objects then go to a separate build folder."""
    nvcc = _nvcc()
    checked = os.environ.get("LDPCGB_CHECKED") == "1"
    build_dir = BUILD + ("_checked" if checked else "")
    os.makedirs(build_dir, exist_ok=True)
    common = _deps()
    flags = FLAGS + list(extra_flags or []) + (["-DLDPC_CHECKED"] if checked else [])
    jobs = []
    objs = []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        if _stale(obj, [sp] + common):
            jobs.append([nvcc, *ARCH, *flags, "-c", sp, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4) or 1) as ex:
        list(ex.map(run, jobs))
    lib = LIB_CHECKED if checked else LIB
    if jobs or _stale(lib, objs):
        run([nvcc, *ARCH, "-shared", "-o", lib, *objs, "-lcudart"])
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
