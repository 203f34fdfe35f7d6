"""Builds the in-tree shared library ``libgg.so`` for sm_103a.

Every translation unit is compiled in parallel with nvcc (one -gencode,
``arch=compute_103a,code=sm_103a``) and linked into
``paper_2511_10353_gb300/libgg.so`` next to this file. Objects go to
``paper_2511_10353_gb300/_build/``. Runs on x86_64 (cross-compiling, no GPU
needed) and on the aarch64 GPU hosts alike; no host-architecture flags.

    python -m paper_2511_10353_gb300.build [--force]
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = [
    "gg_ct_f32.cu",
    "gg_ct_z_f32.cu",
    "gg_ct_f64.cu",
    "gg_ct_z_f64.cu",
    "gg_axis_f32.cu",
    "gg_axis_f64.cu",
    "gg_kernels_f32.cu",
    "gg_kernels_f64.cu",
    "gg_kernels_common.cu",
    "gg_static.cu",
    "gg_persist.cu",
    "gg_cic.cu",
    "gg_refine.cu",
    "gg_merge.cu",
    "gg_stats.cu",
    "gg_api.cpp",
    "gg_cosmo.cpp",
]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgg.so")
    return path


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
            "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _compile(src):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + ARCH + _flags() + ["-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "c++")
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError("compiling %s failed:\n%s\n%s" % (src, " ".join(cmd), proc.stderr))
    return obj


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "gg.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=True):
    """Compile and link libgg.so if any source is newer than it. Returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError("linking libgg.so failed:\n%s" % proc.stderr)
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv)
