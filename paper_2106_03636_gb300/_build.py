"""In-tree build of the native parts of the package.

* ``libo2gen.so``  - the seeded Time-Frame generator (plain C, host only).
* ``libo2tpc.so``  - the tracker: sm_103a CUDA kernels behind the C-ABI
  declared in ``include/o2tpc.h``.

Everything is compiled with explicit ``gcc``/``nvcc`` command lines (no cmake,
no torch extension machinery), in parallel, into ``paper_2106_03636_gb300/_lib``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "_lib")
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")

GEN_SO = os.path.join(LIB, "libo2gen.so")
TPC_SO = os.path.join(LIB, "libo2tpc.so")

CUDA_SOURCES = [
    "o2tpc_capi.cu",
    "k_bin.cu",
    "k_ca.cu",
    "k_track.cu",
    "k_merge.cu",
    "k_cont.cu",
    "k_ctf.cu",
    "k_clu.cu",
    "o2tpc_ctf_host.cu",
    "o2tpc_static.cu",
    "o2tpc_graph.cu",
]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# Per-file flags: the FP32 Kalman kernels use the approximate (MUFU-based)
# division and square root and flush denormals; their results stay far
# inside the single-precision parity tolerances.
FILE_FLAGS = {
    "k_track.cu": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
    "k_merge.cu": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
    "k_cont.cu": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libo2tpc.so")


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def build_gen(force: bool = False) -> str:
    os.makedirs(LIB, exist_ok=True)
    src = os.path.join(PKG, "synth", "o2gen.c")
    dig = os.path.join(PKG, "synth", "o2digits.c")
    if force or _stale(GEN_SO, [src, dig]):
        _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
              "-o", GEN_SO + ".tmp", src, dig, "-lm"])
        os.replace(GEN_SO + ".tmp", GEN_SO)
    return GEN_SO


def build_tpc(force: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(LIB, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in CUDA_SOURCES]
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "o2tpc.h"))
    if not (force or _stale(TPC_SO, srcs + headers)):
        return TPC_SO
    nvcc = _nvcc()
    objdir = os.path.join(LIB, "obj")
    os.makedirs(objdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                    "--expt-relaxed-constexpr", "-rdc=false"] + (extra or [])

    def one(s: str) -> str:
        obj = os.path.join(objdir, os.path.basename(s) + ".o")
        _run([nvcc] + flags + FILE_FLAGS.get(os.path.basename(s), []) + ["-c", s, "-o", obj])
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(one, srcs))
    _run([nvcc] + ARCH + ["-shared", "-o", TPC_SO + ".tmp"] + objs + ["-lcudart"])
    os.replace(TPC_SO + ".tmp", TPC_SO)
    return TPC_SO


def build_all(force: bool = False) -> None:
    build_gen(force)
    build_tpc(force)
