"""Build the sm_103a CUDA library ``liblbmfvm.so`` in place with nvcc.

Eight translation units compiled in parallel, one ``-gencode`` (compute_103a /
sm_103a), static CUDA runtime, so the library loads on a machine without a GPU driver (the driver
is only needed at the first CUDA call).
"""

from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "liblbmfvm.so")
SOURCES = [os.path.join(CSRC, f) for f in ("lbmfvm.cu", "step_f32.cu", "step_f16.cu", "step_f64.cu", "fv_modes.cu",
                                            "residual_noalloc.cu", "surrogate.cu", "conv_tc.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "kernels.cuh"), os.path.join(CSRC, "batch.inl"), os.path.join(CSRC, "checkpoint.inl"),
                  os.path.join(CSRC, "step_shapes.inl"), os.path.join(CSRC, "conv_tc.h"), os.path.join(INCLUDE, "lbmfvm.h"),
                  os.path.join(INCLUDE, "surrogate.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbmfvm.so")


FLAGS = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC"]


def command(out: str = LIB, verbose_ptxas: bool = False) -> list[str]:
    """One nvcc command that compiles and links every source (sequentially)."""
    cmd = [nvcc()] + FLAGS + ["-shared", "-I" + INCLUDE, "-o", out] + SOURCES
    if verbose_ptxas:
        cmd.insert(1, "-Xptxas=-v")
    return cmd


def _compile_parallel(out: str, verbose_ptxas: bool) -> None:
    """Each translation unit compiled by its own nvcc process, then linked."""
    import tempfile

    with tempfile.TemporaryDirectory(prefix="lbmfvm_build_") as tmp:
        objs, procs = [], []
        for src in SOURCES:
            obj = os.path.join(tmp, os.path.basename(src) + ".o")
            cmd = [nvcc()] + FLAGS + ["-I" + INCLUDE, "-c", src, "-o", obj]
            if verbose_ptxas:
                cmd.insert(1, "-Xptxas=-v")
            procs.append(subprocess.Popen(cmd, cwd=ROOT))
            objs.append(obj)
        failed = [p.args for p in procs if p.wait() != 0]
        if failed:
            raise subprocess.CalledProcessError(1, failed[0])
        subprocess.run([nvcc(), ARCH, "-shared", "-o", out] + objs, check=True, cwd=ROOT)


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile liblbmfvm.so if missing or older than its sources; return its path."""
    if force or stale():
        tmp = LIB + ".tmp"
        _compile_parallel(tmp, verbose_ptxas)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose_ptxas=True))
