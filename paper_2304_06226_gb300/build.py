"""Build the native library libtp.so (CUDA for sm_103a) in-tree with nvcc.

The two translation units compile in parallel; the library is rebuilt only
when a source or header is newer than it."""
from __future__ import annotations

import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
LIB = PKG / "libtp.so"
OBJDIR = PKG / "_build"
# (source, object, extra flags): the transport kernels are compiled once per
# precision so that the halves build in parallel
# The transport kernels are compiled once per (precision, kernel family) so
# that the units build in parallel; the FP32 transport takes the hardware's
# division and square root (within 2 ulp) instead of the IEEE-rounded
# sequences: shorter code in the hot loop, far below the FP32 path's own
# geometric rounding.  FP64 keeps IEEE rounding (its histories match the FP64
# oracle to 1e-9).
_F32 = ["-DTP_BUILD_F32", "-prec-div=false", "-prec-sqrt=false"]
UNITS = ([("tp_transport.cu", f"tp_transport_f32_k{k}.o", _F32 + [f"-DTP_BUILD_KERNEL={k}"]) for k in (1, 2, 3)]
         + [("tp_transport.cu", f"tp_transport_f64_k{k}.o", ["-DTP_BUILD_F64", f"-DTP_BUILD_KERNEL={k}"])
            for k in (1, 2, 3)]
         + [("tp_transport.cu", "tp_transport_common.o", ["-DTP_BUILD_COMMON"]),
            ("tp_api.cu", "tp_api.o", []),
            ("tp_peaks.cu", "tp_peaks.o", [])])
SOURCES = sorted({u[0] for u in UNITS})
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtp.so")


def _stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = ([CSRC / f for f in SOURCES] + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h"))
            + [Path(__file__)])
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and not _stale():
        return LIB
    OBJDIR.mkdir(exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}"]
    if verbose:
        flags += ["-Xptxas", "-v"]
    procs = []
    objs = []
    for src, objname, extra in UNITS:
        obj = OBJDIR / objname
        objs.append(obj)
        procs.append((src, subprocess.Popen([nvcc(), *flags, *extra, "-c", str(CSRC / src), "-o", str(obj)],
                                            stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{out}")
        if verbose and out:
            print(out)
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp.so")
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart"],
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
