"""Build libsph.so (CUDA for sm_103a) in-tree with nvcc.

Three translation units compile in parallel: the C ABI, the FP64 engine and the FP32
engine.  The library lands next to this file; a stamp of the sources and flags skips
rebuilds when nothing changed.
"""
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libsph.so")
UNITS = ["sph_capi.cu", "sph_f64.cu", "sph_f32.cu", "sph_static.cu", "sph_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler",
         "-fPIC,-ffp-contract=off", "-I" + os.path.join(ROOT, "include")]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _stamp():
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    with open(os.path.join(ROOT, "include", "sph.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def build(force=False, verbose=False, extra=(), variant=None):
    """Compile and link the library; returns its path.  ``variant``: a name for a build with
    ``extra`` compile flags (e.g. a lowered compile-time limit), kept apart from the in-tree
    library in ``_build/<variant>/libsph.so``."""
    bdir = os.path.join(BUILD, variant) if variant else BUILD
    lib = os.path.join(bdir, "libsph.so") if variant else LIB
    os.makedirs(bdir, exist_ok=True)
    stamp = _stamp() + ("|" + " ".join(extra) if extra else "")
    sfile = os.path.join(bdir, "libsph.stamp")
    if not force and os.path.exists(lib) and os.path.exists(sfile) and open(sfile).read() == stamp:
        return lib

    def compile_unit(u):
        obj = os.path.join(bdir, u.replace(".cu", ".o"))
        cmd = [nvcc()] + ARCH + FLAGS + list(extra) + ["-c", os.path.join(CSRC, u), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (u, " ".join(cmd), r.stderr[-6000:]))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr[-4000:])
    os.replace(tmp, lib)
    with open(sfile, "w") as f:
        f.write(stamp)
    return lib


if __name__ == "__main__":
    args = sys.argv[1:]
    extra = [a for a in args if a.startswith("-X") or a.startswith("--")] if "--ptxas" in args else []
    if "--ptxas" in args:
        extra = ["-Xptxas", "-v"]
    print(build(force="--force" in args, verbose="--ptxas" in args, extra=extra))
