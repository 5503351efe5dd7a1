"""Builds libamg.so (this package) and libsynth.so (the input generator) for sm_103a.

Each .cu file is compiled on its own nvcc process, in parallel, into
``_build/`` at the repository root; the objects are then linked into a
shared library next to the Python module that loads it.  The CUDA runtime is
linked statically, so the libraries need nothing but the driver at run time.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1512_04506_gb300")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _compile(src, obj, extra):
    cmd = [_nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return r.stderr


def _library(name, sources, out, extra=(), verbose=False):
    bdir = os.path.join(ROOT, "_build", name)
    os.makedirs(bdir, exist_ok=True)
    objs = [os.path.join(bdir, os.path.basename(s).replace(".cu", ".o")) for s in sources]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(sources), os.cpu_count() or 4))) as ex:
        futs = [ex.submit(_compile, s, o, list(extra)) for s, o in zip(sources, objs)]
        for f in futs:
            msg = f.result()
            if verbose and msg:
                print(msg)
    tmp = out + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed for %s:\n%s\n%s" % (name, r.stdout, r.stderr))
    os.replace(tmp, out)
    return out


def build(verbose=False, ptxas_info=False):
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    amg_src = sorted(glob.glob(os.path.join(PKG, "csrc", "*.cu")))
    synth_src = sorted(glob.glob(os.path.join(ROOT, "synth", "csrc", "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(_library, "amg", amg_src, os.path.join(PKG, "libamg.so"), extra, verbose or ptxas_info)
        b = ex.submit(_library, "synth", synth_src, os.path.join(ROOT, "synth", "libsynth.so"), extra,
                      verbose or ptxas_info)
        return a.result(), b.result()


if __name__ == "__main__":
    import sys
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
