"""Compile the CUDA sources in csrc/ into the in-tree shared library libamrhydro.so
(sm_103a only).  Objects go to csrc/_build/; translation units compile in parallel."""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libamrhydro.so")
SOURCES = ["octree.cu", "godunov_fp64.cu", "godunov_fp32.cu", "level_ops.cu", "mlp.cu", "ppcg.cu", "refine.cu",
           "diagnostics.cu", "mlp_tc.cu"]
# per-file extra flags: the FP32 kernels use fast single-precision division / square root
EXTRA = {"godunov_fp32.cu": ["--use_fast_math"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + os.path.join(HERE, "..", "include")]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libamrhydro.so")
    return exe


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    inc = os.path.join(HERE, "..", "include")
    files += [os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h")]
    return max(os.path.getmtime(f) for f in files)


def _code_only(text):
    """Source text without comments and blank space (a change of comments leaves the
    compiled kernel, and so its profiler counters, unchanged)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_hash():
    """Hash of the code the z-column update kernels (the benchmark's dominant kernel) are
    compiled from, comments excluded: ties their recorded profiler counters to a kernel
    version."""
    import hashlib
    h = hashlib.sha256()
    for f in ("common.cuh", "godunov_col.cuh", "godunov_pen.cuh", "hydro_math.cuh"):
        h.update(_code_only(open(os.path.join(CSRC, f)).read()).encode())
    return h.hexdigest()[:16]


def library_hash():
    """Hash of the code of every kernel source of the library (comments excluded): the
    version stamp the profile summaries of the other kernels carry."""
    import hashlib
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            h.update(_code_only(open(os.path.join(CSRC, f)).read()).encode())
    return h.hexdigest()[:16]


def build(force=False, verbose=False):
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= _deps():
        return OUT
    bdir = os.path.join(CSRC, "_build")
    os.makedirs(bdir, exist_ok=True)
    exe = nvcc()

    def one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [exe] + ARCH + FLAGS + EXTRA.get(src, []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
