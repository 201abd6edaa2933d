"""Build step of libdgswe: exact reference tables, then nvcc for sm_103a.

    python -m paper_1904_08684_gb300.build        (or build_library() from Python)

Writes ``_build/dg_ref_tables.h`` (gen_tables.py) and links
``_build/libdgswe.so`` from the translation units in ``csrc/``, compiled in
parallel.  Rebuilds only when a source is newer than the library.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, "libdgswe.so")

UNITS = ["dg_fp64.cu", "dg_fp64_gen.cu", "dg_fp32p64.cu", "dg_fp32p64_gen.cu", "dg_fp32p32.cu",
         "dg_fp32p32_gen.cu", "dgswe_api.cu", "dg_project.cu", "dg_noalloc.cu", "dg_batch_fp64.cu",
         "dg_batch_fp32p64.cu", "dg_batch_fp32p32.cu", "dg_batch_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"] + ARCH


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    out = [os.path.join(CSRC, u) for u in UNITS]
    out += [os.path.join(CSRC, f) for f in ("dg_kernels.cuh", "dg_launch.cuh", "dg_batch.cuh", "gen_tables.py")]
    out.append(os.path.join(INCLUDE, "dgswe.h"))
    return out


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _compile(unit):
    src = os.path.join(CSRC, unit)
    obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
    cmd = [_nvcc()] + NVCC_FLAGS + ["-I" + BUILD, "-I" + INCLUDE, "-I" + CSRC, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    with open(obj + ".log", "w") as f:
        f.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s" % (unit, res.stderr[-4000:]))
    return obj


def build_library(force=False, verbose=False):
    """Compile libdgswe.so for sm_103a if missing or stale; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    subprocess.check_call([sys.executable, os.path.join(CSRC, "gen_tables.py"),
                           os.path.join(BUILD, "dg_ref_tables.h")],
                          stdout=subprocess.DEVNULL)
    workers = max(1, min(len(UNITS), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(_compile, UNITS))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose=True)
