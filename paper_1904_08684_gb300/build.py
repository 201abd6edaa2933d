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
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, "libdgswe.so")

# Stage kernels are compiled once per (arithmetic, feature set, order) and the
# batched kernel once per (arithmetic, mode), so that the build is many small
# compilations run in parallel rather than a few long ones.
#   suffix: (state type, velocity-solve type, highest order)
ARITHS = {"fp64": ("double", "double", 4), "fp32p64": ("float", "double", 4),
          "fp32p32": ("float", "float", 4), "fp32pdf": ("float", "df64", 3),
          "fp32pir": ("float", "MixedIR", 4)}
PLAIN_UNITS = ["dgswe_api.cu", "dg_project.cu", "dg_noalloc.cu", "dg_batch_api.cu", "dg_dispatch.cu"]


def _units():
    """(source, object name, -D definitions) of every compilation."""
    out = [(u, u.replace(".cu", ".o"), []) for u in PLAIN_UNITS]
    for sfx, (real, preal, pmax) in ARITHS.items():
        base = ["-DDG_SUFFIX=" + sfx, "-DDG_REAL=" + real, "-DDG_PREAL=" + preal]
        for p in range(0, pmax + 1):
            out.append(("dg_aux_inst.cu", "aux_%s_p%d.o" % (sfx, p), base + ["-DDG_P=%d" % p]))
        for mode in (0, 1):
            out.append(("dg_batch_inst.cu", "batch_%s_m%d.o" % (sfx, mode), base + ["-DDG_MODE=%d" % mode]))
        if real == "float":
            # tile-fused stage kernels (FP32 state, uniform meshes)
            for p in range(0, pmax + 1):
                out.append(("dg_tile_inst.cu", "tile_%s_p%d.o" % (sfx, p), base + ["-DDG_P=%d" % p]))
            for p in (1, 2, 3):
                out.append(("dg_batch_tile_inst.cu", "batch_tile_%s_p%d.o" % (sfx, p), base + ["-DDG_P=%d" % p]))
        # the general-mesh feature set is not built for the double-float solve
        for feat in ((0, 1) if sfx not in ("fp32pdf", "fp32pir") else (0,)):
            name = sfx + ("_gen" if feat else "")
            for p in range(0, pmax + 1):
                out.append(("dg_stage_inst.cu", "stage_%s_p%d.o" % (name, p),
                            ["-DDG_SUFFIX=" + name, "-DDG_REAL=" + real, "-DDG_PREAL=" + preal,
                             "-DDG_FEAT=%d" % feat, "-DDG_P=%d" % p]))
    return out


SOURCES = sorted({u for u, _, _ in _units()})


def _cost(job):
    """Rough compile-time rank, so that the longest compilations start first."""
    unit, _, defs = job
    order = max([int(d.split("=")[1]) for d in defs if d.startswith("-DDG_P=")] or [0])
    return {"dg_stage_inst.cu": 10, "dg_batch_inst.cu": 12, "dg_aux_inst.cu": 9,
            "dg_tile_inst.cu": 11, "dg_batch_tile_inst.cu": 12}.get(unit, 0) + order + \
        2 * ("-DDG_PREAL=df64" in defs)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"] + ARCH


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    return [os.path.join(CSRC, u) for u in SOURCES] + _headers()


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _headers():
    return [os.path.join(CSRC, f) for f in ("dg_kernels.cuh", "dg_launch.cuh", "dg_batch.cuh", "dg_tile.cuh", "dg_nvtx.h",
                                             "gen_tables.py")] + \
        [os.path.join(INCLUDE, "dgswe.h")]


def _compile(job, force=False):
    unit, objname, defs = job
    src = os.path.join(CSRC, unit)
    obj = os.path.join(BUILD, objname)
    if not force and os.path.exists(obj):
        t = os.path.getmtime(obj)
        if all(os.path.getmtime(d) <= t for d in [src] + _headers()):
            return obj
    cmd = [_nvcc()] + NVCC_FLAGS + defs + ["-I" + BUILD, "-I" + INCLUDE, "-I" + CSRC, "-c", src, "-o", obj]
    t0 = time.time()
    res = subprocess.run(cmd, capture_output=True, text=True)
    with open(obj + ".log", "w") as f:
        f.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
        f.write("compile seconds: %.1f\n" % (time.time() - t0))
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
    jobs = sorted(_units(), key=_cost, reverse=True)
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(lambda j: _compile(j, force), jobs))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose=True)
