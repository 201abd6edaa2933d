"""Arithmetic and memory traffic of one RK stage per element (roofline model).

Counts follow the kernel's formulation exactly: every nonzero entry of the
exact reference tensors costs one fused multiply-add (2 flops); additions,
multiplications, divisions and square roots count 1 flop each.  The tensor
nonzero patterns come from the same exact tables the build generates.

The minimal HBM traffic of a stage is the algorithmic byte count of the
fused path: read the state (3K) and the RK base state (3K, stages 2..S),
read the bathymetry (K), write the new state (3K); everything else (velocity,
fluxes, traces) could in principle stay on chip.  The kernel also writes and
re-reads per-element volume integrals (3K) and edge side records
(3 x (6(p+1)+1)); that extra traffic is reported separately.
"""
import functools
import hashlib
import os
import sys

_CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")


@functools.lru_cache(maxsize=None)
def _tables(p):
    sys.path.insert(0, _CSRC)
    try:
        import gen_tables as gt
    finally:
        sys.path.pop(0)
    basis = gt.make_basis()
    leg = gt.shifted_legendre(gt.PMAX)
    K, P1, T, S, R, Lam, Lpt = gt.tables_for(p, basis, leg)
    return K, P1, T, S, R, Lam, Lpt


# Algorithmic work per element and RK stage used for the roofline: FP64 FMAs
# of the velocity solve and FMAs of everything else, counted from the tensor
# nonzeros (nnz T/2 + K^3/6 + 2K^2 for the solve; products, contractions,
# traces, fluxes and lifts for the rest).
ALGORITHMIC_FMA = {1: (28, 478), 2: (160, 1498), 3: (564, 4143), 4: (1588, 10344)}


def algorithmic_flops(p):
    """flops per element and stage (2 per FMA) of the reference count"""
    a, b = ALGORITHMIC_FMA[p]
    return 2 * (a + b)


# the files that define the stage and batch kernels' device code, their
# reference tables and their launch shapes (host-only API code excluded)
KERNEL_SOURCES = ("dg_aux_inst.cu", "dg_batch.cuh", "dg_batch_inst.cu", "dg_dispatch.cu", "dg_kernels.cuh",
                  "dg_launch.cuh", "dg_stage_inst.cu", "dg_tile.cuh", "dg_tile_inst.cu", "dg_batch_tile_inst.cu", "gen_tables.py")


def _code_only(name, text):
    """C/C++ source without its comments and blank-line or trailing-space
    differences (a comment edit changes no kernel); other files verbatim"""
    if not name.endswith((".cu", ".cuh", ".h")):
        return text
    out, i, n = [], 0, len(text)
    while i < n:
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif text[i] == '"':                       # string literal, kept whole
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(text[i])
            i += 1
    lines = [ln.rstrip() for ln in "".join(out).split("\n")]
    return "\n".join(ln for ln in lines if ln)


def source_hash(read=None):
    """hash of the kernel sources' code (comments ignored): measured traffic
    is valid only for it.  read(name) -> text overrides reading csrc/."""
    h = hashlib.sha1()
    for name in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(_CSRC, name), encoding="utf-8") as f:
                text = f.read()
        else:
            text = read(name)
        h.update((name + _code_only(name, text)).encode())
    return h.hexdigest()[:16]


def _nz(x):
    return x != 0.0


@functools.lru_cache(maxsize=None)
def stage_flops(p, mode="stage"):
    """flops per element of one stage kernel launch (mode 'stage': flux +
    lift + RK update + evaluation of the new state; 'eval': evaluation)."""
    K, P1, T, S, R, Lam, Lpt = _tables(p)
    K1 = p * (p + 1) // 2

    def tprod(nout, mlim):
        f = 0
        for n in range(nout):
            for i in range(K):
                c = sum(1 for m in range(mlim) if _nz(T[n][i][m]))
                if c:
                    f += 2 * c + 2
        return f

    ev = 0
    ev += K                                     # H = xi + hb
    # velocity solve: assembly of the lower triangle, LDL^T, two solves
    for j in range(K):
        for i in range(j, K):
            ev += 2 * sum(1 for n in range(K) if _nz(T[n][i][j]))
        ev += 3 * j + 1                          # W_k, d update, 1/d
        ev += (K - 1 - j) * (2 * j + 1)          # L_ij
    ev += 2 * (2 * K * (K - 1) + K)            # forward + diagonal + backward, 2 rhs
    ev += K                                     # xi + 2 hb
    ev += 5 * tprod(K1, K) + 2 * K1             # projected flux products
    ev += 2 * tprod(K, K1)                      # g xi grad h_b source
    for a in range(K):                          # volume rows, 3 fields
        ev += 3 * (2 * (sum(1 for i in range(K1) if _nz(S[0][a][i])) + sum(1 for i in range(K1) if _nz(S[1][a][i])))
                   + 3) + 4
    nnzlam = sum(1 for j in range(P1) for a in range(P1) for b in range(P1) if _nz(Lam[j][a][b]))
    rowslam = sum(1 for j in range(P1) for a in range(P1) if any(_nz(Lam[j][a][b]) for b in range(P1)))
    nnzpt = [sum(1 for j in range(P1) if _nz(Lpt[k][j])) for k in range(3)]
    for n in range(3):                          # side records
        nnzr = sum(1 for j in range(P1) for i in range(K) if _nz(R[n][j][i]))
        ev += 2 * 5 * nnzr                      # 5 traces
        ev += P1 * (3 + 3 + 2 + 1)              # u.n, q.n, xi + 2 hb, H
        ev += 3 * (2 * nnzlam + 2 * rowslam)    # 3 edge products
        ev += 2 + P1 * (1 + 3 + 3)              # scaled record entries
        ev += 2 * 2 * sum(nnzpt) + 3 * 4 + 2    # wave speed at 3 points
    if mode == "eval":
        return ev
    up = 0
    for n in range(3):
        nnzr = sum(1 for j in range(P1) for i in range(K) if _nz(R[n][j][i]))
        up += 2 + 3 * P1 * 4 + 3 * 2 * nnzr     # flux + lift
    up += 3 * K * 5 + 2                         # RK update (stages with a base state)
    return up + ev


def stage_bytes(p, word_bytes, with_base=True):
    """minimal (algorithmic) HBM bytes per element and stage"""
    K = (p + 1) * (p + 2) // 2
    words = 3 * K + K + 3 * K + (3 * K if with_base else 0)
    return words * word_bytes


def stage_bytes_avg(p, word_bytes, rk_order):
    """algorithmic HBM bytes per element and stage, averaged over the stages
    of one SSP-RK step (the first stage reads no RK base state)"""
    S = rk_order
    return (stage_bytes(p, word_bytes, False) + (S - 1) * stage_bytes(p, word_bytes, True)) / S


def stage_bytes_kernel(p, word_bytes, with_base=True):
    """bytes per element and stage the stage kernel moves by design (own and
    neighbour side records, volume integrals, static bathymetry fields)"""
    K = (p + 1) * (p + 2) // 2
    P1 = p + 1
    K1 = p * (p + 1) // 2
    nrec = 6 * P1 + 1
    reads = 3 * K + (3 * K if with_base else 0) + 3 * K + 2 * 3 * nrec + K + 3 * P1 + 2 * K1
    writes = 3 * K + 3 * K + 3 * nrec
    return (reads + writes) * word_bytes
