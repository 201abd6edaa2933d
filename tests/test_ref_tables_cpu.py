"""The reference tensors the CUDA kernels are compiled from
(``csrc/gen_tables.py``, exact rational arithmetic) against their
definitions, recomputed here by Gauss quadrature from the oracle's own basis
(pinned separately against the basis printed in §2.2).

  T[n][i][m]   = int phi^_n phi^_i phi^_m          (triple products, §2.2)
  S[r][a][i]   = int d_r phi^_a phi^_i             (stiffness, Eq. (15))
  R[e][j][i]   = int_0^1 phi^_i(gamma^_e(s)) L_j(s) ds   (edge restriction)
  Lam[j][a][b] = int_0^1 L_j L_a L_b ds            (1D product projection)
  Lpt[k][j]    = L_j(s_k), s = 0, 1/2, 1           (wave-speed points)

on the reference triangle x, y >= 0, x + y <= 1 with counter-clockwise edges
gamma^_0(s) = (1-s, s), gamma^_1(s) = (0, 1-s), gamma^_2(s) = (s, 0) and the
orthonormal Legendre polynomials L_j(s) = sqrt(2j+1) P_j(2s-1) on [0, 1].
Every integrand is a polynomial, so a Gauss rule of enough points is exact
up to rounding.
"""
import os
import re
import subprocess
import sys

import numpy as np
import pytest
from numpy.polynomial import legendre

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEN = os.path.join(ROOT, "paper_1904_08684_gb300", "csrc", "gen_tables.py")
# p <= 3: the printed basis, exact in both; p = 4: the oracle completes the
# basis by Gram-Schmidt in floating point (coefficients up to ~2.5e3, about
# 1e-13 relative rounding), the generator in rational arithmetic
TOL = {0: 2e-14, 1: 2e-14, 2: 2e-14, 3: 2e-14, 4: 1e-12}


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("tables") / "dg_ref_tables.h")
    subprocess.check_call([sys.executable, GEN, out], stdout=subprocess.DEVNULL)
    src = open(out).read()
    res = {}
    for m in re.finditer(r"struct RefTables<(\d)> \{(.*?)\n\};", src, flags=re.S):
        p, body = int(m.group(1)), m.group(2)
        arrs = {}
        for a in re.finditer(r"static constexpr double (\w+)((?:\[\d+\])+) = (\{.*?\});", body, flags=re.S):
            dims = [int(d) for d in re.findall(r"\[(\d+)\]", a.group(2))]
            vals = np.array([float(v) for v in re.findall(r"[-+0-9.eE]+", a.group(3))])
            arrs[a.group(1)] = vals.reshape(dims)
        res[p] = arrs
    m = re.search(r"struct BasisMonomials \{\s*static constexpr double c\[15\]\[5\]\[5\] = (\{.*?\});", src,
                  flags=re.S)
    res["monomials"] = np.array([float(v) for v in re.findall(r"[-+0-9.eE]+", m.group(1))]).reshape(15, 5, 5)
    assert sorted(k for k in res if k != "monomials") == [0, 1, 2, 3, 4]
    return res


@pytest.fixture(scope="module")
def basis(oracle_mod):
    """monomial coefficients c[i][a][b] of phi^_i = sum c x^a y^b (oracle)"""
    return oracle_mod.Oracle(2, 2, 4).basis_table()


def _eval(c, x, y, dx=0, dy=0):
    """phi^_i (or a derivative) at points x, y for every i: (K, npts)"""
    out = np.zeros((c.shape[0],) + np.shape(x))
    for a in range(5):
        for b in range(5 - a):
            if a < dx or b < dy:
                continue
            f = np.prod(np.arange(a - dx + 1, a + 1)) * np.prod(np.arange(b - dy + 1, b + 1))
            out += c[:, a, b][:, None] * f * x ** (a - dx) * y ** (b - dy)
    return out


def _gauss01(n):
    z, w = legendre.leggauss(n)
    return 0.5 * (z + 1.0), 0.5 * w


def _triangle_rule(n=12):
    """collapsed (Duffy) Gauss rule: x = u, y = (1 - u) v, weight (1 - u)"""
    s, w = _gauss01(n)
    u, v = np.meshgrid(s, s, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    return u.ravel(), ((1.0 - u) * v).ravel(), (wu * wv * (1.0 - u)).ravel()


def _L(j, s):
    coef = np.zeros(j + 1)
    coef[j] = 1.0
    return np.sqrt(2 * j + 1) * legendre.legval(2.0 * s - 1.0, coef)


def _K(p):
    return (p + 1) * (p + 2) // 2


def test_monomial_table_is_the_pinned_basis(tables, basis):
    c = tables["monomials"]
    scale = np.abs(c).reshape(15, -1).max(axis=1)
    err = np.abs(c - basis).reshape(15, -1).max(axis=1) / scale
    assert err[:10].max() <= 1e-15      # printed functions (p <= 3)
    assert err[10:].max() <= 1e-14      # degree-4 completion


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_triple_products_and_stiffness(tables, basis, p):
    K = _K(p)
    x, y, w = _triangle_rule()
    phi = _eval(basis[:K], x, y)
    T = np.einsum("nq,iq,mq,q->nim", phi, phi, phi, w)
    S = np.stack([np.einsum("aq,iq,q->ai", _eval(basis[:K], x, y, dx=1 - r, dy=r), phi, w) for r in (0, 1)])
    assert np.abs(tables[p]["T"] - T).max() <= TOL[p]
    assert np.abs(tables[p]["S"] - S).max() <= 4 * TOL[p]
    # sanity of the definitions themselves: T[0] = phi^_0 I (constant phi^_0)
    assert np.allclose(tables[p]["T"][0], np.sqrt(2.0) * np.eye(K), atol=2e-14)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_edge_restriction_and_edge_products(tables, basis, p):
    K, P1 = _K(p), p + 1
    s, w = _gauss01(12)
    gamma = [(1.0 - s, s), (np.zeros_like(s), 1.0 - s), (s, np.zeros_like(s))]
    L = np.stack([_L(j, s) for j in range(P1)])
    R = np.stack([np.einsum("jq,iq,q->ji", L, _eval(basis[:K], gx, gy), w) for gx, gy in gamma])
    Lam = np.einsum("jq,aq,bq,q->jab", L, L, L, w)
    Lpt = np.stack([[_L(j, np.array(sk)) for j in range(P1)] for sk in (0.0, 0.5, 1.0)])
    assert np.abs(tables[p]["R"] - R).max() <= TOL[p]
    assert np.abs(tables[p]["Lam"] - Lam).max() <= 2e-14
    assert np.abs(tables[p]["Lpt"] - Lpt).max() <= 2e-14
    # the restriction reproduces traces: a basis function's edge values are
    # recovered from its Legendre coefficients when its trace has degree <= p
    for (gx, gy), Re in zip(gamma, tables[p]["R"]):
        assert np.abs(Re.T @ L - _eval(basis[:K], gx, gy)).max() <= 50 * TOL[p]


def test_roofline_counts_follow_the_tables(tables):
    """bench.py's algorithmic FMA counts: the velocity solve is
    nnz(T)/2 (assembly of A^H) + K^3/6 (LDL^T) + 2K^2 (two solves), and the
    rest covers at least the five projected products (5 nnz T) and the
    volume contraction (3 nnz S)"""
    from paper_1904_08684_gb300 import flops as FL
    for p in (1, 2, 3, 4):
        K = _K(p)
        nnzT = int(np.count_nonzero(tables[p]["T"]))
        nnzS = int(np.count_nonzero(tables[p]["S"]))
        solve, rest = FL.ALGORITHMIC_FMA[p]
        assert solve == round(nnzT / 2 + K ** 3 / 6 + 2 * K * K)
        assert rest >= 5 * nnzT + 3 * nnzS
        assert FL.algorithmic_flops(p) == 2 * (solve + rest)
