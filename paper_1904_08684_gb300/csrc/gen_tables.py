"""Build step: exact reference tensors of the quadrature-free DG scheme.

The paper evaluates every element and edge integral of basis-function
products analytically with sympy (§2.3, Listing 1).  Here the same integrals
are computed once, exactly, in rational arithmetic: each reference basis
function is phi^_i = R_i * sqrt(sigma_i) with a rational polynomial R_i and a
rational sigma_i, so every tensor entry is (rational) * sqrt(rational) and is
rounded to the nearest double only at the end (60 significant digits).

Written to ``dg_ref_tables.h`` (C++17 constexpr tables, one struct per order
p = 1..4):

  T[n][i][m]   = int_T^ phi^_n phi^_i phi^_m             (§2.2, Eq. (16) kernels)
  S[r][a][i]   = int_T^ d_r phi^_a phi^_i                (§2.2, Eq. (15))
  R[e][j][i]   = int_0^1 phi^_i(gamma^_e(s)) L_j(s) ds    edge restriction
  Lam[j][a][b] = int_0^1 L_j L_a L_b ds                   1D product projection
  Lpt[k][j]    = L_j(s_k), s = 0, 1/2, 1                  wave-speed points
  phi4         = the degree-4 functions (for the set-up projection)

with the reference triangle {x, y >= 0, x + y <= 1}, edges gamma^_0(s) =
(1-s, s), gamma^_1(s) = (0, 1-s), gamma^_2(s) = (s, 0) (counter-clockwise,
edge e opposite vertex e) and L_j(s) = sqrt(2j+1) P_j(2s-1) orthonormal on
[0, 1].  The basis is the one printed in §2.2 for orders 0..3; order 4
continues it by Gram-Schmidt of x^4, x^3 y, x^2 y^2, x y^3, y^4.

Usage: python gen_tables.py OUT_HEADER
"""
import math
import sys
from decimal import Decimal, getcontext
from fractions import Fraction as Fr

getcontext().prec = 60
PMAX = 4


# -- bivariate polynomials: {(a, b): Fraction} for x^a y^b ------------------
def padd(p, q, s=Fr(1)):
    r = dict(p)
    for k, v in q.items():
        r[k] = r.get(k, Fr(0)) + s * v
    return {k: v for k, v in r.items() if v != 0}


def pmul(p, q):
    r = {}
    for (a, b), u in p.items():
        for (c, d), v in q.items():
            k = (a + c, b + d)
            r[k] = r.get(k, Fr(0)) + u * v
    return {k: v for k, v in r.items() if v != 0}


def pdiff(p, r):
    out = {}
    for (a, b), v in p.items():
        if r == 0 and a > 0:
            out[(a - 1, b)] = out.get((a - 1, b), Fr(0)) + a * v
        if r == 1 and b > 0:
            out[(a, b - 1)] = out.get((a, b - 1), Fr(0)) + b * v
    return out


def tri_integral(p):
    """exact integral over the reference triangle: x^a y^b -> a! b! / (a+b+2)!"""
    return sum((v * Fr(math.factorial(a) * math.factorial(b), math.factorial(a + b + 2))
                for (a, b), v in p.items()), Fr(0))


def poly(*terms):
    """poly((c, a, b), ...) = sum c x^a y^b"""
    out = {}
    for c, a, b in terms:
        out[(a, b)] = out.get((a, b), Fr(0)) + Fr(c)
    return out


# -- the printed basis (§2.2): phi^_i = sqrt(sigma_i) * R_i -----------------
PRINTED = [
    (2, poly((1, 0, 0))),
    (1, poly((2, 0, 0), (-6, 1, 0))),
    (12, poly((1, 0, 0), (-1, 1, 0), (-2, 0, 1))),
    (6, poly((1, 0, 0), (-8, 1, 0), (10, 2, 0))),
    (3, poly((-1, 0, 0), (-4, 1, 0), (5, 2, 0), (12, 0, 1), (-15, 0, 2))),
    (45, poly((1, 0, 0), (-4, 1, 0), (3, 2, 0), (-4, 0, 1), (8, 1, 1), (3, 0, 2))),
    (8, poly((-1, 0, 0), (15, 1, 0), (-45, 2, 0), (35, 3, 0))),
    (24, poly((-1, 0, 0), (13, 1, 0), (-33, 2, 0), (21, 3, 0), (2, 0, 1), (-24, 1, 1), (42, 2, 1))),
    (40, poly((-1, 0, 0), (9, 1, 0), (-15, 2, 0), (7, 3, 0), (6, 0, 1), (-48, 1, 1), (42, 2, 1),
              (-6, 0, 2), (42, 1, 2))),
    (56, poly((-1, 0, 0), (3, 1, 0), (-3, 2, 0), (1, 3, 0), (12, 0, 1), (-24, 1, 1), (12, 2, 1),
              (-30, 0, 2), (30, 1, 2), (20, 0, 3))),
]


def make_basis():
    basis = [(Fr(s), R) for s, R in PRINTED]
    for k in range(5):                       # x^4, x^3 y, x^2 y^2, x y^3, y^4
        m = poly((1, 4 - k, k))
        r = dict(m)
        for sig, R in basis:
            r = padd(r, R, -sig * tri_integral(pmul(m, R)))
        rho = tri_integral(pmul(r, r))
        basis.append((1 / rho, r))
    return basis


# -- univariate (edge) polynomials: {k: Fraction} ---------------------------
def umul(p, q):
    r = {}
    for a, u in p.items():
        for b, v in q.items():
            r[a + b] = r.get(a + b, Fr(0)) + u * v
    return r


def uint01(p):
    return sum((v / (k + 1) for k, v in p.items()), Fr(0))


def upow_lin(c0, c1, n):
    """(c0 + c1 s)^n"""
    r = {0: Fr(1)}
    for _ in range(n):
        r = umul(r, {0: Fr(c0), 1: Fr(c1)})
    return r


def restrict(R, edge):
    """R(gamma^_edge(s)) as a polynomial in s"""
    xs = {0: (1, -1, 0, 1), 1: (0, 0, 1, -1), 2: (0, 1, 0, 0)}[edge]   # x = a + b s, y = c + d s
    out = {}
    for (a, b), v in R.items():
        t = umul(upow_lin(xs[0], xs[1], a), upow_lin(xs[2], xs[3], b))
        for k, w in t.items():
            out[k] = out.get(k, Fr(0)) + v * w
    return out


def shifted_legendre(nmax):
    """P_j(2s - 1), j = 0..nmax, by Bonnet's recurrence"""
    P = [{0: Fr(1)}, {0: Fr(-1), 1: Fr(2)}]
    for j in range(1, nmax):
        t = umul({0: Fr(-1), 1: Fr(2)}, P[j])
        nxt = {}
        for k, v in t.items():
            nxt[k] = nxt.get(k, Fr(0)) + Fr(2 * j + 1, j + 1) * v
        for k, v in P[j - 1].items():
            nxt[k] = nxt.get(k, Fr(0)) - Fr(j, j + 1) * v
        P.append(nxt)
    return P[:nmax + 1]


def uval(p, s):
    return sum((v * Fr(s) ** k for k, v in p.items()), Fr(0))


# -- exact value -> double ---------------------------------------------------
def rs(q, sig):
    """q * sqrt(sig), correctly rounded to double"""
    if q == 0 or sig == 0:
        return 0.0
    d = Decimal(q.numerator) / Decimal(q.denominator)
    s = (Decimal(sig.numerator) / Decimal(sig.denominator)).sqrt()
    return float(str(d * s))


def fmt(v):
    if v == 0.0:
        return "0.0"
    return repr(v)


def emit_array(name, arr, shape):
    def rec(a, depth):
        if depth == len(shape) - 1:
            return "{" + ", ".join(fmt(x) for x in a) + "}"
        return "{" + ",\n    ".join(rec(x, depth + 1) for x in a) + "}"
    dims = "".join("[%d]" % n for n in shape)
    return "  static constexpr double %s%s = %s;\n" % (name, dims, rec(arr, 0))


def tables_for(p, basis, leg):
    K = (p + 1) * (p + 2) // 2
    P1 = p + 1
    B = basis[:K]
    T = [[[rs(tri_integral(pmul(pmul(B[n][1], B[i][1]), B[m][1])), B[n][0] * B[i][0] * B[m][0])
           for m in range(K)] for i in range(K)] for n in range(K)]
    S = [[[rs(tri_integral(pmul(pdiff(B[a][1], r), B[i][1])), B[a][0] * B[i][0])
           for i in range(K)] for a in range(K)] for r in range(2)]
    R = [[[rs(uint01(umul(restrict(B[i][1], e), leg[j])), B[i][0] * (2 * j + 1))
           for i in range(K)] for j in range(P1)] for e in range(3)]
    Lam = [[[rs(uint01(umul(umul(leg[j], leg[a]), leg[b])), Fr((2 * j + 1) * (2 * a + 1) * (2 * b + 1)))
             for b in range(P1)] for a in range(P1)] for j in range(P1)]
    Lpt = [[rs(uval(leg[j], s), Fr(2 * j + 1)) for j in range(P1)] for s in (Fr(0), Fr(1, 2), Fr(1))]
    return K, P1, T, S, R, Lam, Lpt


def main(out):
    basis = make_basis()
    leg = shifted_legendre(PMAX)
    parts = ["// Generated by gen_tables.py (exact rational arithmetic); do not edit.\n",
             "#pragma once\n\nnamespace dgswe {\n\ntemplate <int P> struct RefTables;\n\n"]
    counts = []
    for p in range(0, PMAX + 1):
        K, P1, T, S, R, Lam, Lpt = tables_for(p, basis, leg)
        nnz = lambda a: sum(1 for x in _flat(a) if x != 0.0)  # noqa: E731
        counts.append((p, nnz(T), nnz(S[0]), nnz(S[1]), nnz(R), nnz(Lam)))
        parts.append("template <> struct RefTables<%d> {\n" % p)
        parts.append("  static constexpr int K = %d, P1 = %d;\n" % (K, P1))
        parts.append(emit_array("T", T, (K, K, K)))
        parts.append(emit_array("S", S, (2, K, K)))
        parts.append(emit_array("R", R, (3, P1, K)))
        parts.append(emit_array("Lam", Lam, (P1, P1, P1)))
        parts.append(emit_array("Lpt", Lpt, (3, P1)))
        parts.append("};\n\n")
    # monomial tables of the 15 basis functions (host-side set-up projection)
    mono = [[[0.0] * 5 for _ in range(5)] for _ in range(15)]
    for i, (sig, R) in enumerate(basis):
        for (a, b), v in R.items():
            mono[i][a][b] = rs(v, sig)
    parts.append("struct BasisMonomials {\n")
    parts.append(emit_array("c", mono, (15, 5, 5)))
    parts.append("};\n\n")
    parts.append("// nonzeros (p, T, S1, S2, R, Lam): %s\n" % (counts,))
    parts.append("}  // namespace dgswe\n")
    with open(out, "w") as f:
        f.write("".join(parts))
    return counts


def _flat(a):
    if isinstance(a, list):
        for x in a:
            yield from _flat(x)
    else:
        yield a


if __name__ == "__main__":
    print(main(sys.argv[1]))
