"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics, independent of the oracle's own code paths.

Each test names what it pins and why a plausible mistake would fail it.
None of these tests needs a GPU.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1904_08684_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


# ---------------------------------------------------------------- inputs
def test_splitmix64_reference_outputs():
    """The seeded input generator reproduces SplitMix64's published outputs."""
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        ref = [int(t) for t in f.read().split("\n") if t.strip() and not t.startswith("#")]
    got = [int(v) for v in I.splitmix64(1234567, len(ref))]
    assert got == ref


# ---------------------------------------------------------------- basis
def test_basis_vertex_values(oracle_mod):
    """§2.2 printed basis: values at the three reference vertices."""
    o = oracle_mod.Oracle(2, 2, 3, bc="reflective")
    tab = o.basis_table()
    ref = _golden("basis_vertex_values.txt")
    for row in ref:
        i = int(row[0]) - 1
        for (x, y), val in zip(((0, 0), (1, 0), (0, 1)), row[1:]):
            got = sum(tab[i, a, b] * x ** a * y ** b for a in range(5) for b in range(5))
            assert abs(got - val) < 1e-13, (i + 1, x, y, got, val)


def _monomial_integral(a, b):
    """exact integral of x^a y^b over the reference triangle: a! b! / (a+b+2)!"""
    return Fraction(math.factorial(a) * math.factorial(b), math.factorial(a + b + 2))


@pytest.mark.parametrize("p", [3, 4])
def test_basis_orthonormal(oracle_mod, p):
    """Gram matrix of the oracle's basis, integrated with exact monomial
    integrals (not the oracle's quadrature), is the identity (§2.2 basis is
    orthonormal; the degree-4 completion must keep it so)."""
    o = oracle_mod.Oracle(2, 2, p, bc="reflective")
    tab = o.basis_table()
    K = tab.shape[0]
    mono = [[_monomial_integral(a, b) for b in range(9)] for a in range(9)]
    # exact rational arithmetic on the (exactly representable) coefficients
    coef = [[(a, b, Fraction(float(tab[i, a, b]))) for a in range(5) for b in range(5) if tab[i, a, b] != 0]
            for i in range(K)]
    G = np.zeros((K, K))
    for i in range(K):
        for j in range(i, K):
            acc = Fraction(0)
            for a, b, c in coef[i]:
                for a2, b2, c2 in coef[j]:
                    acc += c * c2 * mono[a + a2][b + b2]
            G[i, j] = G[j, i] = float(acc)
    assert np.abs(G - np.eye(K)).max() < 1e-12


# ---------------------------------------------------------------- mesh
def test_mesh_topology_is_geometric(oracle_mod):
    """Every interior edge is shared with its neighbour, traversed in the
    opposite direction; all triangles are counter-clockwise (det B > 0)."""
    for bc in ("periodic", "reflective"):
        o = oracle_mod.Oracle(5, 4, 1, bc=bc, Lx=2.0, Ly=1.5)
        verts, det, nb = o.geometry()
        assert (det > 0).all()
        for e in range(o.E):
            for n in range(3):
                f = nb[e, n]
                if f < 0:
                    assert bc == "reflective"
                    continue
                P, Q = verts[e, (n + 1) % 3], verts[e, (n + 2) % 3]
                # find the neighbour edge with the reversed endpoints, modulo
                # the periodic box
                found = False
                for m in range(3):
                    P2, Q2 = verts[f, (m + 1) % 3], verts[f, (m + 2) % 3]
                    d1 = np.mod(P - Q2 + [1.0, 0.75], [2.0, 1.5]) - [1.0, 0.75]
                    d2 = np.mod(Q - P2 + [1.0, 0.75], [2.0, 1.5]) - [1.0, 0.75]
                    if np.abs(d1).max() < 1e-12 and np.abs(d2).max() < 1e-12:
                        found = True
                        assert m == n
                assert found, (e, n, f)


# ---------------------------------------------------------------- projections
def _rand_poly(rng, deg):
    c = rng.standard_normal((deg + 1, deg + 1))

    def f(x, y):
        out = np.zeros(np.broadcast(x, y).shape)
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                out += c[a, b] * x ** a * y ** b
        return out
    return f


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_projection_reproduces_polynomials(oracle_mod, p):
    """L2 projection onto P^p is the identity on polynomials of degree <= p."""
    rng = np.random.default_rng(10 + p)
    o = oracle_mod.Oracle(3, 2, p, bc="reflective", Lx=1.3, Ly=0.7)
    f = _rand_poly(rng, p)
    c = o.project(f)
    verts, _, _ = o.geometry()
    for e in range(o.E):
        for _ in range(3):
            w = rng.dirichlet([1, 1, 1])
            x, y = w @ verts[e]
            assert abs(o.eval_point(c, e, x, y) - f(x, y)) < 1e-11 * (1 + abs(f(x, y)))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_u_projection_recovers_velocity(oracle_mod, p):
    """Eq. (12): for u, H in P^p and q := Pi_p(u H), the projection returns u."""
    rng = np.random.default_rng(20 + p)
    o = oracle_mod.Oracle(2, 2, p, bc="periodic")
    fu = _rand_poly(rng, p)
    fv = _rand_poly(rng, p)
    hb = o.project_hb(lambda x, y: 5.0 + x + 0.5 * y)
    xi = o.project(lambda x, y: 0.3 * np.sin(x + 2 * y) if p > 0 else 0.1)
    u_true = o.project(fu)
    v_true = o.project(fv)
    xy = o.proj_nodes()
    # evaluate the polynomial fields at the projection nodes via eval_point
    vals = {}
    for name, c in (("xi", xi), ("u", u_true), ("v", v_true)):
        vals[name] = np.array([[o.eval_point(c, e, *xy[e, q]) for q in range(xy.shape[1])]
                               for e in range(o.E)])
    hbv = 5.0 + xy[..., 0] + 0.5 * xy[..., 1]
    Hv = vals["xi"] + hbv
    U = _project_values(o, vals["u"] * Hv)
    V = _project_values(o, vals["v"] * Hv)
    u, v = o.project_u(hb, xi, U, V)
    assert np.abs(u - u_true).max() < 1e-11 * (1 + np.abs(u_true).max())
    assert np.abs(v - v_true).max() < 1e-11 * (1 + np.abs(v_true).max())


def _project_values(o, vals):
    """project point values given at o.proj_nodes() onto P^p"""
    import ctypes
    coef = np.zeros((o.E, o.K))
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    assert o.lib.or_project(o._h, vals.ctypes.data_as(dp), coef.ctypes.data_as(dp)) == 0
    return coef


# ---------------------------------------------------------------- p = 0 is FV
def _fv_rhs(nx, ny, Lx, Ly, bc, xi, U, V, hb, g):
    """Independent first-order finite-volume Rusanov (local Lax-Friedrichs)
    scheme on the same triangles: d mean/dt = -(1/area) sum_edges |E| F^."""
    def vid(i, j):
        if bc == "periodic":
            return (j % ny) * nx + (i % nx)
        return j * (nx + 1) + i

    def vxy(i, j):
        return np.array([Lx * i / nx, Ly * j / ny])
    tris, pts = [], []
    for j in range(ny):
        for i in range(nx):
            tris.append([(i, j), (i + 1, j), (i, j + 1)])
            tris.append([(i + 1, j + 1), (i, j + 1), (i + 1, j)])
    E = len(tris)
    edge_owner = {}
    for e, t in enumerate(tris):
        for k in range(3):
            a, b = t[k], t[(k + 1) % 3]
            edge_owner.setdefault(frozenset((vid(*a), vid(*b))), []).append(e)
    H = xi + hb
    u, v = U / H, V / H
    out = np.zeros((3, E))
    for e, t in enumerate(tris):
        P = [vxy(*q) for q in t]
        area = 0.5 * abs((P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]))
        acc = np.zeros(3)
        for k in range(3):
            a, b = t[k], t[(k + 1) % 3]
            d = P[(k + 1) % 3] - P[k]
            L = np.hypot(*d)
            n = np.array([d[1], -d[0]]) / L
            owners = [f for f in edge_owner[frozenset((vid(*a), vid(*b)))] if f != e]
            if owners:
                f = owners[0]
                cp = np.array([xi[f], U[f], V[f]])
                up = np.array([u[f], v[f]])
                hp = hb[f]
            else:
                qn = U[e] * n[0] + V[e] * n[1]
                un = u[e] * n[0] + v[e] * n[1]
                cp = np.array([xi[e], U[e] - 2 * qn * n[0], V[e] - 2 * qn * n[1]])
                up = np.array([u[e] - 2 * un * n[0], v[e] - 2 * un * n[1]])
                hp = hb[e]
            cm = np.array([xi[e], U[e], V[e]])
            um = np.array([u[e], v[e]])

            def phys(c, uu, h):
                pr = 0.5 * g * c[0] * (c[0] + 2 * h)
                un_ = uu @ n
                return np.array([c[1] * n[0] + c[2] * n[1], c[1] * un_ + pr * n[0], c[2] * un_ + pr * n[1]])
            lam = max(abs(um @ n) + np.sqrt(g * (cm[0] + hb[e])), abs(up @ n) + np.sqrt(g * (cp[0] + hp)))
            F = 0.5 * (phys(cm, um, hb[e]) + phys(cp, up, hp)) + 0.5 * lam * (cm - cp)
            acc += L * F
        out[:, e] = -acc / area
    return out


@pytest.mark.parametrize("bc", ["periodic", "reflective"])
def test_p0_equals_rusanov_finite_volume(oracle_mod, bc):
    """At p = 0 the DG scheme is the first-order Lax-Friedrichs FV scheme
    (the only basis function is sqrt(2): mean value = sqrt(2) c)."""
    nx, ny, Lx, Ly, g = 4, 3, 1.0, 0.8, 9.81
    o = oracle_mod.Oracle(nx, ny, 0, bc=bc, Lx=Lx, Ly=Ly, g=g)
    rng = np.random.default_rng(5)
    E = o.E
    xi = 0.3 * rng.standard_normal(E)
    U = rng.standard_normal(E)
    V = rng.standard_normal(E)
    hbm = 5 + rng.random(E)
    hb = np.zeros((E, o.Kb))
    hb[:, 0] = hbm / math.sqrt(2)
    s2 = math.sqrt(2)
    R = o.rhs(hb, (xi / s2)[:, None], (U / s2)[:, None], (V / s2)[:, None])
    ref = _fv_rhs(nx, ny, Lx, Ly, bc, xi, U, V, hbm, g)
    assert np.allclose(R[:, :, 0] * s2, ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- exactness
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_rhs_integrals_are_exact(oracle_mod, p):
    """Every integrand is a polynomial of degree <= 3p, so adding quadrature
    points must not change the RHS (the quadrature-free claim of §2.2)."""
    rng = np.random.default_rng(30 + p)
    kw = dict(bc="periodic", Lx=1.0, Ly=1.0)
    o1 = oracle_mod.Oracle(3, 3, p, **kw)
    o2 = oracle_mod.Oracle(3, 3, p, quad_extra=3, **kw)
    hb = o1.project_hb(lambda x, y: 8 + np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))
    xi = 0.2 * rng.standard_normal((o1.E, o1.K))
    U = rng.standard_normal((o1.E, o1.K))
    V = rng.standard_normal((o1.E, o1.K))
    xi[:, 1:] *= 0.1
    R1 = o1.rhs(hb, xi, U, V)
    R2 = o2.rhs(hb, xi, U, V)
    assert np.abs(R1 - R2).max() < 1e-11 * np.abs(R1).max()


# ---------------------------------------------------------------- invariants
def _hump_state(o, offset=0.5, amp=0.1, sig=0.15, U0=0.0):
    hb = o.project_hb(lambda x, y: 10 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))
    xi = o.project(lambda x, y: offset + amp * np.exp(-((x - 0.4) ** 2 + (y - 0.55) ** 2) / (2 * sig ** 2)))
    U = o.project(lambda x, y: U0 + 0.0 * x)
    V = o.project(lambda x, y: 0.0 * x)
    return hb, xi, U, V


@pytest.mark.slow
@pytest.mark.parametrize("bc", ["periodic", "reflective"])
def test_mass_conservation(oracle_mod, bc):
    """The mass flux through every interior edge cancels and is zero on
    walls: integral of xi is constant to round-off over 1000 steps."""
    o = oracle_mod.Oracle(6, 6, 2, bc=bc, rk_order=3, cfl=0.2)
    hb, xi, U, V = _hump_state(o, U0=0.3 if bc == "periodic" else 0.0)
    m0, _ = o.diagnostics(hb, xi, U, V)
    xi, U, V, t, _ = o.run(hb, xi, U, V, 1000)
    m1, _ = o.diagnostics(hb, xi, U, V)
    assert abs(m1 - m0) <= 1e-13 * abs(m0)
    assert t > 0


@pytest.mark.parametrize("p,level,lin", [(1, 0.0, False), (2, 0.1, False), (1, 0.1, True), (3, 0.0, True)])
def test_lake_at_rest(oracle_mod, p, level, lin):
    """xi = const, q = 0 stays at rest (flat h_b, and continuous linear h_b,
    which P^p represents exactly for p >= 1: the pressure flux and the
    g xi grad h_b source of Eq. (5) cancel)."""
    o = oracle_mod.Oracle(5, 5, p, bc="reflective", rk_order=3, cfl=0.2)
    hb = o.project_hb((lambda x, y: 10 + 2 * x - 1.5 * y) if lin else (lambda x, y: 10 + 0 * x))
    xi = o.project(lambda x, y: level + 0 * x)
    z = np.zeros_like(xi)
    xi1, U1, V1, t, _ = o.run(hb, xi, z, z, 1000)
    assert np.abs(xi1 - xi).max() <= 1e-12
    assert np.abs(U1).max() <= 1e-12 and np.abs(V1).max() <= 1e-12


@pytest.mark.parametrize("p", [0, 1, 2])
def test_friction_coriolis_uniform_flow(oracle_mod, p):
    """Eq. (2) sources on a uniform flow over flat bathymetry (periodic): all
    fluxes are constant, so the RHS is exactly the source,
    d_t (U, V) = -tau_bf (U, V) + f_c (V, -U), in the constant mode only;
    and the time integration follows the closed-form solution
    (U, V)(t) = e^{-tau t} R(-f t) (U0, V0) to the SSP-RK3 local error."""
    # [0, 1000]^2 in 4 x 4 quads, dt = 0.5: the gravity-wave CFL number is
    # ~0.2, so round-off modes of the uniform state stay bounded
    tau, f, U0, V0, H0, dt = 0.005, 0.02, 0.7, -0.4, 10.0, 0.5
    o = oracle_mod.Oracle(4, 4, p, bc="periodic", rk_order=3, dt=dt, tau_bf=tau, f_c=f, Lx=1000.0, Ly=1000.0)
    hb = o.project_hb(lambda x, y: H0 + 0 * x)
    xi = o.project(lambda x, y: 0 * x)
    U = o.project(lambda x, y: U0 + 0 * x)
    V = o.project(lambda x, y: V0 + 0 * x)
    R = o.rhs(hb, xi, U, V)
    c = np.sqrt(2.0)   # mean = sqrt(2) c_1
    assert np.abs(R[0]).max() <= 1e-13
    assert np.allclose(R[1][:, 0] * c, -tau * U0 + f * V0, rtol=0, atol=1e-13)
    assert np.allclose(R[2][:, 0] * c, -tau * V0 - f * U0, rtol=0, atol=1e-13)
    if o.K > 1:
        assert np.abs(R[1:, :, 1:]).max() <= 1e-13
    n = 200
    _, U1, V1, t, _ = o.run(hb, xi, U, V, n)
    assert abs(t - n * dt) <= 1e-12
    decay = np.exp(-tau * t)
    Ue = decay * (U0 * np.cos(f * t) + V0 * np.sin(f * t))
    Ve = decay * (V0 * np.cos(f * t) - U0 * np.sin(f * t))
    # SSP-RK3 is third order: global error ~ t (|lambda| dt)^3 / 24 with
    # |lambda| = |tau + i f|
    lam = np.hypot(tau, f)
    bound = 2 * t * (lam * dt) ** 3 / 24 * np.hypot(U0, V0)
    assert np.abs(U1[:, 0] * c - Ue).max() <= bound
    assert np.abs(V1[:, 0] * c - Ve).max() <= bound
    assert np.abs(U1[:, 0] * c - Ue).max() > 0      # the bound is not vacuous


def test_mirror_symmetry(oracle_mod):
    """The mesh is invariant under (x, y) -> (y, x); a symmetric hump keeps
    xi(x, y) = xi(y, x) and U(x, y) = V(y, x)."""
    o = oracle_mod.Oracle(8, 8, 2, bc="reflective", rk_order=3, cfl=0.2)
    hb = o.project_hb(lambda x, y: 10 + np.cos(np.pi * x) * np.cos(np.pi * y))
    xi = o.project(lambda x, y: 0.1 * np.exp(-((x - 0.35) ** 2 + (y - 0.35) ** 2) / 0.02))
    z = np.zeros_like(xi)
    xi, U, V, t, _ = o.run(hb, xi, z, z, 60)
    verts, _, _ = o.geometry()
    rng = np.random.default_rng(3)
    # element containing the mirrored point: mirror each element's centroid
    cen = verts.mean(axis=1)
    for e in rng.choice(o.E, 40, replace=False):
        w = rng.dirichlet([1, 1, 1])
        x, y = w @ verts[e]
        f = int(np.argmin(np.hypot(cen[:, 0] - cen[e, 1], cen[:, 1] - cen[e, 0])))
        a = o.eval_point(xi, e, x, y)
        b = o.eval_point(xi, f, y, x)
        assert abs(a - b) < 1e-13
        assert abs(o.eval_point(U, e, x, y) - o.eval_point(V, f, y, x)) < 1e-13
    assert np.abs(U).max() > 1e-3


def test_cfl_time_step(oracle_mod):
    """dt = cfl d_min / ((2p+1) max_e (|u_bar| + sqrt(g H_bar))) from element
    means; with the printed basis the mean of a field is sqrt(2) c_1."""
    o = oracle_mod.Oracle(4, 4, 2, bc="periodic", cfl=0.3, Lx=2.0, Ly=1.0)
    hb, xi, U, V = _hump_state(o, U0=0.7)
    V = V + 0.2
    dt = o.cfl_dt(hb, xi, U, V)
    s2 = math.sqrt(2)
    Hm = s2 * (xi[:, 0] + hb[:, 0])
    lam = np.hypot(s2 * U[:, 0] / Hm, s2 * V[:, 0] / Hm) + np.sqrt(9.81 * Hm)
    h = 0.5   # right triangles with legs 0.5 and 0.25
    a, b = 0.5, 0.25
    dmin = 2 * a * b / (a + b + np.hypot(a, b))
    assert abs(o.dmin() - dmin) < 1e-15
    assert abs(dt - 0.3 * dmin / (5 * lam.max())) < 1e-14 * dt
    del h


# ---------------------------------------------------------------- §3.1
def test_manufactured_force_matches_symbolic(oracle_mod):
    """The body force of the §3.1 test equals d_t q + div(q q^T / H) +
    g H grad xi differentiated symbolically (sympy)."""
    sp = pytest.importorskip("sympy")
    x, y, t = sp.symbols("x y t")
    S = sp.sin(sp.pi * (x + y + sp.Rational(1, 5) * t) / 600)
    ca, ct, ya = sp.Rational(1, 5), sp.Rational(1, 5), sp.Rational(3, 10)
    xi = 2 + ya - 2 * ca * S
    U = 2 * ya + ca * ct * S
    V = ya + ca * ct * S
    hb = 1 + x / 1000 + 2 * y / 1000
    H = xi + hb
    g = sp.Rational(981, 100)
    Fx = sp.diff(U, t) + sp.diff(U * U / H, x) + sp.diff(U * V / H, y) + g * H * sp.diff(xi, x)
    Fy = sp.diff(V, t) + sp.diff(U * V / H, x) + sp.diff(V * V / H, y) + g * H * sp.diff(xi, y)
    mass = sp.simplify(sp.diff(xi, t) + sp.diff(U, x) + sp.diff(V, y))
    assert mass == 0
    fx = sp.lambdify((x, y, t), Fx)
    fy = sp.lambdify((x, y, t), Fy)
    rng = np.random.default_rng(0)
    for _ in range(20):
        px, py, pt = rng.uniform(0, 1000), rng.uniform(0, 1000), rng.uniform(0, 1500)
        out = oracle_mod.ms_point(px, py, pt)
        assert abs(out[0] - I.ms_xi(px, py, pt)) < 1e-14
        assert abs(out[4] - fx(px, py, pt)) < 1e-12
        assert abs(out[5] - fy(px, py, pt)) < 1e-12


def _manufactured_run(oracle_mod, level, p, t_end, perturbed=True):
    w = I.manufactured(level=level, p=p, perturbed=perturbed)
    o = oracle_mod.Oracle(w.nx, w.ny, p, bc="dirichlet", Lx=1000.0, Ly=1000.0, rk_order=3, dt=0.5,
                          vertex_xy=w.vertex_xy, manufactured=True)
    hb = o.project_hb(I.ms_hb)
    xi, U, V = o.project(I.ms_xi), o.project(I.ms_U), o.project(I.ms_V)
    xi, U, V, t, _ = o.run(hb, xi, U, V, int(round(t_end / 0.5)))
    return o.ms_errors(xi, U, V, t)


@pytest.mark.slow
@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_convergence_order(oracle_mod, p):
    """§3.1 / Table 1: the L2 error decays like h^(p+1) on the perturbed
    mesh (experimental order of convergence close to p + 1)."""
    errs = np.array([_manufactured_run(oracle_mod, L, p, 100.0) for L in (2, 3, 4)])
    eoc = np.log2(errs[:-1] / errs[1:])
    assert (eoc[-1] > p + 1 - 0.3).all(), eoc
    assert (eoc[-1] < p + 1 + 0.8).all(), eoc


@pytest.mark.slow
@pytest.mark.parametrize("p,factor", [(0, 10.0), (1, 4.0), (2, 4.0), (3, 10.0)])
def test_table1_error_magnitude(oracle_mod, p, factor):
    """Errors at t = 1500 on the 32-element mesh are of Table 1's magnitude.
    The paper's random mesh is not reproducible: within a factor 4 at
    k = 1, 2.  At k = 0 the U and V errors here are 6x the table's while xi
    is 0.7x (the error in q follows the elevation error through the gravity
    wave speed, |dq| ~ sqrt(g H) |dxi|; neither the time integrator, nor the
    wave-speed point set, nor perturbing the boundary vertices changes that),
    and at k = 3 the xi error is 0.12x the table's: a factor 10 there."""
    ref = _golden("table1_convergence.txt")
    row = ref[(ref[:, 0] == p) & (ref[:, 1] == 32)][0]
    err = _manufactured_run(oracle_mod, 2, p, 1500.0)
    ratio = err / row[2:5]
    assert (ratio > 1.0 / factor).all() and (ratio < factor).all(), (err, row[2:5])


# ---------------------------------------------------------------- LF wave speed
# Reading of the Lax-Friedrichs flux named after Eq. (12) (§2.2): one wave
# speed per edge, lambda = max over both sides and the edge points
# s = 0, 1/2, 1 of |u.n| + sqrt(g H).  The pin below evaluates one edge's
# flux integral independently (numpy, the printed degree-1 basis through its
# vertex values, the mesh's documented vertex layout) and compares the
# change it causes in the neighbouring element's RHS with the oracle's.

_LAM_N, _LAM_L, _LAM_G = 4, 1.0, 9.81


def _p1_vertex_matrix():
    """Phi[k, i] = phi^_i at reference vertex k ((0,0), (1,0), (0,1)),
    printed degree-1 functions of §2.2"""
    ref = _golden("basis_vertex_values.txt")
    return ref[:3, 1:].T


def _lower_triangle(i, j, n=_LAM_N, L=_LAM_L):
    """vertices (v_ij, v_i+1j, v_ij+1) of the lower triangle of quad (i, j)"""
    h = L / n
    return np.array([[i * h, j * h], [(i + 1) * h, j * h], [i * h, (j + 1) * h]])


def _upper_triangle(i, j, n=_LAM_N, L=_LAM_L):
    """vertices (v_i+1j+1, v_ij+1, v_i+1j) of the upper triangle of quad (i, j)"""
    h = L / n
    return np.array([[(i + 1) * h, (j + 1) * h], [i * h, (j + 1) * h], [(i + 1) * h, j * h]])


def _p1_coefficients(f, verts):
    """coefficients of the linear function f in the basis phi^_i o F_e^-1:
    sum_i c_i phi^_i(vertex k) = f(vertex k)"""
    vals = np.array([f(x, y) for x, y in verts])
    return np.linalg.solve(_p1_vertex_matrix(), vals)


def _p1_basis_at(verts, x, y):
    """phi_ei(x, y) by barycentric interpolation of the vertex values"""
    T = np.array([[verts[1, 0] - verts[0, 0], verts[2, 0] - verts[0, 0]],
                  [verts[1, 1] - verts[0, 1], verts[2, 1] - verts[0, 1]]])
    xr, yr = np.linalg.solve(T, np.array([x, y]) - verts[0])
    bary = np.array([1.0 - xr - yr, xr, yr])
    return bary @ _p1_vertex_matrix()


def _lam_case():
    """Flat bathymetry and constant elevation (so H is constant and u = q/H
    exactly); linear discharge everywhere, and in the upper triangle f of
    quad (1, 1) an added discharge along the diagonal's normal that grows
    from 0 at one end of the shared edge to its maximum at the other: the
    wave speed of the shared edge peaks at that endpoint, on f's side."""
    hb0, xi0 = 10.0, 0.05
    e_v, f_v = _lower_triangle(1, 1), _upper_triangle(1, 1)
    P, Q = e_v[1], e_v[2]                      # edge 0 of e: from a2 to a3
    d = Q - P
    n = np.array([d[1], -d[0]]) / np.hypot(*d)  # outward normal of e
    A = 60.0

    def U(x, y):
        return 0.3 + 0.1 * y

    def V(x, y):
        return -0.2 + 0.05 * x

    def ramp(x, y):
        return ((x - P[0]) * d[0] + (y - P[1]) * d[1]) / (d @ d)
    return dict(hb0=hb0, xi0=xi0, e_v=e_v, f_v=f_v, P=P, Q=Q, n=n, U=U, V=V,
                Uf=lambda x, y: U(x, y) + A * n[0] * ramp(x, y),
                Vf=lambda x, y: V(x, y) + A * n[1] * ramp(x, y))


def _lam_oracle_delta(oracle_mod, c, lib=None):
    """oracle RHS of element e (lower triangle of quad (1,1)) with f's
    discharge modified, minus the RHS with the unmodified linear state"""
    o = oracle_mod.Oracle(_LAM_N, _LAM_N, 1, bc="reflective", Lx=_LAM_L, Ly=_LAM_L, g=_LAM_G, lib=lib)
    E = o.E
    e = 2 * (1 * _LAM_N + 1)
    f = e + 1
    hb = np.zeros((E, 3))
    xi = np.zeros((E, 3))
    U = np.zeros((E, 3))
    V = np.zeros((E, 3))
    verts, _, nb = o.geometry()
    assert nb[e, 0] == f
    assert np.allclose(verts[e], c["e_v"]) and np.allclose(verts[f], c["f_v"])
    for k in range(E):
        hb[k] = _p1_coefficients(lambda x, y: c["hb0"], verts[k])
        xi[k] = _p1_coefficients(lambda x, y: c["xi0"], verts[k])
        U[k] = _p1_coefficients(c["U"], verts[k])
        V[k] = _p1_coefficients(c["V"], verts[k])
    R0 = o.rhs(hb, xi, U, V)[:, e]
    U[f] = _p1_coefficients(c["Uf"], verts[f])
    V[f] = _p1_coefficients(c["Vf"], verts[f])
    R1 = o.rhs(hb, xi, U, V)[:, e]
    return R1 - R0


def _lam_numpy_delta(c, points=(0.0, 0.5, 1.0), sides=("in", "out")):
    """the same difference from one edge integral, evaluated here: element
    e's volume term and its other two edges are unchanged, so
    d R_e = -(1 / |det B_e|) (int F^(modified) phi - int F^(linear) phi)"""
    g, H = _LAM_G, c["hb0"] + c["xi0"]
    P, Q, n = c["P"], c["Q"], c["n"]
    length = np.hypot(*(Q - P))
    s_q, w_q = np.polynomial.legendre.leggauss(6)
    s_q, w_q = 0.5 * (s_q + 1.0), 0.5 * w_q
    pres = 0.5 * g * c["xi0"] * (c["xi0"] + 2 * c["hb0"])

    def flux(Uq, Vq):
        un = (Uq * n[0] + Vq * n[1]) / H
        return np.array([Uq * n[0] + Vq * n[1], Uq * un + pres * n[0], Vq * un + pres * n[1]])

    def speed(Uq, Vq):
        return abs((Uq * n[0] + Vq * n[1]) / H) + np.sqrt(g * H)

    def integral(Uf, Vf):
        lam = 0.0
        for s in points:
            x, y = P + s * (Q - P)
            if "in" in sides:
                lam = max(lam, speed(c["U"](x, y), c["V"](x, y)))
            if "out" in sides:
                lam = max(lam, speed(Uf(x, y), Vf(x, y)))
        acc = np.zeros((3, 3))
        for s, w in zip(s_q, w_q):
            x, y = P + s * (Q - P)
            cm = np.array([c["xi0"], c["U"](x, y), c["V"](x, y)])
            cp = np.array([c["xi0"], Uf(x, y), Vf(x, y)])
            F = 0.5 * (flux(cm[1], cm[2]) + flux(cp[1], cp[2])) + 0.5 * lam * (cm - cp)
            acc += w * length * np.outer(F, _p1_basis_at(c["e_v"], x, y))
        return acc, lam
    I1, lam1 = integral(c["Uf"], c["Vf"])
    I0, _ = integral(c["U"], c["V"])
    det = abs(np.linalg.det(np.array([c["e_v"][1] - c["e_v"][0], c["e_v"][2] - c["e_v"][0]]).T))
    return -(I1 - I0) / det, lam1


def test_lf_wave_speed_three_points_both_sides(oracle_mod):
    """λ of the Lax-Friedrichs flux is the maximum over both sides and
    s = 0, 1/2, 1: the oracle's RHS change equals the independent one-edge
    evaluation, and the construction makes the two plausible misreadings
    (midpoint only, interior side only) differ from it clearly."""
    c = _lam_case()
    ref, lam = _lam_numpy_delta(c)
    _, lam_mid = _lam_numpy_delta(c, points=(0.5,))
    _, lam_in = _lam_numpy_delta(c, sides=("in",))
    assert lam > 1.15 * lam_mid and lam > 1.15 * lam_in, (lam, lam_mid, lam_in)
    got = _lam_oracle_delta(oracle_mod, c)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (got, ref)
    for pts, sd in (((0.5,), ("in", "out")), ((0.0, 0.5, 1.0), ("in",))):
        wrong, _ = _lam_numpy_delta(c, points=pts, sides=sd)
        assert np.abs(wrong - ref).max() > 1e-3 * np.abs(ref).max()


# the lines of the oracle's wave-speed loop that the planted mistakes change
_LAM_LOOP = "for (int k = 0; k < 3; ++k) {\n      double s = 0.5 * k;"
_LAM_OUTER = "      if (lb > lam) lam = lb;\n"


@pytest.mark.parametrize("mutation", ["midpoint_only", "interior_only"])
def test_lf_wave_speed_pin_catches_planted_mistakes(oracle_mod, tmp_path, mutation):
    """A copy of the oracle with λ taken at the edge midpoint only, or from
    the interior side only, fails the comparison above."""
    src = oracle_mod.source()
    assert src.count(_LAM_LOOP) == 1 and src.count(_LAM_OUTER) == 1
    if mutation == "midpoint_only":
        src = src.replace(_LAM_LOOP, "for (int k = 1; k < 2; ++k) {\n      double s = 0.5 * k;")
    else:
        src = src.replace(_LAM_OUTER, "")
    lib = oracle_mod.build_variant(src, mutation, str(tmp_path))
    c = _lam_case()
    ref, _ = _lam_numpy_delta(c)
    got = _lam_oracle_delta(oracle_mod, c, lib=lib)
    assert np.abs(got - ref).max() > 1e-3 * np.abs(ref).max()


# ---------------------------------------------------------------- diagnostics
def _linear_square_integral(a, b, c, Lx, Ly):
    """exact integral of (a + b x + c y)^2 over [0, Lx] x [0, Ly]:
    area (mean^2 + b^2 Lx^2 / 12 + c^2 Ly^2 / 12)"""
    mean = a + b * Lx / 2 + c * Ly / 2
    return Lx * Ly * (mean ** 2 + (b * Lx) ** 2 / 12 + (c * Ly) ** 2 / 12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_energy_diagnostic_closed_form(oracle_mod, p):
    """energy = 1/2 integral (g xi^2 + U u + V v) and mass = integral xi, at
    rest, in uniform flow and with linear fields at constant depth (then
    u = q / H exactly): E = 1/2 (g int xi^2 + int (U^2 + V^2) / H)."""
    Lx, Ly, g, H0 = 1.2, 0.8, 9.81, 7.5
    o = oracle_mod.Oracle(3, 4, p, bc="reflective", Lx=Lx, Ly=Ly, g=g)
    cases = [((0.3, 0, 0), (0, 0, 0), (0, 0, 0)),            # at rest
             ((0.3, 0, 0), (0.9, 0, 0), (-0.4, 0, 0)),       # uniform flow
             ((0.2, 0.5, -0.3), (0.6, -0.7, 0.4), (0.1, 0.3, 0.8))]
    for (xa, xb, xc), (ua, ub, uc), (va, vb, vc) in cases:
        hb = o.project_hb(lambda x, y: H0 - (xa + xb * x + xc * y))
        xi = o.project(lambda x, y: xa + xb * x + xc * y)
        U = o.project(lambda x, y: ua + ub * x + uc * y)
        V = o.project(lambda x, y: va + vb * x + vc * y)
        mass, energy = o.diagnostics(hb, xi, U, V)
        m_ref = Lx * Ly * (xa + xb * Lx / 2 + xc * Ly / 2)
        e_ref = 0.5 * (g * _linear_square_integral(xa, xb, xc, Lx, Ly) +
                       (_linear_square_integral(ua, ub, uc, Lx, Ly) +
                        _linear_square_integral(va, vb, vc, Lx, Ly)) / H0)
        assert abs(mass - m_ref) <= 1e-13 * abs(m_ref)
        assert abs(energy - e_ref) <= 1e-13 * e_ref, (energy, e_ref)


_EN_HALF = "en += 0.5 * w *"
_EN_UU = "eval_field(h, U, e, xr, yr) * eval_field(h, u, e, xr, yr)"


@pytest.mark.parametrize("mutation", ["no_half", "U_times_U"])
def test_energy_pin_catches_planted_mistakes(oracle_mod, tmp_path, mutation):
    """A copy of the oracle whose energy drops the factor 1/2, or uses U^2
    instead of U u, fails the closed form of the uniform flow."""
    src = oracle_mod.source()
    assert src.count(_EN_HALF) == 1 and src.count(_EN_UU) == 1
    if mutation == "no_half":
        src = src.replace(_EN_HALF, "en += w *")
    else:
        src = src.replace(_EN_UU, "eval_field(h, U, e, xr, yr) * eval_field(h, U, e, xr, yr)")
    lib = oracle_mod.build_variant(src, mutation, str(tmp_path))
    Lx, Ly, g, H0, xi0, U0 = 1.2, 0.8, 9.81, 7.5, 0.3, 0.9
    o = oracle_mod.Oracle(3, 4, 2, bc="reflective", Lx=Lx, Ly=Ly, g=g, lib=lib)
    hb = o.project_hb(lambda x, y: H0 - xi0 + 0 * x)
    xi = o.project(lambda x, y: xi0 + 0 * x)
    U = o.project(lambda x, y: U0 + 0 * x)
    _, energy = o.diagnostics(hb, xi, U, np.zeros_like(U))
    e_ref = 0.5 * Lx * Ly * (g * xi0 ** 2 + U0 ** 2 / H0)
    assert abs(energy - e_ref) > 1e-3 * e_ref
