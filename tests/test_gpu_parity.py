"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Every input is produced by the oracle's own L2 projection of the seeded
workload fields and handed to both sides unchanged.  Tolerances:
  * FP64 right-hand side: max |GPU - oracle| <= 1e-13 * max |oracle| per field;
  * FP64 time stepping: relative L2 per field <= 1e-12 after 100 steps;
  * FP32 state with FP64 velocity solve: relative L2 per field <= 1e-5 after
    1000 steps.
Relative L2 uses the orthonormal basis: ||a - b|| / ||b|| over all
coefficients (all triangles have the same |det B| on the uniform mesh).
"""
import numpy as np
import pytest

from paper_1904_08684_gb300 import binding as B
from paper_1904_08684_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    yield
    torch.cuda.synchronize()


def _relL2(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def _state(o, wl, U0=0.0, V0=0.0, with_flow=True):
    """oracle-projected inputs of a workload; optional smooth discharge"""
    hb = o.project_hb(wl.hb)
    xi = o.project(wl.xi0)
    if with_flow:
        U = o.project(lambda x, y: U0 + 0.3 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))
        V = o.project(lambda x, y: V0 + 0.2 * np.cos(2 * np.pi * (x + y)))
    else:
        U = np.zeros_like(xi)
        V = np.zeros_like(xi)
    return hb, xi, U, V


def _cfg(wl, precision="fp64", **kw):
    args = dict(bc=wl.bc, precision=precision, rk_order=wl.rk_order, cfl=wl.cfl, dt=wl.dt, g=wl.g,
                x0=wl.x0, y0=wl.y0, Lx=wl.Lx, Ly=wl.Ly)
    args.update(kw)
    return B.make_config(wl.nx, wl.ny, wl.p, **args)


def _to_soa(fields, dtype):
    """list of (E, K) arrays -> torch (F, K, E) on the GPU"""
    a = np.stack([np.asarray(f).T for f in fields])
    return torch.tensor(a, dtype=dtype, device="cuda").contiguous()


def _gpu_rhs(cfg, hb, xi, U, V, dtype=torch.float64):
    ctx = B.dg_init(cfg, hb, xi, U, V)
    try:
        st = _to_soa([xi, U, V], dtype)
        out = torch.empty_like(st)
        B.dg_rhs(ctx, st, out)
        torch.cuda.synchronize()
        return out.double().cpu().numpy().transpose(0, 2, 1)
    finally:
        B.dg_destroy(ctx)


# ------------------------------------------------------------------ RHS
@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("bc", ["periodic", "reflective"])
def test_rhs_matches_oracle_fp64(oracle_mod, p, bc):
    """13 x 11 quads = 286 triangles: several 128-thread blocks and a ragged
    tail.  p = 0 is the degenerate case: a first-order finite-volume
    Lax-Friedrichs scheme, with h_b in P^1 (source and edge depths)."""
    wl = I.waves_p2_512(n=13, p=p, ngauss=3)
    wl.ny = 11
    wl.bc = bc
    o = oracle_mod.Oracle(wl.nx, wl.ny, p, bc=bc)
    hb, xi, U, V = _state(o, wl)
    ref = o.rhs(hb, xi, U, V)
    got = _gpu_rhs(_cfg(wl), hb, xi, U, V)
    # p = 4: the oracle builds the degree-4 functions by Gram-Schmidt in
    # floating point (coefficients up to ~1e3, with cancellation), which adds
    # ~1e-13 relative rounding; the FP64-path bar of 1e-12 applies there
    tol = 1e-13 if p < 4 else 1e-12
    for f in range(3):
        scale = np.abs(ref[f]).max()
        assert np.abs(got[f] - ref[f]).max() <= tol * scale, (f, np.abs(got[f] - ref[f]).max() / scale)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("proj", ["fp64", "fp32", "df64", "mixed"])
def test_rhs_fp32_state(oracle_mod, p, proj):
    """FP32 state and contractions (velocity solve in FP64, FP32,
    double-float, or FP32 with FP64-residual refinement): the RHS agrees with
    the FP64 oracle to FP32 round-off amplified by the Lax-Friedrichs jump
    term (|jump| ~ eps |w|, times lambda / h).  The double-float solve is
    built for p <= 3."""
    if proj == "df64" and p > 3:
        pytest.skip("double-float solve is built for p <= 3")
    wl = I.waves_p2_512(n=13, p=p, ngauss=3)
    wl.ny = 11
    o = oracle_mod.Oracle(wl.nx, wl.ny, p, bc="periodic")
    hb, xi, U, V = _state(o, wl)
    ref = o.rhs(hb, xi, U, V)
    got = _gpu_rhs(_cfg(wl, precision="fp32", proj_precision=proj), hb, xi, U, V, dtype=torch.float32)
    for f in range(3):
        assert _relL2(got[f], ref[f]) <= 2e-5, (f, _relL2(got[f], ref[f]))


def _weighted_mass_condition(o, H, e):
    """condition number of A^H (Eq. (12)) on element e, assembled in FP64 from
    the oracle's own L2 projection: column b = Pi(H phi_b)"""
    xy = o.proj_nodes(np.array([e], dtype=np.int32))[0]
    A = np.zeros((o.K, o.K))
    for b in range(o.K):
        c = np.zeros((o.E, o.K))
        c[e, b] = 1.0
        phib = np.array([o.eval_point(c, e, x, y) for x, y in xy])
        col = np.zeros((o.E, o.K))
        o.project_sub((H(xy[:, 0], xy[:, 1]) * phib)[None, :], [e], col)
        A[:, b] = col[e]
    w = np.linalg.eigvalsh(0.5 * (A + A.T))
    return w[-1] / w[0]


@pytest.mark.parametrize("p", [3, 4])
def test_velocity_solve_ill_conditioned_element(oracle_mod, p):
    """One element whose depth vanishes like lambda_1^p towards an edge
    (H = 1e-3 + 10 lambda_1^p, a beach inside one triangle; depth 10
    elsewhere): A^H of Eq. (12) then has kappa ~ 5e2 (p = 3) and ~ 3e3
    (p = 4).  With the FP64, mixed (refined) and double-float solves the
    momentum RHS of that element and its neighbours stays at the FP32 level
    of the state (bar 2e-6 ~ 30 eps_32: sums of ~30 rounded products); the
    FP32 solve adds an error ~ kappa eps_32, which at p = 4 is more than ten
    times larger: the case the FP64 solve is there for."""
    n, e0 = 8, 54
    vx = np.array([[0.375, 0.375], [0.5, 0.375], [0.375, 0.5]])    # element 54, counter-clockwise

    def lam1(x, y):
        (x1, y1), (x2, y2), (x3, y3) = vx
        det = (x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1)
        l2 = ((x - x1) * (y3 - y1) - (x3 - x1) * (y - y1)) / det
        l3 = ((x2 - x1) * (y - y1) - (x - x1) * (y2 - y1)) / det
        return 1.0 - l2 - l3

    def beach(x, y):
        return 1e-3 + 10.0 * lam1(x, y) ** p

    o = oracle_mod.Oracle(n, n, p, bc="reflective")
    verts, _, nb = o.geometry()
    assert np.allclose(np.sort(verts[e0], axis=0), np.sort(vx, axis=0))
    kappa = _weighted_mass_condition(o, beach, e0)
    assert kappa > (300 if p == 3 else 2000), kappa
    hb = np.zeros((o.E, o.Kb))
    hb[:, 0] = 10.0 / np.sqrt(2.0)          # phi_1 = sqrt(2): depth 10
    xy = o.proj_nodes(np.array([e0], dtype=np.int32))
    o.project_sub(beach(xy[..., 0], xy[..., 1]), [e0], hb, hb=True)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)    # noqa: E731
    hb = f32(hb)
    xi = np.zeros((o.E, o.K))
    U = f32(o.project(lambda x, y: 0.3 + 0.1 * x))
    V = f32(o.project(lambda x, y: -0.2 + 0.05 * y))
    ref = o.rhs(hb, xi, U, V)
    S = np.unique(np.concatenate([[e0], nb[e0][nb[e0] >= 0]]))
    errs = {}
    for proj in ("fp64", "mixed", "df64", "fp32"):
        if proj == "df64" and p > 3:
            continue
        cfg = B.make_config(n, n, p, bc="reflective", precision="fp32", rk_order=3, cfl=0.2,
                            proj_precision=proj)
        got = _gpu_rhs(cfg, hb, xi, U, V, dtype=torch.float32)
        errs[proj] = max(_relL2(got[f][S], ref[f][S]) for f in (1, 2))
    print("p = %d, kappa(A^H) = %.0f: momentum RHS relative L2 near the element per solve %s"
          % (p, kappa, {k: "%.2e" % v for k, v in errs.items()}))
    for proj in ("fp64", "mixed", "df64"):
        if proj in errs:
            assert errs[proj] <= 2e-6, (proj, errs)
    if p == 4:
        assert errs["fp32"] >= 10 * errs["fp64"], errs


@pytest.mark.parametrize("block", [32, 64, 96])
def test_rhs_block_sizes_and_state_pointer(oracle_mod, block):
    """smaller thread blocks (more, ragged blocks) give the same RHS; the
    context's own state (dg_state_device) serves as dg_rhs input"""
    wl = I.waves_p2_512(n=13, p=2, ngauss=3)
    wl.ny = 11
    o = oracle_mod.Oracle(wl.nx, wl.ny, 2, bc="periodic")
    hb, xi, U, V = _state(o, wl)
    ref = o.rhs(hb, xi, U, V)
    cfg = _cfg(wl, block_size=block)
    got = _gpu_rhs(cfg, hb, xi, U, V)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    ctx = B.dg_init(cfg, hb, xi, U, V)
    try:
        out = torch.empty((3, o.K, o.E), dtype=torch.float64, device="cuda")
        B.dg_rhs(ctx, B.dg_state_device(ctx), out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().transpose(0, 2, 1), got)
    finally:
        B.dg_destroy(ctx)


def test_rhs_nonsquare_domain(oracle_mod):
    """hx != hy exercises the diagonal normal and the adj(B) scaling."""
    wl = I.waves_p2_512(n=9, p=2, ngauss=2)
    wl.ny, wl.Lx, wl.Ly = 5, 2.0, 0.7
    wl.xi0 = I.gaussian_sum([0.05], [0.2], [1.0], [0.35], periodic=False)
    for bc in ("periodic", "reflective"):
        o = oracle_mod.Oracle(wl.nx, wl.ny, 2, bc=bc, Lx=2.0, Ly=0.7)
        hb, xi, U, V = _state(o, wl)
        ref = o.rhs(hb, xi, U, V)
        got = _gpu_rhs(_cfg(wl, bc=bc), hb, xi, U, V)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


# ------------------------------------------------------------------ time stepping
def test_run_matches_oracle_hump_p1(oracle_mod):
    """32 x 32 reflective hump, p = 1, SSP-RK2, CFL 0.2, 100 steps."""
    wl = I.hump_p1_32()
    o = oracle_mod.Oracle(wl.nx, wl.ny, 1, bc="reflective", rk_order=2, cfl=0.2)
    hb, xi, U, V = _state(o, wl, with_flow=False)
    xr, Ur, Vr, tr, _ = o.run(hb, xi, U, V, wl.steps)
    ctx = B.dg_init(_cfg(wl), hb, xi, U, V)
    try:
        t = B.dg_run(ctx, wl.steps)
        xg, Ug, Vg = B.dg_get_state(ctx, o.E, o.K)
    finally:
        B.dg_destroy(ctx)
    assert abs(t - tr) <= 1e-13 * tr
    for g_, r_ in ((xg, xr), (Ug, Ur), (Vg, Vr)):
        assert _relL2(g_, r_) <= 1e-12


@pytest.mark.parametrize("p", [0, 2, 3])
def test_run_matches_oracle_waves(oracle_mod, p):
    """periodic waves on sinusoidal bathymetry with a mean flow, SSP-RK3."""
    wl = I.waves_p2_512(n=16, p=p, ngauss=4)
    o = oracle_mod.Oracle(wl.nx, wl.ny, p, bc="periodic", rk_order=3, cfl=0.2)
    hb, xi, U, V = _state(o, wl, U0=0.5, V0=-0.3)
    xr, Ur, Vr, tr, _ = o.run(hb, xi, U, V, 100)
    ctx = B.dg_init(_cfg(wl), hb, xi, U, V)
    try:
        t = B.dg_run(ctx, 100)
        xg, Ug, Vg = B.dg_get_state(ctx, o.E, o.K)
    finally:
        B.dg_destroy(ctx)
    assert abs(t - tr) <= 1e-13 * tr
    for g_, r_ in ((xg, xr), (Ug, Ur), (Vg, Vr)):
        assert _relL2(g_, r_) <= 1e-12


def test_fixed_dt_rk1_step(oracle_mod):
    """forward Euler with a fixed dt: w' = w + dt R(w) exactly as the oracle."""
    wl = I.waves_p2_512(n=6, p=2, ngauss=2)
    wl.rk_order, wl.dt = 1, 1e-4
    o = oracle_mod.Oracle(6, 6, 2, bc="periodic", rk_order=1, dt=1e-4)
    hb, xi, U, V = _state(o, wl)
    xr, Ur, Vr, tr, _ = o.run(hb, xi, U, V, 3)
    ctx = B.dg_init(_cfg(wl, rk_order=1, dt=1e-4), hb, xi, U, V)
    try:
        assert B.dg_rk_step(ctx, want_dt=True) == 1e-4
        B.dg_rk_step(ctx)
        t = B.dg_run(ctx, 1)
        xg, Ug, Vg = B.dg_get_state(ctx, o.E, o.K)
    finally:
        B.dg_destroy(ctx)
    assert abs(t - 3e-4) < 1e-18
    for g_, r_ in ((xg, xr), (Ug, Ur), (Vg, Vr)):
        assert _relL2(g_, r_) <= 1e-13


# ------------------------------------------------------------------ FP32 state
@pytest.mark.slow
@pytest.mark.parametrize("proj", ["fp64", "df64", "mixed"])
def test_fp32_mixed_hump_p3_1000_steps(oracle_mod, proj):
    """FP32 state and contractions, FP64 (or double-float) velocity solve,
    p = 3, 1000 SSP-RK3 steps against the FP64 oracle: relative L2 per field
    <= 1e-5."""
    wl = I.hump_p3_32()
    o = oracle_mod.Oracle(wl.nx, wl.ny, 3, bc="reflective", rk_order=3, cfl=0.2)
    hb, xi, U, V = _state(o, wl, with_flow=False)
    xr, Ur, Vr, tr, _ = o.run(hb, xi, U, V, wl.steps)
    ctx = B.dg_init(_cfg(wl, precision="fp32", proj_precision=proj), hb, xi, U, V)
    try:
        m0, _ = B.dg_diagnostics(ctx)
        t = B.dg_run(ctx, wl.steps)
        m1, _ = B.dg_diagnostics(ctx)
        xg, Ug, Vg = B.dg_get_state(ctx, o.E, o.K)
    finally:
        B.dg_destroy(ctx)
    assert abs(t - tr) <= 1e-5 * tr
    errs = [_relL2(g_, r_) for g_, r_ in ((xg, xr), (Ug, Ur), (Vg, Vr))]
    print("hump-p3-32 FP32 state, %s solve, %d steps: relative L2 (xi, qx, qy) %s, mass drift %.2e"
          % (proj, wl.steps, ["%.2e" % v for v in errs], (m1 - m0) / m0))
    # xi is measured around its mean state: the hump is the signal
    assert max(errs) <= 1e-5, errs
    assert abs(m1 - m0) <= 1e-5 * abs(m0)


# ------------------------------------------------------------------ invariants on the GPU
def test_lake_at_rest_gpu():
    """xi = 0.1, q = 0 on flat bathymetry stays at rest (1000 steps, FP64)."""
    wl = I.hump_p1_32(p=2, rk=3)
    E, K = wl.E, wl.K
    xi = np.zeros((E, K))
    xi[:, 0] = 0.1 * np.sqrt(2.0)       # constant 0.1 (phi_1 = sqrt 2)
    hb = np.zeros((E, K))
    hb[:, 0] = 10.0 * np.sqrt(2.0)
    z = np.zeros((E, K))
    ctx = B.dg_init(_cfg(wl), hb, xi, z, z)
    try:
        B.dg_run(ctx, 1000)
        xg, Ug, Vg = B.dg_get_state(ctx, E, K)
    finally:
        B.dg_destroy(ctx)
    assert np.abs(xg - xi).max() <= 1e-12
    assert np.abs(Ug).max() <= 1e-12 and np.abs(Vg).max() <= 1e-12


def test_deterministic_and_checkpoint_resume(oracle_mod):
    """Two runs are bit-identical; 2N steps == N steps, save, restore, N steps."""
    wl = I.waves_p2_512(n=12, p=2, ngauss=3)
    o = oracle_mod.Oracle(12, 12, 2, bc="periodic")
    hb, xi, U, V = _state(o, wl)
    cfg = _cfg(wl)
    outs = []
    for _ in range(2):
        ctx = B.dg_init(cfg, hb, xi, U, V)
        t = B.dg_run(ctx, 20)
        outs.append((B.dg_get_state(ctx, o.E, o.K), t))
        B.dg_destroy(ctx)
    for a, b in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(a, b)
    ctx = B.dg_init(cfg, hb, xi, U, V)
    t1 = B.dg_run(ctx, 10)
    saved = B.dg_get_state(ctx, o.E, o.K)
    B.dg_destroy(ctx)
    ctx = B.dg_init(cfg, hb, *saved)
    B.dg_set_state(ctx, *saved, t=t1)
    t2 = B.dg_run(ctx, 10)
    res = B.dg_get_state(ctx, o.E, o.K)
    B.dg_destroy(ctx)
    assert t2 == outs[0][1]
    for a, b in zip(res, outs[0][0]):
        assert np.array_equal(a, b)


def _pinned_views(E, K, n=3, offset=5):
    """n (E, K) float64 arrays inside one page-locked buffer, the first
    starting ``offset`` words in (an interior pointer of the allocation)"""
    buf = torch.empty(offset + n * E * K + 7, dtype=torch.float64).pin_memory().numpy()
    buf[:] = np.nan
    return buf, [buf[offset + k * E * K: offset + (k + 1) * E * K].reshape(E, K) for k in range(n)]


@pytest.mark.parametrize("precision,proj", [("fp64", "fp64"), ("fp32", "mixed")])
def test_state_through_page_locked_host_arrays(oracle_mod, precision, proj):
    """dg_get_state / dg_set_state with page-locked arrays (read and written
    in place by the conversion kernels over the host link) give the bits of
    pageable arrays (staged copies), on a ragged 13 x 11 mesh; the words
    around the arrays stay untouched; a run continued from a state set
    through page-locked arrays equals one continued from pageable arrays."""
    wl = I.waves_p2_512(n=13, p=2, ngauss=3)
    wl.ny = 11
    o = oracle_mod.Oracle(13, 11, 2, bc="periodic")
    hb, xi, U, V = _state(o, wl)
    cfg = _cfg(wl, precision=precision, proj_precision=proj)
    E, K = o.E, o.K
    ctx = B.dg_init(cfg, hb, xi, U, V)
    try:
        t = B.dg_run(ctx, 7)
        ref = B.dg_get_state(ctx, E, K)
        buf, views = _pinned_views(E, K)
        B.dg_get_state(ctx, E, K, out=views)
        for a, r in zip(views, ref):
            assert np.array_equal(a, r)
        assert np.isnan(buf[:5]).all() and np.isnan(buf[5 + 3 * E * K:]).all()
        # a perturbed state set through each kind of array, then 3 steps
        new = [r * (1.0 + 1e-3 * np.cos(np.arange(r.size)).reshape(r.shape)) for r in ref]
        B.dg_set_state(ctx, *new, t=t)
        B.dg_run(ctx, 3)
        want = B.dg_get_state(ctx, E, K)
        for v, a in zip(views, new):
            v[:] = a
        B.dg_set_state(ctx, *views, t=t)
        B.dg_run(ctx, 3)
        got = B.dg_get_state(ctx, E, K, out=_pinned_views(E, K, offset=0)[1])
        for a, r in zip(got, want):
            assert np.array_equal(a, r)
    finally:
        B.dg_destroy(ctx)


def test_diagnostics_match_oracle(oracle_mod):
    wl = I.waves_p2_512(n=10, p=2, ngauss=3)
    o = oracle_mod.Oracle(10, 10, 2, bc="periodic")
    hb, xi, U, V = _state(o, wl, U0=0.4)
    m_ref, e_ref = o.diagnostics(hb, xi, U, V)
    ctx = B.dg_init(_cfg(wl), hb, xi, U, V)
    try:
        m, e = B.dg_diagnostics(ctx)
    finally:
        B.dg_destroy(ctx)
    assert abs(m - m_ref) <= 1e-13 * abs(m_ref)
    assert abs(e - e_ref) <= 1e-13 * abs(e_ref)


def test_setup_projection_exact_on_polynomials(oracle_mod):
    """dg_project reproduces the oracle's projection of a polynomial of
    degree p (both exact), and of a smooth field to quadrature accuracy."""
    for p in (1, 2, 3, 4):
        cfg = B.make_config(5, 4, p, Lx=1.5, Ly=1.0)
        o = oracle_mod.Oracle(5, 4, p, bc="periodic", Lx=1.5, Ly=1.0)
        f = lambda x, y: 1.0 + 0.5 * x - 0.25 * y + 0.3 * x * y ** (p - 1)  # noqa: E731
        Q = B.dg_proj_num_nodes(p)
        E = o.E
        xy = torch.empty((2, Q, E), dtype=torch.float64, device="cuda")
        B.dg_proj_nodes(cfg, xy)
        vals = f(xy[0], xy[1]).contiguous()
        coef = torch.empty((o.K, E), dtype=torch.float64, device="cuda")
        B.dg_project(cfg, vals, coef)
        torch.cuda.synchronize()
        got = coef.cpu().numpy().T
        ref = o.project(f)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("precision,proj", [("fp64", "fp64"), ("fp32", "fp64"), ("fp32", "mixed"),
                                             ("fp32", "df64"), ("fp32", "fp32")])
def test_dry_state_is_reported(precision, proj):
    """A negative depth in the input is reported as DG_ERR_DRY, not a hang or
    a fault, and the context stays usable; in every arithmetic (the mixed
    solve's FP32 pivots fail there and it hands the element to the FP64
    solve, which reports it)."""
    wl = I.hump_p1_32(n=8)
    E, K = wl.E, wl.K
    xi = np.zeros((E, K))
    hb = np.zeros((E, K))
    hb[:, 0] = 10.0 * np.sqrt(2.0)
    hb[5, 0] = -3.0 * np.sqrt(2.0)      # one element with negative depth
    z = np.zeros((E, K))
    ctx = B.dg_init(_cfg(wl, precision=precision, proj_precision=proj, dt=1e-4), hb, xi, z, z)
    try:
        with pytest.raises(B.DGError) as ei:
            B.dg_run(ctx, 1)
        assert ei.value.status in (B.DG_ERR_DRY, B.DG_ERR_NONFINITE)
        xg, _, _ = B.dg_get_state(ctx, E, K)
        assert xg.shape == (E, K)
    finally:
        B.dg_destroy(ctx)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rhs_of_a_dry_trial_state_leaves_the_time_loop_clean(precision):
    """dg_rhs of some other (here dry) state has its own error word: the
    context's next dg_run, on its own healthy state, reports DG_OK, and the
    state it reaches equals a context that never saw the dry right-hand side"""
    wl = I.hump_p1_32(n=8)
    E, K = wl.E, wl.K
    hb = np.zeros((E, K))
    hb[:, 0] = 10.0 * np.sqrt(2.0)
    xi = np.zeros((E, K))
    xi[:, 0] = 0.01 * np.sin(np.arange(E))
    z = np.zeros((E, K))
    dry = xi.copy()
    dry[5, 0] = -12.0 * np.sqrt(2.0)      # H < 0 on element 5
    dtype = torch.float64 if precision == "fp64" else torch.float32
    cfg = _cfg(wl, precision=precision, dt=1e-4)
    ctx = B.dg_init(cfg, hb, xi, z, z)
    ref = B.dg_init(cfg, hb, xi, z, z)
    try:
        st = _to_soa([dry, z, z], dtype)
        out = torch.empty_like(st)
        B.dg_rhs(ctx, st, out)
        torch.cuda.synchronize()
        B.dg_run(ctx, 2)                      # raises on a reported error
        B.dg_run(ref, 2)
        for a, b in zip(B.dg_get_state(ctx, E, K), B.dg_get_state(ref, E, K)):
            assert np.array_equal(a, b)
    finally:
        B.dg_destroy(ctx)
        B.dg_destroy(ref)


def test_nonfinite_state_is_reported():
    """a NaN in the input discharge is reported as DG_ERR_NONFINITE"""
    wl = I.hump_p1_32(n=8)
    E, K = wl.E, wl.K
    hb = np.zeros((E, K))
    hb[:, 0] = 10.0 * np.sqrt(2.0)
    z = np.zeros((E, K))
    U = np.zeros((E, K))
    U[7, 1] = np.nan
    ctx = B.dg_init(_cfg(wl, dt=1e-4), hb, z, U, z)
    try:
        with pytest.raises(B.DGError) as ei:
            B.dg_run(ctx, 1)
        assert ei.value.status == B.DG_ERR_NONFINITE
    finally:
        B.dg_destroy(ctx)


def test_device_allocation_failure_is_reported():
    """a configuration whose buffers cannot fit is refused with DG_ERR_OOM
    before any input is read (the host arrays are never touched)"""
    import ctypes
    cfg = B.make_config(30000, 30000, 4, bc="periodic", precision="fp64")   # ~1.8e9 triangles, p = 4
    h = ctypes.c_void_p()
    z = (ctypes.c_double * 1)()
    assert B.load().dg_init(ctypes.byref(cfg), z, z, z, z, None, ctypes.byref(h)) == B.DG_ERR_OOM
    torch.cuda.synchronize()
    # the device stays usable
    small = B.make_config(4, 4, 1)
    E, K = B.dg_num_elements(small), 3
    hb = np.zeros((E, K))
    hb[:, 0] = 10.0
    ctx = B.dg_init(small, hb, np.zeros((E, K)), np.zeros((E, K)), np.zeros((E, K)))
    B.dg_destroy(ctx)


def test_checkpoint_resume_through_file(oracle_mod, tmp_path):
    """N steps, checkpoint to .npz, a new context resumes: bit-identical to 2N"""
    from paper_1904_08684_gb300 import checkpoint
    wl = I.waves_p2_512(n=10, p=2, ngauss=2)
    o = oracle_mod.Oracle(wl.nx, wl.ny, 2, bc="periodic")
    hb, xi, U, V = _state(o, wl)
    for precision in ("fp64", "fp32"):
        cfg = _cfg(wl, precision=precision)
        ref = B.dg_init(cfg, hb, xi, U, V)
        a = B.dg_init(cfg, hb, xi, U, V)
        b = B.dg_init(cfg, hb, xi, U, V)
        try:
            t_ref = B.dg_run(ref, 20)
            B.dg_run(a, 10)
            path = str(tmp_path / ("ck_%s.npz" % precision))
            checkpoint.save(path, a, cfg)
            assert checkpoint.load(path, b, cfg) == B.dg_run(a, 0)
            t_b = B.dg_run(b, 10)
            assert t_b == t_ref
            for x, y in zip(B.dg_get_state(b, o.E, o.K), B.dg_get_state(ref, o.E, o.K)):
                assert np.array_equal(x, y)
        finally:
            for c in (ref, a, b):
                B.dg_destroy(c)


def test_rhs_friction_coriolis(oracle_mod):
    """bottom friction tau_bf and Coriolis f_c of Eq. (2) (source r of Eq. (5))"""
    wl = I.waves_p2_512(n=9, p=2, ngauss=2)
    wl.ny = 7
    for bc in ("periodic", "reflective"):
        o = oracle_mod.Oracle(9, 7, 2, bc=bc, tau_bf=0.03, f_c=1.2e-4 * 1000)
        hb, xi, U, V = _state(o, wl, U0=0.3, V0=-0.2)
        ref = o.rhs(hb, xi, U, V)
        got = _gpu_rhs(_cfg(wl, bc=bc, tau_bf=0.03, f_c=0.12), hb, xi, U, V)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
