"""dg_rhs_noalloc: the allocation-free right-hand side must equal dg_rhs.

Callers that cannot call cudaMalloc (graph capture in progress, fixed device
budgets) use dg_rhs_noalloc, which keeps its intermediates in a fixed array
inside the library.  It runs the same kernels as dg_rhs on the same inputs,
so the two results are compared bit for bit, on two calls in a row.  This
file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It must pass both alone in
a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_1904_08684_gb300 import binding as B
from paper_1904_08684_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _fields(wl, seed, depth_shift=0.0):
    """seeded smooth fields sampled at the library's set-up nodes and
    projected with dg_project (device FP64 SoA (K, E)); depth_shift is
    added to the bathymetry"""
    cfg = B.make_config(wl.nx, wl.ny, wl.p, bc=wl.bc)
    Q, E, K = B.dg_proj_num_nodes(wl.p), wl.E, wl.K
    xy = torch.empty((2, Q, E), dtype=torch.float64, device="cuda")
    B.dg_proj_nodes(cfg, xy)
    r = I.uniform(seed, 4)
    fields = [lambda x, y: wl.hb(x, y) + depth_shift, I.gaussian_sum([0.05 + 0.05 * r[0]], [0.08], [r[1]], [r[2]]),
              lambda x, y: 0.2 + 0.1 * torch.sin(2 * np.pi * (x + r[3])),
              lambda x, y: -0.1 + 0.05 * torch.cos(2 * np.pi * y)]
    out = []
    for k, f in enumerate(fields):
        if k == 0 and wl.p == 0:
            # h_b lives in P^max(p,1): project it with an order-1 rule
            cfg1 = B.make_config(wl.nx, wl.ny, 1, bc=wl.bc)
            xy1 = torch.empty((2, B.dg_proj_num_nodes(1), E), dtype=torch.float64, device="cuda")
            B.dg_proj_nodes(cfg1, xy1)
            c = torch.empty((B.dg_num_basis_bathymetry(0), E), dtype=torch.float64, device="cuda")
            B.dg_project(cfg1, f(xy1[0], xy1[1]).contiguous(), c)
        else:
            c = torch.empty((K, E), dtype=torch.float64, device="cuda")
            B.dg_project(cfg, f(xy[0], xy[1]).contiguous(), c)
        out.append(c)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision,p,proj,bc", [
    ("fp64", 2, "fp64", "periodic"), ("fp64", 3, "fp64", "reflective"), ("fp32", 3, "fp64", "periodic"),
    ("fp64", 0, "fp64", "reflective"), ("fp64", 1, "fp64", "periodic"), ("fp32", 4, "fp64", "reflective"),
    ("fp32", 3, "mixed", "periodic"), ("fp32", 2, "df64", "reflective"), ("fp32", 1, "fp32", "periodic")])
def test_noalloc_rhs_equals_dg_rhs_twice(precision, p, proj, bc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = I.waves_p2_512(n=37 if p < 4 else 21, p=p, ngauss=2)
    wl.ny = 29 if p < 4 else 17                  # ragged last block
    wl.bc = bc
    cfg = B.make_config(wl.nx, wl.ny, p, bc=bc, precision=precision, rk_order=3, cfl=0.2,
                        proj_precision=proj)
    dt = torch.float64 if precision == "fp64" else torch.float32
    refs, inputs = [], []
    for seed in (11, 12):                        # two different inputs
        hb, xi, U, V = _fields(wl, seed)
        state = torch.stack([xi, U, V]).to(dt).contiguous()
        ctx = B.dg_init_device(cfg, hb, xi, U, V)
        try:
            ref = torch.empty_like(state)
            B.dg_rhs(ctx, state, ref)
            torch.cuda.synchronize()
        finally:
            B.dg_destroy(ctx)
        refs.append(ref)
        inputs.append((hb, state))
    outs = []
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    for hb, state in inputs:                     # two calls in a row
        out = torch.full_like(state, float("nan"))
        B.dg_rhs_noalloc(cfg, hb, state, out, d_flags=flags)
        outs.append(out)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    for call, (o, r) in enumerate(zip(outs, refs)):
        o = o.cpu().numpy()
        r = r.cpu().numpy()
        assert np.isfinite(o).all()
        # the same kernels on the same inputs: identical bits
        assert np.array_equal(o, r), (call, np.abs(o - r).max())


def test_noalloc_reports_a_dry_state_through_the_flag_word():
    """a bathymetry lowered below the surface (H <= 0 everywhere) sets
    DG_FLAG_DRY in the caller's word; without a word the call still returns
    DG_OK (nothing is read back); a wet state leaves the word at zero"""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = I.waves_p2_512(n=9, p=2, ngauss=1)
    cfg = B.make_config(wl.nx, wl.ny, 2, bc="periodic", precision="fp64")
    for shift, want in ((-40.0, B.DG_FLAG_DRY), (0.0, 0)):
        hb, xi, U, V = _fields(wl, 5, depth_shift=shift)
        state = torch.stack([xi, U, V]).contiguous()
        out = torch.empty_like(state)
        flags = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.dg_rhs_noalloc(cfg, hb, state, out, d_flags=flags)
        B.dg_rhs_noalloc(cfg, hb, state, out)
        torch.cuda.synchronize()
        assert int(flags.item()) & B.DG_FLAG_DRY == want


def test_noalloc_rejects_oversized_mesh():
    cfg = B.make_config(400, 400, 2, bc="periodic")       # 320,000 triangles > 32 MiB
    with pytest.raises(B.DGError) as ei:
        B.dg_rhs_noalloc(cfg, 1, 2, 3)                      # rejected before touching pointers
    assert ei.value.status == B.DG_ERR_ARG
