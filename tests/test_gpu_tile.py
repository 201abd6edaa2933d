"""The tile-fused FP32 stage kernels (tile_shape 1, 2, 3: tiles of 8 x 8,
16 x 8 and 8 x 4 quads evaluating each stage's input in shared memory, with
the neighbours across the tile boundary recomputed as a halo; the default
0 takes 8 x 8 tiles at p <= 3).

* Every tile shape gives the same bits: the per-element arithmetic does not
  depend on which thread or tile computes it, a halo triangle's side record
  included.
* The tile kernels and the per-element kernels (tile_shape -1, side records
  through HBM) agree to FP32 rounding.
* The tile path follows the FP64 oracle within the FP32 bar.
Meshes are ragged on purpose: partial tiles, meshes smaller than one tile
(the periodic neighbour of a tile-boundary triangle lies in the same tile),
a single column of quads between walls.
"""
import numpy as np
import pytest

from paper_1904_08684_gb300 import binding as B
from paper_1904_08684_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [(13, 11, "periodic"), (10, 9, "reflective"), (3, 2, "periodic"), (9, 17, "periodic"),
         (1, 5, "reflective"), (17, 4, "reflective")]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


def _relL2(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def _inputs(oracle_mod, nx, ny, p, bc):
    o = oracle_mod.Oracle(nx, ny, p, bc=bc, rk_order=3, cfl=0.2)
    periodic = bc == "periodic"
    hb = o.project_hb(lambda x, y: 10 + 2 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))
    xi = o.project(I.gaussian_sum([0.08], [0.15], [0.4], [0.55], periodic=periodic))
    if periodic:
        U = o.project(lambda x, y: 0.3 + 0.2 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))
        V = o.project(lambda x, y: -0.2 + 0.1 * np.cos(2 * np.pi * (x + y)))
    else:
        U = o.project(lambda x, y: 0.2 * np.sin(np.pi * x) * np.sin(np.pi * y))
        V = o.project(lambda x, y: -0.1 * np.sin(np.pi * x) * np.sin(2 * np.pi * y))
    return o, (hb, xi, U, V)


def _run(nx, ny, p, bc, fields, steps, tile, proj="fp64"):
    cfg = B.make_config(nx, ny, p, bc=bc, precision="fp32", rk_order=3, cfl=0.2, proj_precision=proj,
                        tile_shape=tile)
    ctx = B.dg_init(cfg, *fields)
    try:
        t = B.dg_run(ctx, steps)
        st = B.dg_get_state(ctx, 2 * nx * ny, B.dg_num_basis(p))
    finally:
        B.dg_destroy(ctx)
    return t, st


@pytest.mark.parametrize("p,proj", [(0, "fp64"), (1, "fp64"), (2, "mixed"), (3, "mixed"), (3, "fp64"),
                                    (2, "df64"), (4, "mixed"), (1, "fp32")])
def test_tile_shapes_give_identical_bits(oracle_mod, p, proj):
    for nx, ny, bc in SIZES:
        if bc == "periodic" and min(nx, ny) < 2:
            continue
        _, fields = _inputs(oracle_mod, nx, ny, p, bc)
        ref = _run(nx, ny, p, bc, fields, 12, 1, proj)
        for shape in (2, 3):
            got = _run(nx, ny, p, bc, fields, 12, shape, proj)
            assert got[0] == ref[0], (nx, ny, bc, shape)
            for a, r in zip(got[1], ref[1]):
                assert np.array_equal(a, r), (nx, ny, bc, shape, np.abs(a - r).max())


@pytest.mark.parametrize("p,proj", [(0, "fp64"), (1, "fp64"), (2, "fp64"), (2, "mixed"), (3, "mixed"),
                                    (4, "fp64")])
def test_tile_and_per_element_kernels_agree(oracle_mod, p, proj):
    """the same scheme through two kernel forms: equal to FP32 rounding
    (20 steps, relative L2 <= 2e-6 per field, same time to 1e-6)"""
    for nx, ny, bc in SIZES[:4]:
        _, fields = _inputs(oracle_mod, nx, ny, p, bc)
        t1, a = _run(nx, ny, p, bc, fields, 20, 1, proj)
        t2, b = _run(nx, ny, p, bc, fields, 20, -1, proj)
        assert abs(t1 - t2) <= 1e-6 * t2
        for x, y in zip(a, b):
            assert _relL2(x, y) <= 2e-6, (nx, ny, bc, _relL2(x, y))


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_tile_run_matches_oracle(oracle_mod, p):
    """FP32 tile path (mixed solve; p = 0 and 4 with the FP64 solve too)
    against the FP64 oracle after 60 SSP-RK3 steps: relative L2 <= 1e-5
    per field on a ragged periodic and a ragged reflective mesh"""
    for nx, ny, bc in (SIZES[0], SIZES[1]):
        o, fields = _inputs(oracle_mod, nx, ny, p, bc)
        xr, Ur, Vr, tr, _ = o.run(*fields, 60)
        for proj in (("mixed", "fp64") if p in (0, 4) else ("mixed",)):
            t, (xg, Ug, Vg) = _run(nx, ny, p, bc, fields, 60, 1, proj)
            assert abs(t - tr) <= 1e-6 * tr
            for g_, r_ in ((xg, xr), (Ug, Ur), (Vg, Vr)):
                assert _relL2(g_, r_) <= 1e-5, (nx, ny, bc, proj, _relL2(g_, r_))


def test_tile_lake_at_rest():
    """constant elevation over flat bathymetry, q = 0, 50 steps.  With
    xi = 0 every flux vanishes identically: the state stays exactly at rest.
    With xi = 0.25 the constant pressure flux and the volume term cancel
    only to FP32 rounding: drift <= 1e-6 in xi and 1e-5 in q, the level of
    the per-element kernels on the same state."""
    nx, ny, p = 11, 9, 2
    K, E = B.dg_num_basis(p), 2 * nx * ny
    hb = np.zeros((E, K))
    hb[:, 0] = 10.0 / np.sqrt(2.0)
    z = np.zeros((E, K))
    for bc in ("periodic", "reflective"):
        t, (x1, U1, V1) = _run(nx, ny, p, bc, (hb, z, z, z), 50, 1, "mixed")
        assert t > 0 and not x1.any() and not U1.any() and not V1.any()
        xi = np.zeros((E, K))
        xi[:, 0] = 0.25 / np.sqrt(2.0)
        x0 = np.float32(xi).astype(np.float64)
        for tile in (1, -1):
            t, (x1, U1, V1) = _run(nx, ny, p, bc, (hb, xi, z, z), 50, tile, "mixed")
            assert np.abs(x1 - x0).max() <= 1e-6, (bc, tile, np.abs(x1 - x0).max())
            assert np.abs(U1).max() <= 1e-5 and np.abs(V1).max() <= 1e-5, (bc, tile)


def test_default_kernel_form(oracle_mod):
    """tile_shape 0 takes 8 x 8 tiles with the mixed and FP32 solves at
    p <= 3, 8 x 4 tiles with the FP32 solve at p = 4 and the per-element
    kernels otherwise: identical bits to the explicit choice in each case"""
    nx, ny, bc = SIZES[0]
    for p, proj, explicit in ((2, "mixed", 1), (3, "fp32", 1), (2, "fp64", -1), (3, "df64", -1), (4, "mixed", -1),
                              (4, "fp32", 3)):
        _, fields = _inputs(oracle_mod, nx, ny, p, bc)
        t0, a = _run(nx, ny, p, bc, fields, 8, 0, proj)
        t1, b = _run(nx, ny, p, bc, fields, 8, explicit, proj)
        assert t0 == t1, (p, proj)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), (p, proj)
