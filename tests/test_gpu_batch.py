"""Batched instances (one persistent launch per RK stage) against separate
single-instance contexts (bit-identical: the element code is shared) and,
for one instance, against the FP64 oracle."""
import numpy as np
import pytest

from paper_1904_08684_gb300 import binding as B
from paper_1904_08684_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (nx, ny, p, bc): uneven sizes and orders, ragged work items
SPECS = [(7, 5, 3, "periodic"), (12, 9, 1, "reflective"), (5, 6, 2, "periodic"), (11, 13, 2, "reflective"),
         (9, 4, 1, "periodic"), (6, 6, 3, "reflective")]


def _instance(k, nx, ny, p, bc, precision, proj="fp64", tile=0):
    r = I.uniform(100 + k, 6)
    wl = I.Workload("b%d" % k, nx, ny, p, bc, 3, 0.2, 0, precision,
                    hb=I.fourier_bathymetry(12.0, [1.5 * r[0], 1.0 * r[1]], [1, 0], [1, 2], [0, 1]),
                    xi0=I.gaussian_sum([0.02 + 0.05 * r[2]], [0.1], [r[3]], [r[4]], periodic=(bc == "periodic")))
    cfg = B.make_config(nx, ny, p, bc=bc, precision=precision, rk_order=3, cfl=0.2 + 0.1 * r[5],
                        proj_precision=proj, tile_shape=tile)
    Q, E, K = B.dg_proj_num_nodes(p), wl.E, wl.K
    xy = torch.empty((2, Q, E), dtype=torch.float64, device="cuda")
    B.dg_proj_nodes(cfg, xy)
    fields = []
    for f in (wl.hb, wl.xi0, lambda x, y: 0.1 * torch.sin(2 * np.pi * x), lambda x, y: 0.0 * x - 0.05):
        c = torch.empty((K, E), dtype=torch.float64, device="cuda")
        B.dg_project(cfg, f(xy[0], xy[1]).contiguous(), c)
        fields.append(c)
    torch.cuda.synchronize()
    return cfg, fields, E, K


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


@pytest.mark.parametrize("precision,proj", [("fp64", "fp64"), ("fp32", "fp64"), ("fp32", "fp32"), ("fp32", "df64"),
                                             ("fp32", "mixed")])
@pytest.mark.parametrize("tile", [1, -1])
def test_batch_equals_single_contexts(precision, proj, tile):
    """the batched persistent kernel reproduces single contexts bit for bit
    (FP32: tile-fused and per-element kernel forms)"""
    if precision == "fp64" and tile < 0:
        pytest.skip("FP64 has one kernel form")
    inst = [_instance(k, *s, precision, proj, tile=tile) for k, s in enumerate(SPECS)]
    steps = 15
    ref = []
    for cfg, f, E, K in inst:
        ctx = B.dg_init_device(cfg, *f)
        t = B.dg_run(ctx, steps)
        ref.append((B.dg_get_state(ctx, E, K), t))
        B.dg_destroy(ctx)
    b = B.dg_batch_init_device([c for c, *_ in inst], [f[0] for _, f, _, _ in inst], [f[1] for _, f, _, _ in inst],
                        [f[2] for _, f, _, _ in inst], [f[3] for _, f, _, _ in inst])
    try:
        assert B.dg_batch_dofs(b) == sum(3 * K * E for _, _, E, K in inst)
        t = B.dg_batch_run(b, steps)
        for i, (cfg, f, E, K) in enumerate(inst):
            st = B.dg_batch_get_state(b, i, E, K)
            assert t[i] == ref[i][1]
            for a, r in zip(st, ref[i][0]):
                assert np.array_equal(a, r), (i, np.abs(a - r).max())
    finally:
        B.dg_batch_destroy(b)


def test_batch_set_state_resumes_bit_exactly():
    """5 steps, every instance's state and time copied out and into a fresh
    batch, 5 more steps: identical to 10 uninterrupted steps"""
    inst = [_instance(k, *s, "fp32") for k, s in enumerate(SPECS)]
    args = ([c for c, *_ in inst], [f[0] for _, f, _, _ in inst], [f[1] for _, f, _, _ in inst],
            [f[2] for _, f, _, _ in inst], [f[3] for _, f, _, _ in inst])
    b1 = B.dg_batch_init_device(*args)
    b2 = B.dg_batch_init_device(*args)
    try:
        t5 = B.dg_batch_run(b1, 5)
        for i, (_, _, E, K) in enumerate(inst):
            B.dg_batch_set_state(b2, i, *B.dg_batch_get_state(b1, i, E, K), t=float(t5[i]))
        t1 = B.dg_batch_run(b1, 5)
        t2 = B.dg_batch_run(b2, 5)
        assert np.array_equal(t1, t2)
        for i, (_, _, E, K) in enumerate(inst):
            for a, r in zip(B.dg_batch_get_state(b2, i, E, K), B.dg_batch_get_state(b1, i, E, K)):
                assert np.array_equal(a, r)
    finally:
        B.dg_batch_destroy(b1)
        B.dg_batch_destroy(b2)


def test_batch_state_through_page_locked_host_arrays():
    """dg_batch_get_state / dg_batch_set_state with page-locked host arrays
    (in place, one conversion kernel each) agree bit for bit with pageable
    arrays (staged copies), FP32 and FP64 batches; dg_batch_get_states
    (all instances, one synchronisation) returns the same bits"""
    for precision in ("fp32", "fp64"):
        inst = [_instance(k, *s, precision) for k, s in enumerate(SPECS)]
        args = ([c for c, *_ in inst], [f[0] for _, f, _, _ in inst], [f[1] for _, f, _, _ in inst],
                [f[2] for _, f, _, _ in inst], [f[3] for _, f, _, _ in inst])
        b1 = B.dg_batch_init_device(*args)
        b2 = B.dg_batch_init_device(*args)
        try:
            t4 = B.dg_batch_run(b1, 4)
            pinned = []
            for i, (_, _, E, K) in enumerate(inst):
                ref = B.dg_batch_get_state(b1, i, E, K)
                pv = [torch.full((E, K), float("nan"), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
                B.dg_batch_get_state(b1, i, E, K, out=pv)
                for a, r in zip(pv, ref):
                    assert np.array_equal(a, r), (precision, i)
                pinned.append(pv)
                B.dg_batch_set_state(b2, i, *pv, t=float(t4[i]))
            t1 = B.dg_batch_run(b1, 3)
            t2 = B.dg_batch_run(b2, 3)
            assert np.array_equal(t1, t2)
            shapes = [(E, K) for _, _, E, K in inst]
            # every instance at once, into page-locked and into pageable arrays
            for got in (B.dg_batch_get_states(b2, shapes, out=pinned), B.dg_batch_get_states(b2, shapes)):
                for i, (_, _, E, K) in enumerate(inst):
                    for a, r in zip(got[i], B.dg_batch_get_state(b1, i, E, K)):
                        assert np.array_equal(a, r), (precision, i)
        finally:
            B.dg_batch_destroy(b1)
            B.dg_batch_destroy(b2)


@pytest.mark.parametrize("precision,proj", [("fp32", "mixed"), ("fp32", "fp64"), ("fp64", "fp64")])
def test_batch_step_host_matches_set_run_get(precision, proj):
    """dg_batch_step_host (pipelined per order class in the tile-fused FP32
    batch, one group in the per-element ones) gives the bits of
    dg_batch_set_state for every instance + dg_batch_run(b, 1) +
    dg_batch_get_states, over three consecutive steps: page-locked inputs
    with pageable outputs, pageable inputs with the output aliasing them,
    page-locked inputs and outputs (prebuilt HostStates)"""
    inst = [_instance(k, *s, precision, proj) for k, s in enumerate(SPECS)]
    args = ([c for c, *_ in inst], [f[0] for _, f, _, _ in inst], [f[1] for _, f, _, _ in inst],
            [f[2] for _, f, _, _ in inst], [f[3] for _, f, _, _ in inst])
    shapes = [(E, K) for _, _, E, K in inst]
    b1 = B.dg_batch_init_device(*args)
    b2 = B.dg_batch_init_device(*args)

    def pinned_copy(states):
        return [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in st] for st in states]
    try:
        B.dg_batch_run(b1, 2)
        B.dg_batch_run(b2, 2)
        ref = B.dg_batch_get_states(b1, shapes)
        cur2 = pinned_copy(ref)
        for step in range(3):
            tnow = B.dg_batch_run(b1, 0)
            for i in range(len(inst)):
                B.dg_batch_set_state(b1, i, *ref[i], t=float(tnow[i]))
            t1 = B.dg_batch_run(b1, 1)
            ref = B.dg_batch_get_states(b1, shapes)
            if step == 0:
                got, t2 = B.dg_batch_step_host(b2, shapes, cur2)
            elif step == 1:
                got, t2 = B.dg_batch_step_host(b2, shapes, cur2, out=cur2)
            else:
                got, t2 = B.dg_batch_step_host(b2, shapes, B.HostStates(shapes, pinned_copy(cur2)),
                                               out=B.HostStates(shapes, pinned=True))
            assert np.array_equal(t1, t2), (step, t1, t2)
            for i in range(len(inst)):
                for a, r in zip(got[i], ref[i]):
                    assert np.array_equal(a, r), (precision, proj, step, i)
            cur2 = [[np.array(a) for a in st] for st in got]
    finally:
        B.dg_batch_destroy(b1)
        B.dg_batch_destroy(b2)


@pytest.mark.parametrize("tile", [1, -1])
def test_batch_autotune_keeps_state(tile):
    """the autotuner (tile shapes of a tile-fused batch, elements per work
    item of a per-element batch) leaves state and times as they were"""
    inst = [_instance(k, *s, "fp32", tile=tile) for k, s in enumerate(SPECS)]
    args = ([c for c, *_ in inst], [f[0] for _, f, _, _ in inst], [f[1] for _, f, _, _ in inst],
            [f[2] for _, f, _, _ in inst], [f[3] for _, f, _, _ in inst])
    b1 = B.dg_batch_init_device(*args)
    b2 = B.dg_batch_init_device(*args)
    try:
        t1 = B.dg_batch_run(b1, 5)
        blk, ms = B.dg_batch_autotune(b2, 2)
        if tile >= 0:
            assert blk in (1, 2, 3) and (ms[:3] > 0).all() and ms[3] == 0
        else:
            assert blk in (32, 64, 96, 128) and (ms > 0).all()
        t2 = B.dg_batch_run(b2, 5)
        assert np.array_equal(t1, t2)
        for i, (_, _, E, K) in enumerate(inst):
            for a, r in zip(B.dg_batch_get_state(b2, i, E, K), B.dg_batch_get_state(b1, i, E, K)):
                assert np.array_equal(a, r)
        for blk in ((2, 3) if tile >= 0 else (32, 96)):
            B.dg_batch_set_block(b1, blk)
            B.dg_batch_run(b1, 1)
        with pytest.raises(B.DGError):
            B.dg_batch_set_block(b1, 64 if tile >= 0 else 2)   # a shape of the other kernel form
    finally:
        B.dg_batch_destroy(b1)
        B.dg_batch_destroy(b2)


def test_batch_instance_matches_oracle(oracle_mod):
    """one FP64 batch instance against the oracle (20 steps, <= 1e-12)."""
    nx, ny, p, bc = SPECS[3]
    o = oracle_mod.Oracle(nx, ny, p, bc=bc, rk_order=3, cfl=0.25)
    wl = I.waves_p2_512(n=nx, p=p, ngauss=2)
    hb = o.project_hb(wl.hb)
    xi = o.project(wl.xi0)
    U = o.project(lambda x, y: 0.2 + 0.1 * np.cos(2 * np.pi * y))
    V = np.zeros_like(xi)
    xr, Ur, Vr, tr, _ = o.run(hb, xi, U, V, 20)
    cfg = B.make_config(nx, ny, p, bc=bc, precision="fp64", rk_order=3, cfl=0.25)
    dev = [torch.tensor(a.T.copy(), dtype=torch.float64, device="cuda").contiguous() for a in (hb, xi, U, V)]
    other = _instance(0, *SPECS[0], "fp64")
    b = B.dg_batch_init_device([other[0], cfg], [other[1][0], dev[0]], [other[1][1], dev[1]],
                        [other[1][2], dev[2]], [other[1][3], dev[3]])
    try:
        t = B.dg_batch_run(b, 20)
        xg, Ug, Vg = B.dg_batch_get_state(b, 1, o.E, o.K)
    finally:
        B.dg_batch_destroy(b)
    assert abs(t[1] - tr) <= 1e-13 * tr
    for g_, r_ in ((xg, xr), (Ug, Ur), (Vg, Vr)):
        assert np.linalg.norm(g_ - r_) <= 1e-12 * np.linalg.norm(r_)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_host_and_device_forms_identical(precision):
    """dg_batch_init from host FP64 AoS arrays (the §8(b) form) and
    dg_batch_init_device from device SoA arrays build the same batch: after
    10 steps every instance's state and time agree bit for bit"""
    inst = [_instance(k, *s, precision) for k, s in enumerate(SPECS)]
    cfgs = [c for c, *_ in inst]
    dev = [[f[k] for _, f, _, _ in inst] for k in range(4)]
    host = [[f[k].t().contiguous().cpu().numpy() for _, f, _, _ in inst] for k in range(4)]
    b1 = B.dg_batch_init_device(cfgs, *dev)
    b2 = B.dg_batch_init(cfgs, *host)
    try:
        t1 = B.dg_batch_run(b1, 10)
        t2 = B.dg_batch_run(b2, 10)
        assert np.array_equal(t1, t2)
        for i, (_, _, E, K) in enumerate(inst):
            for a, r in zip(B.dg_batch_get_state(b2, i, E, K), B.dg_batch_get_state(b1, i, E, K)):
                assert np.array_equal(a, r)
    finally:
        B.dg_batch_destroy(b1)
        B.dg_batch_destroy(b2)
