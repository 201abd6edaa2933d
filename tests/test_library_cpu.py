"""CPU-side checks of the C-ABI library: it builds, loads and exports every
entry point declared in include/dgswe.h; argument validation needs no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dgswe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1904_08684_gb300 import binding
    return binding.load()


def test_header_lists_the_abi():
    names = _declared()
    for n in ("dg_init", "dg_rhs", "dg_rk_step", "dg_run"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1904_08684_gb300 import binding
    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(dg_[a-z_0-9]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    assert set(binding.EXPORTS) <= exported
    for n in _declared():
        assert hasattr(lib, n)


def test_counts_and_status_strings(lib):
    from paper_1904_08684_gb300 import binding as B
    assert [B.dg_num_basis(p) for p in range(5)] == [1, 3, 6, 10, 15]
    assert B.dg_num_basis(5) == 0
    # h_b lives in P^max(p,1)
    assert [B.dg_num_basis_bathymetry(p) for p in range(6)] == [3, 3, 6, 10, 15, 0]
    assert B.dg_num_elements(B.make_config(7, 5, 2)) == 70
    assert B.dg_proj_num_nodes(2) == 25
    assert B.dg_status_str(B.DG_ERR_DRY) == "DG_ERR_DRY"
    assert B.dg_status_str(99) == "DG_ERR_UNKNOWN"


def test_config_struct_layout(lib):
    from paper_1904_08684_gb300 import binding as B
    # int,int | 4 double | ptr | int(+pad) | double | 3 int(+pad) | 2 double | 2 int | 2 double
    assert ctypes.sizeof(B.dg_config) == 128
    assert B.dg_config.g.offset == 56 and B.dg_config.cfl.offset == 80 and B.dg_config.tau_bf.offset == 104


@pytest.mark.parametrize("bad", [dict(nx=0), dict(p=5), dict(rk_order=4), dict(Lx=-1.0),
                                 dict(cfl=0.0, dt=0.0), dict(block_size=33)])
def test_invalid_configs_rejected_without_gpu(lib, bad):
    """Validation happens before any CUDA call, so these run on a CPU host."""
    from paper_1904_08684_gb300 import binding as B
    kw = dict(nx=4, ny=4, p=1, bc="periodic")
    kw.update(bad)
    cfg = B.make_config(**kw)
    h = ctypes.c_void_p()
    z = (ctypes.c_double * 1)()
    assert B.load().dg_init(ctypes.byref(cfg), z, z, z, z, None, ctypes.byref(h)) == B.DG_ERR_ARG
    assert B.load().dg_init(None, z, z, z, z, None, ctypes.byref(h)) == B.DG_ERR_ARG


def test_unsupported_configs(lib):
    import numpy as np
    from paper_1904_08684_gb300 import binding as B
    for kw in (dict(bc="dirichlet"), dict(bc="periodic", vertex_xy=np.zeros((25, 2)))):
        base = dict(nx=4, ny=4, p=1, bc="periodic")
        base.update(kw)
        cfg = B.make_config(**base)
        n = B.dg_num_elements(cfg) * B.dg_num_basis(cfg.p)
        z = np.zeros(n)
        with pytest.raises(B.DGError) as ei:
            B.dg_init(cfg, z, z, z, z)
        assert ei.value.status == B.DG_ERR_UNSUPPORTED


def test_batch_rejects_mixed_or_unsupported_without_gpu(lib):
    """Batch validation runs before any CUDA call."""
    from paper_1904_08684_gb300 import binding as B
    a = B.make_config(4, 4, 2, precision="fp64")
    b = B.make_config(4, 4, 1, precision="fp32")
    c = B.make_config(4, 4, 4)
    one = [1, 1]
    with pytest.raises(B.DGError) as ei:
        B.dg_batch_init_device([a, b], one, one, one, one)
    assert ei.value.status == B.DG_ERR_ARG
    for unsupported in (c, B.make_config(4, 4, 0)):      # the batched kernel holds p = 1..3
        with pytest.raises(B.DGError) as ei:
            B.dg_batch_init_device([unsupported], [1], [1], [1], [1])
        assert ei.value.status == B.DG_ERR_UNSUPPORTED
    with pytest.raises(B.DGError) as ei:
        B.dg_batch_init_device([], [], [], [], [])
    assert ei.value.status == B.DG_ERR_ARG


def test_batch_host_form_validates_before_any_gpu_work(lib):
    """dg_batch_init (host FP64 AoS arrays, the §8(b) form) applies the same
    checks as the device form before touching any array or the GPU"""
    from paper_1904_08684_gb300 import binding as B
    L = B.load()
    dp = ctypes.POINTER(ctypes.c_double)
    fake = ctypes.cast(ctypes.c_void_p(0x1000), dp)          # never dereferenced

    def call(cfgs, ptrs=None, n=None):
        n = len(cfgs) if n is None else n
        carr = (B.dg_config * max(1, len(cfgs)))(*cfgs)
        arrs = []
        for _ in range(4):
            a = (dp * max(1, len(cfgs)))()
            for k in range(len(cfgs)):
                a[k] = fake if ptrs is None else ptrs[k]
            arrs.append(a)
        h = ctypes.c_void_p()
        return L.dg_batch_init(n, carr, *arrs, None, ctypes.byref(h)), h
    a = B.make_config(4, 4, 2, precision="fp64")
    b = B.make_config(4, 4, 1, precision="fp32")
    assert call([a, b])[0] == B.DG_ERR_ARG                   # mixed precisions
    assert call([B.make_config(4, 4, 4)])[0] == B.DG_ERR_UNSUPPORTED
    assert call([B.make_config(4, 4, 0)])[0] == B.DG_ERR_UNSUPPORTED
    assert call([B.make_config(4, 4, 1, bc="dirichlet", forcing=1)])[0] == B.DG_ERR_UNSUPPORTED
    assert call([a], n=0)[0] == B.DG_ERR_ARG
    st, h = call([a], ptrs=[ctypes.cast(None, dp)])             # NULL field array
    assert st == B.DG_ERR_ARG and not h.value
    h = ctypes.c_void_p()
    assert L.dg_batch_init(1, ctypes.byref(a), None, None, None, None, None, ctypes.byref(h)) == B.DG_ERR_ARG


def test_plain_c_program_uses_the_abi(lib, tmp_path):
    """include/dgswe.h is valid C99 on its own, and a C program links the
    library and gets the documented answers from the host-side calls"""
    import shutil
    import subprocess
    from paper_1904_08684_gb300 import build as BLD
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    here = os.path.dirname(os.path.abspath(__file__))
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.dirname(BLD.LIB)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", BLD.INCLUDE,
                           os.path.join(here, "c_abi_check.c"), "-L", libdir, "-ldgswe",
                           "-Wl,-rpath," + libdir, "-o", exe])
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0 and res.stdout.strip() == "OK", (res.stdout, res.stderr)


@pytest.mark.parametrize("bad,status", [
    (dict(tau_bf=-1.0), "ARG"), (dict(tau_bf=float("nan")), "ARG"), (dict(f_c=float("inf")), "ARG"),
    (dict(p=5), "ARG"), (dict(bc="dirichlet"), "ARG"), (dict(nx=1, ny=1, bc="periodic"), "ARG"),
    (dict(block_size=48), "ARG"), (dict(forcing=1), "UNSUPPORTED"),
    (dict(precision="fp32", proj_precision="df64", p=4), "UNSUPPORTED"),
    (dict(nx=8000, ny=8000), "ARG"),            # beyond the entry point's mesh limit
    (dict(nx=200, ny=200, p=2), "ARG"),         # 80,000 FP64 triangles: beyond the fixed array
])
def test_noalloc_rhs_rejects_before_any_gpu_work(lib, bad, status):
    """the allocation-free RHS validates its configuration and checks that
    the mesh fits its fixed array before any CUDA call (so on a CPU host)"""
    from paper_1904_08684_gb300 import binding as B
    kw = dict(nx=4, ny=4, p=1, bc="periodic")
    kw.update(bad)
    cfg = B.make_config(**kw)
    fake = [ctypes.c_void_p(0x1000 * (k + 1)) for k in range(3)]   # never dereferenced
    got = B.load().dg_rhs_noalloc(ctypes.byref(cfg), fake[0], fake[1], fake[2], None, None)
    assert got == getattr(B, "DG_ERR_" + status)
    # the same pointer as input and output is refused
    ok_cfg = B.make_config(4, 4, 1)
    assert B.load().dg_rhs_noalloc(ctypes.byref(ok_cfg), fake[0], fake[1], fake[1], None, None) == B.DG_ERR_ARG


def test_null_handles_are_rejected(lib):
    """every entry point taking a context or batch refuses NULL on the host"""
    from paper_1904_08684_gb300 import binding as B
    L = B.load()
    d = ctypes.c_double()
    p = ctypes.c_void_p(0x1000)
    assert L.dg_rhs(None, p, ctypes.c_void_p(0x2000)) == B.DG_ERR_ARG
    assert L.dg_run(None, 1, ctypes.byref(d)) == B.DG_ERR_ARG
    assert L.dg_rk_step(None, ctypes.byref(d)) == B.DG_ERR_ARG
    assert L.dg_get_state(None, None, None, None) == B.DG_ERR_ARG
    assert L.dg_set_state(None, None, None, None, 0.0) == B.DG_ERR_ARG
    assert L.dg_diagnostics(None, ctypes.byref(d), ctypes.byref(d)) == B.DG_ERR_ARG
    assert L.dg_state_device(None, ctypes.byref(ctypes.c_void_p())) == B.DG_ERR_ARG
    assert L.dg_batch_run(None, 1, None) == B.DG_ERR_ARG
    assert L.dg_batch_set_block(None, 64) == B.DG_ERR_ARG
    assert L.dg_batch_get_state(None, 0, None, None, None) == B.DG_ERR_ARG
    assert L.dg_batch_get_states(None, None, None, None) == B.DG_ERR_ARG
    assert L.dg_batch_step_host(None, None, None, None, None, None, None, None) == B.DG_ERR_ARG
    assert L.dg_batch_set_state(None, 0, None, None, None, 0.0) == B.DG_ERR_ARG
    assert L.dg_batch_autotune(None, 1, None, None) == B.DG_ERR_ARG
    assert L.dg_batch_dofs(None) == 0
    assert L.dg_batch_tile_shape(None, 3) == 0
    L.dg_destroy(None)
    L.dg_batch_destroy(None)


def test_friction_must_be_a_finite_nonnegative_number(lib):
    from paper_1904_08684_gb300 import binding as B
    z = (ctypes.c_double * 1)()
    h = ctypes.c_void_p()
    for kw in (dict(tau_bf=-0.1), dict(tau_bf=float("nan")), dict(f_c=float("nan"))):
        cfg = B.make_config(4, 4, 1, **kw)
        assert B.load().dg_init(ctypes.byref(cfg), z, z, z, z, None, ctypes.byref(h)) == B.DG_ERR_ARG


def test_tile_shape_is_validated(lib):
    """dg_config.tile_shape outside -1..3 is refused before any CUDA call"""
    from paper_1904_08684_gb300 import binding as B
    z = (ctypes.c_double * 1)()
    h = ctypes.c_void_p()
    for bad in (-2, 4):
        cfg = B.make_config(4, 4, 1, precision="fp32", tile_shape=bad)
        assert B.load().dg_init(ctypes.byref(cfg), z, z, z, z, None, ctypes.byref(h)) == B.DG_ERR_ARG


def test_kernel_source_fingerprint_ignores_comments_only():
    """the fingerprint that ties measured DRAM traffic to the kernel sources
    is unchanged by comment and blank-line edits and changed by any code
    edit (including one inside a line that also holds a comment)"""
    from paper_1904_08684_gb300 import flops as FL
    base = {n: "" for n in FL.KERNEL_SOURCES}
    base["dg_tile.cuh"] = 'int a = 1;  // one\n/* block\n comment */\nconst char* s = "// not a comment";\n'
    h0 = FL.source_hash(lambda n: base[n])
    cmt = dict(base, **{"dg_tile.cuh": 'int a = 1;  // other words\n\n/* x */\nconst char* s = "// not a comment";\n'})
    assert FL.source_hash(lambda n: cmt[n]) == h0
    code = dict(base, **{"dg_tile.cuh": 'int a = 2;  // one\n/* block\n comment */\nconst char* s = "// not a comment";\n'})
    assert FL.source_hash(lambda n: code[n]) != h0
    lit = dict(base, **{"dg_tile.cuh": 'int a = 1;  // one\n/* block\n comment */\nconst char* s = "// changed";\n'})
    assert FL.source_hash(lambda n: lit[n]) != h0
    py = dict(base, **{"gen_tables.py": "# a comment\n"})
    assert FL.source_hash(lambda n: py[n]) != h0        # non-C files are hashed verbatim
