"""Thin ctypes binding of libdgswe (include/dgswe.h): same names, argument
marshalling only.  Every computation runs in the library's CUDA kernels; if
the library is missing this module raises instead of falling back.

Host arrays are numpy float64, element-major (E, K).  Device arrays are
torch CUDA tensors (or raw integer device pointers) in the library's SoA
layout: state (3, K, E), single fields (K, E).
"""
import ctypes
import os

import numpy as np

from . import build as _build

DG_OK, DG_ERR_ARG, DG_ERR_UNSUPPORTED, DG_ERR_OOM, DG_ERR_CUDA, DG_ERR_DRY, DG_ERR_NONFINITE, DG_ERR_TIMEOUT = range(8)
DG_BC_PERIODIC, DG_BC_REFLECTIVE, DG_BC_DIRICHLET = 0, 1, 2
DG_PREC_FP64, DG_PREC_FP32_MIXED = 0, 1
DG_PROJ_FP64, DG_PROJ_FP32, DG_PROJ_DF64, DG_PROJ_MIXED = 0, 1, 2, 3
PROJ = {"fp64": DG_PROJ_FP64, "fp32": DG_PROJ_FP32, "df64": DG_PROJ_DF64, "mixed": DG_PROJ_MIXED}

BC = {"periodic": DG_BC_PERIODIC, "reflective": DG_BC_REFLECTIVE, "dirichlet": DG_BC_DIRICHLET}
PREC = {"fp64": DG_PREC_FP64, "fp32": DG_PREC_FP32_MIXED}

# every entry point declared in include/dgswe.h
EXPORTS = ["dg_num_basis", "dg_num_basis_bathymetry", "dg_num_elements", "dg_init", "dg_init_device", "dg_rhs", "dg_rk_step", "dg_run",
           "dg_get_state", "dg_set_state", "dg_state_device", "dg_diagnostics", "dg_proj_num_nodes",
           "dg_proj_nodes", "dg_project", "dg_destroy", "dg_status_str", "dg_rhs_noalloc",
           "dg_batch_init", "dg_batch_init_device", "dg_batch_run", "dg_batch_get_state", "dg_batch_get_states", "dg_batch_set_state", "dg_batch_step_host",
           "dg_batch_autotune",
           "dg_batch_set_block", "dg_batch_tile_shape", "dg_batch_dofs", "dg_batch_destroy"]


class DGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s" % (where, _status_name(status)))


class dg_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
                ("vertex_xy", ctypes.POINTER(ctypes.c_double)),
                ("p", ctypes.c_int), ("g", ctypes.c_double),
                ("bc", ctypes.c_int), ("precision", ctypes.c_int), ("rk_order", ctypes.c_int),
                ("cfl", ctypes.c_double), ("dt", ctypes.c_double),
                ("proj_precision", ctypes.c_int), ("block_size", ctypes.c_int),
                ("tau_bf", ctypes.c_double), ("f_c", ctypes.c_double), ("forcing", ctypes.c_int),
                ("tile_shape", ctypes.c_int)]


def make_config(nx, ny, p, bc="periodic", precision="fp64", rk_order=3, cfl=0.2, dt=0.0, g=9.81,
                x0=0.0, y0=0.0, Lx=1.0, Ly=1.0, proj_precision="fp64", block_size=0, tau_bf=0.0, f_c=0.0,
                vertex_xy=None, forcing=0, tile_shape=0):
    vxy = None
    if vertex_xy is not None:
        _keep = np.ascontiguousarray(vertex_xy, dtype=np.float64).ravel()
        vxy = _keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg = dg_config(nx, ny, x0, y0, Lx, Ly, vxy, p, g,
                     BC[bc] if isinstance(bc, str) else int(bc),
                     PREC[precision] if isinstance(precision, str) else int(precision),
                     rk_order, cfl, dt,
                     PROJ[proj_precision] if isinstance(proj_precision, str) else int(proj_precision), block_size,
                     float(tau_bf), float(f_c), int(forcing), int(tile_shape))
    if vertex_xy is not None:
        cfg._vertex_keep = _keep   # keep the vertex array alive with the struct
    return cfg


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libdgswe.so (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build_library()
    if not os.path.exists(path):
        raise RuntimeError("libdgswe.so is not built (%s); run paper_1904_08684_gb300.build" % path)
    lib = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    cp = ctypes.POINTER(dg_config)
    lib.dg_num_basis.argtypes = [ctypes.c_int]
    lib.dg_num_basis_bathymetry.argtypes = [ctypes.c_int]
    lib.dg_num_elements.argtypes = [cp]
    lib.dg_num_elements.restype = ctypes.c_longlong
    lib.dg_init.argtypes = [cp, dp, dp, dp, dp, vp, ctypes.POINTER(vp)]
    lib.dg_init_device.argtypes = [cp, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]
    lib.dg_rhs.argtypes = [vp, vp, vp]
    lib.dg_rk_step.argtypes = [vp, dp]
    lib.dg_run.argtypes = [vp, ctypes.c_int, dp]
    lib.dg_get_state.argtypes = [vp, dp, dp, dp]
    lib.dg_set_state.argtypes = [vp, dp, dp, dp, ctypes.c_double]
    lib.dg_state_device.argtypes = [vp, ctypes.POINTER(vp)]
    lib.dg_diagnostics.argtypes = [vp, dp, dp]
    lib.dg_proj_num_nodes.argtypes = [ctypes.c_int]
    lib.dg_proj_nodes.argtypes = [cp, vp, vp]
    lib.dg_project.argtypes = [cp, vp, vp, vp]
    lib.dg_rhs_noalloc.argtypes = [cp, vp, vp, vp, vp, vp]
    vpp = ctypes.POINTER(ctypes.c_void_p)
    dpp = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))
    lib.dg_batch_init.argtypes = [ctypes.c_int, cp, dpp, dpp, dpp, dpp, vp, ctypes.POINTER(vp)]
    lib.dg_batch_init_device.argtypes = [ctypes.c_int, cp, vpp, vpp, vpp, vpp, vp, ctypes.POINTER(vp)]
    lib.dg_batch_run.argtypes = [vp, ctypes.c_int, dp]
    lib.dg_batch_get_state.argtypes = [vp, ctypes.c_int, dp, dp, dp]
    lib.dg_batch_get_states.argtypes = [vp, dpp, dpp, dpp]
    lib.dg_batch_step_host.argtypes = [vp, vpp, vpp, vpp, vpp, vpp, vpp, dp]
    lib.dg_batch_set_state.argtypes = [vp, ctypes.c_int, dp, dp, dp, ctypes.c_double]
    lib.dg_batch_autotune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]
    lib.dg_batch_set_block.argtypes = [vp, ctypes.c_int]
    lib.dg_batch_tile_shape.argtypes = [vp, ctypes.c_int]
    lib.dg_batch_dofs.argtypes = [vp]
    lib.dg_batch_dofs.restype = ctypes.c_longlong
    lib.dg_batch_destroy.argtypes = [vp]
    lib.dg_batch_destroy.restype = None
    lib.dg_destroy.argtypes = [vp]
    lib.dg_destroy.restype = None
    lib.dg_status_str.argtypes = [ctypes.c_int]
    lib.dg_status_str.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _status_name(s):
    try:
        return load(False).dg_status_str(s).decode()
    except Exception:  # library not loadable: numeric code only
        return "status %d" % s


def _check(s, where):
    if s != DG_OK:
        raise DGError(s, where)


def _dptr(x):
    """device pointer of a torch tensor or an int"""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return ctypes.c_void_p(x.data_ptr())


def _hptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _host(a, E, K):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != E * K:
        raise ValueError("expected %d x %d coefficients, got shape %s" % (E, K, a.shape))
    return a


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- entry points
def dg_num_basis(p):
    return load().dg_num_basis(int(p))


def dg_num_basis_bathymetry(p):
    return load().dg_num_basis_bathymetry(int(p))


def dg_num_elements(cfg):
    return load().dg_num_elements(ctypes.byref(cfg))


def dg_init(cfg, hb, xi, qx, qy, stream=None):
    """Context from host FP64 arrays, hb (E, Kb) and the state (E, K);
    returns an opaque handle."""
    lib = load()
    E, K, Kb = dg_num_elements(cfg), dg_num_basis(cfg.p), dg_num_basis_bathymetry(cfg.p)
    arrs = [_host(hb, E, Kb)] + [_host(a, E, K) for a in (xi, qx, qy)]
    h = ctypes.c_void_p()
    _check(lib.dg_init(ctypes.byref(cfg), *[_hptr(a) for a in arrs], _stream(stream), ctypes.byref(h)),
           "dg_init")
    return h


def dg_init_device(cfg, d_hb, d_xi, d_qx, d_qy, stream=None):
    """Context from device FP64 (K, E) arrays."""
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.dg_init_device(ctypes.byref(cfg), _dptr(d_hb), _dptr(d_xi), _dptr(d_qx), _dptr(d_qy),
                              _stream(stream), ctypes.byref(h)), "dg_init_device")
    return h


def dg_rhs(ctx, d_state_in, d_rhs_out):
    _check(load().dg_rhs(ctx, _dptr(d_state_in), _dptr(d_rhs_out)), "dg_rhs")


def dg_rk_step(ctx, want_dt=False):
    dt = ctypes.c_double(0.0)
    _check(load().dg_rk_step(ctx, ctypes.byref(dt) if want_dt else None), "dg_rk_step")
    return dt.value if want_dt else None


def dg_run(ctx, nsteps):
    t = ctypes.c_double(0.0)
    _check(load().dg_run(ctx, int(nsteps), ctypes.byref(t)), "dg_run")
    return t.value


def dg_get_state(ctx, E, K, out=None):
    """state as three host (E, K) FP64 arrays (written into ``out`` if given,
    e.g. page-locked buffers)"""
    if out is None:
        out = [np.zeros((E, K)) for _ in range(3)]
    for a in out:
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != E * K:
            raise ValueError("out arrays must be contiguous float64 of %d x %d" % (E, K))
    _check(load().dg_get_state(ctx, *[_hptr(a) for a in out]), "dg_get_state")
    return out


def dg_set_state(ctx, xi, qx, qy, t=0.0):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (xi, qx, qy)]
    _check(load().dg_set_state(ctx, *[_hptr(a) for a in arrs], float(t)), "dg_set_state")


def dg_state_device(ctx):
    p = ctypes.c_void_p()
    _check(load().dg_state_device(ctx, ctypes.byref(p)), "dg_state_device")
    return p.value


def dg_diagnostics(ctx):
    m, e = ctypes.c_double(), ctypes.c_double()
    _check(load().dg_diagnostics(ctx, ctypes.byref(m), ctypes.byref(e)), "dg_diagnostics")
    return m.value, e.value


def dg_proj_num_nodes(p):
    return load().dg_proj_num_nodes(int(p))


def dg_proj_nodes(cfg, d_xy, stream=None):
    _check(load().dg_proj_nodes(ctypes.byref(cfg), _dptr(d_xy), _stream(stream)), "dg_proj_nodes")


def dg_project(cfg, d_vals, d_coef, stream=None):
    _check(load().dg_project(ctypes.byref(cfg), _dptr(d_vals), _dptr(d_coef), _stream(stream)), "dg_project")


DG_FLAG_DRY = 1


def dg_rhs_noalloc(cfg, d_hb, d_state_in, d_rhs_out, d_flags=None, stream=None):
    """dg_rhs without device allocation (fixed in-library scratch array);
    d_flags: None or a device int32 word the call ORs DG_FLAG_DRY into."""
    _check(load().dg_rhs_noalloc(ctypes.byref(cfg), _dptr(d_hb), _dptr(d_state_in), _dptr(d_rhs_out),
                                 _dptr(d_flags), _stream(stream)), "dg_rhs_noalloc")


def _ptr_array(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for k, t in enumerate(ts):
        arr[k] = t if isinstance(t, int) else t.data_ptr()
    return arr


def dg_batch_init(cfgs, hb, xi, qx, qy, stream=None):
    """Batch of instances from host FP64 (E_i, K_i) arrays (lists)."""
    n = len(cfgs)
    carr = (dg_config * n)(*cfgs)
    keep = []
    arrs = []
    for lst in (hb, xi, qx, qy):
        ptrs = (ctypes.POINTER(ctypes.c_double) * n)()
        for k, (cfg, a) in enumerate(zip(cfgs, lst)):
            nb = dg_num_basis_bathymetry(cfg.p) if lst is hb else dg_num_basis(cfg.p)
            a = _host(a, dg_num_elements(cfg), nb)
            keep.append(a)
            ptrs[k] = _hptr(a)
        arrs.append(ptrs)
    h = ctypes.c_void_p()
    _check(load().dg_batch_init(n, carr, *arrs, _stream(stream), ctypes.byref(h)), "dg_batch_init")
    h._n = n
    return h


def dg_batch_init_device(cfgs, d_hb, d_xi, d_qx, d_qy, stream=None):
    """Batch of instances from device FP64 (K_i, E_i) arrays (lists)."""
    n = len(cfgs)
    carr = (dg_config * n)(*cfgs)
    h = ctypes.c_void_p()
    _check(load().dg_batch_init_device(n, carr, _ptr_array(d_hb), _ptr_array(d_xi), _ptr_array(d_qx),
                                       _ptr_array(d_qy), _stream(stream), ctypes.byref(h)),
           "dg_batch_init_device")
    h._n = n
    return h


def dg_batch_run(b, nsteps):
    t = np.zeros(b._n)
    _check(load().dg_batch_run(b, int(nsteps), _hptr(t)), "dg_batch_run")
    return t


def dg_batch_get_state(b, i, E, K, out=None):
    """state of instance i as three host (E, K) FP64 arrays (written into
    ``out`` if given, e.g. page-locked buffers)"""
    if out is None:
        out = [np.zeros((E, K)) for _ in range(3)]
    for a in out:
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == E * K
    _check(load().dg_batch_get_state(b, int(i), *[_hptr(a) for a in out]), "dg_batch_get_state")
    return out


def dg_batch_get_states(b, shapes, out=None):
    """every instance's state (one synchronisation): shapes = [(E_i, K_i)];
    returns [[xi, qx, qy] per instance] as host (E_i, K_i) FP64 arrays
    (written into ``out`` if given, e.g. page-locked buffers)"""
    n = len(shapes)
    if out is None:
        out = [[np.zeros((E, K)) for _ in range(3)] for E, K in shapes]
    if len(out) != n:
        raise ValueError("expected %d instances, got %d" % (n, len(out)))
    ptrs = [(ctypes.POINTER(ctypes.c_double) * n)() for _ in range(3)]
    for i, ((E, K), arrs) in enumerate(zip(shapes, out)):
        for f, a in enumerate(arrs):
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == E * K
            ptrs[f][i] = _hptr(a)
    _check(load().dg_batch_get_states(b, *ptrs), "dg_batch_get_states")
    return out


class HostStates:
    """Host states of every instance of a batch, [[xi, qx, qy] per
    instance] as (E_i, K_i) FP64 arrays, with the C pointer arrays of
    dg_batch_step_host built once (the arrays must stay alive and in place;
    reuse the object across steps to skip the marshalling)."""

    def __init__(self, shapes, arrays=None, pinned=False):
        if arrays is None:
            if pinned:
                import torch
                arrays = [[torch.zeros((E, K), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
                          for E, K in shapes]
            else:
                arrays = [[np.zeros((E, K)) for _ in range(3)] for E, K in shapes]
        if len(arrays) != len(shapes):
            raise ValueError("expected %d instances, got %d" % (len(shapes), len(arrays)))
        n = len(shapes)
        cols = [[0] * n for _ in range(3)]
        for i, ((E, K), st) in enumerate(zip(shapes, arrays)):
            for f, a in enumerate(st):
                if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != E * K:
                    raise ValueError("instance %d: expected contiguous float64 of %d x %d" % (i, E, K))
                cols[f][i] = a.ctypes.data
        self.arrays = arrays
        self.ptrs = [(ctypes.c_void_p * n)(*c) for c in cols]


def dg_batch_step_host(b, shapes, states, out=None):
    """one step of every instance from host states to host states: states
    and out are HostStates or lists [[xi, qx, qy] per instance] of host
    (E_i, K_i) FP64 arrays (out may be the same object as states; None:
    new pageable arrays).  Returns (out arrays, t after the step)."""
    if not isinstance(states, HostStates):
        states = HostStates(shapes, [[np.ascontiguousarray(a, dtype=np.float64) for a in st] for st in states])
    if out is None:
        out = HostStates(shapes)
    elif not isinstance(out, HostStates):
        out = HostStates(shapes, out)
    t = np.zeros(len(shapes))
    _check(load().dg_batch_step_host(b, *states.ptrs, *out.ptrs, _hptr(t)), "dg_batch_step_host")
    return out.arrays, t


def dg_batch_set_state(b, i, xi, qx, qy, t=0.0):
    """replace the state (host (E, K) FP64 arrays) and time of instance i"""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (xi, qx, qy)]
    _check(load().dg_batch_set_state(b, int(i), *[_hptr(a) for a in arrs], float(t)), "dg_batch_set_state")


def dg_batch_autotune(b, trial_steps=2):
    """-> (block, ms per step of blocks 32, 64, 96, 128)"""
    blk = ctypes.c_int(0)
    ms = np.zeros(4)
    _check(load().dg_batch_autotune(b, int(trial_steps), ctypes.byref(blk), _hptr(ms)), "dg_batch_autotune")
    return blk.value, ms


def dg_batch_set_block(b, block):
    _check(load().dg_batch_set_block(b, int(block)), "dg_batch_set_block")


def dg_batch_tile_shape(b, p):
    return load().dg_batch_tile_shape(b, int(p))


def dg_batch_dofs(b):
    return load().dg_batch_dofs(b)


def dg_batch_destroy(b):
    if b:
        load().dg_batch_destroy(b)


def dg_destroy(ctx):
    if ctx:
        load().dg_destroy(ctx)


def dg_status_str(s):
    return load().dg_status_str(int(s)).decode()
