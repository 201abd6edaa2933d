"""ctypes wrapper of ``dg_oracle.c`` (plain FP64 CPU reference).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` use this module; the library never does.

Arrays follow the library's host convention: one array per field, shape
(E, K) (element-major, coefficient of basis function i of element e at
[e, i]), element e = 2 (j nx + i) + t.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libdgoracle.so")

BC = {"periodic": 0, "reflective": 1, "dirichlet": 2}


def build_oracle(force=False):
    """Compile the oracle with gcc (plain -O2, OpenMP) if it is missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
                ("vertex_xy", ctypes.POINTER(ctypes.c_double)),
                ("p", ctypes.c_int), ("g", ctypes.c_double), ("bc", ctypes.c_int),
                ("rk_order", ctypes.c_int), ("cfl", ctypes.c_double), ("dt", ctypes.c_double),
                ("tau_bf", ctypes.c_double), ("f_c", ctypes.c_double),
                ("manufactured", ctypes.c_int), ("quad_extra", ctypes.c_int)]


_lib = None


def build_variant(src_text, tag, outdir):
    """Compile a modified copy of the oracle source into ``outdir`` and load
    it: tests plant a deliberate mistake in the oracle this way (on the CPU)
    to check that a pin catches it.  Returns a library handle for
    ``Oracle(..., lib=...)``."""
    os.makedirs(outdir, exist_ok=True)
    src = os.path.join(outdir, "dg_oracle_%s.c" % tag)
    so = os.path.join(outdir, "libdgoracle_%s.so" % tag)
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c11", "-shared", "-fPIC", "-o", so, src, "-lm"])
    return _configure(ctypes.CDLL(so))


def source():
    """text of the oracle's C source"""
    with open(_SRC) as f:
        return f.read()


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build_oracle()))
    return _lib


def _configure(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    vp = ctypes.c_void_p
    lib.or_create.restype = vp
    lib.or_create.argtypes = [ctypes.POINTER(_Cfg)]
    lib.or_destroy.argtypes = [vp]
    lib.or_set_threads.argtypes = [vp, ctypes.c_int]
    lib.or_threads.argtypes = [vp]
    lib.or_num_elems.argtypes = [vp]
    lib.or_K.argtypes = [vp]
    lib.or_Kb.argtypes = [vp]
    lib.or_project_hb.argtypes = [vp, dp, dp]
    lib.or_dmin.argtypes = [vp]
    lib.or_dmin.restype = ctypes.c_double
    lib.or_basis_table.argtypes = [vp, dp]
    lib.or_geometry.argtypes = [vp, dp, dp, ip]
    lib.or_eval_point.argtypes = [vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.or_eval_point.restype = ctypes.c_double
    lib.or_num_proj_nodes.argtypes = [vp]
    lib.or_proj_nodes.argtypes = [vp, dp]
    lib.or_proj_nodes_sub.argtypes = [vp, ip, ctypes.c_int, dp]
    lib.or_project.argtypes = [vp, dp, dp]
    lib.or_project_sub.argtypes = [vp, ctypes.c_int, ip, ctypes.c_int, dp, dp]
    lib.or_project_u.argtypes = [vp, dp, dp, dp, dp, dp, dp]
    lib.or_rhs.argtypes = [vp, dp, dp, dp, dp, ctypes.c_double, ip, ctypes.c_int, dp, dp, dp]
    lib.or_max_wave_speed.argtypes = [vp, dp, dp, dp, dp]
    lib.or_max_wave_speed.restype = ctypes.c_double
    lib.or_cfl_dt.argtypes = [vp, dp, dp, dp, dp]
    lib.or_cfl_dt.restype = ctypes.c_double
    lib.or_run.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int, dp, dp]
    lib.or_diagnostics.argtypes = [vp, dp, dp, dp, dp, dp, dp]
    lib.or_ms_errors.argtypes = [vp, dp, dp, dp, ctypes.c_double, dp]
    lib.or_ms_point.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, dp]
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def ms_point(x, y, t, g=9.81):
    """§3.1 manufactured (xi, U, V, h_b, F_x, F_y) at one point."""
    out = np.zeros(6)
    _load().or_ms_point(float(x), float(y), float(t), float(g), _ptr(out))
    return out


class Oracle:
    """One mesh + order + boundary setting of the FP64 reference scheme."""

    def __init__(self, nx, ny, p, bc="periodic", x0=0.0, y0=0.0, Lx=1.0, Ly=1.0, g=9.81,
                 rk_order=3, cfl=0.2, dt=0.0, vertex_xy=None, tau_bf=0.0, f_c=0.0,
                 manufactured=False, threads=0, quad_extra=0, lib=None):
        lib = lib if lib is not None else _load()
        self._vxy = None if vertex_xy is None else _f64(vertex_xy).ravel()
        cfg = _Cfg(nx, ny, x0, y0, Lx, Ly,
                   None if self._vxy is None else _ptr(self._vxy),
                   p, g, BC[bc] if isinstance(bc, str) else int(bc), rk_order, cfl, dt,
                   tau_bf, f_c, 1 if manufactured else 0, int(quad_extra))
        self._h = lib.or_create(ctypes.byref(cfg))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.lib = lib
        self.nx, self.ny, self.p = nx, ny, p
        self.E = lib.or_num_elems(self._h)
        self.K = lib.or_K(self._h)
        self.Kb = lib.or_Kb(self._h)
        self.g = g
        if threads:
            lib.or_set_threads(self._h, int(threads))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.or_destroy(h)
            self._h = None

    def set_threads(self, n):
        self.lib.or_set_threads(self._h, int(n))

    def threads(self):
        """threads the element loops run on"""
        return int(self.lib.or_threads(self._h))

    # ---- geometry / basis -------------------------------------------------
    def basis_table(self):
        out = np.zeros((self.K, 5, 5))
        self.lib.or_basis_table(self._h, _ptr(out))
        return out

    def geometry(self):
        verts = np.zeros((self.E, 3, 2))
        det = np.zeros(self.E)
        nb = np.zeros((self.E, 3), dtype=np.int32)
        self.lib.or_geometry(self._h, _ptr(verts), _ptr(det),
                             nb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return verts, det, nb

    def dmin(self):
        return self.lib.or_dmin(self._h)

    def eval_point(self, coef, e, x, y):
        coef = _f64(coef, (self.E, self.K))
        return self.lib.or_eval_point(self._h, _ptr(coef), int(e), float(x), float(y))

    # ---- projection ---------------------------------------------------------
    def proj_nodes(self, elems=None):
        """physical projection nodes, shape (E, Q, 2), or (len(elems), Q, 2)"""
        Q = self.lib.or_num_proj_nodes(self._h)
        if elems is None:
            xy = np.zeros((self.E, Q, 2))
            self.lib.or_proj_nodes(self._h, _ptr(xy))
            return xy
        el = np.ascontiguousarray(elems, dtype=np.int32)
        xy = np.zeros((len(el), Q, 2))
        self.lib.or_proj_nodes_sub(self._h, el.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(el), _ptr(xy))
        return xy

    def project_sub(self, vals, elems, out, hb=False):
        """L2 projection of values at proj_nodes(elems) (shape (len(elems), Q))
        into rows ``elems`` of ``out`` (shape (E, K), or (E, Kb) with hb)"""
        el = np.ascontiguousarray(elems, dtype=np.int32)
        vals = _f64(vals)
        nf = self.Kb if hb else self.K
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == (self.E, nf)
        if self.lib.or_project_sub(self._h, nf, el.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(el),
                                   _ptr(vals), _ptr(out)):
            raise RuntimeError("oracle projection failed")
        return out

    def project(self, f):
        """L2 projection of the function f(x, y) (numpy-vectorised) onto P^p."""
        xy = self.proj_nodes()
        vals = _f64(f(xy[..., 0], xy[..., 1]))
        coef = np.zeros((self.E, self.K))
        st = self.lib.or_project(self._h, _ptr(vals), _ptr(coef))
        if st:
            raise RuntimeError("oracle projection failed")
        return coef

    def project_values(self, vals):
        """L2 projection onto P^p of values given at proj_nodes(), shape (E, Q)."""
        vals = _f64(vals)
        coef = np.zeros((self.E, self.K))
        if self.lib.or_project(self._h, _ptr(vals), _ptr(coef)):
            raise RuntimeError("oracle projection failed")
        return coef

    def project_hb_values(self, vals):
        """as project_values, onto the bathymetry space P^max(p,1)"""
        vals = _f64(vals)
        coef = np.zeros((self.E, self.Kb))
        if self.lib.or_project_hb(self._h, _ptr(vals), _ptr(coef)):
            raise RuntimeError("oracle projection failed")
        return coef

    def project_hb(self, f):
        """L2 projection of the bathymetry f(x, y) onto P^max(p,1)."""
        xy = self.proj_nodes()
        vals = _f64(f(xy[..., 0], xy[..., 1]))
        coef = np.zeros((self.E, self.Kb))
        if self.lib.or_project_hb(self._h, _ptr(vals), _ptr(coef)):
            raise RuntimeError("oracle projection failed")
        return coef

    def _hbs(self, hb, *fields):
        return [_f64(hb, (self.E, self.Kb))] + [_f64(a, (self.E, self.K)) for a in fields]

    def project_u(self, hb, xi, U, V):
        arrs = self._hbs(hb, xi, U, V)
        u = np.zeros((self.E, self.K))
        v = np.zeros((self.E, self.K))
        st = self.lib.or_project_u(self._h, *[_ptr(a) for a in arrs], _ptr(u), _ptr(v))
        if st:
            raise RuntimeError("oracle u-projection failed (status %d)" % st)
        return u, v

    # ---- the scheme -----------------------------------------------------------
    def rhs(self, hb, xi, U, V, t=0.0, elems=None):
        """d_t (xi, U, V) coefficients, shape (3, E, K); rows of unlisted
        elements are zero when ``elems`` is given."""
        arrs = self._hbs(hb, xi, U, V)
        R = np.zeros((3, self.E, self.K))
        if elems is None:
            ep, ne = None, 0
        else:
            el = np.ascontiguousarray(elems, dtype=np.int32)
            ep, ne = el.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(el)
        st = self.lib.or_rhs(self._h, *[_ptr(a) for a in arrs], float(t), ep, ne,
                             _ptr(R[0]), _ptr(R[1]), _ptr(R[2]))
        if st:
            raise RuntimeError("oracle rhs failed (status %d)" % st)
        return R

    def max_wave_speed(self, hb, xi, U, V):
        arrs = self._hbs(hb, xi, U, V)
        return self.lib.or_max_wave_speed(self._h, *[_ptr(a) for a in arrs])

    def cfl_dt(self, hb, xi, U, V):
        arrs = self._hbs(hb, xi, U, V)
        return self.lib.or_cfl_dt(self._h, *[_ptr(a) for a in arrs])

    def run(self, hb, xi, U, V, nsteps, t=0.0):
        """Advance nsteps SSP-RK steps; returns (xi, U, V, t, dt_last)."""
        hb = _f64(hb, (self.E, self.Kb))
        xi, U, V = (np.array(a, dtype=np.float64).reshape(self.E, self.K) for a in (xi, U, V))
        tt = np.array([t], dtype=np.float64)
        dtl = np.zeros(1)
        st = self.lib.or_run(self._h, _ptr(hb), _ptr(xi), _ptr(U), _ptr(V), int(nsteps),
                             _ptr(tt), _ptr(dtl))
        if st:
            raise RuntimeError("oracle run failed (status %d)" % st)
        return xi, U, V, float(tt[0]), float(dtl[0])

    def diagnostics(self, hb, xi, U, V):
        arrs = self._hbs(hb, xi, U, V)
        m = np.zeros(1)
        en = np.zeros(1)
        st = self.lib.or_diagnostics(self._h, *[_ptr(a) for a in arrs], _ptr(m), _ptr(en))
        if st:
            raise RuntimeError("oracle diagnostics failed")
        return float(m[0]), float(en[0])

    def ms_errors(self, xi, U, V, t):
        arrs = [_f64(a, (self.E, self.K)) for a in (xi, U, V)]
        err = np.zeros(3)
        self.lib.or_ms_errors(self._h, *[_ptr(a) for a in arrs], float(t), _ptr(err))
        return err
