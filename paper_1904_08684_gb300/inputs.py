"""Seeded synthetic inputs: meshes, bathymetries and initial states.

This module holds no part of the numerical method: it only defines the
point-wise fields (bathymetry h_b(x, y), initial elevation xi_0(x, y) and
discharge q_0 = 0) and the mesh parameters of each workload, and draws their
random parameters from SplitMix64 streams.  Both the library's set-up path
and the test oracle project these fields onto their own polynomial bases.

Workloads (names are descriptive; sizes in quads, triangles = 2 nx ny):

* ``hump-p1-32``   : 32 x 32 quads on the unit square, p = 1, reflective
  walls, flat h_b = 10 m, Gaussian hump (amplitude 0.1 m, sigma 0.1) at the
  centre, q = 0, SSP-RK2, CFL 0.2, 100 steps, FP64.
* ``waves-p2-512`` : 512 x 512 quads, p = 2, periodic, h_b = 10 +
  2 sin(2 pi x) cos(2 pi y), sum of 8 seeded Gaussians (amplitude U[0.01,
  0.1] m, sigma U[0.03, 0.1], centres U[0,1]^2, periodic images), SSP-RK3,
  CFL 0.2, 1000 steps, FP64.
* ``hump-p3-32``   : the first mesh at p = 3, SSP-RK3, FP32 state.
* ``ensemble-256`` : 256 instances, nx, ny uniform in {64..384}, p uniform in
  {1, 2, 3}, smooth periodic h_b between 5 and 20 m, one Gaussian hump each.
* ``waves-p4-2048``: 2048 x 2048 quads, p = 4, periodic, the bathymetry of
  ``waves-p2-512`` and 8 Gaussians drawn with seed 5, SSP-RK3, FP32 state.
* ``manufactured`` : §3.1 test of the paper: [0, 1000]^2, analytic solution
  with C_a = C_t = 0.2, y_a = 0.3, h_b = 1 + x/1000 + 2 y/1000, dt = 0.5.
"""
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

_MASK = (1 << 64) - 1


def _xp(x):
    """numpy, or torch when the coordinates are torch tensors (fields can then
    be sampled directly on a GPU)"""
    if type(x).__module__.startswith("torch"):
        import torch
        return torch
    return np


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of Vigna's SplitMix64 generator started from ``seed``
    (output k mixes the counter seed + (k + 1) * 0x9E3779B97F4A7C15)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return lo + (hi - lo) * u


def uniform_int(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform in {lo, ..., hi}."""
    u = uniform(seed, n)
    return np.minimum(lo + np.floor(u * (hi - lo + 1)).astype(np.int64), hi)


# --------------------------------------------------------------------------
# fields

def gaussian_sum(amps, sigmas, cx, cy, periodic=True, L=1.0):
    """xi_0 = sum_k A_k exp(-d_k^2 / (2 sigma_k^2)); with ``periodic`` the sum
    runs over the 3 x 3 periodic images of each centre (separable in x, y)."""
    amps, sigmas, cx, cy = (np.asarray(a, dtype=np.float64) for a in (amps, sigmas, cx, cy))

    def f(x, y):
        xp = _xp(x)
        out = 0.0 * x + 0.0 * y
        shifts = (-L, 0.0, L) if periodic else (0.0,)
        for A, s, ax, ay in zip(amps, sigmas, cx, cy):
            c = -1.0 / (2.0 * s * s)
            gx = sum(xp.exp(c * (x - ax - sx) ** 2) for sx in shifts)
            gy = sum(xp.exp(c * (y - ay - sy) ** 2) for sy in shifts)
            out = out + A * gx * gy
        return out
    return f


def constant(c):
    def f(x, y):
        return 0.0 * x + 0.0 * y + float(c)
    return f


def sin_cos_bathymetry(x, y):
    """h_b = 10 + 2 sin(2 pi x) cos(2 pi y)."""
    xp = _xp(x)
    return 10.0 + 2.0 * xp.sin(2 * np.pi * x) * xp.cos(2 * np.pi * y)


def fourier_bathymetry(mean, amps, ms, ns, kinds):
    """h_b = mean + sum_k a_k trig_k(2 pi (m_k x + n_k y)), trig = sin or cos."""
    def f(x, y):
        xp = _xp(x)
        out = 0.0 * x + 0.0 * y + float(mean)
        for a, m, n, kd in zip(amps, ms, ns, kinds):
            arg = 2 * np.pi * (float(m) * x + float(n) * y)
            out = out + float(a) * (xp.sin(arg) if kd == 0 else xp.cos(arg))
        return out
    return f


# §3.1 analytic solution of the paper (the body force that makes it exact is
# derived where the scheme is; here only the fields).
MS_CA, MS_CT, MS_YA = 0.2, 0.2, 0.3


def ms_xi(x, y, t=0.0):
    return 2.0 + MS_YA - 2.0 * MS_CA * _xp(x).sin(np.pi * (x + y + MS_CT * t) / 600.0)


def ms_U(x, y, t=0.0):
    return 2.0 * MS_YA + MS_CA * MS_CT * _xp(x).sin(np.pi * (x + y + MS_CT * t) / 600.0)


def ms_V(x, y, t=0.0):
    return MS_YA + MS_CA * MS_CT * _xp(x).sin(np.pi * (x + y + MS_CT * t) / 600.0)


def ms_hb(x, y):
    return 1.0 + x / 1000.0 + 2.0 * y / 1000.0


def perturbed_vertices(nx, ny, Lx, Ly, frac=0.2, seed=7, x0=0.0, y0=0.0):
    """Regular vertex lattice with every vertex moved by a random vector of
    length up to ``frac`` of the cell width (§3.1's randomly perturbed mesh:
    perturbation of up to 20 % of the edge length).  Boundary vertices move
    only along the boundary, corners stay.  Shape ((ny+1)(nx+1), 2), row j
    major."""
    hx, hy = Lx / nx, Ly / ny
    i = np.arange(nx + 1)[None, :].repeat(ny + 1, 0)
    j = np.arange(ny + 1)[:, None].repeat(nx + 1, 1)
    r = uniform(seed, 2 * (nx + 1) * (ny + 1)).reshape(ny + 1, nx + 1, 2)
    rad = frac * r[..., 0]
    ang = 2.0 * np.pi * r[..., 1]
    dx = rad * np.cos(ang) * hx
    dy = rad * np.sin(ang) * hy
    dx[:, 0] = 0.0
    dx[:, -1] = 0.0
    dy[0, :] = 0.0
    dy[-1, :] = 0.0
    x = x0 + i * hx + dx
    y = y0 + j * hy + dy
    return np.stack([x, y], axis=-1).reshape(-1, 2)


# --------------------------------------------------------------------------
# workloads

@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    p: int
    bc: str
    rk_order: int
    cfl: float
    steps: int
    precision: str                      # "fp64" or "fp32"
    hb: Callable = field(repr=False)
    xi0: Callable = field(repr=False)
    x0: float = 0.0
    y0: float = 0.0
    Lx: float = 1.0
    Ly: float = 1.0
    g: float = 9.81
    dt: float = 0.0
    vertex_xy: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def E(self):
        return 2 * self.nx * self.ny

    @property
    def K(self):
        return (self.p + 1) * (self.p + 2) // 2

    def dofs(self):
        """degrees of freedom updated per RK stage: 3 fields x K x E"""
        return 3 * self.K * self.E


def _gaussians(seed, n, periodic=True):
    r = uniform(seed, 5 * n)
    A = 0.01 + 0.09 * r[0:n]
    s = 0.03 + 0.07 * r[n:2 * n]
    cx = r[2 * n:3 * n]
    cy = r[3 * n:4 * n]
    return gaussian_sum(A, s, cx, cy, periodic=periodic)


def hump_p1_32(p=1, rk=2, steps=100, precision="fp64", n=32):
    return Workload("hump-p%d-%d" % (p, n), n, n, p, "reflective", rk, 0.2, steps, precision,
                    hb=constant(10.0),
                    xi0=gaussian_sum([0.1], [0.1], [0.5], [0.5], periodic=False))


def waves_p2_512(n=512, p=2, seed=2, steps=1000, precision="fp64", ngauss=8):
    return Workload("waves-p%d-%d" % (p, n), n, n, p, "periodic", 3, 0.2, steps, precision,
                    hb=sin_cos_bathymetry, xi0=_gaussians(seed, ngauss))


def hump_p3_32(steps=1000, precision="fp32"):
    return hump_p1_32(p=3, rk=3, steps=steps, precision=precision)


def waves_p4_2048(n=2048, steps=200, precision="fp32"):
    return waves_p2_512(n=n, p=4, seed=5, steps=steps, precision=precision)


def ensemble(n=256, seed=4, nmin=64, nmax=384, pset=(1, 2, 3), steps=100, precision="fp32"):
    """Independent instances of uneven size and order (ensemble bathymetries
    and humps)."""
    nxs = uniform_int(seed, n, nmin, nmax)
    nys = uniform_int(seed + 1, n, nmin, nmax)
    ps = np.asarray(pset)[uniform_int(seed + 2, n, 0, len(pset) - 1)]
    out: List[Workload] = []
    for k in range(n):
        s = 1000 * (seed + 1) + 16 * k
        r = uniform(s, 3)
        amps = r * (7.5 / 3.0)                 # sum |a| <= 7.5 -> depth in [5, 20]
        mn = uniform_int(s + 1, 6, 0, 3).reshape(3, 2)
        mn[(mn[:, 0] == 0) & (mn[:, 1] == 0), 0] = 1
        kinds = uniform_int(s + 2, 3, 0, 1)
        hb = fourier_bathymetry(12.5, amps, mn[:, 0], mn[:, 1], kinds)
        g = uniform(s + 3, 5)
        xi0 = gaussian_sum([0.01 + 0.09 * g[0]], [0.03 + 0.07 * g[1]], [g[2]], [g[3]])
        out.append(Workload("ensemble-%d" % k, int(nxs[k]), int(nys[k]), int(ps[k]), "periodic", 3, 0.2,
                            steps, precision, hb=hb, xi0=xi0))
    return out


def manufactured(level=2, p=1, perturbed=True, seed=7, rk=3, dt=0.5):
    """§3.1 convergence test: level L has 2^L x 2^L quads on [0, 1000]^2."""
    n = 2 ** level
    vxy = perturbed_vertices(n, n, 1000.0, 1000.0, 0.2, seed) if perturbed else None
    return Workload("manufactured-L%d-p%d" % (level, p), n, n, p, "dirichlet", rk, 0.0, 0, "fp64",
                    hb=ms_hb, xi0=ms_xi, Lx=1000.0, Ly=1000.0, dt=dt, vertex_xy=vxy)


WORKLOADS = {
    "hump-p1-32": hump_p1_32,
    "waves-p2-512": waves_p2_512,
    "hump-p3-32": hump_p3_32,
    "waves-p4-2048": waves_p4_2048,
}
