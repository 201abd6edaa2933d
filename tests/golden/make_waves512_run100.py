#!/usr/bin/env python
"""Writes tests/golden/waves512_run100.npz: the FP64 oracle's state after
100 SSP-RK3 steps of the 512 x 512-quad, p = 2, periodic waves workload
(524,288 triangles, h_b = 10 + 2 sin(2 pi x) cos(2 pi y), eight seeded
Gaussians, q = 0, CFL 0.2), at a fixed set of sampled elements.

Calls only oracle/ (the FP64 CPU reference of the scheme, paper §2.2) and
the seeded field definitions of paper_1904_08684_gb300.inputs; nothing of
the CUDA library.  The whole mesh has to be advanced (every element's
domain of dependence grows by one neighbour per stage), which takes about
50 minutes on 8 host cores.

At h = 1/512 the FP64 round-off of the scheme itself is no longer ~1e-16:
the volume and edge integrals are O(h) and cancel to O(h^2) before the
division by |det B| = O(h^2), and 300 stages accumulate it.  To measure
that floor the oracle is run a second time with two extra Gauss points per
direction (still exact for the degree-3p integrands, so the same scheme in
exact arithmetic, with different rounding); the two runs' disagreement is
the oracle's own noise at this size.

Stored arrays:
  elems   int32 (S,)      sampled element indices (random + periodic seams)
  xi, U, V  float64 (S, 6)  coefficients of the samples after 100 steps
  xi_q2, U_q2, V_q2        the same from the run with two extra points
  t, t_q2 float64 ()      simulation time after 100 steps (CFL steps)
  dt_last float64 ()      the last step's dt
  mass0, mass  float64 () mass before and after (oracle diagnostics)

    python tests/golden/make_waves512_run100.py            # both runs
    python tests/golden/make_waves512_run100.py --append-q2  # second run only,
                                                   added to an existing file
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1904_08684_gb300 import inputs as I  # noqa: E402

STEPS = 100
OUT = os.path.join(HERE, "waves512_run100.npz")


def initial_state(o, wl):
    """the oracle's L2 projection of the seeded fields (q = 0)"""
    xy = o.proj_nodes()
    hb = o.project_hb_values(wl.hb(xy[..., 0], xy[..., 1]))
    xi = o.project_values(wl.xi0(xy[..., 0], xy[..., 1]))
    return hb, xi


def samples(E, nx):
    """2000 distinct pseudo-random elements (SplitMix64, seed 512100) plus
    the periodic seams and corners of the mesh"""
    picks = np.unique(I.uniform_int(512100, 2600, 0, E - 1))[:2000]
    seam = [0, 1, 2 * (nx - 1), 2 * (nx - 1) + 1, E - 1, E - 2, E - 2 * nx, E - 2 * nx + 1]
    return np.unique(np.concatenate([picks, seam])).astype(np.int32)


def run(quad_extra):
    wl = I.waves_p2_512()
    o = oracle.Oracle(wl.nx, wl.ny, wl.p, bc="periodic", rk_order=3, cfl=wl.cfl, quad_extra=quad_extra)
    hb, xi = initial_state(o, wl)
    z = np.zeros_like(xi)
    m0, _ = o.diagnostics(hb, xi, z, z)
    t0 = time.time()
    xr, Ur, Vr, t, dtl = o.run(hb, xi, z, z, STEPS)
    el = time.time() - t0
    m1, _ = o.diagnostics(hb, xr, Ur, Vr)
    print("quad_extra %d: t = %.17g, %d oracle threads, %.0f s" % (quad_extra, t, o.threads(), el))
    return o, wl, xr, Ur, Vr, t, dtl, m0, m1


def main():
    if "--append-q2" in sys.argv:
        base = dict(np.load(OUT))
    else:
        o, wl, xr, Ur, Vr, t, dtl, m0, m1 = run(0)
        S = samples(o.E, wl.nx)
        base = dict(elems=S, xi=xr[S], U=Ur[S], V=Vr[S], t=np.float64(t), dt_last=np.float64(dtl),
                    mass0=np.float64(m0), mass=np.float64(m1))
    S = base["elems"]
    _, _, x2, U2, V2, t2, _, _, _ = run(2)
    base.update(xi_q2=x2[S], U_q2=U2[S], V_q2=V2[S], t_q2=np.float64(t2))
    np.savez_compressed(OUT, **base)
    print("wrote %s: %d samples" % (OUT, len(S)))


if __name__ == "__main__":
    main()
