"""Checkpoint / resume of a dgswe context: the state coefficients (host FP64,
element-major) and the model time in one .npz file.  A resumed run continues
bit-identically (the state is held exactly; FP32 contexts store their FP32
values widened to FP64, which round back exactly)."""
import numpy as np

from . import binding as B


def save(path, ctx, cfg):
    """write the context's state and time to ``path`` (.npz)"""
    E, K = B.dg_num_elements(cfg), B.dg_num_basis(cfg.p)
    xi, qx, qy = B.dg_get_state(ctx, E, K)
    t = B.dg_run(ctx, 0)      # zero steps: returns the model time
    np.savez(path, xi=xi, qx=qx, qy=qy, t=np.float64(t), p=np.int64(cfg.p),
             nx=np.int64(cfg.nx), ny=np.int64(cfg.ny))


def load(path, ctx, cfg):
    """restore a state written by ``save`` into a context of the same mesh and
    order; returns the restored time"""
    with np.load(path) as f:
        if (int(f["p"]), int(f["nx"]), int(f["ny"])) != (cfg.p, cfg.nx, cfg.ny):
            raise ValueError("checkpoint of another mesh or order")
        t = float(f["t"])
        B.dg_set_state(ctx, f["xi"], f["qx"], f["qy"], t=t)
    return t
