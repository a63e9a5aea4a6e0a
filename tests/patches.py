"""One oracle step on a patch of a larger grid (test helper): the whole step for the cell at the
patch centre needs the fields within 3 cells of it (the finite differences of the cell's
neighbours reach 2 further, the pull of their populations 1) and, in a closed domain, the
thermodynamic pressure after the step, which the caller supplies (oracle.step.first_step_pressure)."""
import copy

import numpy as np

FIELDS = ("T", "Y", "u", "P_h", "g", "rho", "lam")


def _slice(a, dims, lo, hi):
    nx, ny, nz = dims
    lead = a.shape[:-1]
    v = a.reshape(*lead, nz, ny, nx)[..., lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    return v.reshape(*lead, -1)


def patch_step(wl, r, P1, store_round=None, rad=3):
    from oracle.step import Oracle
    cfg = wl.cfg
    dims = (cfg["nx"], cfg["ny"], cfg["nz"])
    c = (r % dims[0], (r // dims[0]) % dims[1], r // (dims[0] * dims[1]))
    lo = [max(0, c[a] - rad) for a in range(3)]
    hi = [min(dims[a], c[a] + rad + 1) for a in range(3)]
    sub = copy.deepcopy(cfg)
    sub["nx"], sub["ny"], sub["nz"] = (hi[a] - lo[a] for a in range(3))
    for a, name in enumerate("xyz"):
        b_lo, b_hi = cfg["bc"][name]
        # a cut face gets a wall: the sampled cell's step never reaches it
        sub["bc"][name] = (b_lo if lo[a] == 0 else "wall", b_hi if hi[a] == dims[a] else "wall")
    mask = _slice(np.asarray(wl.mask).reshape(-1), dims, lo, hi)
    face = np.asarray(wl.inlet_u).reshape(3, dims[2], dims[1])[:, lo[2]:hi[2], lo[1]:hi[1]].reshape(3, -1)
    o = Oracle(sub, mask, face, store_round=store_round)
    g_pert = None if wl.g_pert is None else _slice(np.asarray(wl.g_pert), dims, lo, hi)
    st = o.round_state(o.init_state(T=_slice(wl.T, dims, lo, hi), Y=_slice(wl.Y, dims, lo, hi),
                                    u=_slice(wl.u, dims, lo, hi), P_h=_slice(wl.P_h, dims, lo, hi), g_pert=g_pert))
    st = o.round_state(o.step(st, P_next=P1))
    rc = (c[0] - lo[0]) + sub["nx"] * ((c[1] - lo[1]) + sub["ny"] * (c[2] - lo[2]))
    return {k: st[k].numpy()[..., rc] for k in FIELDS}


