"""Helpers shared by the GPU parity tests: run the same seeded workload through the CUDA
library and the FP64 oracle, and compare fields with the relative L-infinity metric

    err(field) = max_fluid |gpu - oracle| / max_fluid |oracle - reference|

where the reference is the field's rest value (0 for P_h, u and Y_k, T_ref for T, w_i P_ref for
the populations), so that the denominator is the size of the field's deviation."""
import numpy as np
import torch

from oracle.step import Oracle


def oracle_run(wl, steps, store_round=None):
    o = Oracle(wl.cfg, wl.mask, wl.inlet_u, store_round=store_round)
    st = o.init_state(T=wl.T, Y=wl.Y, u=wl.u, P_h=wl.P_h, g_pert=wl.g_pert)
    st = o.round_state(st)
    st = o.run(st, steps)
    return o, st


def as_fields(st):
    """Oracle state in the layout of the GPU output."""
    out = {"u": st["u"].numpy(), "P_h": st["P_h"].numpy(), "g": st["g"].numpy()}
    for k in ("T", "Y", "rho", "lam"):
        if k in st:
            out[k] = st[k].numpy()
    return out


def storage_floor(wl, steps, st_exact, metric=None, store_round="f32"):
    """Per-field error of the FP64 oracle whose state is rounded to the storage precision after
    every step, against the exact oracle: the accuracy limit of that storage format."""
    _, st_r = oracle_run(wl, steps, store_round=store_round)
    return compare(wl, as_fields(st_r), st_exact, metric=metric or rel_linf)


def gpu_run(wl, steps, **kw):
    from paper_2207_11567_gb300 import from_workload
    s = from_workload(wl, **kw)
    s.step(steps)
    out = s.fields()
    out["links"] = s.links()
    out["stencil_words"] = s.stencil_words()
    out["scalars"] = s.scalars()
    s.close()
    return out


def rel_linf(a, b, fluid, ref=0.0):
    a = np.asarray(a)[..., fluid]
    b = np.asarray(b)[..., fluid]
    den = np.max(np.abs(b - ref))
    return float(np.max(np.abs(a - b)) / max(den, 1e-300))


def rel_l2(a, b, fluid, ref=0.0):
    a = np.asarray(a)[..., fluid]
    b = np.asarray(b)[..., fluid]
    den = np.sqrt(np.sum((b - ref) ** 2))
    return float(np.sqrt(np.sum((a - b) ** 2)) / max(den, 1e-300))


def compare(wl, gpu, st, metric=rel_linf):
    """Per-field errors (dict) between the GPU output and the oracle state."""
    fluid = np.asarray(wl.mask).reshape(-1) == 0
    errs = {"u": metric(gpu["u"], st["u"].numpy(), fluid),
            "P_h": metric(gpu["P_h"], st["P_h"].numpy(), fluid)}
    g_o = st["g"].numpy()
    errs["g"] = max(metric(gpu["g"][i], g_o[i], fluid) for i in range(g_o.shape[0]))
    if wl.cfg.get("thermal"):
        errs["T"] = metric(gpu["T"], st["T"].numpy(), fluid, ref=wl.cfg["T_ref"])
        Yo = st["Y"].numpy()
        errs["Y"] = max(metric(gpu["Y"][k], Yo[k], fluid) for k in range(Yo.shape[0]))
        errs["rho"] = metric(gpu["rho"], st["rho"].numpy(), fluid, ref=0.0)
        errs["lam"] = metric(gpu["lam"], st["lam"].numpy(), fluid)
    return errs
