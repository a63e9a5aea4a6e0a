"""The benchmark's full-size workload, the reactive swirl burner 384 x 192 x 192 (14.2 M cells,
FP32 storage and arithmetic, closed-domain pressure, flame sensor), one step in the launch
configuration bench.py times, against the FP64 oracle on sampled cells.

The oracle cannot hold the full grid's populations, so it forms what the step needs globally,
the thermodynamic pressure after the step (finite-difference update over the whole grid and the
mass balance, oracle.step.first_step_pressure), and runs the whole step on a 7 x 7 x 7 patch
around each sampled cell (radius 2 for the finite differences of the cell's neighbours, 1 for the
pull of their populations) with that pressure. Samples: random fluid cells, cells on the inlet
and outlet faces and cells next to walls. Bound per field: max(1e-5, 3 x the storage floor), the
floor being the same patch step with the state rounded to the storage type before and after."""
import copy

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("T", "Y", "u", "P_h", "g", "rho", "lam")


def _slice(a, dims, lo, hi):
    nx, ny, nz = dims
    lead = a.shape[:-1]
    v = a.reshape(*lead, nz, ny, nx)[..., lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    return v.reshape(*lead, -1)


def _patch_step(wl, r, P1, store_round=None, rad=3):
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


def _samples(wl, rng):
    nx, ny, nz = wl.cfg["nx"], wl.cfg["ny"], wl.cfg["nz"]
    m = np.asarray(wl.mask).reshape(nz, ny, nx) != 0
    fluid = ~m
    near = np.zeros_like(fluid)
    for ax in range(3):
        for sh in (-1, 1):
            near |= np.roll(m, sh, axis=ax)
    near &= fluid
    flat = lambda b: np.nonzero(b.reshape(-1))[0]
    inlet = fluid.copy()
    inlet[:, :, 1:] = False
    outlet = fluid.copy()
    outlet[:, :, :-1] = False
    pick = lambda idx, n: rng.choice(idx, size=min(n, idx.size), replace=False)
    return np.concatenate([pick(flat(fluid), 40), pick(flat(inlet), 12), pick(flat(outlet), 12),
                           pick(flat(near), 24)])


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_c4_full_size_one_step_on_sampled_cells(storage):
    """FP32 arithmetic with FP32 or FP16 population storage (the benchmark's two variants); the
    floor rounds the oracle's state to the same storage."""
    from oracle.step import first_step_pressure
    from paper_2207_11567_gb300 import from_workload
    wl = W.make("c4_swirl_reactive_3d")
    assert wl.cfg["storage"] == "f32" and wl.cfg["closed_domain"] and wl.cfg["flame_sensor"]
    wl.cfg["storage"] = storage
    s = from_workload(wl)
    s.step(1)
    gpu = s.fields()
    P_gpu = s.scalars()["P_th"]
    s.close()
    P1 = first_step_pressure(wl.cfg, wl.mask, wl.inlet_u, wl.T, wl.Y, wl.u)
    assert abs(P_gpu - P1) / P1 < 1e-6, (P_gpu, P1)  # FP32 fields, exact fixed-point sum
    cells = _samples(wl, np.random.default_rng(2207))
    ref = {k: [] for k in FIELDS}
    rnd = {k: [] for k in FIELDS}
    got = {k: [] for k in FIELDS}
    for r in cells:
        a = _patch_step(wl, int(r), P1)
        b = _patch_step(wl, int(r), P1, store_round=storage)
        for k in FIELDS:
            ref[k].append(a[k])
            rnd[k].append(b[k])
            got[k].append(np.asarray(gpu[k])[..., r])
    bad = {}
    for k in FIELDS:
        o, f, gv = np.array(ref[k]), np.array(rnd[k]), np.array(got[k])
        base = wl.cfg["T_ref"] if k == "T" else 0.0
        scale = np.abs(o - base).max() + 1e-300
        err = np.abs(gv - o).max() / scale
        floor = np.abs(f - o).max() / scale
        if not err <= max(1e-5, 3.0 * floor):
            bad[k] = (err, floor)
    assert not bad, bad
