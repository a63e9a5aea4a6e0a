"""The benchmark's full-size workload, the reactive swirl burner 384 x 192 x 192 (14.2 M cells,
FP32 storage and arithmetic, closed-domain pressure, flame sensor), one step in the launch
configuration bench.py times, against the FP64 oracle on sampled cells.

The oracle cannot hold the full grid's populations, so it forms what the step needs globally,
the thermodynamic pressure after the step (finite-difference update over the whole grid and the
mass balance, oracle.step.first_step_pressure), and runs the whole step on a 7 x 7 x 7 patch
around each sampled cell (radius 2 for the finite differences of the cell's neighbours, 1 for the
pull of their populations) with that pressure. Samples: random fluid cells, cells on the inlet
and outlet faces and cells next to walls. Bound per field: max(1e-5, 3 x the storage floor), the
floor being the same patch step with the state rounded to the storage type before and after.
The patch method itself is checked against whole-grid oracle steps in test_oracle_patch.py."""
import numpy as np
import pytest

import workloads as W
from tests.patches import FIELDS, patch_step as _patch_step

pytestmark = pytest.mark.gpu


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
