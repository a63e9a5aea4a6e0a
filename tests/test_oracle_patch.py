"""The method of the full-size check, checked on a grid the oracle can step whole: the reactive
burner 24 x 16 x 16 (closed domain, flame sensor). The thermodynamic pressure after the first step
from oracle.step.first_step_pressure (the FD update and mass balance alone) equals the full step's,
and the whole step run on a 7 x 7 x 7 patch around a cell with that pressure gives the full step's
values at the cell (inner cells, cells on the inlet and outlet faces, cells next to walls)."""
import numpy as np

import workloads as W
from oracle.step import Oracle, first_step_pressure
from tests.patches import FIELDS, patch_step


def test_patch_steps_reproduce_the_full_step():
    wl = W.generate.swirl_3d(24, 16, 16, reactive=True, storage="f64", seed=21)
    assert wl.cfg["closed_domain"] and wl.cfg["flame_sensor"]
    o = Oracle(wl.cfg, wl.mask, wl.inlet_u)
    st = o.init_state(T=wl.T, Y=wl.Y, u=wl.u, P_h=wl.P_h, g_pert=wl.g_pert)
    full = o.step(st)
    P1 = first_step_pressure(wl.cfg, wl.mask, wl.inlet_u, wl.T, wl.Y, wl.u)
    assert abs(P1 - full["P_th"]) <= 1e-13 * P1
    nx, ny = wl.cfg["nx"], wl.cfg["ny"]
    fluid = np.nonzero(np.asarray(wl.mask).reshape(-1) == 0)[0]
    x = fluid % nx
    m = np.asarray(wl.mask).reshape(-1) != 0
    near = [r for r in fluid if any(m[r + d] for d in (1, -1, nx, -nx, nx * ny, -nx * ny) if 0 <= r + d < m.size)]
    rng = np.random.default_rng(3)
    cells = np.concatenate([rng.choice(fluid, 6, replace=False), rng.choice(fluid[x == 0], 3, replace=False),
                            rng.choice(fluid[x == nx - 1], 3, replace=False), rng.choice(near, 6, replace=False)])
    for r in cells:
        a = patch_step(wl, int(r), P1)
        for k in FIELDS:
            ref = full[k].numpy()[..., r]
            scale = max(np.abs(full[k].numpy()).max(), 1e-300)
            assert np.abs(a[k] - ref).max() <= 1e-12 * scale, (int(r), k, np.abs(a[k] - ref).max() / scale)
