"""The finite-difference stencil kinds are symmetric, which the FD adjoint uses to find, from a
cell's own stencil word, the cells whose stencils hold it: for every fluid cell s, axis, side and
distance d in {1, 2}, the cell q at distance d on the opposite side has s as its real point (fluid,
inside the domain or across a periodic face) on that side exactly when s's own word marks its
points on the opposite side up to distance d as real. Checked on the oracle's stencil words (equal
bit for bit to the library's, tests/test_gpu_parity.py) for 2-D and 3-D workloads with walls,
obstacles, an inlet, an outlet and periodic faces."""
import numpy as np
import pytest

import workloads as W
from oracle.step import Oracle


def _cases():
    return {
        "chamber_2d": W.generate.chamber_2d(nx=48, ny=24, inlet=True, seed=2, n_rows=1, per_row=2),
        "flame_2d_periodic_y": W.generate.flame_2d(nx=40, ny=6),
        "swirl_3d": W.generate.swirl_3d(24, 16, 16, reactive=True, seed=3),
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_stencil_kinds_are_symmetric(name):
    wl = _cases()[name]
    o = Oracle(wl.cfg, wl.mask, wl.inlet_u)
    w = o.stencil_words_packed().numpy().astype(np.int64)
    D = wl.cfg["dim"]
    dims = [wl.cfg["nx"], wl.cfg["ny"], wl.cfg["nz"]][:D]
    strides = [1, dims[0], dims[0] * dims[1]][:D]
    idx = np.arange(w.size)
    pos = [idx % dims[0], (idx // dims[0]) % dims[1], idx // (dims[0] * dims[1])][:D]
    bc = wl.cfg["bc"]
    fluid = ((w >> 31) & 1) == 1
    owners = 0
    for ax, name_ax in enumerate("xyz"[:D]):
        periodic = bc[name_ax][0] == "periodic"
        for sd in (0, 1):
            sg = 1 if sd else -1
            opp = (w >> (4 * (2 * ax + (1 - sd)))) & 15  # s's kinds toward -sg
            for dist in (1, 2):
                own_view = ((opp & 3) == 0) if dist == 1 else (opp == 0)
                qd = pos[ax] - dist * sg
                inside = (qd >= 0) & (qd < dims[ax])
                if periodic:
                    qd = qd % dims[ax]
                    inside = np.ones_like(inside)
                q = idx + (np.where(inside, qd, pos[ax]) - pos[ax]) * strides[ax]
                wq = w[q]
                owner_view = inside & (((wq >> 31) & 1) == 1) & \
                    (((wq >> (4 * (2 * ax + sd) + 2 * (dist - 1))) & 3) == 0)
                assert np.array_equal(owner_view[fluid], own_view[fluid]), (name_ax, sd, dist)
                owners += int(owner_view[fluid].sum())
    assert owners > 0
