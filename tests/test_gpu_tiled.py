"""The tiled FD update (3-D FP32) at its edges, against the FP64 oracle: partial tiles in x and y
(the last x tile holds the outlet column), a single z chunk shorter than the default plane count,
and cells with ghost-point wall weights, which a second launch of the general kernel updates (its
thermodynamic-pressure partial sums follow the tiled kernel's). Bound per field: max(1e-5, 3 x the
FP32 storage floor), and for the interpolated walls, whose FP32 interpolation drifts P_h slowly,
max(3e-5, 3 x floor), as in the other curved-wall FP32 tests."""
import numpy as np
import pytest

import workloads as W
from tests.parity import compare, gpu_run, oracle_run, storage_floor

pytestmark = pytest.mark.gpu


def _check(wl, errs, floor, tol):
    print(f"{wl.name}: FP32 relative L-inf", {k: f"{v:.2e} (floor {floor[k]:.2e})" for k, v in errs.items()})
    bad = {k: (v, floor[k]) for k, v in errs.items() if not v <= max(tol, 3.0 * floor[k])}
    assert not bad, f"errors above max({tol}, 3 x floor): {bad}"


def test_tiled_fd_partial_tiles_and_single_chunk_f32():
    """36 x 20 x 13: tiles of 32 x 8 leave 4 columns in x (with the outlet at x = 35, whose ghost
    values go into the tile's interior columns) and 4 rows in y; 13 planes make one z chunk."""
    wl = W.generate.swirl_3d(36, 20, 13, reactive=True, seed=21, dt=2e-6)
    assert wl.cfg["flame_sensor"] and wl.cfg["closed_domain"]
    o, st = oracle_run(wl, 20)
    gpu = gpu_run(wl, 20)
    assert np.array_equal(gpu["stencil_words"].astype(np.int64), o.stencil_words_packed().numpy())
    _check(wl, compare(wl, gpu, st), storage_floor(wl, 20, st), 1e-5)
    assert abs(gpu["scalars"]["P_th"] - st["P_th"]) <= 1e-12 * st["P_th"]
    assert abs(gpu["scalars"]["M"] - st["M"]) <= 1e-6 * abs(st["M"])


def test_tiled_fd_with_ghost_point_walls_f32():
    """The reactive burner with interpolated walls on the injector cylinders and the exhaust cone,
    flame sensor and closed domain: the wall cells go to the general kernel's walls-only launch."""
    from oracle.step import Oracle
    wl = W.generate.swirl_3d(32, 18, 18, reactive=True, curved=True, storage="f32", seed=6, dt=2e-6)
    c, d, q = wl.info["wall_links"]
    q = np.asarray(q, dtype=np.float32).astype(np.float64)
    wl.info["wall_links"] = (c, d, q)
    dense = np.zeros((27, wl.N))
    dense[d, c] = q

    def run(store_round=None):
        o = Oracle(wl.cfg, wl.mask, wl.inlet_u, store_round=store_round, qwall=dense)
        st = o.round_state(o.init_state(T=wl.T, Y=wl.Y, u=wl.u, P_h=wl.P_h, g_pert=wl.g_pert))
        return o, o.run(st, 20)

    o, st = run()
    gpu = gpu_run(wl, 20)
    words = gpu["stencil_words"].astype(np.int64)
    assert np.array_equal(words, o.stencil_words_packed().numpy())
    assert ((words >> 30) & 1).sum() > 50  # cells with ghost-point weights exist
    _, st32 = run("f32")
    fields = {"u": st32["u"].numpy(), "P_h": st32["P_h"].numpy(), "g": st32["g"].numpy(), "T": st32["T"].numpy(),
              "Y": st32["Y"].numpy(), "rho": st32["rho"].numpy(), "lam": st32["lam"].numpy()}
    _check(wl, compare(wl, gpu, st), compare(wl, fields, st), 3e-5)
    assert abs(gpu["scalars"]["M"] - st["M"]) <= 1e-6 * abs(st["M"])
