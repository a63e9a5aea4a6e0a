"""Mixture-averaged species diffusion (lbm_set_transport) on the GPU against the FP64 oracle with the
same option: element-by-element parity in FP64 (2-D chamber with obstacles, an inlet and an outlet;
3-D reactive burner with the flame sensor), FP32 within the storage-floor bound, the option is live
(the species differ from the constant-Lewis run), and the combinations it does not support are
refused."""
import numpy as np
import pytest

import workloads as W
from tests.parity import compare, gpu_run, oracle_run, storage_floor
from workloads.configs import mixture_averaged

pytestmark = pytest.mark.gpu


def _case(which, storage):
    if which == "chamber2d":
        wl = W.generate.chamber_2d(nx=64, ny=32, inlet=True, dt=5e-7, storage=storage, seed=4, u_init=0.01,
                                   n_rows=1, per_row=2)
        return wl, 100
    wl = W.generate.swirl_3d(28, 16, 16, reactive=True, storage=storage, seed=5)
    wl.cfg["closed_domain"] = False
    return wl, 20


@pytest.mark.parametrize("which", ["chamber2d", "swirl3d"])
def test_mixture_averaged_f64(which):
    wl, steps = _case(which, "f64")
    mixture_averaged(wl.cfg)
    o, st = oracle_run(wl, steps)
    gpu = gpu_run(wl, steps)
    errs = compare(wl, gpu, st)
    bad = {k: v for k, v in errs.items() if not v <= 1e-10}
    assert not bad, f"errors above 1e-10: {bad} (all: {errs})"


@pytest.mark.parametrize("which", ["chamber2d", "swirl3d"])
def test_mixture_averaged_f32(which):
    """FP32 storage and arithmetic: per field max(1e-5, 3 x the FP32 storage floor of the same run),
    capped at 5e-5 (P_h, g, Lambda) and 1e-5 (u, T, Y, rho) unless the floor itself is above the cap."""
    wl, steps = _case(which, "f32")
    mixture_averaged(wl.cfg)
    o, st = oracle_run(wl, steps)
    gpu = gpu_run(wl, steps)
    errs = compare(wl, gpu, st)
    floor = storage_floor(wl, steps, st)
    print({k: f"{errs[k]:.2e} (floor {floor[k]:.2e})" for k in errs})
    bad = {k: (v, floor[k]) for k, v in errs.items() if not v <= max(1e-5, 3.0 * floor[k])}
    assert not bad, f"FP32 errors above max(1e-5, 3 x floor): {bad}"


def test_mixture_averaged_is_live():
    wl, steps = _case("chamber2d", "f64")
    a = gpu_run(wl, steps)
    mixture_averaged(wl.cfg)
    b = gpu_run(wl, steps)
    fluid = wl.mask.reshape(-1) == 0
    dY = np.abs(a["Y"][:, fluid] - b["Y"][:, fluid]).max()
    assert dY > 1e-4, dY


def test_mixture_averaged_refuses_unsupported_combinations():
    from paper_2207_11567_gb300 import _lib as L
    from paper_2207_11567_gb300 import from_workload
    from workloads.configs import variable_cp
    wl, _ = _case("chamber2d", "f64")
    s = from_workload(wl)
    Le = np.asarray(mixture_averaged(dict(wl.cfg))["Le_pair"])
    bad = Le.copy()
    bad[0, 1] = -1.0
    with pytest.raises(L.HLBMError) as e:
        s.set_transport(bad)
    assert e.value.status == L.LBM_ERR_ARG
    s.set_thermo([sp["cp_poly"] for sp in variable_cp(dict(wl.cfg, species=[dict(x) for x in wl.cfg["species"]]))
                  ["species"]])
    with pytest.raises(L.HLBMError) as e:
        s.set_transport(Le)
    assert e.value.status == L.LBM_ERR_UNSUPPORTED
    s.set_thermo(None)
    s.set_transport(Le)
    s.step(2)
    s.close()
