"""Variable heat capacities (lbm_set_thermo) on the GPU against the FP64 oracle with the same
option: element-by-element parity in FP64 (2-D chamber with obstacles and an inlet, planar flame,
3-D reactive burner with the flame sensor and closed-domain pressure), FP32 at the storage floor,
and the converged planar flame's burnt temperature at the closed-form adiabatic value of the
variable-c_p enthalpy balance."""
import numpy as np
import pytest

import workloads as W
from tests.parity import compare, gpu_run, oracle_run, storage_floor
from workloads.configs import variable_cp

pytestmark = pytest.mark.gpu


def _check(errs, tol):
    bad = {k: v for k, v in errs.items() if not (v <= tol)}
    assert not bad, f"errors above {tol}: {bad} (all: {errs})"


@pytest.mark.parametrize("case", ["chamber2d", "flame2d", "swirl3d_sensor", "swirl3d_closed"])
def test_variable_cp_f64(case):
    """The reactive burner runs once with the flame sensor (open domain) and once with the
    closed-domain pressure (no sensor): with both at once this case is ill-conditioned already
    with constant c_p (GPU and oracle part at 1e-8..5e-7 within 20 steps, measured on GB300,
    while each alone agrees to 1e-13)."""
    if case == "chamber2d":
        wl = W.generate.chamber_2d(nx=64, ny=32, inlet=True, dt=5e-7, storage="f64", seed=4, u_init=0.01,
                                   n_rows=1, per_row=2)
        steps = 100
    elif case == "flame2d":
        wl = W.generate.flame_2d(nx=96, ny=4, storage="f64", seed=3)
        steps = 60
    else:
        wl = W.generate.swirl_3d(28, 16, 16, reactive=True, storage="f64", seed=5)
        wl.cfg["flame_sensor"] = case == "swirl3d_sensor"
        wl.cfg["closed_domain"] = case == "swirl3d_closed"
        steps = 20
    variable_cp(wl.cfg)
    o, st = oracle_run(wl, steps)
    gpu = gpu_run(wl, steps)
    _check(compare(wl, gpu, st), 1e-10)


def test_variable_cp_changes_the_temperature():
    """The option is live: the same chamber run with constant c_p differs in T by far more than the
    parity tolerance."""
    wl = W.generate.chamber_2d(nx=64, ny=32, inlet=True, dt=5e-7, storage="f64", seed=4, u_init=0.01,
                               n_rows=1, per_row=2)
    a = gpu_run(wl, 100)
    variable_cp(wl.cfg)
    b = gpu_run(wl, 100)
    fluid = wl.mask == 0
    assert np.abs(a["T"][fluid] - b["T"][fluid]).max() > 1.0


def test_variable_cp_f32():
    """FP32 within max(1e-5, 3 x storage floor) per field on the closed chamber (200 steps); with an
    inlet and a moving initial state the constant-c_p FP32 path already sits at ~15x the floor in
    P_h (1.5e-5, measured on GB300), so there the variable-c_p run is held to that: at most 1.5x
    the constant-c_p run's error, field by field."""
    wl = W.generate.chamber_2d(nx=97, ny=41, dt=5e-7, storage="f32", seed=3)
    variable_cp(wl.cfg)
    o, st = oracle_run(wl, 200)
    errs = compare(wl, gpu_run(wl, 200), st)
    floor = storage_floor(wl, 200, st)
    bad = {k: (v, floor[k]) for k, v in errs.items() if not (v <= max(1e-5, 3.0 * floor[k]))}
    assert not bad, (errs, floor)

    def inlet_case(vcp):
        wl = W.generate.chamber_2d(nx=64, ny=32, inlet=True, dt=5e-7, storage="f32", seed=4, u_init=0.01,
                                   n_rows=1, per_row=2)
        if vcp:
            variable_cp(wl.cfg)
        o, st = oracle_run(wl, 150)
        return compare(wl, gpu_run(wl, 150), st), storage_floor(wl, 150, st)
    (ev, fv), (ec, _) = inlet_case(True), inlet_case(False)
    bad = {k: (v, ec[k]) for k, v in ev.items() if not (v <= max(1e-5, 3.0 * fv[k], 1.5 * ec[k]))}
    assert not bad, (ev, ec, fv)


def test_variable_cp_adjoint_is_unsupported():
    import torch
    from paper_2207_11567_gb300 import _lib as L
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.chamber_2d(nx=24, ny=12, inlet=True, storage="f32", seed=2, n_rows=1, per_row=1)
    variable_cp(wl.cfg)
    s = from_workload(wl)
    s.step(2)
    state = s.save_state()
    adj = torch.zeros(s.state_bytes() // 4, dtype=torch.float32, device="cuda")
    gin = torch.zeros(2 * wl.cfg["ny"], dtype=torch.float32, device="cuda")
    with pytest.raises(L.HLBMError) as e:
        s.adjoint_step(state, adj, gin)
    assert e.value.status == L.LBM_ERR_UNSUPPORTED
    s.set_thermo(None)  # back to constant c_p: the adjoint runs
    s.adjoint_step(state, adj, gin)
    s.synchronize()
    assert torch.isfinite(adj).all()
    s.close()


def test_free_flame_reaches_variable_cp_adiabatic_temperature():
    """Planar flame thickened by F = 3 with c_p,k(T): burnt temperature within 1e-3 of the root of
    the enthalpy balance of complete combustion (unity Lewis numbers), 2064 K, far from the
    constant-c_p 1952 K. (At F = 4 the hotter burnt gas's thickened diffusivity exceeds the
    explicit limit of this time step: dt F lambda / (rho c_p dx^2) reaches 0.5 near 2060 K.)"""
    from paper_2207_11567_gb300 import from_workload
    from paper_2207_11567_gb300.flame1d import free_flame
    from tests.test_oracle_pins import _T_ad_variable_cp
    from workloads.configs import burnt_mixture
    wl = W.generate.flame_2d(nx=256, ny=1, storage="f64", seed=0, width_cells=60.0)
    wl.cfg["thicken_F"] = 3.0
    variable_cp(wl.cfg)
    s = from_workload(wl)
    sol = free_flame(s, chunk=200, max_steps=400000)
    s.close()
    names = W.SPECIES["4sp"]
    T_ad = _T_ad_variable_cp(wl.cfg, wl.cfg["T_in"], wl.cfg["Y_in"], burnt_mixture(names, 0.83))
    assert sol.converged
    assert abs(sol.T_b - T_ad) / T_ad < 1e-3, (sol.T_b, T_ad)
    assert abs(T_ad - 1951.7) > 100.0
