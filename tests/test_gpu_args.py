"""Argument and state checks of the newer entry points (no kernel reaches bad data): each refusal is
an lbm_status with a message, and the context keeps working afterwards."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _solver(thermal=True, storage="f32"):
    from paper_2207_11567_gb300 import from_workload
    if thermal:
        wl = W.generate.chamber_2d(nx=32, ny=16, inlet=True, storage=storage, seed=1, n_rows=1, per_row=1)
    else:
        wl = W.generate.box(2, 16, storage=storage, seed=1)
    return wl, from_workload(wl)


def test_flame_properties_and_thermo_arguments():
    from paper_2207_11567_gb300 import _lib as L
    wl, s = _solver(thermal=False)
    with pytest.raises(L.HLBMError) as e:
        s.flame_properties(0)
    assert e.value.status == L.LBM_ERR_ARG
    s.close()
    wl, s = _solver()
    with pytest.raises(L.HLBMError) as e:
        s.flame_properties(7)  # no such species
    assert e.value.status == L.LBM_ERR_ARG
    bad = [[1000.0, float("nan"), 0, 0, 0]] + [[1000.0, 0, 0, 0, 0]] * 5
    with pytest.raises(L.HLBMError) as e:
        s.set_thermo(bad)
    assert e.value.status == L.LBM_ERR_ARG
    with pytest.raises(ValueError):
        s.set_inlet(np.zeros(3))  # wrong size (checked by the binding)
    s.step(2)
    assert np.isfinite(s.fields(L.F_T)["T"]).all()
    s.close()


def test_probe_and_spectrum_arguments():
    from paper_2207_11567_gb300 import _lib as L
    wl, s = _solver()
    with pytest.raises(L.HLBMError) as e:
        s.probes()  # no probes set
    assert e.value.status == L.LBM_ERR_STATE
    with pytest.raises(L.HLBMError):
        s.set_probes([wl.N + 5])
    fluid = np.nonzero(wl.mask == 0)[0]
    s.set_probes(fluid[:2], capacity=8)
    s.step(4)
    with pytest.raises(L.HLBMError) as e:
        s.probe_spectrum(0, 0, 16)  # more than the 4 samples recorded
    assert e.value.status == L.LBM_ERR_ARG
    with pytest.raises(L.HLBMError):
        s.probe_spectrum(2, 0, 4)  # no probe 2
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(L.HLBMError):
        s.welch_psd(x, 1e-3, 5)  # odd segment
    with pytest.raises(L.HLBMError):
        s.welch_psd(x, 1e-3, 16)  # longer than the series
    f, p = s.probe_spectrum(0, 0, 4)
    assert p.shape == (3,) and np.isfinite(p).all()
    s.close()


def test_adjoint_sweep_arguments():
    from paper_2207_11567_gb300 import _lib as L
    wl, s = _solver()
    s.step(1)
    ck = [s.save_state(), s.save_state()]
    adj = torch.zeros(s.state_bytes() // 4, dtype=torch.float32, device="cuda")
    gin = torch.zeros(2 * wl.cfg["ny"], dtype=torch.float32, device="cuda")
    for C, K in ((4, 4), (4, 9), (0, 4)):  # 2 segments need 4 < K <= 8
        with pytest.raises(L.HLBMError) as e:
            s.adjoint_sweep(ck, C, K, adj, gin)
        assert e.value.status == L.LBM_ERR_ARG
    s.adjoint_sweep(ck, 4, 6, adj, gin)
    s.synchronize()
    assert torch.isfinite(adj).all()
    s.close()
