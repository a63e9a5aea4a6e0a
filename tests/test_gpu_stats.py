"""On-device diagnostics against the FP64 oracle: running mean / RMS of u, P_h and T over sampled
steps, and the flame length (marching squares on the progress variable) of the GPU's own
temperature field."""
import numpy as np
import pytest

import workloads as W
from oracle.stats import flame_length, running_stats
from oracle.step import Oracle

pytestmark = pytest.mark.gpu


def _oracle_samples(wl, steps, interval):
    o = Oracle(wl.cfg, wl.mask, wl.inlet_u)
    st = o.init_state(T=wl.T, Y=wl.Y, u=wl.u, P_h=wl.P_h, g_pert=wl.g_pert)
    out = []
    for n in range(1, steps + 1):
        st = o.step(st)
        if n % interval == 0:
            f = [st["u"][a].numpy() for a in range(wl.cfg["dim"])] + [st["P_h"].numpy()]
            if wl.cfg.get("thermal"):
                f.append(st["T"].numpy())
            out.append(np.stack(f))
    return out


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_running_statistics_chamber(storage):
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.chamber_2d(nx=40, ny=20, inlet=True, dt=5e-7, storage=storage, seed=9, n_rows=1, per_row=1)
    s = from_workload(wl)
    s.stats_control(0)
    s.stats_control(1, 3)
    s.step(30)
    s.stats_control(2)
    s.step(4)  # not sampled
    mean, rms, n = s.stats()
    s.close()
    assert n == 10
    ref_mean, ref_rms = running_stats(_oracle_samples(wl, 30, 3))
    fluid = np.asarray(wl.mask).reshape(-1) == 0
    tol = 2e-6 if storage == "f64" else 2e-5  # FP32 accumulators; FP32 fields in the f32 run
    for f in range(mean.shape[0]):
        scale = np.abs(ref_mean[f][fluid]).max()
        assert np.abs(mean[f][fluid] - ref_mean[f][fluid]).max() <= tol * scale, f
        rscale = max(np.abs(ref_rms[f][fluid]).max(), 1e-300)
        # M2 in FP32: the RMS carries the mean's rounding relative to the fluctuation size
        assert np.abs(rms[f][fluid] - ref_rms[f][fluid]).max() <= 1e-3 * rscale + tol * scale, f


def test_running_statistics_swirl3d_cold():
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.swirl_3d(24, 16, 16, reactive=False, storage="f64", seed=2)
    s = from_workload(wl)
    s.stats_control(1, 2)
    s.step(12)
    mean, rms, n = s.stats()
    s.close()
    assert n == 6
    ref_mean, ref_rms = running_stats(_oracle_samples(wl, 12, 2))
    fluid = np.asarray(wl.mask).reshape(-1) == 0
    for f in range(mean.shape[0]):
        scale = np.abs(ref_mean[f][fluid]).max()
        assert np.abs(mean[f][fluid] - ref_mean[f][fluid]).max() <= 2e-6 * max(scale, 1e-12), f


@pytest.mark.parametrize("storage,level", [("f64", 0.5), ("f32", 0.2), ("f32", 0.8)])
def test_flame_length_matches_marching_squares(storage, level):
    from paper_2207_11567_gb300 import _lib as L
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.chamber_2d(nx=96, ny=48, storage=storage, seed=5, n_rows=1, per_row=2, hot_radius=60.0)
    s = from_workload(wl)
    s.step(10)
    T = s.fields(L.F_T)["T"]
    Tu, Tb = 300.0, 1950.0
    got = s.flame_length(level, Tu, Tb)
    s.close()
    nx, ny = wl.cfg["nx"], wl.cfg["ny"]
    ref = flame_length(((T - Tu) / (Tb - Tu)).reshape(ny, nx), (np.asarray(wl.mask) == 0).reshape(ny, nx), level)
    assert ref > 10.0
    assert abs(got - ref) <= 1e-10 * ref, (got, ref)
