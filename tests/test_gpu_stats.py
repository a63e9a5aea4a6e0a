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


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_probe_series_match_oracle(storage):
    """Probes at fluid cells of the chamber with an inlet, sampled every 2nd step for 30 steps, with
    statistics on at the same time: the GPU series equal the oracle's field values at those cells
    (FP64 to 1e-10 of each field's range; FP32 to the storage floor), and a probe on a solid cell
    is refused."""
    from paper_2207_11567_gb300 import _lib as L
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.chamber_2d(nx=40, ny=20, inlet=True, dt=5e-7, storage=storage, seed=9, n_rows=1, per_row=1)
    fluid = np.nonzero(wl.mask == 0)[0]
    cells = fluid[[3, 150, 400, len(fluid) - 5]]
    s = from_workload(wl)
    with pytest.raises(L.HLBMError):
        s.set_probes([int(np.nonzero(wl.mask)[0][0])])
    s.set_probes(cells, capacity=64, interval=2)
    s.stats_control(1, 5)
    s.step(30)
    ser = s.probes()
    s.close()
    ref = np.stack([o[:, cells].T for o in _oracle_samples(wl, 30, 2)])  # [n][probe][field]
    assert ser.shape == ref.shape == (15, 4, 4)
    scale = np.abs(ref).max(axis=(0, 1)) + 1e-300
    err = (np.abs(ser - ref).max(axis=(0, 1)) / scale).max()
    assert err < (1e-10 if storage == "f64" else 1e-4), err


def test_probe_ring_keeps_the_latest_samples_in_order():
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.chamber_2d(nx=40, ny=20, inlet=True, dt=5e-7, storage="f64", seed=9, n_rows=1, per_row=1)
    fluid = np.nonzero(wl.mask == 0)[0]
    s = from_workload(wl)
    s.set_probes(fluid[[10, 20]], capacity=64, interval=1)
    s.step(40)
    full = s.probes()
    s2 = from_workload(wl)
    s2.set_probes(fluid[[10, 20]], capacity=16, interval=1)
    s2.step(40)
    ring = s2.probes()
    s.close()
    s2.close()
    assert full.shape[0] == 40 and ring.shape[0] == 16
    assert np.array_equal(ring, full[-16:])


def test_welch_psd_matches_oracle():
    """Seeded series (a tone between bins plus noise) handed to the device: lbm_welch_psd equals
    the oracle's numpy estimate, also over a strided view."""
    import torch
    from oracle.stats import welch_psd
    from paper_2207_11567_gb300 import from_workload
    rng = np.random.default_rng(5)
    dt, n = 2e-5, 6000
    t = np.arange(n) * dt
    x = 3.0 + np.sin(2 * np.pi * 517.3 * t) + 0.2 * rng.standard_normal(n)
    s = from_workload(W.generate.box(2, 8, storage="f64"))
    for L in (64, 512):
        f, p = s.welch_psd(torch.tensor(x, dtype=torch.float64, device="cuda"), dt, L)
        fo, po = welch_psd(x, dt, L)
        assert np.allclose(f, fo, rtol=1e-15, atol=0)
        assert np.abs(p - po).max() < 1e-11 * po.max()
    xx = np.stack([x, -x, 2 * x], axis=1).reshape(-1)
    f, p = s.welch_psd(torch.tensor(xx, dtype=torch.float64, device="cuda"), dt, 256, stride=3)
    fo, po = welch_psd(x, dt, 256)
    assert np.abs(p - po).max() < 1e-11 * po.max()
    s.close()


def test_probe_spectrum_matches_oracle():
    """lbm_probe_spectrum over a wrapped ring (130 samples every 2nd step into 96 slots) against the
    oracle's Welch estimate of the oracle's own series at that cell over the same 96 samples: the
    ordering of the ring, the sampling interval and the estimate together."""
    from oracle.stats import welch_psd
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.chamber_2d(nx=40, ny=20, inlet=True, dt=5e-7, storage="f64", seed=9, n_rows=1, per_row=1)
    fluid = np.nonzero(wl.mask == 0)[0]
    cells = fluid[[50, 300]]
    s = from_workload(wl)
    s.set_probes(cells, capacity=96, interval=2)
    s.step(260)
    f, p = s.probe_spectrum(1, 2, 32)
    s.close()
    ref = np.array([o[2, cells[1]] for o in _oracle_samples(wl, 260, 2)])[-96:]  # P_h at probe 1
    fo, po = welch_psd(ref, 2 * wl.cfg["dt"], 32)
    assert np.allclose(f, fo, rtol=1e-15, atol=0)
    assert np.abs(p - po).max() < 1e-7 * po.max(), np.abs(p - po).max() / po.max()
