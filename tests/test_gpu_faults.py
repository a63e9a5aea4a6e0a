"""Failure reporting of the library, with every failure made on the host (no device fault):
an allocator that returns NULL, calls out of order, a NaN injected into the initial fields on
the host (the device's non-finite flag must come back as LBM_ERR_NONFINITE), and recovery of the
same context after new fields are set."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def test_allocator_returning_null_gives_alloc_error():
    from paper_2207_11567_gb300 import _lib as L
    wl = W.generate.box(2, 16, storage="f32", seed=1)
    calls = {"alloc": 0, "free": 0}

    def alloc(nbytes, user):
        calls["alloc"] += 1
        return None

    def free(ptr, user):
        calls["free"] += 1

    fa, ff = L.ALLOC_FN(alloc), L.FREE_FN(free)
    stream = torch.cuda.Stream()
    cfg = L.config_from_dict(wl.cfg, C.c_void_p(stream.cuda_stream))
    cfg.alloc, cfg.free = fa, ff
    ctx = C.c_void_p()
    st = L.lib.lbm_init(C.byref(cfg), C.byref(ctx))
    assert st == L.LBM_ERR_ALLOC
    assert calls["alloc"] >= 1
    assert "alloc" in L.lib.lbm_last_error(ctx).decode().lower() if ctx else True
    L.lib.lbm_destroy(ctx)


def test_allocator_failing_later_is_reported_and_context_survives(monkeypatch):
    """Allocations succeed at set-up; the adjoint's workspace allocation fails (the torch
    allocator raises, the hook returns NULL): the call reports LBM_ERR_ALLOC, and once the
    allocator works again the same context steps and computes the adjoint."""
    from paper_2207_11567_gb300 import _lib as L
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.chamber_2d(nx=24, ny=12, inlet=True, storage="f32", seed=2, n_rows=1, per_row=1)
    s = from_workload(wl)
    s.step(2)
    state = s.save_state()
    adj = torch.zeros(s.state_bytes() // 4, dtype=torch.float32, device="cuda")
    gin = torch.zeros(2 * wl.cfg["ny"], dtype=torch.float32, device="cuda")

    def refuse(*args, **kw):
        raise RuntimeError("allocation refused by the test")

    with monkeypatch.context() as m:
        m.setattr(torch.cuda, "caching_allocator_alloc", refuse)
        with pytest.raises(L.HLBMError) as e:
            s.adjoint_step(state, adj, gin)
        assert e.value.status == L.LBM_ERR_ALLOC
    s.step(1)
    s.adjoint_step(state, adj, gin)
    s.synchronize()
    assert torch.isfinite(adj).all()
    s.close()


def test_step_before_fields_is_a_state_error():
    from paper_2207_11567_gb300 import _lib as L
    from paper_2207_11567_gb300.solver import Solver
    wl = W.generate.box(2, 16, storage="f32", seed=1)
    s = Solver(wl.cfg, wl.mask, wl.inlet_u)
    assert L.lib.lbm_step(s.ctx, 1) == L.LBM_ERR_STATE
    assert "set_fields" in L.lib.lbm_last_error(s.ctx).decode()
    s.close()


@pytest.mark.parametrize("field", ["T", "u"])
def test_nan_injected_on_host_is_reported_as_nonfinite(field):
    from paper_2207_11567_gb300 import _lib as L
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.chamber_2d(nx=32, ny=16, inlet=True, storage="f32", seed=3, n_rows=1, per_row=1)
    s = from_workload(wl)
    s.step(3)
    s.fields(L.F_T)  # clean run: no error
    bad = {"T": np.array(wl.T, dtype=np.float64), "u": np.array(wl.u, dtype=np.float64)}
    fluid = np.nonzero(np.asarray(wl.mask).reshape(-1) == 0)[0]
    r = int(fluid[len(fluid) // 2])
    if field == "T":
        bad["T"][r] = np.nan
    else:
        bad["u"][0, r] = np.nan
    s.set_fields(T=bad["T"], Y=wl.Y, u=bad["u"], P_h=wl.P_h)
    s.step(2)
    with pytest.raises(L.HLBMError) as e:
        s.fields(L.F_T)
    assert e.value.status == L.LBM_ERR_NONFINITE
    # the flag is cleared once reported; fresh finite fields run clean on the same context
    s.set_fields(T=wl.T, Y=wl.Y, u=wl.u, P_h=wl.P_h)
    s.step(2)
    f = s.fields(L.F_T | L.F_U)
    assert np.isfinite(f["T"]).all() and np.isfinite(f["u"]).all()
    s.close()
