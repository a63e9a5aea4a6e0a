"""Host I/O paths of the C ABI: fields given in pinned host memory are read by the kernels in
place and fields read back into pinned host memory are written in place; pageable memory goes
through a device staging buffer. Both paths give the same bits."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _pinned(a):
    t = torch.empty(np.asarray(a).size, dtype=torch.float64, pin_memory=True)
    v = t.numpy()
    v[:] = np.asarray(a, dtype=np.float64).reshape(-1)
    return v


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_pinned_and_pageable_io_agree(storage):
    from paper_2207_11567_gb300 import Solver
    from paper_2207_11567_gb300 import _lib as L
    wl = W.generate.chamber_2d(nx=48, ny=24, inlet=True, storage=storage, seed=11, n_rows=1, per_row=1)
    bits = L.F_T | L.F_Y | L.F_U | L.F_PH | L.F_G
    res = []
    for pin in (False, True):
        s = Solver(wl.cfg, wl.mask, wl.inlet_u)
        conv = _pinned if pin else (lambda a: np.array(a, dtype=np.float64))
        s.set_fields(T=conv(wl.T), Y=conv(wl.Y), u=conv(wl.u), P_h=conv(wl.P_h))
        s.step(7)
        n = L.lib.lbm_fields_size(s.ctx, bits)
        out = _pinned(np.zeros(n)) if pin else np.zeros(n)
        s.fields(bits, out=out)
        res.append(np.array(out))
        s.close()
    assert np.array_equal(res[0], res[1])
