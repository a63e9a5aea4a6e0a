"""The allocation-free thermodynamic-pressure integral, for callers that cannot allocate device
memory: its result equals the FP64 oracle's integral of the same FP32 fields on two calls in a
row (its static scratch array is shared and reused between calls), for the chemistry's molar
masses and for light and heavy ones; a fluid cell at T = 0 gives NaN; sizes beyond its scratch
are refused."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import geometry as geo
from oracle.step import pth_integral
from oracle.units import Params

pytestmark = pytest.mark.gpu


def _noalloc(L, T32, Y32, mask, N, W, T_ref, rho_ref, out, stream):
    err = C.create_string_buffer(256)
    Wa = (C.c_double * len(W))(*W)
    st = L.lib.lbm_pth_integral_noalloc(C.c_void_p(T32.data_ptr()), C.c_void_p(Y32.data_ptr()),
                                        C.c_void_p(mask.data_ptr()), N, len(W), Wa, T_ref, rho_ref,
                                        C.c_void_p(out.data_ptr()), C.c_void_p(stream), err, 256)
    return st, err.value.decode()


def _fields(wl, Wk, seed):
    """Seeded FP32 temperature (300-2200 K) and mass fractions (a random point of the simplex per
    cell) on the workload's mask."""
    rng = np.random.default_rng(seed)
    N, K = wl.N, len(Wk)
    T = rng.uniform(300.0, 2200.0, N).astype(np.float32)
    Y = rng.dirichlet(np.ones(K), N).T.astype(np.float32)
    return T, Y


def _oracle_integral(wl, Wk, T, Y):
    cfg = dict(wl.cfg)
    cfg["species"] = [{"W": w, "Le": 1.0, "hf": 0.0} for w in Wk]
    p = Params(cfg)
    grid = geo.Grid(cfg, wl.mask)
    return pth_integral(p, grid, torch.as_tensor(T.astype(np.float64)), torch.as_tensor(Y.astype(np.float64)))


@pytest.mark.parametrize("which", ["chemistry", "light", "heavy"])
def test_noalloc_integral_matches_oracle(which):
    import __graft_entry__
    __graft_entry__.build()
    import workloads as W
    from paper_2207_11567_gb300 import _lib as L

    wl = W.generate.swirl_3d(40, 24, 24, reactive=True, seed=4)
    Wk = {"chemistry": [sp["W"] for sp in wl.cfg["species"]],
          "light": [0.002016, 0.004003, 0.018015, 0.028014],
          "heavy": [0.1, 0.2, 0.3]}[which]
    T, Y = _fields(wl, Wk, seed=len(Wk))
    I_ref = _oracle_integral(wl, Wk, T, Y)
    N = wl.N
    T32 = torch.as_tensor(T, device="cuda")
    Y32 = torch.as_tensor(Y, device="cuda").contiguous()
    mask = torch.as_tensor(np.asarray(wl.mask, np.uint8), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(-1.0)
        st, msg = _noalloc(L, T32, Y32, mask, N, Wk, wl.cfg["T_ref"], wl.cfg["rho_ref"], out, stream)
        assert st == L.LBM_OK, msg
        torch.cuda.synchronize()
        # per-cell FP32 terms (rounding 6e-8 relative) summed exactly: 1e-6 relative covers it
        assert abs(out.item() - I_ref) <= 1e-6 * I_ref, (out.item(), I_ref)


def test_noalloc_zero_temperature_gives_nan():
    import __graft_entry__
    __graft_entry__.build()
    import workloads as W
    from paper_2207_11567_gb300 import _lib as L

    wl = W.generate.swirl_3d(40, 24, 24, reactive=True, seed=4)
    Wk = [sp["W"] for sp in wl.cfg["species"]]
    T, Y = _fields(wl, Wk, seed=3)
    fluid = np.nonzero(np.asarray(wl.mask).reshape(-1) == 0)[0]
    T[fluid[len(fluid) // 2]] = 0.0
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    mask = torch.as_tensor(np.asarray(wl.mask, np.uint8), device="cuda")
    st, msg = _noalloc(L, torch.as_tensor(T, device="cuda"), torch.as_tensor(Y, device="cuda").contiguous(), mask,
                       wl.N, Wk, wl.cfg["T_ref"], wl.cfg["rho_ref"], out, torch.cuda.current_stream().cuda_stream)
    assert st == L.LBM_OK, msg
    torch.cuda.synchronize()
    assert np.isnan(out.item())
    # the next call on valid fields is clean again (the counter is cleared per call)
    T[fluid[len(fluid) // 2]] = 800.0
    st, msg = _noalloc(L, torch.as_tensor(T, device="cuda"), torch.as_tensor(Y, device="cuda").contiguous(), mask,
                       wl.N, Wk, wl.cfg["T_ref"], wl.cfg["rho_ref"], out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == L.LBM_OK and np.isfinite(out.item())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11567_gb300 import _lib as L
    t = torch.zeros(4, device="cuda")
    m = torch.zeros(4, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, msg = _noalloc(L, t, t, m, 1 << 25, [0.028], 300.0, 1.17, out, 0)
    assert st == L.LBM_ERR_ARG and "static scratch" in msg
