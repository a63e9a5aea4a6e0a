"""The allocation-free thermodynamic-pressure integral (for callers that cannot allocate device
memory) gives the same integral as a context's own set-up reduction, on two calls in a row
(its static scratch array is shared and reused between calls)."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(L, T32, Y32, mask, N, W, T_ref, rho_ref, out, stream):
    err = C.create_string_buffer(256)
    Wa = (C.c_double * len(W))(*W)
    st = L.lib.lbm_pth_integral_noalloc(C.c_void_p(T32.data_ptr()), C.c_void_p(Y32.data_ptr()),
                                        C.c_void_p(mask.data_ptr()), N, len(W), Wa, T_ref, rho_ref,
                                        C.c_void_p(out.data_ptr()), C.c_void_p(stream), err, 256)
    return st, err.value.decode()


def test_noalloc_integral_matches_context_reduction():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import workloads as W
    from paper_2207_11567_gb300 import _lib as L
    from paper_2207_11567_gb300 import from_workload

    wl = W.generate.swirl_3d(40, 24, 24, reactive=True, seed=4)
    s = from_workload(wl)
    sc = s.scalars()
    I_ref = sc["M"] / sc["P_th"]  # the context's set-up reduction: M = P_th0 * I
    f = s.fields(L.F_T | L.F_Y, device=True)
    N, K = wl.N, len(wl.cfg["species"])
    T32 = f["T"].float().contiguous()
    Y32 = f["Y"].float().contiguous()
    mask = torch.as_tensor(np.asarray(wl.mask, np.uint8), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    Wk = [sp["W"] for sp in wl.cfg["species"]]
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.zero_()
        st, msg = _noalloc(L, T32, Y32, mask, N, Wk, wl.cfg["T_ref"], wl.cfg["rho_ref"], out, stream)
        assert st == L.LBM_OK, msg
        torch.cuda.synchronize()
        assert abs(out.item() - I_ref) <= 1e-12 * I_ref, (out.item(), I_ref)
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11567_gb300 import _lib as L
    t = torch.zeros(4, device="cuda")
    m = torch.zeros(4, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, msg = _noalloc(L, t, t, m, 1 << 25, [0.028], 300.0, 1.17, out, 0)
    assert st == L.LBM_ERR_ARG and "static scratch" in msg
