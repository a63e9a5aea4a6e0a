"""Discrete adjoint on the GPU: one step against the oracle's reverse mode (autograd through the
FP64 oracle step) at the same state, and the gradient of the fuel-consumption functional over
several steps with checkpointing, against the oracle's gradient and against central finite
differences of the GPU's own FP64 forward run. Case: 2-D reactive chamber with a velocity inlet,
pressure outlet, walls and an obstacle row, 6 species, two-step chemistry."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.adjoint_util import (oracle_fuel_gradient, oracle_vjp, pack_adjoint, seeded_adjoint,
                                state_from_buffer, unpack_adjoint)

pytestmark = pytest.mark.gpu

FUEL = 0  # CH4


def _case(storage="f64", nx=34, ny=18, smooth=True):
    """smooth: seeded initial flow, jittered inlet and a trace of every product, so that no upwind
    choice and no max(Y, 0) sits on its switch and J is differentiable at the point; otherwise the
    gas starts at rest with zero CO (roundoff then decides some upwind choices)."""
    extra = dict(inlet_jitter=0.1, u_init=0.01, y_trace=1e-4) if smooth else {}
    wl = W.generate.chamber_2d(nx=nx, ny=ny, inlet=True, u_in=0.02, dt=5e-7, storage=storage, seed=21,
                               n_rows=1, per_row=1, **extra)
    assert wl.cfg["species"][FUEL]["name"] == "CH4"
    return wl


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _one_step(storage, smooth=True, wl=None):
    from oracle.step import Oracle
    from paper_2207_11567_gb300 import from_workload
    wl = _case(storage, smooth=smooth) if wl is None else wl
    dt = torch.float64 if storage == "f64" else torch.float32
    s = from_workload(wl)
    s.step(3)
    state = s.save_state()
    o = Oracle(wl.cfg, wl.mask, wl.inlet_u)
    st = state_from_buffer(o, wl, state, dt)
    lam = seeded_adjoint(wl, seed=5)
    ref = oracle_vjp(o, st, lam)
    adj = torch.zeros(s.state_bytes() // dt.itemsize, dtype=dt, device="cuda")
    packed = torch.as_tensor(pack_adjoint(o, lam))
    adj[: packed.numel()] = packed.to(device="cuda", dtype=dt)
    gin = torch.zeros(2 * wl.cfg["ny"], dtype=dt, device="cuda")
    s.adjoint_step(state, adj, gin)
    got = unpack_adjoint(o, wl, adj.double().cpu().numpy())
    got["inlet"] = gin.double().cpu().numpy().reshape(2, -1)
    s.close()
    return {k: _rel(got[k], ref[k]) for k in ref}


def _flame_case(storage, extra_species=False):
    """Planar flame, 40 x 6, periodic in y (the slot sums wrap there), one-step chemistry with 4
    species, or 5 with a trace of H2O taken from N2 (the field-count-generic adjoint kernel); a
    seeded transverse velocity keeps the y-face velocities off zero."""
    from workloads.configs import species
    wl = W.generate.flame_2d(nx=40, ny=6, storage=storage, seed=3)
    rng = np.random.default_rng(9)
    wl.u[1] = 0.001 * rng.standard_normal(wl.N)
    if extra_species:
        tr = 1e-3
        wl.cfg["species"] = list(wl.cfg["species"]) + species(["H2O"])
        wl.Y = np.vstack([wl.Y, np.full((1, wl.N), tr)])
        wl.Y[3] -= tr
        y_in = list(wl.cfg["Y_in"]) + [tr]
        y_in[3] -= tr
        wl.cfg["Y_in"] = y_in
    return wl


@pytest.mark.parametrize("extra_species", [False, True])
def test_one_step_adjoint_planar_flame_f64(extra_species):
    wl = _flame_case("f64", extra_species)
    assert len(wl.cfg["species"]) == (5 if extra_species else 4)
    errs = _one_step("f64", wl=wl)
    assert max(errs.values()) < 1e-10, errs


def test_one_step_adjoint_f64():
    errs = _one_step("f64")
    assert max(errs.values()) < 1e-10, errs


def test_one_step_adjoint_at_rest_f64():
    # at the same state both sides take the same upwind choices, ties included
    errs = _one_step("f64", smooth=False)
    assert max(errs.values()) < 1e-10, errs


def test_chain_at_rest_matches_oracle_vjps_at_the_same_states():
    """Gas at rest, CO at zero: J is not differentiable at the point (upwind ties, max(Y, 0)), so
    compare the chained reverse with the oracle's reverse taken at the GPU's own states."""
    from oracle import fd as ofd
    from oracle.step import Oracle
    from paper_2207_11567_gb300 import from_workload
    wl = _case("f64", smooth=False)
    s = from_workload(wl)
    states = [s.save_state()]
    for _ in range(3):
        s.step(1)
        states.append(s.save_state())
    adj = torch.zeros(s.state_bytes() // 8, dtype=torch.float64, device="cuda")
    s.fuel_objective(FUEL, adj)
    gin = torch.zeros(2 * wl.cfg["ny"], dtype=torch.float64, device="cuda")
    for n in (2, 1, 0):
        s.adjoint_step(states[n], adj, gin)
    got = adj.cpu().numpy()
    o = Oracle(wl.cfg, wl.mask, wl.inlet_u)
    st = state_from_buffer(o, wl, states[3], torch.float64)
    T, Y = st["T"].clone().requires_grad_(), st["Y"].clone().requires_grad_()
    ofd.fuel_consumption(o.p, T, Y, st["P_th"], o.grid.fluid, FUEL).backward()
    lam = {"g": np.zeros((wl.Q, wl.N)), "u": np.zeros((2, wl.N)), "T": T.grad.numpy(), "Y": Y.grad.numpy()}
    inlet = 0.0
    for n in (2, 1, 0):
        o = Oracle(wl.cfg, wl.mask, wl.inlet_u)
        r = oracle_vjp(o, state_from_buffer(o, wl, states[n], torch.float64), lam)
        inlet = inlet + r["inlet"]
        lam = {k: r[k] for k in ("g", "u", "T", "Y")}
    s.close()
    ref = pack_adjoint(o, lam)
    assert _rel(got[: ref.size], ref) < 1e-10
    assert _rel(gin.cpu().numpy().reshape(2, -1), inlet) < 1e-10


def test_one_step_adjoint_isothermal_box_f64():
    """Isothermal mode (rho = 1, Lambda = 0): periodic box with a random flow, Smagorinsky on."""
    from oracle.step import Oracle
    from paper_2207_11567_gb300 import from_workload
    wl = W.generate.box(2, (20, 12), storage="f64", seed=3, pert=1e-3, U=0.03)
    wl.cfg["smag_cs"] = 0.17
    s = from_workload(wl)
    s.step(2)
    state = s.save_state()
    o = Oracle(wl.cfg, wl.mask, wl.inlet_u)
    st = state_from_buffer(o, wl, state, torch.float64)
    lam = seeded_adjoint(wl, seed=8)
    ref = oracle_vjp(o, st, lam)
    adj = torch.zeros(s.state_bytes() // 8, dtype=torch.float64, device="cuda")
    packed = torch.as_tensor(pack_adjoint(o, lam))
    adj[: packed.numel()] = packed.cuda()
    gin = torch.zeros(2 * wl.cfg["ny"], dtype=torch.float64, device="cuda")
    s.adjoint_step(state, adj, gin)
    got = unpack_adjoint(o, wl, adj.cpu().numpy())
    s.close()
    errs = {k: _rel(got[k], ref[k]) for k in ("g", "u")}
    assert max(errs.values()) < 1e-10, errs


def test_one_step_adjoint_f32():
    # same state, FP32 arithmetic: a few ulps of 2^-24 per operation through ~100 dependent
    # operations, amplified by the WENO weight derivatives (1/eps with eps = 1e-6 on Y)
    errs = _one_step("f32")
    assert max(errs.values()) < 2e-4, errs


def _problem(wl, n_steps, C):
    from paper_2207_11567_gb300 import AdjointProblem
    return AdjointProblem(wl.cfg, wl.mask, wl.Y, u0=wl.u, P_h0=wl.P_h, g_pert=wl.g_pert, n_steps=n_steps,
                          checkpoint_every=C, fuel=FUEL)


def test_fuel_gradient_matches_oracle_f64():
    wl = _case("f64")
    n_steps = 12
    J_ref, gin_ref, gT_ref = oracle_fuel_gradient(wl, n_steps, FUEL)
    pb = _problem(wl, n_steps, C=5)  # segments 5, 5, 2
    J = pb.forward(wl.inlet_u, wl.T)
    gin, gT = pb.backward()
    pb.close()
    assert abs(J - J_ref) <= 1e-11 * abs(J_ref)
    assert _rel(gin.cpu().numpy(), gin_ref) < 1e-9
    assert _rel(gT.cpu().numpy(), gT_ref) < 1e-9


def test_fuel_gradient_matches_finite_differences_f64():
    """Directional derivatives along seeded random directions (inlet: N(0, 1) x 10 % of the peak
    inlet velocity per row; T0: N(0, 1) x 10 K per fluid cell) vs central differences with
    h = 1e-4 of the GPU's own FP64 forward run. The error is measured against the sum of the
    magnitudes of the gradient-direction products, which a directional derivative can cancel."""
    wl = _case("f64")
    n_steps = 20
    pb = _problem(wl, n_steps, C=8)  # segments 8, 8, 4
    inlet0 = np.asarray(wl.inlet_u, dtype=np.float64).reshape(2, -1)
    T0 = np.asarray(wl.T, dtype=np.float64).reshape(-1)
    pb.forward(inlet0, T0)
    gin, gT = pb.backward()
    gin, gT = gin.cpu().numpy(), gT.cpu().numpy()
    rng = np.random.default_rng(1234)
    fluid = (np.asarray(wl.mask).reshape(-1) == 0).astype(np.float64)
    h = 1e-4
    worst = 0.0
    for _ in range(4):
        di = rng.standard_normal(inlet0.shape) * (inlet0 != 0) * 0.1 * np.abs(inlet0).max()
        dT = rng.standard_normal(T0.shape) * fluid * 10.0
        fd = (pb.forward(inlet0 + h * di, T0 + h * dT) - pb.forward(inlet0 - h * di, T0 - h * dT)) / (2 * h)
        ad = float((gin * di).sum() + (gT * dT).sum())
        scale = float(np.abs(gin * di).sum() + np.abs(gT * dT).sum())
        worst = max(worst, abs(ad - fd) / scale)
    pb.close()
    # O(h^2) truncation, about 1e-10 on this tie-free case; a kink crossed inside [-h, h]
    # (a species reaching zero, a face velocity changing sign) would show as 1e-6 or more
    assert worst < 1e-8, worst


def test_fuel_gradient_f32_close_to_f64():
    res = {}
    for storage in ("f64", "f32"):
        wl = _case(storage)
        pb = _problem(wl, 12, C=5)
        J = pb.forward(wl.inlet_u, wl.T)
        gin, gT = pb.backward()
        res[storage] = (J, gin.double().cpu().numpy(), gT.double().cpu().numpy())
        pb.close()
    (J64, gi64, gT64), (J32, gi32, gT32) = res["f64"], res["f32"]
    assert abs(J32 - J64) <= 1e-4 * abs(J64)
    assert np.linalg.norm(gi32 - gi64) <= 1e-3 * np.linalg.norm(gi64)
    assert np.linalg.norm(gT32 - gT64) <= 1e-3 * np.linalg.norm(gT64)


def test_autograd_function():
    from paper_2207_11567_gb300 import HybridStepFn
    wl = _case("f64")
    pb = _problem(wl, 6, C=4)
    inlet = torch.tensor(np.asarray(wl.inlet_u, dtype=np.float64).reshape(2, -1), requires_grad=True)
    T0 = torch.tensor(np.asarray(wl.T, dtype=np.float64).reshape(-1), requires_grad=True)
    J = HybridStepFn.apply(inlet, T0, pb)
    (2.0 * J).backward()
    J_ref, gin_ref, gT_ref = oracle_fuel_gradient(wl, 6, FUEL)
    pb.close()
    assert abs(J.item() - J_ref) <= 1e-11 * abs(J_ref)
    assert _rel(inlet.grad.numpy(), 2.0 * gin_ref) < 1e-9
    assert _rel(T0.grad.numpy(), 2.0 * gT_ref) < 1e-9


def test_autograd_two_graphs_reversed_in_any_order():
    """Two forward calls on the same problem with different inlet velocities and initial
    temperatures, each through HybridStepFn; the backward of the first graph, taken after the
    second forward, must still give the first call's gradient (oracle reverse mode)."""
    from paper_2207_11567_gb300 import HybridStepFn
    wl = _case("f64")
    pb = _problem(wl, 6, C=4)
    inlet0 = np.asarray(wl.inlet_u, dtype=np.float64).reshape(2, -1)
    T00 = np.asarray(wl.T, dtype=np.float64).reshape(-1)
    fluid = np.asarray(wl.mask).reshape(-1) == 0
    ia = torch.tensor(inlet0, requires_grad=True)
    ta = torch.tensor(T00, requires_grad=True)
    ib = torch.tensor(1.1 * inlet0, requires_grad=True)
    tb = torch.tensor(np.where(fluid, T00 + 5.0, T00), requires_grad=True)
    Ja = HybridStepFn.apply(ia, ta, pb)
    Jb = HybridStepFn.apply(ib, tb, pb)
    Ja.backward()
    Jb.backward()
    pb.close()
    ref_a = oracle_fuel_gradient(wl, 6, FUEL)
    ref_b = oracle_fuel_gradient(wl, 6, FUEL, inlet_u=1.1 * inlet0, T0=np.where(fluid, T00 + 5.0, T00))
    for J, gi, gt, (J_ref, gin_ref, gT_ref) in ((Ja, ia.grad, ta.grad, ref_a), (Jb, ib.grad, tb.grad, ref_b)):
        assert abs(J.item() - J_ref) <= 1e-11 * abs(J_ref)
        assert _rel(gi.numpy(), gin_ref) < 1e-9
        assert _rel(gt.numpy(), gT_ref) < 1e-9


def test_adjoint_rejects_unsupported_configs():
    from paper_2207_11567_gb300 import _lib as L, from_workload
    wl = W.generate.swirl_3d(nx=16, ny=12, nz=12, reactive=False, storage="f32", seed=1)
    s = from_workload(wl)
    state = s.save_state()
    adj = torch.zeros(s.state_bytes() // 4, dtype=torch.float32, device="cuda")
    gin = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(L.HLBMError):
        s.adjoint_step(state, adj, gin)
    s.close()


@pytest.mark.parametrize("n,case", [(3, "chamber"), (4, "chamber"), (4, "flame")])
def test_adjoint_segment_equals_single_steps(n, case):
    """lbm_adjoint_segment (recompute in the library, reverse over stored states, alternating
    buffers, the T and Y adjoints passed between steps in slot form) gives the same bits as n
    lbm_adjoint_step calls on saved states."""
    from paper_2207_11567_gb300 import from_workload
    wl = _case("f32") if case == "chamber" else _flame_case("f32")
    s = from_workload(wl)
    s.step(2)
    states = [s.save_state()]
    for _ in range(n):
        s.step(1)
        states.append(s.save_state())
    adj0 = torch.zeros(s.state_bytes() // 4, dtype=torch.float32, device="cuda")
    s.fuel_objective(FUEL, adj0)
    a1, g1 = adj0.clone(), torch.zeros(2 * wl.cfg["ny"], dtype=torch.float32, device="cuda")
    for k in reversed(range(n)):
        s.adjoint_step(states[k], a1, g1)
    a2, g2 = adj0.clone(), torch.zeros_like(g1)
    s.adjoint_segment(states[0], n, a2, g2)
    s.close()
    nw = (wl.Q + 2 + 1 + len(wl.cfg["species"])) * wl.N
    assert torch.equal(a1[:nw], a2[:nw])
    assert torch.equal(g1, g2)


@pytest.mark.parametrize("K,C", [(11, 4), (12, 4), (5, 5), (7, 3)])
def test_adjoint_sweep_equals_segments(K, C):
    """lbm_adjoint_sweep (recompute of the next segment on a second stream, two-segment workspace)
    gives the same bits as lbm_adjoint_segment over the segments from last to first, including
    a shorter last segment and a single segment."""
    from paper_2207_11567_gb300 import from_workload
    wl = _case("f32")
    s = from_workload(wl)
    s.step(2)
    ckpts = []
    for n in range(K):
        if n % C == 0:
            ckpts.append(s.save_state())
        s.step(1)
    adjK = torch.zeros(s.state_bytes() // 4, dtype=torch.float32, device="cuda")
    s.fuel_objective(FUEL, adjK)
    a1, g1 = adjK.clone(), torch.zeros(2 * wl.cfg["ny"], dtype=torch.float32, device="cuda")
    for seg in reversed(range(len(ckpts))):
        s.adjoint_segment(ckpts[seg], min(C, K - seg * C), a1, g1)
    a2, g2 = adjK.clone(), torch.zeros_like(g1)
    s.adjoint_sweep(ckpts, C, K, a2, g2)
    s.close()
    nw = (wl.Q + 2 + 1 + len(wl.cfg["species"])) * wl.N
    assert torch.equal(a1[:nw], a2[:nw])
    assert torch.equal(g1, g2)


def test_chamber_512x128_full_horizon_gradient():
    """The 512 x 128 chamber from its fields 400 steps after ignition, K = 2000, checkpoints every
    100 steps: the FP32 gradient is finite and within 1e-3 (relative L2) of the FP64 one, and the
    FP64 gradient agrees with central differences (h = 1e-6) along 4 Philox directions to 1e-3 of
    sum |grad_i d_i|. (At h = 1e-4 the secants cross kinks of the discrete map, such as upwind
    switches and the max(Y, 0) of the rate law, and differ from the gradient by ~1e-3.)"""
    from paper_2207_11567_gb300 import AdjointProblem, Solver
    from paper_2207_11567_gb300 import _lib as L
    wl = W.make("c5_adjoint_2d")
    inlet0 = np.asarray(wl.inlet_u, dtype=np.float64).reshape(2, -1)
    s = Solver(dict(wl.cfg, storage="f64"), wl.mask, inlet0)
    s.set_fields(T=wl.T, Y=wl.Y, u=wl.u, P_h=wl.P_h)
    s.step(400)
    f = s.fields(L.F_T | L.F_Y | L.F_U | L.F_PH)
    s.close()
    fluid = (np.asarray(wl.mask).reshape(-1) == 0).astype(np.float64)
    grads = {}
    for storage in ("f32", "f64"):
        p = AdjointProblem(dict(wl.cfg, storage=storage), wl.mask, f["Y"], u0=f["u"], P_h0=f["P_h"], n_steps=2000,
                           checkpoint_every=100, fuel=FUEL)
        p.forward(inlet0, f["T"])
        gi, gt = (v.double().cpu().numpy() for v in p.backward())
        grads[storage] = np.concatenate([gi.ravel(), gt.ravel()])
        if storage == "f64":
            rng = np.random.Generator(np.random.Philox(2207))
            h = 1e-6
            for _ in range(4):
                di = rng.standard_normal(inlet0.shape) * (inlet0 != 0) * 0.1 * np.abs(inlet0).max()
                dT = rng.standard_normal(f["T"].shape) * fluid * 10.0
                fd = (p.forward(inlet0 + h * di, f["T"] + h * dT) - p.forward(inlet0 - h * di, f["T"] - h * dT)) / (2 * h)
                ad = float((gi * di).sum() + (gt * dT).sum())
                err = abs(ad - fd) / float(np.abs(gi * di).sum() + np.abs(gt * dT).sum())
                assert err <= 1e-3, (ad, fd, err)
        p.close()
    g32, g64 = grads["f32"], grads["f64"]
    assert np.isfinite(g32).all()
    rel = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    print("FP32 vs FP64 gradient, relative L2:", rel)
    assert rel <= 1e-3, rel
