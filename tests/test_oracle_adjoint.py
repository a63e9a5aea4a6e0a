"""Pins of the oracle's reverse mode (the reference of the GPU adjoint): the objective against
the species update it comes from, and autograd gradients through several oracle steps against
central finite differences of the oracle itself."""
import numpy as np
import torch

import workloads as W
from oracle import fd as ofd
from oracle.step import Oracle
from oracle.units import R_GAS
from tests.adjoint_util import oracle_fuel_gradient

FUEL = 0


def test_fuel_consumption_is_the_fuel_mass_rate_of_a_uniform_update():
    """In a uniform field at rest the FD update reduces to explicit chemistry,
    Y_F^{n+1} = Y_F + dt omega_F / (rho F), so J = -sum rho F (Y_F^{n+1} - Y_F) / dt."""
    wl = W.generate.chamber_2d(nx=8, ny=6, storage="f64", seed=3, n_rows=1, per_row=1)
    o = Oracle(wl.cfg, np.zeros_like(np.asarray(wl.mask)), None)
    p = o.p
    N = o.grid.N
    T = torch.full((N,), 1500.0, dtype=torch.float64)
    Y = torch.as_tensor(p.Y_in, dtype=torch.float64)[:, None].repeat(1, N)
    u = torch.zeros(p.dim, N, dtype=torch.float64)
    T1, Y1, rho, _ = ofd.fd_update(p, o.grid, o.nb, T, Y, u, torch.zeros(p.dim, N, dtype=torch.float64),
                                   p.P_th0, 0.0)
    rho_phys = p.P_th0 * ofd.mean_molar_mass(p, Y) / (R_GAS * T)
    J = ofd.fuel_consumption(p, T, Y, p.P_th0, o.grid.fluid, FUEL).item()
    J_update = (-(rho_phys * p.F * (Y1[FUEL] - Y[FUEL]) / p.dt)).sum().item()
    assert J > 0
    assert abs(J - J_update) <= 1e-9 * J


def test_oracle_gradient_matches_central_differences():
    wl = W.generate.chamber_2d(nx=16, ny=8, inlet=True, u_in=0.02, dt=5e-7, storage="f64", seed=21,
                               n_rows=1, per_row=1, inlet_jitter=0.1, u_init=0.01, y_trace=1e-4)
    n = 4
    J0, gin, gT = oracle_fuel_gradient(wl, n, FUEL)
    inlet0 = np.asarray(wl.inlet_u, dtype=np.float64).reshape(2, -1)
    T0 = np.asarray(wl.T, dtype=np.float64).reshape(-1)
    fluid = (np.asarray(wl.mask).reshape(-1) == 0).astype(np.float64)
    rng = np.random.default_rng(7)
    h = 1e-4
    for _ in range(3):
        di = rng.standard_normal(inlet0.shape) * (inlet0 != 0) * np.abs(inlet0).max()
        dT = rng.standard_normal(T0.shape) * fluid * 100.0
        Jp, _, _ = oracle_fuel_gradient(wl, n, FUEL, inlet_u=inlet0 + h * di, T0=T0 + h * dT)
        Jm, _, _ = oracle_fuel_gradient(wl, n, FUEL, inlet_u=inlet0 - h * di, T0=T0 - h * dT)
        fd = (Jp - Jm) / (2 * h)
        ad = float((gin * di).sum() + (gT * dT).sum())
        scale = float(np.abs(gin * di).sum() + np.abs(gT * dT).sum())
        # O(h^2) truncation only (about 1e-10 here). The case is built without ties: an exact
        # upwind tie (gas at rest, or a mirror-symmetric state) or a species at exactly zero (the
        # max(Y, 0) of the rate law) puts a kink at the point, and central differences then
        # average the one-sided derivatives: a gap of 1e-7 to 1e-6 at every h
        assert abs(ad - fd) <= 1e-8 * scale, (ad, fd, scale)
