"""Properties of a planar premixed flame, FP64 (test infrastructure like the rest of the oracle;
only the tests and the benchmark's CPU baseline use it).

Section 3.1 takes the burnt-gas composition, the adiabatic temperature and the interface
thickness of its initial fields from a 1-D freely propagating flame computed with the same scheme
and mixture; Section 3.2.2 gives that flame's speed S_L and its thickness as the temperature rise
divided by the largest temperature gradient. For a flame that propagates along x through the
grid, with column means taken over the fluid cells of each x column (the y and z directions):

* consumption speed (reading: the paper names S_L without saying how it is measured; the
  consumption speed is the flame speed that follows from the fuel balance of a steady 1-D flame,
  S_c rho_u Y_F,u = integral of the fuel consumption rate over x):
      S_c = sum over fluid cells of (-omega_F / F_loc) dx / (rho_u Y_F,u A)
  with A the ny nz cells of the cross-section, rho_u = P_th W_u / (R T_in) and Y_F,u = Y_in[F]
  the inlet (unburnt) state, omega_F the fuel rate of the rate law of ``fd`` and F_loc the
  thickening factor of the update at this state (the rate the species equation actually sees;
  the thickened flame burns F times slower over an F times wider front, so S_c stays);
* thickness  delta_L = (T_max - T_min) / max |dT/dx|, T_min and T_max the extremes of the
  column-mean temperature and dT/dx its centred difference (T(x+1) - T(x-1)) / (2 dx) at the
  columns whose two neighbours hold fluid;
* flame position x_f: the first crossing, going up in x, of the mid temperature
  (T_min + T_max)/2 by the column means, placed linearly between column centres x dx;
* burnt state: the column means of T and Y_k at the last column (largest x) holding fluid.

Parity pins: closed forms on tanh profiles and on uniform states (tests/test_oracle_pins.py).
"""
import numpy as np
import torch

from . import fd as fdm
from .units import R_GAS


def column_means(grid, f):
    """Mean over the fluid cells of each x column of f [N]; returns (means [nx], counts [nx]),
    0 where a column holds no fluid."""
    nx, ny, nz = grid.shape
    v = np.asarray(f, dtype=np.float64).reshape(nz, ny, nx)
    fl = grid.fluid.numpy().reshape(nz, ny, nx)
    n = fl.sum(axis=(0, 1)).astype(np.float64)
    s = np.where(fl, v, 0.0).sum(axis=(0, 1))
    return np.where(n > 0, s / np.where(n > 0, n, 1.0), 0.0), n


def fuel_rate(p, T, Y, P_th, fuel):
    """-omega_F / F_loc per cell [kg/(m^3 s)]: the fuel source of the update, rho = P_th W / (R T)."""
    T = torch.as_tensor(np.asarray(T, dtype=np.float64))
    Y = torch.as_tensor(np.asarray(Y, dtype=np.float64))
    rho_phys = P_th * fdm.mean_molar_mass(p, Y) / (R_GAS * T)
    om = fdm.species_rates(p, fdm.reaction_rates(p, T, Y, rho_phys))[fuel]
    return -(om.expand_as(T) / fdm.thickening(p, T, Y)).numpy()


def profile_properties(Tm, n, dx):
    """delta_L, x_f, T_min, T_max from column means Tm [nx] and fluid counts n [nx]."""
    has = n > 0
    Tmin, Tmax = Tm[has].min(), Tm[has].max()
    gmax = 0.0
    for x in range(1, len(Tm) - 1):
        if has[x - 1] and has[x + 1]:
            gmax = max(gmax, abs(Tm[x + 1] - Tm[x - 1]) / (2.0 * dx))
    delta = (Tmax - Tmin) / gmax if gmax > 0 else 0.0
    mid = 0.5 * (Tmin + Tmax)
    xf = -1.0
    for x in range(len(Tm) - 1):
        if not (has[x] and has[x + 1]):
            continue
        a, b = Tm[x] - mid, Tm[x + 1] - mid
        if a != b and ((a <= 0 <= b) or (a >= 0 >= b)):
            xf = dx * (x + a / (a - b))
            break
    return delta, xf, Tmin, Tmax


def flame_properties(p, grid, T, Y, P_th, fuel):
    """Dict S_c (m/s), delta_L (m), x_f (m), T_min, T_max, T_b, Y_b [K] and the column means
    T, w_F (-omega_F / F_loc) and Y [K][nx] of the state (T [N], Y [K][N], P_th in Pa)."""
    dx = p.cfg["dx"]
    nx, ny, nz = grid.shape
    T = np.asarray(T, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    w = fuel_rate(p, T, Y, P_th, fuel)
    Tm, n = column_means(grid, T)
    wm, _ = column_means(grid, w)
    Ym = np.stack([column_means(grid, Y[k])[0] for k in range(p.K)])
    W_u = 1.0 / sum(p.Y_in[k] / p.W[k] for k in range(p.K))
    rho_u = P_th * W_u / (R_GAS * p.T_in)
    fl = grid.fluid.numpy()
    S_c = w[fl].sum() * dx / (rho_u * p.Y_in[fuel] * ny * nz)
    delta, xf, Tmin, Tmax = profile_properties(Tm, n, dx)
    last = int(np.nonzero(n > 0)[0].max())
    return {"S_c": S_c, "delta_L": delta, "x_f": xf, "T_min": Tmin, "T_max": Tmax,
            "T_b": Tm[last], "Y_b": Ym[:, last].copy(), "T": Tm, "w_F": wm, "Y": Ym}
