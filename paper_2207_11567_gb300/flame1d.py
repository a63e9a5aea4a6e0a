"""1-D freely propagating premixed flame: laminar flame speed, thickness and burnt state.

Section 3.1 sets up its reacting run with the burnt-gas composition, the adiabatic temperature
and the interface thickness of a 1-D freely propagating flame computed with the same scheme and
mixture; Section 3.2.2 quotes S_L and delta_L = (T_max - T_min) / max dT/dx of such a flame. Here
that flame is the library's own planar flame: a channel that is periodic across (y, z), fresh
gas entering at x = 0 with the inlet velocity, burnt gas leaving at the high-x outlet.

A free flame moves against the fresh gas at S_L; to keep it inside the channel the inlet
velocity follows the measured consumption speed S_c (lbm_flame_properties), with a
proportional correction that pulls the flame position x_f back to a target:
    u_in = <S_c> - gain (x_f - x_target) / tau_f                (velocities in m/s)
applied every ``chunk`` steps (lbm_set_inlet), with <S_c> the mean consumption speed over the
last flame time tau_f = delta_L / S_c. With the fresh gas arriving at <S_c> the position error
decays as exp(-gain t / tau_f): slow against the flame's own response (about one flame time),
so that the loop does not ring, and blind to the small oscillation of S_c as a thin front
crosses grid cells. The run has converged when the means of S_c over the last two windows of one
flame time (at least ``window`` chunks each) differ by less than ``tol``, x_f has stayed within
two cells of the target over both, and the gas burnt since the start has swept the channel behind
the flame twice (burnt-gas velocity estimated as <S_c> T_max / T_min), so that the outlet holds
the flame's own burnt state; S_L is the mean of the last window. Every step and every
measurement runs in the library's kernels; this module only chooses the inlet velocity and
keeps the history.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class FlameSolution:
    S_L: float             # consumption speed (m/s) at convergence
    delta_L: float         # (T_max - T_min) / max dT/dx (m)
    T_b: float             # burnt temperature (K): column mean at the outlet
    Y_b: np.ndarray        # burnt mass fractions [K]
    T_u: float             # fresh-gas temperature (K)
    x_f: float             # flame position (m): mid-temperature crossing
    x: np.ndarray          # column centres (m)
    T: np.ndarray          # column-mean temperature [nx]
    Y: np.ndarray          # column-mean mass fractions [K][nx]
    w_F: np.ndarray        # column-mean fuel consumption rate -omega_F [nx] (kg/(m^3 s))
    steps: int
    converged: bool
    history: list = field(default_factory=list)  # (step, S_c, x_f, u_in) per chunk

    def fields_at(self, distance):
        """T and Y at signed distances (m) from the mid-temperature point, positive towards the
        burnt gas: the converged profile, held constant beyond its ends. Gives initial fields
        with the flame's own interface for a reacting run (e.g. a burnt-gas pocket with
        distance = r - r_0 turned inside out: pass r_0 - r)."""
        d = np.asarray(distance, dtype=np.float64)
        xs = self.x_f + d
        T = np.interp(xs, self.x, self.T)
        Y = np.stack([np.interp(xs, self.x, self.Y[k]) for k in range(self.Y.shape[0])])
        return T, Y


def free_flame(solver, fuel=0, x_target=None, chunk=200, gain=0.2, tol=2e-3, window=5, max_steps=400000,
               u_max=None):
    """Run the planar flame held by ``solver`` (a ``Solver`` whose fields are already set: inlet at
    low x, outlet at high x, periodic across) until its consumption speed is steady.

    x_target: where the flame is held (m), default the initial flame position. u_max: upper
    bound of the inlet velocity (m/s), default a lattice Mach number of 0.1. Raises RuntimeError
    if the flame leaves the channel or is extinguished."""
    cfg = solver.cfg
    dx, dt = cfg["dx"], cfg["dt"]
    nx = cfg["nx"]
    n_face = solver.N // nx
    lat = dt / dx  # m/s -> lattice velocity
    if u_max is None:
        u_max = 0.1 / np.sqrt(3.0) / lat
    p = solver.flame_properties(fuel)
    if p["x_f"] < 0:
        raise RuntimeError("no flame in the initial fields (no mid-temperature crossing)")
    if x_target is None:
        x_target = p["x_f"]
    hist = []
    steps = 0
    converged = False
    S_L = p["S_c"]
    while steps < max_steps:
        solver.step(chunk)
        steps += chunk
        p = solver.flame_properties(fuel)
        S, xf = p["S_c"], p["x_f"]
        if not np.isfinite(S) or xf < 0 or xf > (nx - 1) * dx:
            raise RuntimeError(f"flame left the channel or went out after {steps} steps (x_f={xf}, S_c={S})")
        if S <= 0 or p["T_max"] - p["T_min"] < 1e-3 * p["T_min"]:
            raise RuntimeError(f"flame extinguished after {steps} steps")
        hist.append((steps, S, xf, 0.0))
        tau = max(p["delta_L"], dx) / S
        L = max(window, int(np.ceil(tau / (chunk * dt))))
        S_bar = float(np.mean([h[1] for h in hist[-L:]]))
        u = float(np.clip(S_bar - gain * (xf - x_target) / tau, 0.0, u_max))
        hist[-1] = (steps, S, xf, u)
        solver.set_inlet(np.concatenate([np.full(n_face, u * lat), np.zeros((solver.dim - 1) * n_face)]))
        if len(hist) >= 2 * L:
            a = np.mean([h[1] for h in hist[-L:]])
            b = np.mean([h[1] for h in hist[-2 * L:-L]])
            pos = np.array([h[2] for h in hist[-2 * L:]])
            flushed = steps * dt * a * p["T_max"] / p["T_min"] >= 2.0 * ((nx - 1) * dx - xf)
            if abs(a - b) <= tol * a and np.abs(pos - x_target).max() <= 2 * dx and flushed:
                converged = True
                S_L = float(a)
                break
        S_L = S_bar
    p = solver.flame_properties(fuel, profile=True)
    return FlameSolution(S_L=S_L, delta_L=p["delta_L"], T_b=p["T_b"], Y_b=p["Y_b"], T_u=cfg["T_in"],
                         x_f=p["x_f"], x=np.arange(nx) * dx, T=p["T"], Y=p["Y"], w_F=p["w_F"], steps=steps,
                         converged=converged, history=hist)
