"""1-D freely propagating premixed flame: laminar flame speed, thickness and burnt state.

Section 3.1 sets up its reacting run with the burnt-gas composition, the adiabatic temperature
and the interface thickness of a 1-D freely propagating flame computed with the same scheme and
mixture; Section 3.2.2 quotes S_L and delta_L = (T_max - T_min) / max dT/dx of such a flame. Here
that flame is the library's own planar flame: a channel that is periodic across (y, z), fresh
gas entering at x = 0 with the inlet velocity, burnt gas leaving at the high-x outlet.

A free flame moves against the fresh gas at S_L; to keep it inside the channel the inlet
velocity follows the measured consumption speed S_c (lbm_flame_properties), with a
proportional correction that pulls the flame position x_f back to a target:
    u_in = S_c - gain (x_f - x_target) / (chunk dt)        (velocities in m/s)
applied every ``chunk`` steps (lbm_set_inlet). In the flame's frame the fresh gas then arrives
at S_c, and the position error decays by the factor (1 - gain) per chunk. The run has converged
when, over the last ``window`` chunks and at least one flame time delta_L / S_c, S_c varies by
less than ``tol`` of its mean and x_f stays within one cell of the target (a transient that
decays on the flame time then leaves an error of a few tol). Every step and every measurement runs in the library's kernels;
this module only chooses the inlet velocity and keeps the history.
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


def free_flame(solver, fuel=0, x_target=None, chunk=200, gain=0.5, tol=2e-3, window=5, max_steps=400000,
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
    while steps < max_steps:
        solver.step(chunk)
        steps += chunk
        p = solver.flame_properties(fuel)
        S, xf = p["S_c"], p["x_f"]
        if not np.isfinite(S) or xf < 0 or xf > (nx - 1) * dx:
            raise RuntimeError(f"flame left the channel or went out after {steps} steps (x_f={xf}, S_c={S})")
        if S <= 0 or p["T_max"] - p["T_min"] < 1e-3 * p["T_min"]:
            raise RuntimeError(f"flame extinguished after {steps} steps")
        u = float(np.clip(S - gain * (xf - x_target) / (chunk * dt), 0.0, u_max))
        solver.set_inlet(np.concatenate([np.full(n_face, u * lat), np.zeros((solver.dim - 1) * n_face)]))
        hist.append((steps, S, xf, u))
        span = max(window, int(np.ceil(p["delta_L"] / S / (chunk * dt))) + 1)
        if len(hist) >= span:
            last = np.array([h[1] for h in hist[-span:]])
            pos = np.array([h[2] for h in hist[-span:]])
            if np.ptp(last) <= tol * abs(last.mean()) and np.abs(pos - x_target).max() <= dx:
                converged = True
                break
    p = solver.flame_properties(fuel, profile=True)
    return FlameSolution(S_L=p["S_c"], delta_L=p["delta_L"], T_b=p["T_b"], Y_b=p["Y_b"], T_u=cfg["T_in"],
                         x_f=p["x_f"], x=np.arange(nx) * dx, T=p["T"], Y=p["Y"], w_F=p["w_F"], steps=steps,
                         converged=converged, history=hist)
