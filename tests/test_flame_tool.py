"""Host logic of the 1-D free-flame tool (paper_2207_11567_gb300.flame1d) on a scripted flame,
no GPU: the inlet-velocity control holds the flame at its target and converges to its speed,
a flame that leaves the channel raises, and the profile lookup of the solution."""
import numpy as np
import pytest

from paper_2207_11567_gb300.flame1d import FlameSolution, free_flame


class ScriptedFlame:
    """A planar front at x_f moving at u_in - S through a channel (m, s), whose measured
    consumption speed relaxes to S from 30% above with time constant tau."""

    def __init__(self, S=0.35, x0=3e-3, nx=256, ny=4, dx=5e-5, dt=5e-7, tau=1e-3):
        self.cfg = {"nx": nx, "ny": ny, "dx": dx, "dt": dt, "T_in": 300.0}
        self.dim, self.N = 2, nx * ny
        self.S, self.x, self.t, self.tau = S, x0, 0.0, tau
        self.u = 0.2  # m/s, too slow at first: the flame moves upstream
        self.inlets = []

    def step(self, n):
        for _ in range(n):
            self.x += (self.u - self.S) * self.cfg["dt"]
            self.t += self.cfg["dt"]

    def set_inlet(self, inlet):
        a = np.asarray(inlet)
        assert a.shape == (self.dim * self.cfg["ny"],)
        assert np.all(a[self.cfg["ny"]:] == 0) and np.ptp(a[: self.cfg["ny"]]) == 0
        self.u = a[0] * self.cfg["dx"] / self.cfg["dt"]
        self.inlets.append(self.u)

    def flame_properties(self, fuel=0, profile=False):
        S_c = self.S * (1.0 + 0.3 * np.exp(-self.t / self.tau))
        out = {"S_c": S_c, "x_f": self.x, "delta_L": 4e-4, "T_min": 300.0, "T_max": 2000.0, "T_b": 2000.0,
               "Y_b": np.array([0.0, 0.05])}
        if profile:
            x = np.arange(self.cfg["nx"]) * self.cfg["dx"]
            T = 300.0 + 1700.0 * 0.5 * (1 + np.tanh((x - self.x) / 2e-4))
            out.update({"T": T, "w_F": np.zeros_like(T), "Y": np.stack([0.05 * (2000 - T) / 1700, 0.05 + 0 * T])})
        return out


def test_control_holds_the_flame_and_converges_to_its_speed():
    f = ScriptedFlame()
    sol = free_flame(f, x_target=3e-3, chunk=100, tol=1e-3, window=5)
    assert sol.converged
    # the scripted transient decays on about one flame time: a few tol of error remain
    assert abs(sol.S_L - f.S) < 3e-3 * f.S
    assert abs(sol.x_f - 3e-3) <= 2 * f.cfg["dx"]
    # the fresh gas arrives at the flame speed, up to the correction of a position error of at
    # most two cells (gain 0.2 over one flame time delta_L / S)
    assert abs(f.u - f.S) <= 0.2 * 2 * f.cfg["dx"] / (4e-4 / f.S) + 3e-3 * f.S
    assert len(sol.history) == sol.steps // 100


def test_flame_that_leaves_the_channel_raises():
    f = ScriptedFlame(S=5.0)  # far faster than any inlet velocity the tool allows: blows upstream
    with pytest.raises(RuntimeError, match="left the channel"):
        free_flame(f, chunk=100, u_max=1.0)


def test_fields_at_distance():
    x = np.linspace(0.0, 1e-2, 101)
    T = 300.0 + 1700.0 * (x >= 5e-3)
    sol = FlameSolution(S_L=0.3, delta_L=4e-4, T_b=2000.0, Y_b=np.zeros(1), T_u=300.0, x_f=4.95e-3, x=x,
                        T=np.interp(x, [0, 4.9e-3, 5e-3, 1e-2], [300, 300, 2000, 2000]), Y=np.zeros((1, 101)),
                        w_F=np.zeros(101), steps=0, converged=True)
    Td, Yd = sol.fields_at(np.array([-1.0, 0.0, 1.0]))
    assert Td[0] == 300.0 and Td[2] == 2000.0 and abs(Td[1] - 1150.0) < 1e-9
    assert Yd.shape == (1, 3)
