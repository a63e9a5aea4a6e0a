"""Gradient of a combustion functional through K steps of the hybrid solver: discrete adjoint
(reverse mode) with checkpointing, behind ``torch.autograd.Function``.

The paper computes no gradients; this is the exact transpose of the discrete step the library
runs (lbm_adjoint_step), chained over the steps. The functional is the fuel consumption at the
last step, J = sum over fluid cells of -omega_F(T^K, Y^K) (lbm_fuel_objective); its parameters
are the inlet-face velocity (the boundary data of the inlet rule) and the initial temperature
field T0 (which sets T^0 and, through rho = P_th W / (R T) of Eq. 13, the initial equilibrium
populations of Eq. 6).

Forward: set the inlet and the initial fields, run K steps, saving the state every C steps.
Backward: lbm_adjoint_sweep takes the segments last first: for each, the library recomputes and
keeps the segment's states from its checkpoint, then applies the adjoint step from the segment's
last step down to its first, adding the inlet-velocity adjoint; the recompute of the next
segment runs on a second stream while the current one is reversed. lbm_initial_T_adjoint turns
the adjoint of state 0 into dJ/dT0. Memory: K/C checkpoints of ``Solver.state_bytes()`` plus the
library's workspace of two segments (2 C states with their rho and Lambda).

Each forward call returns J and keeps a tape of its own (inlet velocity, checkpoints, adjoint of
the last state), so that several forward calls may be reversed later in any order: the backward
of a tape sets that forward's inlet velocity again before its recompute. The backward leaves the
solver in an unspecified state (its recompute and lbm_initial_T_adjoint load checkpoints): call
forward again before stepping the solver for another purpose.
Every arithmetic step runs in the library's CUDA kernels; this module only orders the calls.
"""
import numpy as np
import torch

from .solver import Solver


class AdjointProblem:
    """A fixed geometry, initial composition, velocity and pressure, step count and checkpoint
    interval; J and its gradient are functions of the inlet velocity and of T0."""

    def __init__(self, cfg, mask, Y0, u0=None, P_h0=None, g_pert=None, n_steps=100, checkpoint_every=100,
                 fuel=0, device=None):
        if not cfg.get("thermal"):
            raise ValueError("the fuel-consumption functional needs a thermal configuration")
        self.cfg = cfg
        self.mask = np.asarray(mask)
        self.Y0, self.u0, self.P_h0, self.g_pert = Y0, u0, P_h0, g_pert
        self.n_steps = int(n_steps)
        self.C = max(1, int(checkpoint_every))
        self.fuel = int(fuel)
        self.solver = Solver(cfg, self.mask, None, device=device)
        self.dtype = torch.float64 if cfg.get("storage", "f32") == "f64" else torch.float32
        esize = 8 if self.dtype == torch.float64 else 4
        self.n_words = (self.solver.state_bytes() + esize - 1) // esize
        self.dim, self.ny = cfg["dim"], cfg["ny"]
        self.tape = None  # the last forward call's tape

    def close(self):
        self.solver.close()

    def _zeros(self, n):
        return torch.zeros(n, dtype=self.dtype, device=self.solver.device)

    def forward(self, inlet_u, T0):
        """Run the K steps from (inlet_u [dim][ny], T0 [N]); returns J. The call's tape
        (``self.tape``) holds what its backward needs."""
        s = self.solver
        inlet = np.array(inlet_u, dtype=np.float64).reshape(self.dim, self.ny)
        s.set_geometry(self.mask, inlet)
        s.set_fields(T=np.asarray(T0, dtype=np.float64), Y=self.Y0, u=self.u0, P_h=self.P_h0, g_pert=self.g_pert)
        ckpt = []
        for n0 in range(0, self.n_steps, self.C):
            ckpt.append(s.save_state())
            s.step(min(self.C, self.n_steps - n0))
        adjK = self._zeros(self.n_words)
        J = s.fuel_objective(self.fuel, adjK)
        self.tape = {"inlet": inlet, "ckpt": ckpt, "adjK": adjK}
        return J

    def backward(self, scale=1.0, tape=None):
        """dJ/d(inlet_u) [dim][ny] and dJ/dT0 [N] (storage type) of the forward call that made
        ``tape`` (default: the last one)."""
        tape = self.tape if tape is None else tape
        if tape is None:
            raise RuntimeError("backward needs a forward call first")
        s = self.solver
        s.set_inlet(tape["inlet"])
        adj = tape["adjK"] * scale
        gin = self._zeros(self.dim * self.ny)
        s.adjoint_sweep(tape["ckpt"], self.C, self.n_steps, adj, gin)
        gT = self._zeros(s.N)
        s.initial_T_adjoint(tape["ckpt"][0], adj, gT)
        return gin.reshape(self.dim, self.ny), gT


class HybridStepFn(torch.autograd.Function):
    """J = HybridStepFn.apply(inlet_u, T0, problem): the fuel consumption after the problem's K
    steps, differentiable with respect to the inlet-face velocity and the initial temperature."""

    @staticmethod
    def forward(ctx, inlet_u, T0, problem):
        ctx.problem = problem
        ctx.meta = (inlet_u.dtype, inlet_u.device, T0.dtype, T0.device)
        J = problem.forward(inlet_u.detach().cpu().numpy(), T0.detach().cpu().numpy())
        ctx.tape = problem.tape  # this call's own checkpoints: later forward calls do not touch them
        return torch.tensor(J, dtype=torch.float64, device=inlet_u.device)

    @staticmethod
    def backward(ctx, gJ):
        gin, gT = ctx.problem.backward(float(gJ), tape=ctx.tape)
        idt, idev, tdt, tdev = ctx.meta
        return gin.to(dtype=idt, device=idev), gT.to(dtype=tdt, device=tdev), None
