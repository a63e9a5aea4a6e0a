"""Discrete velocity sets (Section 2.1, the paragraph after Eq. 7: first-neighbour stencils
from third-order quadrature, D2Q9 and D3Q27, with c_s = dr / (sqrt(3) dt)).

Both sets are tensor products of the one-dimensional three-point Gauss-Hermite rule with
abscissae {-1, 0, 1} and weights {1/6, 2/3, 1/6}. Direction i has velocity (cx, cy[, cz]) with
    i = (cx + 1) + 3 (cy + 1) [+ 9 (cz + 1)],
so the rest velocity is i = (Q - 1) / 2 and the opposite of i is Q - 1 - i.
"""
import torch

CS2 = 1.0 / 3.0  # c_s^2 in lattice units (dr = dt = 1)
_W1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}


class Lattice:
    """Velocities ``c`` [Q, dim] (float64), weights ``w`` [Q], opposite index ``opp`` [Q]."""

    def __init__(self, dim):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim = dim
        self.Q = 3 ** dim
        vel, wts = [], []
        for i in range(self.Q):
            comps = [(i // 3 ** a) % 3 - 1 for a in range(dim)]
            vel.append(comps)
            wt = 1.0
            for ca in comps:
                wt *= _W1[ca]
            wts.append(wt)
        self.c = torch.tensor(vel, dtype=torch.float64)
        self.ci = torch.tensor(vel, dtype=torch.int64)
        self.w = torch.tensor(wts, dtype=torch.float64)
        self.opp = torch.tensor([self.Q - 1 - i for i in range(self.Q)], dtype=torch.int64)
        self.rest = (self.Q - 1) // 2
