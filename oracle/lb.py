"""Lattice Boltzmann part of the step (Section 2.1 and 2.2), lattice units dr = dt = 1.

Per fluid cell, in the order of the paper:
  1. pull streaming, Eq. 1, with the boundary links of ``geometry``;
  2. moments, Eq. 7: P_h = sum g + (1/2) rho c_s^2 Lambda, rho u = (1/c_s^2) sum c g;
  3. equilibrium f^eq, Eq. 4, and source Xi, Eq. 2;
  4. pre-conditioning, Eq. 13: f' = g / (rho c_s^2) + Xi / (2 rho c_s^2);
  5. collision of f' (BGK, or cumulants, Eq. 9-12 with the readings below);
  6. post-collision, Eq. 8: g* = rho c_s^2 f'* + Xi / 2.

Readings (the paper defers the operator to supplementary material that is not available):
  * Eq. 9 is read as the standard relaxation f'* = M^-1 [(I - W) K' + W K'^eq].
  * Eq. 12 gives a relaxation time: tau = nu / c_s^2 + 1/2, omega = 1 / tau.
  * The pre-conditioned populations carry zeroth moment p' = sum f' and first moment u; by Eq. 4,
    6 and 13 their equilibrium is (p' - 1) w_i + f^eq_i(rho = 1, u). The collision therefore acts
    on h = f' - (p' - 1) w, a distribution with unit density and velocity u, and adds the rest
    part back afterwards. This keeps the momentum flux of Eq. 6 at equilibrium for any P_h/rho.
  * Cumulant relaxation: second order split into trace (bulk rate omega_b, equilibrium
    d c_s^2) and deviatoric part (shear rate omega_s, equilibrium 0); every cumulant of order
    n = 3..6 relaxes to 0 with rate omega_hi[n - 3] (all 1 by default).
  * BGK: every moment of h relaxes with omega_s towards f^eq(1, u) (the single-rate case of
    Eq. 9; it shares Eq. 8 and Eq. 13).
  * Smagorinsky (named in Section 1, no formula given): nu_t = (C_s dr)^2 |S| with |S| from the
    deviatoric non-equilibrium second moment Pi of h, giving
    tau_eff = (tau_0 + sqrt(tau_0^2 + 18 sqrt(2) C_s^2 |Pi|)) / 2.
"""
import math

import torch

from .lattice import CS2


def f_eq(lat, rho, u):
    """Eq. 4: second-order equilibrium, [Q, N]."""
    cu = lat.c @ u
    usq = (u * u).sum(0)
    return lat.w[:, None] * rho[None, :] * (
        1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq[None, :] / (2.0 * CS2))


def g_eq(lat, P_h, rho, u):
    """Eq. 6: g^eq = w (P_h - rho c_s^2) + c_s^2 f^eq."""
    return lat.w[:, None] * (P_h - rho * CS2)[None, :] + CS2 * f_eq(lat, rho, u)


def source_xi(lat, rho, u, grad_rho, lam):
    """Eq. 2: Xi_i = c_s^2 (f^eq_i / rho - w_i)(c_i - u).grad(rho) + w_i rho c_s^2 Lambda."""
    feq = f_eq(lat, rho, u)
    proj = lat.c @ grad_rho - (u * grad_rho).sum(0)[None, :]
    return CS2 * (feq / rho[None, :] - lat.w[:, None]) * proj + lat.w[:, None] * (rho * CS2 * lam)[None, :]


def moments(lat, g, rho, lam):
    """Eq. 7: (P_h, u)."""
    P_h = g.sum(0) + 0.5 * rho * CS2 * lam
    u = (lat.c.T @ g) / (CS2 * rho[None, :])
    return P_h, u


def stream(g_post, code, src, lat, rho, uin_at_r, u_prev, P_out, wall=None):
    """Pull streaming with boundary links (Eq. 1 read as pull).

    g_post [Q, N] are the post-collision populations of the previous step. uin_at_r [dim, N]
    is the inlet velocity of the face element next to each cell (code 2: moving-wall
    bounce-back g_i = g*_opp + 2 w_i rho c_i.u_w, the first-order part of Eq. 6 doubled).
    Code 3 (outlet): anti-bounce-back g_i = -g*_opp + 2 w_i (P_out + rho (1.5 (c_i.u)^2 - 0.5 u^2)),
    twice the even part of Eq. 6 at the outlet pressure, with u the previous-step velocity.
    wall (optional): {"q": [Q, N] wall fractions, "far": [Q, N] index of r + c_i or -1} for
    interpolated bounce-back on code-1 links (see ``interp_bounce_back``).
    """
    Q = lat.Q
    g = torch.empty_like(g_post)
    usq = (u_prev * u_prev).sum(0)
    for i in range(Q):
        pulled = g_post[i][src[i]]
        bb = g_post[lat.opp[i]]
        inlet_term = 2.0 * lat.w[i] * rho * (lat.c[i] @ uin_at_r)
        cu = lat.c[i] @ u_prev
        abb = -bb + 2.0 * lat.w[i] * (P_out + rho * (1.5 * cu * cu - 0.5 * usq))
        wbb = bb if wall is None else interp_bounce_back(g_post, lat, i, wall["q"][i], wall["far"][i])
        g[i] = torch.where(code[i] == 0, pulled, torch.where(code[i] == 1, wbb,
                           torch.where(code[i] == 2, bb + inlet_term, abb)))
    return g


def interp_bounce_back(g_post, lat, i, q, far):
    """Linearly interpolated bounce-back (the curved-wall treatment; the paper names it without
    formulas, reading c21) for the population i entering a fluid node r whose link r - c_i crosses
    a wall at the fraction q of the link from r, o = opposite of i:
        q <  1/2:  g_i(r) = 2q g*_o(r) + (1 - 2q) g*_o(r + c_i)
        q >= 1/2:  g_i(r) = g*_o(r) / (2q) + (2q - 1) / (2q) g*_i(r)
    q = 1/2 is half-way bounce-back. Where r + c_i is not a fluid node (far < 0) a link with
    q < 1/2 falls back to half-way bounce-back."""
    o = lat.opp[i]
    own_o, own_i = g_post[o], g_post[i]
    far_o = g_post[o][far.clamp(min=0)]
    near = 2.0 * q * own_o + (1.0 - 2.0 * q) * far_o
    away = own_o / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * own_i
    return torch.where(q < 0.5, torch.where(far >= 0, near, own_o), away)


def tau_smagorinsky(lat, h, u, tau0, cs_smag):
    """Effective relaxation time with the Smagorinsky eddy viscosity (reading in module doc)."""
    if cs_smag == 0.0:
        return tau0
    heq = f_eq(lat, torch.ones_like(u[0]), u)
    d = lat.dim
    neq = h - heq
    Pi = torch.stack([torch.stack([(lat.c[:, a, None] * lat.c[:, b, None] * neq).sum(0)
                                   for b in range(d)]) for a in range(d)])  # [d, d, N]
    tr = sum(Pi[a, a] for a in range(d)) / d
    for a in range(d):
        Pi[a, a] = Pi[a, a] - tr
    n2 = (Pi * Pi).sum((0, 1))
    # |Pi|, with derivative 0 where Pi = 0 (square root of a positive placeholder there)
    norm = torch.where(n2 > 0, torch.sqrt(torch.where(n2 > 0, n2, torch.ones_like(n2))), torch.zeros_like(n2))
    return 0.5 * (tau0 + torch.sqrt(tau0 * tau0 + 18.0 * math.sqrt(2.0) * cs_smag ** 2 * norm))


def relax_cumulants(cs, C, omega_s, omega_b, omega_hi):
    """Cumulant relaxation (reading in module doc). C [Q, N] in storage order."""
    d = cs.dim
    Cs = C.clone()
    diag = [cs.idx.index(tuple(2 if k == a else 0 for k in range(d))) for a in range(d)]
    k0 = C[0]
    A = sum(C[j] for j in diag)
    A_star = A + omega_b * (d * CS2 * k0 - A)
    for j in diag:
        Cs[j] = (1.0 - omega_s) * (C[j] - A / d) + A_star / d
    for j, a in enumerate(cs.idx):
        n = sum(a)
        if n == 2 and max(a) == 1:
            Cs[j] = (1.0 - omega_s) * C[j]
        elif n >= 3:
            Cs[j] = (1.0 - omega_hi[n - 3]) * C[j]
    return Cs


def collide(lat, cs, g, rho, u, xi, tau0, params):
    """Steps 4-6 of the module doc: returns g* [Q, N]."""
    fp = (g + 0.5 * xi) / (rho * CS2)[None, :]
    p = fp.sum(0)
    h = fp - (p - 1.0)[None, :] * lat.w[:, None]
    tau = tau_smagorinsky(lat, h, u, tau0, params["smag_cs"])
    omega = 1.0 / tau
    if params["collision"] == "bgk":
        h_star = h - omega[None, :] * (h - f_eq(lat, torch.ones_like(rho), u))
    else:
        k = cs.central_moments(h, u)
        C = cs.cumulants_from_central(k)
        Cs = relax_cumulants(cs, C, omega, params["omega_bulk"], params["omega_hi"])
        h_star = cs.populations_from_central(cs.central_from_cumulants(Cs), u)
    fp_star = h_star + (p - 1.0)[None, :] * lat.w[:, None]
    return (rho * CS2)[None, :] * fp_star + 0.5 * xi
