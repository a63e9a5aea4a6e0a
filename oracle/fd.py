"""Energy and species balance by finite differences (Section 2.3): explicit Euler in time,
third-order WENO for advection, centred second-order diffusion; two-step (or one-step)
Arrhenius chemistry; thickened flame (Section 1 and 3.2.2, factor written E in the paper).

Equations, lattice units of length and time (see ``units``), for phi in {T, Y_k}:
    phi^{n+1} = phi^n - A_phi + N_phi
    A_phi = sum_axes u_a(r) (phi_hat(r + e_a/2) - phi_hat(r - e_a/2))      (WENO3 faces)
    N_phi = (1/rho) sum_axes [G(r+e/2)(phi(r+e) - phi(r)) - G(r-e/2)(phi(r) - phi(r-e))]
            + chemistry (+ pressure work for T)
with G_T = F_loc mu / Pr, G_k = F_loc mu / (Pr Le_k) and the face value G = arithmetic mean.
Readings (the paper gives no formulas for these):
  * WENO3 (Jiang-Shu): candidate faces -a/2 + 3b/2 and (b + c)/2, smoothness (b - a)^2 and
    (c - b)^2, ideal weights 1/3 and 2/3, eps = 1e-6 in units of the field scale (T_ref^2 for T,
    1 for Y); the upwind side is chosen by the sign of the face velocity (u(r) + u(r+e))/2,
    a zero face velocity counting as positive.
  * Chemistry: q_j = A_j T^beta_j exp(-E_j/(R T)) prod_k [X_k]^n_jk with [X_k] = rho max(Y_k,0)/W_k,
    omega_k = W_k sum_j nu_kj q_j, heat release -sum_k h_f,k omega_k, constant c_p.
  * Thickening (Colin type, efficiency 1): diffusivities times F_loc, rates divided by F_loc.
    F_loc = F, or with the flame sensor F_loc = 1 + (F - 1) tanh(beta Omega / Omega_0) with
    Omega = max(Y_F, 0) max(Y_O, 0) exp(-T_s / T) (fuel and oxidizer mass fractions, reduced
    activation temperature T_s): a sensor linear in the reactants, which stays smooth where
    the fuel vanishes (a sensor built on the fractional-order rate would switch F_loc on fuel
    residues at round-off level).
  * Lambda (Eq. 3) uses the non-advective right-hand side: Lambda = N_T / T + sum (W/W_k) N_k.
  * Thermodynamic pressure: rho = P_th W / (R T); the energy equation gains the pressure work
    dP_th/(rho c_p) of the previous step.
  * Variable heat capacities (option; the paper couples a thermochemistry library that is not
    available): c_p,k(T) a polynomial per species, h_k(T) = h_f,k + integral of c_p,k from T0,
    c_p = sum Y_k c_p,k. The temperature equation becomes
        N_T = [sum_faces lambda_face (T_n - T) + F mu/Pr sum_k (c_p,k - c_p)/Le_k grad Y_k . grad T]
              / (rho c_p) + dt (-sum_k h_k omega_k) / (rho c_p F) + dP/(rho c_p)
    with lambda = F mu c_p / Pr per cell (face value the arithmetic mean; a ghost neighbour's c_p
    from its ghost T and Y), centred gradients (phi(r+e) - phi(r-e))/2 of the ghost-extended
    fields, and the species-enthalpy flux written with the diffusion fluxes relative to the
    mass-averaged velocity (c_p,k - c_p), so that equal species heat capacities give back the
    constant-c_p update exactly.
  * Mixture-averaged species diffusion (option; the paper's transport library is not available,
    so binary diffusion data are given as pair Lewis numbers, rho D_kj = (mu / Pr) / Le_kj):
    the Hirschfelder-Curtiss coefficient rho D_k = (1 - X_k) / sum_{j!=k} X_j / (rho D_kj), written
    per cell as G_k = F_loc mu / (Pr Le_k^mix), Le_k^mix = sum_{j!=k} (X_j + d) Le_kj /
    sum_{j!=k} (X_j + d) with the mole fractions X_j = Y_j W / W_j clipped at 0 and d = 1e-10
    (a pure species keeps a finite coefficient), and the mass flux of the mole-fraction form with
    a correction velocity, j_k = -rho D_k (W_k / W) grad X_k + rho Y_k V_c,
    V_c = sum_j D_j (W_j / W) grad X_j. With (W_k / W) grad X_k = grad Y_k + Y_k grad(ln W), per
    face (arithmetic means G_k,f and Y_k,f, differences dY_k, dlnW = (W_n - W_r) / mean W):
        J_k,f = G_k,f (dY_k + Y_k,f dlnW) - Y_k,f sum_j G_j,f (dY_j + Y_j,f dlnW).
    The J_k,f sum to zero over the species (sum_k Y_k = 1), and equal pair Lewis numbers give
    J_k,f = G_f dY_k, the constant-Lewis flux, exactly. Ghost neighbours take their ghost T and
    Y (and the fluid cell's F_loc) as in the constant-Lewis case.
"""
import math

import torch

from .units import R_GAS


def weno3(a, b, c, eps):
    """Face value from upwind-far a, upwind b, downwind c (Jiang-Shu WENO3)."""
    q0 = -0.5 * a + 1.5 * b
    q1 = 0.5 * b + 0.5 * c
    beta0 = (b - a) ** 2
    beta1 = (c - b) ** 2
    a0 = (1.0 / 3.0) / (eps + beta0) ** 2
    a1 = (2.0 / 3.0) / (eps + beta1) ** 2
    return (a0 * q0 + a1 * q1) / (a0 + a1)


def mean_molar_mass(p, Y):
    return 1.0 / sum(Y[k] / p.W[k] for k in range(p.K))


def reaction_rates(p, T, Y, rho_phys):
    """q_j [mol/(m^3 s)] for every reaction, list of [N] tensors.

    [X]^n is taken as 0 where Y <= 0, with derivative 0 there (the base is replaced by 1
    before the power so that reverse-mode differentiation stays finite)."""
    out = []
    for rx in p.reactions:
        q = rx["A"] * T ** rx["beta"] * torch.exp(-rx["E"] / (R_GAS * T))
        for k, n in rx["order"].items():
            pos = Y[k] > 0
            conc = rho_phys * torch.where(pos, Y[k], torch.ones_like(Y[k])) / p.W[k]
            q = q * torch.where(pos, conc ** n, torch.zeros_like(conc))
        out.append(q)
    return out


def species_rates(p, q):
    """omega_k [kg/(m^3 s)] from reaction rates."""
    om = []
    for k in range(p.K):
        acc = torch.zeros_like(q[0]) if q else torch.zeros(())
        for j, rx in enumerate(p.reactions):
            nu = rx["nu"].get(k, 0.0)
            if nu != 0.0:
                acc = acc + p.W[k] * nu * q[j]
        om.append(acc)
    return om


def cp_species(p, k, T):
    """c_p,k(T) [J/(kg K)]."""
    a = p.cp_poly[k]
    return sum(a[m] * T ** m for m in range(len(a)))


def h_species(p, k, T):
    """h_k(T) = h_f,k + integral from T0 to T of c_p,k [J/kg]."""
    a = p.cp_poly[k]
    T0 = p.T0_thermo
    return p.hf[k] + sum(a[m] * (T ** (m + 1) - T0 ** (m + 1)) / (m + 1) for m in range(len(a)))


def cp_mixture(p, T, Y):
    return sum(Y[k] * cp_species(p, k, T) for k in range(p.K))


def thickening(p, T, Y):
    """F_loc per cell."""
    if not p.sensor:
        return torch.full_like(T, p.F)
    om = torch.clamp(Y[p.sensor_species], min=0.0) * torch.clamp(Y[p.sensor_oxidizer], min=0.0) \
        * torch.exp(-p.sensor_Ta / T)
    return 1.0 + (p.F - 1.0) * torch.tanh(p.sensor_beta * om / p.sensor_wref)


def lewis_mixture(p, Y):
    """Le_k^mix per cell for every species (mixture-averaged option, see the module notes)."""
    W = mean_molar_mass(p, Y)
    X = [torch.clamp(Y[j] * W / p.W[j], min=0.0) + 1e-10 for j in range(p.K)]
    out = []
    for k in range(p.K):
        num = sum(X[j] * p.Le_pair[k][j] for j in range(p.K) if j != k)
        den = sum(X[j] for j in range(p.K) if j != k)
        out.append(num / den)
    return out


def _species_diffusion_mixavg(p, nb, T, Y, Floc, mu):
    """sum over faces of J_k,f for every species (mixture-averaged option): list of [N]."""
    W = mean_molar_mass(p, Y)
    Lr = lewis_mixture(p, Y)
    Gr = [Floc * mu / (p.Pr * Lr[k]) for k in range(p.K)]
    dif = [torch.zeros_like(T) for _ in range(p.K)]
    for a in range(nb.grid.dim):
        for sigma in (-1, 1):
            Tn = nb.value(T, p.T_in, a, sigma, 1)
            Yn = torch.stack([nb.value(Y[k], p.Y_in[k], a, sigma, 1) for k in range(p.K)])
            kn, i_n = nb.kind1(a, sigma), nb.index1(a, sigma)
            Fn = torch.where(kn == 0, Floc[i_n], Floc)
            mun = p.nu_lat * (Tn / p.T_ref) ** p.mu_exp
            Ln = lewis_mixture(p, Yn)
            Wn = mean_molar_mass(p, Yn)
            dlnW = (Wn - W) / (0.5 * (Wn + W))
            Gf = [0.5 * (Gr[k] + Fn * mun / (p.Pr * Ln[k])) for k in range(p.K)]
            Yf = [0.5 * (Y[k] + Yn[k]) for k in range(p.K)]
            dY = [Yn[k] - Y[k] for k in range(p.K)]
            corr = sum(Gf[j] * (dY[j] + Yf[j] * dlnW) for j in range(p.K))
            for k in range(p.K):
                J = Gf[k] * (dY[k] + Yf[k] * dlnW) - Yf[k] * corr
                # with differences neighbour minus cell, both faces of an axis enter with + sign
                dif[k] = dif[k] + J
    return dif


def fd_update(p, grid, nb, T, Y, u, uin_r, P_th, dP_lag):
    """One explicit Euler step of T and Y. Returns (T1, Y1, rho_lat, lam_fd)."""
    W = mean_molar_mass(p, Y)
    rho_phys = P_th * W / (R_GAS * T)
    rho = rho_phys / p.rho_ref
    q = reaction_rates(p, T, Y, rho_phys)
    om = [o.expand_as(T) for o in species_rates(p, q)]
    Floc = thickening(p, T, Y)
    mu = p.nu_lat * (T / p.T_ref) ** p.mu_exp

    fields = [T] + [Y[k] for k in range(p.K)]
    inlet_vals = [p.T_in] + p.Y_in
    Les = [1.0] + p.Le
    epss = [p.weno_eps_T] + [p.weno_eps_Y] * p.K
    N_out = []
    A_out = []
    for f, (phi, phin, Le, eps) in enumerate(zip(fields, inlet_vals, Les, epss)):
        G = Floc * mu / (p.Pr * Le)
        adv = torch.zeros_like(phi)
        dif = torch.zeros_like(phi)
        for a in range(grid.dim):
            pm2 = nb.value(phi, phin, a, -1, 2)
            pm1 = nb.value(phi, phin, a, -1, 1)
            pp1 = nb.value(phi, phin, a, +1, 1)
            pp2 = nb.value(phi, phin, a, +1, 2)
            um = nb.velocity(u[a], uin_r[a], a, -1)
            up = nb.velocity(u[a], uin_r[a], a, +1)
            uf_p = 0.5 * (u[a] + up)
            uf_m = 0.5 * (um + u[a])
            face_p = torch.where(uf_p >= 0, weno3(pm1, phi, pp1, eps), weno3(pp2, pp1, phi, eps))
            face_m = torch.where(uf_m >= 0, weno3(pm2, pm1, phi, eps), weno3(pp1, phi, pm1, eps))
            adv = adv + u[a] * (face_p - face_m)
            # ghost diffusion coefficients: temperature of the ghost, F_loc of the fluid cell
            Tm = nb.value(T, p.T_in, a, -1, 1)
            Tp = nb.value(T, p.T_in, a, +1, 1)
            km, im = nb.kind1(a, -1), nb.index1(a, -1)
            kp, ip = nb.kind1(a, +1), nb.index1(a, +1)
            Fm = torch.where(km == 0, Floc[im], Floc)
            Fp = torch.where(kp == 0, Floc[ip], Floc)
            Gm = Fm * p.nu_lat * (Tm / p.T_ref) ** p.mu_exp / (p.Pr * Le)
            Gp = Fp * p.nu_lat * (Tp / p.T_ref) ** p.mu_exp / (p.Pr * Le)
            dif = dif + 0.5 * (G + Gp) * (pp1 - phi) - 0.5 * (G + Gm) * (phi - pm1)
        if f > 0 and p.mixavg:
            if f == 1:
                dif_mix = _species_diffusion_mixavg(p, nb, T, Y, Floc, mu)
            dif = dif_mix[f - 1]
        dif = dif / rho
        if f == 0 and p.varcp:
            dif, src = _energy_varcp(p, nb, T, Y, Floc, mu, rho, rho_phys, om, dP_lag)
        elif f == 0:
            qdot = -sum(p.hf[k] * om[k] for k in range(p.K)) if p.K else torch.zeros_like(T)
            src = p.dt * qdot / (rho_phys * p.cp * Floc) + dP_lag / (rho_phys * p.cp)
        else:
            src = p.dt * om[f - 1] / (rho_phys * Floc) if p.reactions else torch.zeros_like(phi)
        N_out.append(dif + src)
        A_out.append(adv)
    T1 = T - A_out[0] + N_out[0]
    Y1 = torch.stack([Y[k] - A_out[k + 1] + N_out[k + 1] for k in range(p.K)])
    lam = N_out[0] / T + sum((W / p.W[k]) * N_out[k + 1] for k in range(p.K))
    return T1, Y1, rho, lam


def _energy_varcp(p, nb, T, Y, Floc, mu, rho, rho_phys, om, dP_lag):
    """Diffusion and source parts of N_T with variable heat capacities (see the module notes)."""
    cp = cp_mixture(p, T, Y)
    lam_r = Floc * mu * cp / p.Pr
    dif = torch.zeros_like(T)
    flux = torch.zeros_like(T)  # sum_k (c_p,k - c_p)/Le_k grad Y_k . grad T
    cpk = [cp_species(p, k, T) for k in range(p.K)]
    for a in range(nb.grid.dim):
        Tm = nb.value(T, p.T_in, a, -1, 1)
        Tp = nb.value(T, p.T_in, a, +1, 1)
        Ym = [nb.value(Y[k], p.Y_in[k], a, -1, 1) for k in range(p.K)]
        Yp = [nb.value(Y[k], p.Y_in[k], a, +1, 1) for k in range(p.K)]
        km, im = nb.kind1(a, -1), nb.index1(a, -1)
        kp, ip = nb.kind1(a, +1), nb.index1(a, +1)
        Fm = torch.where(km == 0, Floc[im], Floc)
        Fp = torch.where(kp == 0, Floc[ip], Floc)
        cpm = sum(Ym[k] * cp_species(p, k, Tm) for k in range(p.K))
        cpp = sum(Yp[k] * cp_species(p, k, Tp) for k in range(p.K))
        lam_m = Fm * p.nu_lat * (Tm / p.T_ref) ** p.mu_exp * cpm / p.Pr
        lam_p = Fp * p.nu_lat * (Tp / p.T_ref) ** p.mu_exp * cpp / p.Pr
        dif = dif + 0.5 * (lam_r + lam_p) * (Tp - T) - 0.5 * (lam_r + lam_m) * (T - Tm)
        gT = 0.5 * (Tp - Tm)
        for k in range(p.K):
            flux = flux + (cpk[k] - cp) / p.Le[k] * 0.5 * (Yp[k] - Ym[k]) * gT
    dif = (dif + Floc * mu / p.Pr * flux) / (rho * cp)
    qdot = -sum(h_species(p, k, T) * om[k] for k in range(p.K))
    src = p.dt * qdot / (rho_phys * cp * Floc) + dP_lag / (rho_phys * cp)
    return dif, src


def pth_integrand(p, T, Y):
    """W / (R T rho_ref): thermodynamic-pressure integrand per fluid cell (cell volume 1)."""
    return mean_molar_mass(p, Y) / (R_GAS * T * p.rho_ref)


def fuel_consumption(p, T, Y, P_th, fluid, fuel):
    """Objective of the adjoint tests (not in the paper): J = sum over fluid cells of the fuel
    consumption rate -omega_F [kg/(m^3 s)] of the rate law above, cell volume 1."""
    W = mean_molar_mass(p, Y)
    rho_phys = P_th * W / (R_GAS * T)
    om = species_rates(p, reaction_rates(p, T, Y, rho_phys))[fuel]
    return -(om.expand_as(T)[fluid]).sum()
