"""One full hybrid time step, FP64 (Section 2): finite-difference energy/species update
(Section 2.3) -> thermodynamic pressure -> lattice Boltzmann stream and collide (Section
2.1-2.2). The paper does not state the order; the reading taken is:

  1. FD: from (T^n, Y^n, u^n) compute T^{n+1}, Y^{n+1}, and rho^n, Lambda^n at level n.
  2. Thermodynamic pressure (not in the paper; Eq. 3 assumes it constant). Closed domain:
     P^{n+1} = M^{n+1} / I^{n+1}, I = sum_fluid W / (R T rho_ref), M^{n+1} = M^n + inlet mass
     flux - outlet mass flux (lattice mass per step). Open domain: P constant. A closed domain
     with a pressure outlet is open to the ambient through it: P stays at its initial (ambient)
     value, while M and I are still reduced every step (the mass balance of the domain). Coupling
     P = M / I to the outlet flux instead drifts: the outflow answers the expansion only after an
     acoustic delay, P rises and the reactive burner turns non-finite within a few thousand steps.
     Lambda used by the LB gets -(P^{n+1} - P^n) / P^n; the FD energy equation uses the
     increment of the previous step.
  3. LB: pull g* of the previous step, moments with rho^n, source with grad rho^n (central
     differences, mirrored into non-fluid neighbours) and Lambda^n, collide, store g*, u^{n+1}.
Isothermal mode (no FD): rho = 1, Lambda = 0, grad rho = 0, constant viscosity.

Solid cells keep whatever values they had; only fluid cells are updated.
"""
import torch

from . import fd as fdm
from . import geometry as geo
from . import lb
from .cumulant import CumulantSpace
from .lattice import CS2, Lattice
from .units import R_GAS, Params


class Oracle:
    """FP64 oracle of the full step.

    ``store_round`` (None, "f32" or "f16") rounds the state after every step to the storage
    precision of a GPU configuration (populations in the shifted form (g - w P_ref) / w, fields
    T, Y, u in FP32 for both): the arithmetic stays FP64, so the difference from the unrounded
    oracle is the error floor that storage precision alone imposes.
    """

    def __init__(self, cfg, mask, inlet_u=None, store_round=None, qwall=None):
        self.cfg = cfg
        self.store_round = store_round
        self.p = Params(cfg)
        self.lat = Lattice(cfg["dim"])
        self.cs = CumulantSpace(self.lat)
        self.grid = geo.Grid(cfg, mask)
        self.code, self.src = geo.lb_links(self.lat, self.grid)
        self.wall = None if qwall is None else geo.wall_links(self.lat, self.grid, self.code, self.src, qwall)
        self.nb = geo.FDNeighbours(self.grid, self.wall, self.lat)
        d = cfg["dim"]
        ny = cfg["ny"]
        nz = cfg["nz"] if d == 3 else 1
        if inlet_u is None:
            inlet_u = torch.zeros(d, nz * ny, dtype=torch.float64)
        self.inlet_face = torch.as_tensor(inlet_u, dtype=torch.float64).reshape(d, -1)
        self.uin_r = self.inlet_face[:, self.grid.face_index()]  # [dim, N]
        g = self.grid
        self.at_inlet = g.fluid & (g.coord[0] == 0) & torch.tensor(g.bc[0][0] == geo.INLET)
        self.at_outlet = g.fluid & (g.coord[0] == g.shape[0] - 1) & torch.tensor(g.bc[0][1] == geo.OUTLET)

    def links_packed(self):
        return geo.pack_links(self.code, self.grid, self.wall)

    def stencil_words_packed(self):
        return geo.pack_stencil_words(self.grid, self.nb)

    # ----------------------------------------------------------------- state
    def density(self, T, Y, P_th):
        W = fdm.mean_molar_mass(self.p, Y)
        return P_th * W / (R_GAS * T * self.p.rho_ref)

    def init_state(self, T=None, Y=None, u=None, P_h=None, g_pert=None):
        """Populations at equilibrium (Eq. 6) of the given fields, plus an optional perturbation."""
        N, p = self.grid.N, self.p
        f64 = torch.float64
        u = torch.zeros(p.dim, N, dtype=f64) if u is None else torch.as_tensor(u, dtype=f64).reshape(p.dim, N)
        P_h = torch.zeros(N, dtype=f64) if P_h is None else torch.as_tensor(P_h, dtype=f64).reshape(N)
        st = {"u": u.clone(), "P_th": p.P_th0, "dP_lag": 0.0, "M": 0.0}
        if p.thermal:
            T = torch.as_tensor(T, dtype=f64).reshape(N)
            Y = torch.as_tensor(Y, dtype=f64).reshape(p.K, N)
            rho = self.density(T, Y, p.P_th0)
            st["T"], st["Y"] = T.clone(), Y.clone()
            I = self._integral(T, Y)
            st["M"] = p.P_th0 * I
        else:
            rho = torch.ones(N, dtype=f64)
        g = lb.g_eq(self.lat, P_h, rho, u)
        if g_pert is not None:
            g = g + torch.as_tensor(g_pert, dtype=f64).reshape(self.lat.Q, N)
        st["g"] = g
        st["P_h"] = P_h.clone()
        return st

    def _integral(self, T, Y):
        return pth_integral(self.p, self.grid, T, Y)

    def _mass_flux(self, st, rho):
        return boundary_mass_flux(self.p, self.at_inlet, self.at_outlet, self.uin_r, st, rho)

    # ------------------------------------------------------------------ step
    def grad_rho(self, rho):
        out = []
        for a in range(self.p.dim):
            vals = []
            for sigma in (-1, 1):
                k1, i1 = self.nb.kind1(a, sigma), self.nb.index1(a, sigma)
                vals.append(torch.where(k1 == geo.K_FLUID, rho[i1], rho))
            out.append(0.5 * (vals[1] - vals[0]))
        return torch.stack(out)

    def step(self, st, P_next=None):
        """One step. P_next: thermodynamic pressure after the step, given from outside (a patch
        of a larger closed domain, whose integral the patch cannot form)."""
        p, fluid = self.p, self.grid.fluid
        N = self.grid.N
        new = dict(st)
        if p.thermal:
            T1, Y1, rho, lam_fd = fdm.fd_update(p, self.grid, self.nb, st["T"], st["Y"], st["u"],
                                                self.uin_r, st["P_th"], st["dP_lag"])
            if P_next is not None:
                M1, P1 = st["M"], P_next
            elif p.closed:
                M1 = st["M"] + self._mass_flux(st, rho)
                I1 = self._integral(torch.where(fluid, T1, st["T"]), torch.where(fluid, Y1, st["Y"]))
                P1 = st["P_th"] if p.outlet else M1 / I1
                new["I"] = I1
            else:
                M1, P1 = st["M"], st["P_th"]
            dP = P1 - st["P_th"]
            lam = lam_fd - dP / st["P_th"]
            grad = self.grad_rho(rho)
            mu = p.nu_lat * (st["T"] / p.T_ref) ** p.mu_exp
            tau0 = mu / rho / CS2 + 0.5
            new["T"] = torch.where(fluid, T1, st["T"])
            new["Y"] = torch.where(fluid, Y1, st["Y"])
            new["M"], new["P_th"], new["dP_lag"] = M1, P1, dP
            new["rho"], new["lam"] = rho, lam
        else:
            rho = torch.ones(N, dtype=torch.float64)
            lam = torch.zeros(N, dtype=torch.float64)
            grad = torch.zeros(p.dim, N, dtype=torch.float64)
            tau0 = torch.full((N,), p.nu_lat / CS2 + 0.5, dtype=torch.float64)
        new["g"], new["u"], new["P_h"] = self.lb_update(st["g"], st["u"], st["P_h"], rho, lam, grad, tau0)
        return new

    def lb_update(self, g_post, u_prev, P_prev, rho, lam, grad, tau0):
        """Step 3 of the module doc (Section 2.1-2.2) with the density rho, its gradient grad, the
        dilatation lam and the relaxation time tau0 given per cell: returns (g*, u, P_h); non-fluid
        cells keep g_post, u_prev and P_prev."""
        lat, fluid = self.lat, self.grid.fluid
        g = lb.stream(g_post, self.code, self.src, lat, rho, self.uin_r, u_prev, self.cfg.get("P_ref", 0.0),
                      self.wall)
        P_h, u = lb.moments(lat, g, rho, lam)
        xi = lb.source_xi(lat, rho, u, grad, lam)
        gs = lb.collide(lat, self.cs, g, rho, u, xi, tau0, self.p.as_lb())
        return (torch.where(fluid[None, :], gs, g_post), torch.where(fluid[None, :], u, u_prev),
                torch.where(fluid, P_h, P_prev))

    def round_state(self, st):
        if self.store_round is None:
            return st
        pop_t = torch.float16 if self.store_round == "f16" else torch.float32
        P_ref = self.cfg.get("P_ref", 0.0)
        w = self.lat.w[:, None]
        out = dict(st)
        out["g"] = w * ((st["g"] / w - P_ref).to(pop_t).to(torch.float64) + P_ref)
        for k in ("T", "Y", "u"):
            if k in st:
                out[k] = st[k].to(torch.float32).to(torch.float64)
        return out

    def run(self, st, n):
        for _ in range(n):
            st = self.round_state(self.step(st))
        return st


def pth_integral(p, grid, T, Y):
    """I = sum over fluid cells of W / (R T rho_ref) (cell volume 1): P_th = M / I (reading c5)."""
    return fdm.pth_integrand(p, T, Y)[grid.fluid].sum().item()


def boundary_mass_flux(p, at_inlet, at_outlet, uin_r, st, rho):
    """Inlet minus outlet mass per step (lattice units), level n."""
    m = 0.0
    if at_inlet.any():
        W_in = 1.0 / sum(p.Y_in[k] / p.W[k] for k in range(p.K))
        rho_in = st["P_th"] * W_in / (R_GAS * p.T_in * p.rho_ref)
        m += (rho_in * uin_r[0][at_inlet]).sum().item()
    if at_outlet.any():
        m -= (rho[at_outlet] * st["u"][0][at_outlet]).sum().item()
    return m


def first_step_pressure(cfg, mask, inlet_u, T, Y, u):
    """Thermodynamic pressure after the first step of a closed domain from the initial fields: the
    finite-difference update over the whole grid and the mass balance, without the lattice
    Boltzmann part (a full-size grid's populations would not fit the oracle's memory). Used with
    Oracle.step(P_next=...) on patches of that grid."""
    p = Params(cfg)
    grid = geo.Grid(cfg, mask)
    nb = geo.FDNeighbours(grid)
    d = cfg["dim"]
    nz = cfg["nz"] if d == 3 else 1
    face = torch.as_tensor(inlet_u, dtype=torch.float64).reshape(d, cfg["ny"] * nz)
    uin_r = face[:, grid.face_index()]
    at_inlet = grid.fluid & (grid.coord[0] == 0) & torch.tensor(grid.bc[0][0] == geo.INLET)
    at_outlet = grid.fluid & (grid.coord[0] == grid.shape[0] - 1) & torch.tensor(grid.bc[0][1] == geo.OUTLET)
    T = torch.as_tensor(T, dtype=torch.float64)
    Y = torch.as_tensor(Y, dtype=torch.float64)
    u = torch.as_tensor(u, dtype=torch.float64).reshape(d, grid.N)
    st = {"P_th": p.P_th0, "u": u}
    M0 = p.P_th0 * pth_integral(p, grid, T, Y)
    T1, Y1, rho, _ = fdm.fd_update(p, grid, nb, T, Y, u, uin_r, p.P_th0, 0.0)
    M1 = M0 + boundary_mass_flux(p, at_inlet, at_outlet, uin_r, st, rho)
    I1 = pth_integral(p, grid, torch.where(grid.fluid, T1, T), torch.where(grid.fluid, Y1, Y))
    return p.P_th0 if p.outlet else M1 / I1
