"""Physical (SI) configuration -> lattice units (dr = dt = 1, c_s^2 = 1/3; Section 2.1 ties
c_s to dr and dt by c_s = dr / (sqrt(3) dt)).

Temperatures stay in kelvin, mass fractions are dimensionless, densities are expressed in
units of the configuration's reference density rho_ref, the thermodynamic pressure stays in
pascal. Transport (reading: the paper's mixture-averaged module is not available):
    mu(T) = mu_ref (T / T_ref)^mu_exp, lambda / c_p = mu / Pr, rho D_k = mu / (Pr Le_k)
so that in lattice units mu_lat(T) = nu_ref dt / dr^2 (T / T_ref)^mu_exp.
"""

R_GAS = 8.314462618  # J / (mol K)


class Params:
    def __init__(self, cfg):
        self.cfg = cfg
        self.dim = cfg["dim"]
        self.thermal = bool(cfg.get("thermal", False))
        self.nu_lat = cfg["nu_ref"] * cfg["dt"] / cfg["dx"] ** 2
        self.T_ref = cfg.get("T_ref", 300.0)
        self.mu_exp = cfg.get("mu_exp", 0.7)
        self.Pr = cfg.get("Pr", 0.7)
        self.cp = cfg.get("cp", 1400.0)
        self.rho_ref = cfg.get("rho_ref", 1.0)
        self.P_th0 = cfg.get("P_th0", 101325.0)
        self.closed = bool(cfg.get("closed_domain", False))
        # a pressure outlet holds the thermodynamic pressure at its ambient (initial) value
        self.outlet = cfg.get("bc", {}).get("x", ("", ""))[1] == "outlet"
        self.dt = cfg["dt"]
        self.smag_cs = cfg.get("smag_cs", 0.0)
        self.collision = cfg.get("collision", "cumulant")
        self.omega_bulk = cfg.get("omega_bulk", 1.0)
        self.omega_hi = list(cfg.get("omega_hi", (1.0, 1.0, 1.0, 1.0)))
        self.F = cfg.get("thicken_F", 1.0)
        self.sensor = bool(cfg.get("flame_sensor", False))
        self.sensor_beta = cfg.get("sensor_beta", 10.0)
        self.sensor_wref = cfg.get("sensor_wref", 1.0)
        self.sensor_species = cfg.get("sensor_species", 0)
        self.sensor_oxidizer = cfg.get("sensor_oxidizer", 1)
        self.sensor_Ta = cfg.get("sensor_Ta", 8400.0)
        sp = cfg.get("species", [])
        self.K = len(sp)
        self.W = [s["W"] for s in sp]
        self.Le = [s["Le"] for s in sp]
        self.hf = [s["hf"] for s in sp]
        self.reactions = cfg.get("reactions", [])
        # variable heat capacities (NEXT-2 reading): c_p,k(T) = sum_m a_km T^m, J/(kg K); the
        # formation enthalpies hf hold at T0_thermo
        self.varcp = bool(cfg.get("variable_cp", False))
        self.cp_poly = [list(s.get("cp_poly", [self.cp, 0.0, 0.0, 0.0, 0.0])) for s in sp]
        self.T0_thermo = cfg.get("T0_thermo", 298.15)
        # mixture-averaged species diffusion (option): pair Lewis numbers Le_kj, rho D_kj = mu/(Pr Le_kj)
        self.mixavg = bool(cfg.get("mixture_averaged", False))
        self.Le_pair = cfg.get("Le_pair")
        if self.mixavg and (self.Le_pair is None or len(self.Le_pair) != self.K):
            raise ValueError("mixture-averaged diffusion needs Le_pair [K][K]")
        self.T_in = cfg.get("T_in", self.T_ref)
        self.Y_in = list(cfg.get("Y_in", [0.0] * self.K))
        self.weno_eps_T = 1e-6 * self.T_ref ** 2
        self.weno_eps_Y = 1e-6

    def as_lb(self):
        return {"smag_cs": self.smag_cs, "collision": self.collision,
                "omega_bulk": self.omega_bulk, "omega_hi": self.omega_hi}
