"""Seeded generators of the synthetic workloads (masks, inlet profiles, initial fields).

Shapes follow the paper's cases (Section 3): a 2-D chamber with rows of rectangular
obstacles and a burnt-gas semicircle at the closed end (Section 3.1), and a swirl burner with an
annular swirling inlet, a square confined chamber and a contracting exhaust (Section 3.2), plus
a planar premixed flame. The paper's own geometry files and measurements are not available; these
inputs stand in for them. Randomness: numpy PCG64 seeded by the ``seed`` argument.

Units: lengths in cells, velocities and pressures in lattice units, temperatures in kelvin, mass
fractions dimensionless. The ``cfg`` dictionary carries the SI parameters of the run.
Cell index r = x + nx (y + ny z); fields are [..., N] with x fastest.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from .configs import SPECIES, burnt_mixture, chemistry_1step, chemistry_2step, mixture_phi, species


@dataclass
class Workload:
    name: str
    cfg: dict
    mask: np.ndarray
    inlet_u: np.ndarray
    u: np.ndarray
    P_h: np.ndarray
    T: np.ndarray = None
    Y: np.ndarray = None
    g_pert: np.ndarray = None
    qwall: np.ndarray = None  # [Q][N] wall fraction of bounce-back links (interpolated walls)
    steps: int = 0
    info: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.mask.size

    @property
    def Q(self):
        return 3 ** self.cfg["dim"]


def _base_cfg(dim, nx, ny, nz, storage, collision="cumulant"):
    return {"dim": dim, "nx": nx, "ny": ny, "nz": nz if dim == 3 else 1,
            "storage": storage, "collision": collision,
            "T_ref": 300.0, "mu_exp": 0.7, "Pr": 0.7, "cp": 1400.0, "rho_ref": 1.17,
            "P_th0": 101325.0, "P_ref": 0.0, "omega_bulk": 1.0, "omega_hi": [1.0, 1.0, 1.0, 1.0],
            "smag_cs": 0.0, "thicken_F": 1.0, "flame_sensor": False, "sensor_beta": 10.0,
            "sensor_wref": 1e-5, "sensor_species": 0, "sensor_oxidizer": 1, "sensor_Ta": 8400.0,
            "closed_domain": False, "thermal": False,
            "species": [], "reactions": [], "T_in": 300.0, "Y_in": []}


def _tanh_blend(s, width):
    return 0.5 * (1.0 + np.tanh(s / width))


def _coords(nx, ny, nz):
    r = np.arange(nx * ny * nz)
    return r % nx, (r // nx) % ny, r // (nx * ny)


def perturbation(rng, Q, N, amp):
    """Seeded non-equilibrium perturbation added to the initial populations (both sides)."""
    return amp * rng.standard_normal((Q, N))


# --------------------------------------------------------------------------- planar flame
def flame_2d(nx=256, ny=8, storage="f64", seed=0, collision="cumulant", u_in=0.0034,
             A=1.0e9, steps=2000, dx=5e-5, dt=5e-7, width_cells=20.0, T_u=300.0, T_hot=1950.0,
             unity_lewis=True):
    """Planar premixed flame: inflow at low x, outflow at high x, periodic in y; one-step
    chemistry with 4 species; tanh profile of T and Y over ``width_cells`` cells, position
    jittered by the seed within +-2 cells."""
    rng = np.random.default_rng(seed)
    names = SPECIES["4sp"]
    cfg = _base_cfg(2, nx, ny, 1, storage, collision)
    cfg.update({"bc": {"x": ("inlet", "outlet"), "y": ("periodic", "periodic")},
                "dx": dx, "dt": dt, "nu_ref": 1.8e-5 / 1.17, "thermal": True,
                "species": species(names, unity_lewis), "reactions": chemistry_1step(A),
                "T_in": T_u, "Y_in": mixture_phi(names, 0.83)})
    x, y, _ = _coords(nx, ny, 1)
    x0 = nx / 4.0 + rng.uniform(-2.0, 2.0)
    b = _tanh_blend(x + 0.5 - x0, width_cells / 4.0)
    Yu, Yb = np.array(mixture_phi(names, 0.83)), np.array(burnt_mixture(names, 0.83))
    T = T_u + (T_hot - T_u) * b
    Y = Yu[:, None] * (1 - b)[None, :] + Yb[:, None] * b[None, :]
    u = np.zeros((2, nx * ny))
    u[0] = u_in * T / T_u
    inlet = np.zeros((2, ny))
    inlet[0] = u_in
    return Workload("flame_2d", cfg, np.zeros(nx * ny, np.uint8), inlet, u, np.zeros(nx * ny),
                    T=T, Y=Y, steps=steps, info={"x0": x0})


# ------------------------------------------------------------------------ 2-D chamber
def chamber_2d(nx=1024, ny=256, storage="f32", seed=0, collision="cumulant", F=5.0, smag=0.17,
               obstacle=(16, 48), n_rows=3, per_row=3, inlet=False, u_in=0.02, steps=20000,
               dx=1e-4, dt=5e-8, A1=1.0e9, A2=5.0e6, hot_radius=10.0, T_u=300.0, T_hot=1950.0,
               inlet_jitter=0.0, u_init=0.0, y_trace=0.0, y_floor=0.0):
    """Confined 2-D chamber: closed left end (or an inlet when ``inlet``), open right end, walls
    top and bottom, ``n_rows`` rows of ``per_row`` rectangular obstacles at seeded positions,
    hot burnt-gas semicircle at the left end; 2-step chemistry, 6 species, phi = 0.83.
    The inlet profile is parabolic, times (1 + inlet_jitter N(0, 1)) per row when inlet_jitter
    is set (a seeded profile without the mirror symmetry of the parabola). With u_init the gas
    starts moving: u_x = u_init (1 + 0.2 N(0, 1)), u_y = 0.2 u_init N(0, 1) per cell (a state
    whose face velocities are nowhere zero, so that no upwind choice sits on its switch).
    y_trace adds that mass fraction of each product (CO, CO2, H2O), taken from N2, to the fresh
    and burnt gas and to the inlet mixture (no species then starts at the max(Y, 0) switch of
    the rate law). Mass fractions below y_floor are set to 0 (the tanh blend otherwise leaves
    tails down to 1e-22 of the fresh fuel inside the burnt kernel, where the fractional-order
    rate law has slopes of order Y^-1/2)."""
    rng = np.random.default_rng(seed)
    names = SPECIES["6sp"]
    cfg = _base_cfg(2, nx, ny, 1, storage, collision)
    cfg.update({"bc": {"x": ("inlet" if inlet else "wall", "outlet"), "y": ("wall", "wall")},
                "dx": dx, "dt": dt, "nu_ref": 1.8e-5 / 1.17, "thermal": True, "smag_cs": smag,
                "thicken_F": F, "species": species(names), "reactions": chemistry_2step(A1, A2),
                "T_in": T_u, "Y_in": mixture_phi(names, 0.83)})
    x, y, _ = _coords(nx, ny, 1)
    mask = np.zeros(nx * ny, np.uint8)
    ow = max(2, round(obstacle[0] * nx / 1024))
    oh = max(2, round(obstacle[1] * ny / 256))
    rows = []
    for k in range(n_rows):
        xc = int(nx * (0.25 + 0.22 * k) + rng.integers(-nx // 32, nx // 32 + 1))
        band = ny / per_row
        for j in range(per_row):
            lo = int(j * band + 1)
            hi = int((j + 1) * band - oh - 1)
            yc = int(rng.integers(lo, max(lo, hi) + 1))
            sel = (x >= xc) & (x < xc + ow) & (y >= yc) & (y < yc + oh)
            mask[sel] = 1
            rows.append((xc, yc))
    rad = max(3.0, hot_radius * ny / 256)
    dist = np.sqrt((x + 0.5) ** 2 + (y + 0.5 - ny / 2.0) ** 2)
    b = _tanh_blend(rad - dist, 1.0)
    Yu, Yb = np.array(mixture_phi(names, 0.83)), np.array(burnt_mixture(names, 0.83))
    if y_trace:
        for Ym in (Yu, Yb):
            for nm in ("CO", "CO2", "H2O"):
                Ym[names.index(nm)] += y_trace
            Ym[names.index("N2")] -= 3.0 * y_trace
        cfg["Y_in"] = [float(v) for v in Yu]
    T = T_u + (T_hot - T_u) * b
    Y = Yu[:, None] * (1 - b)[None, :] + Yb[:, None] * b[None, :]
    if y_floor:
        Y[Y < y_floor] = 0.0
    u = np.zeros((2, nx * ny))
    inlet_u = np.zeros((2, ny))
    if inlet:
        yy = np.arange(ny) + 0.5
        inlet_u[0] = u_in * 4.0 * yy * (ny - yy) / ny ** 2
        if inlet_jitter:
            inlet_u[0] *= 1.0 + inlet_jitter * rng.standard_normal(ny)
    if u_init:
        u[0] = u_init * (1.0 + 0.2 * rng.standard_normal(nx * ny))
        u[1] = 0.2 * u_init * rng.standard_normal(nx * ny)
        u[:, mask == 1] = 0.0
    return Workload("chamber_2d", cfg, mask, inlet_u, u, np.zeros(nx * ny), T=T, Y=Y,
                    steps=steps, info={"obstacles": rows})


# -------------------------------------------------------------------------- 3-D swirl
def swirl_k(S, Ri, Ro):
    """Tangential/axial velocity ratio giving swirl number S for uniform axial and tangential
    velocity across an annulus Ri < r < Ro: S = k * 2 (Ro^3 - Ri^3) / (3 Ro (Ro^2 - Ri^2))."""
    return S * 3.0 * Ro * (Ro ** 2 - Ri ** 2) / (2.0 * (Ro ** 3 - Ri ** 3))


def swirl_3d(nx=256, ny=128, nz=128, reactive=False, storage="f32", seed=0,
             collision="cumulant", u_axial=0.05, swirl=0.6, noise=0.05, smag=0.17, F=8.0,
             steps=None, dx=None, dt=None, A1=1.0e9, A2=5.0e6, T_in=320.0, T_hot=1970.0,
             sensor_wref=1e-5, curved=False):
    """Swirl-burner-like domain along x: annular swirling inlet (radii 8 and 16 cells at the
    128-cell scale) through an injector duct, square confined chamber, contracting exhaust to
    an outlet; cold (LB only) or reactive (2-step chemistry, thickened flame with sensor,
    closed-domain thermodynamic pressure). curved: wall fractions of every link toward the
    injector cylinders and the exhaust cone (info["wall_links"] = cells, directions, fractions),
    found by bisection on the continuous shapes of which the mask samples the cell centres."""
    rng = np.random.default_rng(seed)
    s = ny / 128.0
    cfg = _base_cfg(3, nx, ny, nz, storage, collision)
    if dx is None:
        dx = 1e-3 if not reactive else 5e-4
    if dt is None:
        dt = 3e-6 if not reactive else 1e-6
    cfg.update({"bc": {"x": ("inlet", "outlet"), "y": ("wall", "wall"), "z": ("wall", "wall")},
                "dx": dx, "dt": dt, "nu_ref": 1.8e-5 / 1.17, "smag_cs": smag})
    x, y, z = _coords(nx, ny, nz)
    yc, zc = ny / 2.0, nz / 2.0
    r = np.sqrt((y + 0.5 - yc) ** 2 + (z + 0.5 - zc) ** 2)
    Ri, Ro = 8.0 * s, 16.0 * s
    L1 = int(round(24 * s * nx / (2 * ny))) + int(rng.integers(-2, 3))
    L2 = int(round(nx * 0.8)) + int(rng.integers(-4, 5))
    Re = 24.0 * s + rng.uniform(-2.0, 2.0) * s
    Rc = min(ny, nz) / 2.0 - 1.0
    mask = np.zeros(nx * ny * nz, np.uint8)
    inj = x < L1
    mask[inj & ((r < Ri) | (r > Ro))] = 1
    cone = x >= L2
    frac = (x - L2) / max(1, nx - 1 - L2)
    Rx = Rc + (Re - Rc) * frac
    mask[cone & (r > Rx)] = 1
    # inlet face (y, z) values
    fy = (np.arange(ny * nz) % ny) + 0.5 - yc
    fz = (np.arange(ny * nz) // ny) + 0.5 - zc
    fr = np.sqrt(fy ** 2 + fz ** 2)
    ann = (fr >= Ri) & (fr <= Ro)
    k = swirl_k(swirl, Ri, Ro)
    inlet = np.zeros((3, ny * nz))
    inlet[0] = np.where(ann, u_axial, 0.0)
    ut = k * u_axial
    safe = np.where(fr > 0, fr, 1.0)
    inlet[1] = np.where(ann, -ut * fz / safe, 0.0)
    inlet[2] = np.where(ann, ut * fy / safe, 0.0)
    inlet += np.where(ann, 1.0, 0.0)[None, :] * noise * u_axial * rng.standard_normal((3, ny * nz))
    N = nx * ny * nz
    u = np.zeros((3, N))
    wl = Workload("swirl_3d", cfg, mask, inlet, u, np.zeros(N),
                  steps=steps or (5000 if reactive else 10000),
                  info={"L1": L1, "L2": L2, "Re": Re, "swirl_k": k})
    if curved:
        span = max(1, nx - 1 - L2)

        def solid(X, Y, Z):
            rr = np.sqrt((Y - yc) ** 2 + (Z - zc) ** 2)
            return ((X < L1) & ((rr < Ri) | (rr > Ro))) | ((X >= L2) & (rr > Rc + (Re - Rc) * (X - 0.5 - L2) / span))

        assert np.array_equal(solid(x + 0.5, y + 0.5, z + 0.5), mask.astype(bool))
        wl.info["wall_links"] = link_fractions(mask, (nx, ny, nz), solid)
    if reactive:
        names = SPECIES["6sp"]
        Yu, Yb = np.array(mixture_phi(names, 0.83)), np.array(burnt_mixture(names, 0.83))
        xf = L1 + 16 * s
        b = _tanh_blend(x + 0.5 - xf, 4.0 * s)
        cfg.update({"thermal": True, "thicken_F": F, "flame_sensor": True,
                    "sensor_beta": 10.0, "sensor_wref": sensor_wref, "sensor_species": 0,
                    "sensor_oxidizer": 1, "sensor_Ta": 8400.0,
                    "closed_domain": True, "species": species(names),
                    "reactions": chemistry_2step(A1, A2), "T_in": T_in, "T_ref": 300.0,
                    "Y_in": list(Yu)})
        wl.T = T_in + (T_hot - T_in) * b
        wl.Y = Yu[:, None] * (1 - b)[None, :] + Yb[:, None] * b[None, :]
    return wl


def link_fractions(mask, dims, solid, iters=40):
    """Links from fluid cells to solid cells inside the grid, as (cells, directions, fractions):
    for pull direction i the link r -> r - c_i, fraction t in (0, 1] where the segment from the
    centre of r enters the solid region solid(X, Y, Z) (continuous coordinates, cell centres at
    index + 0.5), by bisection. D3Q27 order: c = (i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1)."""
    nx, ny, nz = dims
    m = np.asarray(mask).astype(bool)
    x, y, z = _coords(nx, ny, nz)
    cells, dirs, qs = [], [], []
    for i in range(27):
        cx, cy, cz = i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1
        if cx == 0 and cy == 0 and cz == 0:
            continue
        sx, sy, sz = x - cx, y - cy, z - cz
        ins = (sx >= 0) & (sx < nx) & (sy >= 0) & (sy < ny) & (sz >= 0) & (sz < nz)
        sel = np.zeros(m.size, bool)
        sel[ins] = m[(sx + nx * (sy + ny * sz))[ins]]
        sel &= ~m
        r = np.nonzero(sel)[0]
        if r.size == 0:
            continue
        X0, Y0, Z0 = x[r] + 0.5, y[r] + 0.5, z[r] + 0.5
        lo, hi = np.zeros(r.size), np.ones(r.size)
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            inside = solid(X0 - mid * cx, Y0 - mid * cy, Z0 - mid * cz)
            hi = np.where(inside, mid, hi)
            lo = np.where(inside, lo, mid)
        cells.append(r)
        dirs.append(np.full(r.size, i))
        qs.append(np.clip(hi, 1e-3, 1.0))
    if not cells:
        return np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0)
    return (np.concatenate(cells).astype(np.int32), np.concatenate(dirs).astype(np.int32), np.concatenate(qs))


# ------------------------------------------------------------------------ periodic box
def box(dim, n, storage="f64", collision="cumulant", tau=0.8, seed=0, pert=0.0, U=0.0):
    """Isothermal periodic box with a seeded random velocity field and population noise."""
    rng = np.random.default_rng(seed)
    ns = [n] * dim if np.isscalar(n) else list(n)
    nx, ny = ns[0], ns[1]
    nz = ns[2] if dim == 3 else 1
    cfg = _base_cfg(dim, nx, ny, nz, storage, collision)
    bc = {"x": ("periodic", "periodic"), "y": ("periodic", "periodic")}
    if dim == 3:
        bc["z"] = ("periodic", "periodic")
    cfg.update({"bc": bc, "dx": 1.0, "dt": 1.0, "nu_ref": (tau - 0.5) / 3.0})
    N = nx * ny * nz
    u = U * rng.standard_normal((dim, N))
    wl = Workload("box", cfg, np.zeros(N, np.uint8), np.zeros((dim, ny * nz)), u,
                  np.zeros(N), steps=100)
    if pert:
        wl.g_pert = perturbation(rng, 3 ** dim, N, pert)
    return wl


# ------------------------------------------------------------------- curved/offset walls
_D2 = [(cx, cy) for cy in (-1, 0, 1) for cx in (-1, 0, 1)]  # D2Q9 order of the library (x fastest)


def channel_2d(H=16, nx=64, q=0.5, U=0.01, tau=0.8, collision="bgk", storage="f64"):
    """Plane channel, velocity inlet (low x), pressure outlet (high x), walls in y placed at the
    fraction q of the boundary links (walls at y = 0.5 - q and y = H - 0.5 + q in cell units,
    cell centres at j + 0.5): the fully developed Poiseuille parabola of that width as inlet
    profile and initial state (pressure gradient included)."""
    cfg = _base_cfg(2, nx, H, 1, storage, collision)
    nu = (tau - 0.5) / 3.0
    cfg.update({"bc": {"x": ("inlet", "outlet"), "y": ("wall", "wall")}, "dx": 1.0, "dt": 1.0, "nu_ref": nu})
    lo, hi = 0.5 - q, H - 0.5 + q
    Wd = hi - lo
    yy = np.arange(H) + 0.5
    prof = 4.0 * U * (yy - lo) * (hi - yy) / Wd ** 2
    N = nx * H
    x, y, _ = _coords(nx, H, 1)
    u = np.zeros((2, N))
    u[0] = prof[y]
    P = 8.0 * nu * U / Wd ** 2 * (nx - 0.5 - x)
    inlet = np.zeros((2, H))
    inlet[0] = prof
    qw = np.zeros((9, N))
    for i, (cx, cy) in enumerate(_D2):
        # pull direction i: the link r - c_i leaves through the low wall when cy = +1 at y = 0
        qw[i, (y == 0) & (cy == 1)] = q
        qw[i, (y == H - 1) & (cy == -1)] = q
    return Workload("channel_2d", cfg, np.zeros(N, np.uint8), inlet, u, P, qwall=qw,
                    info={"profile": prof, "walls": (lo, hi)})


def cylinder_2d(nx=96, ny=48, radius=7.3, center=None, U=0.02, tau=0.6, collision="cumulant", storage="f32",
                seed=0):
    """Channel with a circular cylinder: solid cells are those whose centre lies inside the
    circle; every bounce-back link toward the cylinder gets the exact fraction at which the
    segment from the fluid node to its solid neighbour enters the circle. Walls in y half-way,
    parabolic inlet, pressure outlet; a seeded offset of the centre breaks the symmetry."""
    rng = np.random.default_rng(seed)
    cfg = _base_cfg(2, nx, ny, 1, storage, collision)
    nu = (tau - 0.5) / 3.0
    cfg.update({"bc": {"x": ("inlet", "outlet"), "y": ("wall", "wall")}, "dx": 1.0, "dt": 1.0, "nu_ref": nu,
                "smag_cs": 0.17})
    if center is None:
        center = (nx * 0.3 + rng.uniform(-0.5, 0.5), ny * 0.5 + rng.uniform(-0.5, 0.5))
    xc, yc = center
    N = nx * ny
    x, y, _ = _coords(nx, ny, 1)
    px, py = x + 0.5, y + 0.5
    solid = (px - xc) ** 2 + (py - yc) ** 2 < radius ** 2
    mask = solid.astype(np.uint8)
    qw = np.zeros((9, N))
    for i, (cx, cy) in enumerate(_D2):
        if cx == 0 and cy == 0:
            continue
        # the link from r to r - c_i; solve |p - t c - center| = R for the entering t in (0, 1]
        sx, sy = x - cx, y - cy
        inside = (sx >= 0) & (sx < nx) & (sy >= 0) & (sy < ny)
        nb_solid = np.zeros(N, bool)
        nb_solid[inside] = solid[(sy * nx + sx)[inside]]
        sel = (~solid) & nb_solid
        dx_, dy_ = px - xc, py - yc
        a = cx * cx + cy * cy
        b = -2.0 * (dx_ * cx + dy_ * cy)
        c = dx_ * dx_ + dy_ * dy_ - radius ** 2
        disc = np.maximum(b * b - 4 * a * c, 0.0)
        t = (-b - np.sqrt(disc)) / (2 * a)
        qw[i, sel] = np.clip(t[sel], 1e-3, 1.0)
    yy = np.arange(ny) + 0.5
    prof = 4.0 * U * yy * (ny - yy) / ny ** 2
    inlet = np.zeros((2, ny))
    inlet[0] = prof
    u = np.zeros((2, N))
    u[0] = np.where(solid, 0.0, prof[y])
    return Workload("cylinder_2d", cfg, mask, inlet, u, np.zeros(N), qwall=qw, steps=2000,
                    info={"center": center, "radius": radius})


def duct_3d(nx=32, ny=12, nz=8, q=0.3, U=0.01, tau=0.8, collision="cumulant", storage="f64"):
    """3-D duct: velocity inlet / pressure outlet in x, walls in y at the fraction q of the
    boundary links (as channel_2d), periodic in z; plane Poiseuille initial state."""
    cfg = _base_cfg(3, nx, ny, nz, storage, collision)
    nu = (tau - 0.5) / 3.0
    cfg.update({"bc": {"x": ("inlet", "outlet"), "y": ("wall", "wall"), "z": ("periodic", "periodic")},
                "dx": 1.0, "dt": 1.0, "nu_ref": nu})
    lo, hi = 0.5 - q, ny - 0.5 + q
    Wd = hi - lo
    yy = np.arange(ny) + 0.5
    prof = 4.0 * U * (yy - lo) * (hi - yy) / Wd ** 2
    N = nx * ny * nz
    x, y, z = _coords(nx, ny, nz)
    u = np.zeros((3, N))
    u[0] = prof[y]
    P = 8.0 * nu * U / Wd ** 2 * (nx - 0.5 - x)
    inlet = np.zeros((3, ny * nz))
    inlet[0] = np.tile(prof, nz)
    qw = np.zeros((27, N))
    for i in range(27):
        cy = (i // 3) % 3 - 1
        qw[i, (y == 0) & (cy == 1)] = q
        qw[i, (y == ny - 1) & (cy == -1)] = q
    return Workload("duct_3d", cfg, np.zeros(N, np.uint8), inlet, u, P, qwall=qw,
                    info={"profile": prof, "walls": (lo, hi)})


_NAMED = {
    "c1_flame_2d": lambda seed=0: flame_2d(seed=seed),
    "c2_chamber_2d": lambda seed=0: chamber_2d(seed=seed),
    "c3_swirl_cold_3d": lambda seed=0: swirl_3d(seed=seed),
    "c4_swirl_reactive_3d": lambda seed=0: swirl_3d(384, 192, 192, reactive=True, seed=seed),
    # C2 family at 512 x 128 with an inlet; a hot kernel of 24 cells (smaller ones quench under
    # the thickening within the 2000 steps); a seeded initial flow, jittered inlet profile and a
    # trace of products keep J differentiable at the point (no upwind tie, no species at 0)
    "c5_adjoint_2d": lambda seed=0: chamber_2d(512, 128, inlet=True, steps=2000, seed=seed, hot_radius=48.0,
                                               inlet_jitter=0.1, u_init=0.005, y_trace=1e-4),
}


def names():
    return list(_NAMED)


def make(name, seed=0):
    return _NAMED[name](seed)
