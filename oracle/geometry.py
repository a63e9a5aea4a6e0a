"""Boundary handling of the oracle: lattice Boltzmann links and finite-difference ghosts.

The paper states only that walls are no-slip / zero-flux / adiabatic (Section 3.1) and that
"proper treatment" of boundaries is used (Section 1). Readings taken here:

Lattice Boltzmann (pull form of Eq. 1): the population i arriving at fluid cell r comes from
s = r - c_i.
  * x below 0: periodic -> wrap; wall -> halfway bounce-back; inlet -> bounce-back from a wall
    moving with the inlet velocity of the face element next to r (takes precedence over every
    other rule).
  * x at or above nx: periodic -> wrap; wall -> bounce-back; outlet -> anti-bounce-back from the
    half-way face with the outlet pressure P_h = P_ref and the wall velocity equal to the
    velocity of the outlet cell at the previous step (an open end at ambient pressure).
  * inlet and outlet rules of the x faces take precedence over the walls of other faces.
  * y, z: periodic -> wrap; wall -> bounce-back.
  * s inside the domain but solid (mask != 0) -> bounce-back.
Codes: 0 pull from ``src``, 1 bounce-back, 2 bounce-back plus inlet term, 3 outlet
anti-bounce-back. Inlets are allowed on the low-x face only, outlets on the high-x face only.

Finite differences (Section 2.3): a stencil point that is not a fluid cell takes a ghost value.
  * wall or solid: zero gradient (value of the last fluid cell on the line; velocity 0), or, with
    sub-cell wall positions, the ghost-point value of ``FDNeighbours``;
  * inlet: the inlet state (Dirichlet; velocity = inlet velocity of the face element next to r);
  * outlet: zero gradient (value and velocity of the last fluid cell).

Packed link word used to compare with the GPU library bit for bit: for a fluid cell, bit i is
set when direction i is not a plain pull (code 1, 2 or 3) and bit 31 is set; a solid cell has
word 0.

Packed stencil word of the finite-difference update: for axis a and side s (0: -, 1: +) the
four bits at 4 (2a + s) hold the kind of the distance-1 point (bits 0-1: 0 fluid, 1 wall or
solid, 2 inlet, 3 outlet) and of the distance-2 point (bits 2-3: 0 fluid, 1 zero-gradient copy
of the distance-1 value, 2 inlet); bit 30 marks a cell with ghost-point wall weights; bit 31
marks a fluid cell, a solid cell has word 0.
"""
import torch

PERIODIC, WALL, INLET, OUTLET = 0, 1, 2, 3
BC_NAMES = {"periodic": PERIODIC, "wall": WALL, "inlet": INLET, "outlet": OUTLET}
K_FLUID, K_SOLID, K_INLET, K_OUTLET = 0, 1, 2, 3


def bc_codes(cfg):
    out = []
    for ax in ("x", "y", "z")[: cfg["dim"]]:
        lo, hi = cfg["bc"][ax]
        out.append((BC_NAMES[lo], BC_NAMES[hi]))
    return out


class Grid:
    def __init__(self, cfg, mask):
        self.dim = cfg["dim"]
        self.shape = (cfg["nx"], cfg["ny"], cfg["nz"] if self.dim == 3 else 1)
        nx, ny, nz = self.shape
        self.N = nx * ny * nz
        self.bc = bc_codes(cfg)
        self.mask = torch.as_tensor(mask).reshape(-1).to(torch.int64)
        assert self.mask.numel() == self.N
        self.fluid = self.mask == 0
        r = torch.arange(self.N)
        self.coord = [r % nx, (r // nx) % ny, r // (nx * ny)][: self.dim]
        for a in range(self.dim):
            lo, hi = self.bc[a]
            if (lo == OUTLET) or (hi == INLET) or (a > 0 and (lo in (INLET, OUTLET) or hi in (INLET, OUTLET))):
                raise ValueError("inlet only on low x, outlet only on high x")

    def index(self, coords):
        nx, ny, _ = self.shape
        r = coords[0] + nx * coords[1]
        if self.dim == 3:
            r = r + nx * ny * coords[2]
        return r

    def face_index(self):
        """Index of the low-x face element (y[, z]) next to each cell: y + ny z."""
        ny = self.shape[1]
        f = self.coord[1].clone()
        if self.dim == 3:
            f = f + ny * self.coord[2]
        return f


def lb_links(lat, grid):
    """Per direction and cell: code [Q, N] (0 pull, 1 bounce-back, 2 inlet) and source [Q, N]."""
    Q, N = lat.Q, grid.N
    code = torch.zeros(Q, N, dtype=torch.int64)
    src = torch.zeros(Q, N, dtype=torch.int64)
    r = torch.arange(N)
    for i in range(Q):
        inlet = torch.zeros(N, dtype=torch.bool)
        outlet = torch.zeros(N, dtype=torch.bool)
        wall = torch.zeros(N, dtype=torch.bool)
        s = []
        for a in range(grid.dim):
            n = grid.shape[a]
            lo, hi = grid.bc[a]
            sa = grid.coord[a] - lat.ci[i, a]
            below, above = sa < 0, sa >= n
            if lo == PERIODIC:
                sa = torch.where(below, sa + n, sa)
            elif lo == WALL:
                wall |= below
            elif lo == INLET:
                inlet |= below
            if hi == PERIODIC:
                sa = torch.where(above, sa - n, sa)
            elif hi == WALL:
                wall |= above
            elif hi == OUTLET:
                outlet |= above
            s.append(sa.clamp(0, n - 1))
        sidx = grid.index(s)
        solid_src = grid.mask[sidx] != 0
        c = torch.where(inlet, 2, torch.where(outlet, 3, torch.where(wall | solid_src, 1, 0)))
        code[i] = c
        src[i] = torch.where(c == 0, sidx, r)
    code[:, ~grid.fluid] = 0
    return code, src


def wall_links(lat, grid, code, src, qwall):
    """Interpolated bounce-back data: wall fraction q [Q, N] of each code-1 link (0.5 elsewhere and
    where no fraction is given) and the index of r + c_i when that node is fluid (else -1). The
    node r + c_i is the pull source of the opposite direction."""
    q = torch.as_tensor(qwall, dtype=torch.float64).reshape(lat.Q, grid.N).clone()
    bb = code == 1
    q = torch.where(bb & (q > 0) & (q <= 1), q, torch.full_like(q, 0.5))
    far = torch.full((lat.Q, grid.N), -1, dtype=torch.int64)
    for i in range(lat.Q):
        o = int(lat.opp[i])
        ok = code[o] == 0  # r + c_i = r - c_o is the pull source of direction o, a fluid node
        far[i] = torch.where(ok, src[o], torch.full_like(src[o], -1))
    return {"q": q, "far": far}


def pack_links(code, grid, wall=None):
    """Packed link words (int64 holding the uint32 bit pattern); bit 30 marks cells with an
    interpolated bounce-back link (a code-1 link whose effective fraction is not 1/2)."""
    Q = code.shape[0]
    word = torch.zeros(grid.N, dtype=torch.int64)
    for i in range(Q):
        word |= (code[i] != 0).to(torch.int64) << i
    if wall is not None:
        eff = torch.where((wall["q"] < 0.5) & (wall["far"] < 0), torch.full_like(wall["q"], 0.5), wall["q"])
        interp = ((code == 1) & (eff != 0.5)).any(0)
        word |= interp.to(torch.int64) << 30
    word |= grid.fluid.to(torch.int64) << 31
    word[~grid.fluid] = 0
    return word


def _classify(grid, axis, sigma, base):
    """Kind and index of base + sigma e_axis (kind: fluid, solid, inlet, outlet)."""
    n = grid.shape[axis]
    lo, hi = grid.bc[axis]
    # base is an index array; recover its coordinates
    nx, ny, _ = grid.shape
    bc_ = [base % nx, (base // nx) % ny, base // (nx * ny)][: grid.dim]
    pa = bc_[axis] + sigma
    kind = torch.full_like(base, K_FLUID)
    out_lo, out_hi = pa < 0, pa >= n
    if sigma < 0:
        if lo == PERIODIC:
            pa = torch.where(out_lo, pa + n, pa)
        elif lo == INLET:
            kind = torch.where(out_lo, K_INLET, kind)
        else:
            kind = torch.where(out_lo, K_SOLID, kind)
    else:
        if hi == PERIODIC:
            pa = torch.where(out_hi, pa - n, pa)
        elif hi == OUTLET:
            kind = torch.where(out_hi, K_OUTLET, kind)
        else:
            kind = torch.where(out_hi, K_SOLID, kind)
    bc_[axis] = pa.clamp(0, n - 1)
    idx = grid.index(bc_)
    inside = kind == K_FLUID
    kind = torch.where(inside & (grid.mask[idx] != 0), K_SOLID, kind)
    idx = torch.where(kind == K_FLUID, idx, base)
    return kind, idx


class FDNeighbours:
    """Ghost resolution of the radius-2 line stencils, for each axis and side.

    Walls with sub-cell positions (reading of the paper's curved-boundary treatment for the
    finite differences: ghost points): where the distance-1 point along an axis is a wall or a
    solid cell, the interpolated bounce-back data give the wall at the fraction q of the link, and
    the point opposite is fluid, the ghost value is taken from the parabola through the cell and
    its opposite neighbour whose derivative along the axis vanishes at the wall (adiabatic,
    zero flux): ghost = phi_r + w (phi_opp - phi_r), w = (1 - 2q) / (1 + 2q). A distance-2 point
    beyond such a ghost copies it; a distance-2 wall point seen past a fluid neighbour takes that
    neighbour's ghost, phi_1 + w_1 (phi_r - phi_1). q = 1/2 (w = 0) is the zero-gradient ghost."""

    def __init__(self, grid, wall=None, lat=None):
        self.grid = grid
        r = torch.arange(grid.N)
        self.lines = {}
        for axis in range(grid.dim):
            for sigma in (-1, 1):
                k1, i1 = _classify(grid, axis, sigma, r)
                k2, i2 = _classify(grid, axis, sigma, i1)
                # distance-2 point: if the first point is a ghost, repeat the first ghost
                ghost1 = k1 != K_FLUID
                k2 = torch.where(ghost1, k1, k2)
                i2 = torch.where(ghost1, r, i2)
                # a zero-gradient ghost at distance 2 copies the fluid point at distance 1
                self.lines[(axis, sigma)] = (k1, i1, k2, i2)
        self.w1, self.w2 = None, None
        if wall is not None:
            self.w1, self.w2 = {}, {}
            for axis in range(grid.dim):
                for sigma in (-1, 1):
                    c = [0, 0, 0]
                    c[axis] = -sigma  # pull direction whose source is r + sigma e_axis
                    i = sum((c[a] + 1) * 3 ** a for a in range(grid.dim))
                    q = wall["q"][i]
                    q = torch.where((q < 0.5) & (wall["far"][i] < 0), torch.full_like(q, 0.5), q)
                    k1 = self.lines[(axis, sigma)][0]
                    kopp = self.lines[(axis, -sigma)][0]
                    use = (k1 == K_SOLID) & (kopp == K_FLUID) & grid.fluid
                    self.w1[(axis, sigma)] = torch.where(use, (1 - 2 * q) / (1 + 2 * q), torch.zeros_like(q))
            for axis in range(grid.dim):
                for sigma in (-1, 1):
                    k1, i1, k2, _ = self.lines[(axis, sigma)]
                    beyond = (k1 == K_FLUID) & (k2 == K_SOLID)
                    self.w2[(axis, sigma)] = torch.where(beyond, self.w1[(axis, sigma)][i1],
                                                         torch.zeros(grid.N, dtype=torch.float64))

    def value(self, phi, phi_in, axis, sigma, dist):
        """phi at r + dist*sigma*e_axis with ghosts (zero gradient or inlet Dirichlet, or the
        ghost-point value at walls with sub-cell positions)."""
        k1, i1, k2, i2 = self.lines[(axis, sigma)]
        k, i = (k1, i1) if dist == 1 else (k2, i2)
        v = torch.where(k == K_INLET, torch.as_tensor(phi_in, dtype=phi.dtype), phi[i])
        if self.w1 is None:
            return v
        w1 = self.w1[(axis, sigma)]
        opp = phi[self.lines[(axis, -sigma)][1]]
        g1 = phi + w1 * (opp - phi)  # ghost-point value; the zero-gradient one where w1 = 0
        if dist == 1:
            return torch.where(k1 == K_SOLID, g1, v)
        v = torch.where(k1 == K_SOLID, g1, v)  # beyond a ghost: its copy
        p1 = phi[i1]
        w2 = self.w2[(axis, sigma)]
        return torch.where(w2 != 0, p1 + w2 * (phi - p1), v)

    def velocity(self, u_axis, uin_axis_at_r, axis, sigma):
        """Velocity component at r + sigma e_axis: fluid value, 0 at walls, inlet value, or
        the value at r for an outlet."""
        k1, i1, _, _ = self.lines[(axis, sigma)]
        r = torch.arange(self.grid.N)
        v = u_axis[i1]
        v = torch.where(k1 == K_SOLID, torch.zeros_like(v), v)
        v = torch.where(k1 == K_INLET, uin_axis_at_r, v)
        v = torch.where(k1 == K_OUTLET, u_axis[r], v)
        return v

    def kind1(self, axis, sigma):
        return self.lines[(axis, sigma)][0]

    def index1(self, axis, sigma):
        return self.lines[(axis, sigma)][1]


def pack_stencil_words(grid, nb):
    """Packed finite-difference stencil words (int64 holding the uint32 bit pattern)."""
    word = torch.zeros(grid.N, dtype=torch.int64)
    for axis in range(grid.dim):
        for side, sigma in enumerate((-1, 1)):
            k1, _, k2, _ = nb.lines[(axis, sigma)]
            # distance-2 kind relative to the rule: fluid, zero-gradient copy, or inlet
            d2 = torch.where(k2 == K_FLUID, 0, torch.where(k2 == K_INLET, 2, 1))
            word |= (k1 | (d2 << 2)) << (4 * (2 * axis + side))
    if nb.w1 is not None:
        # bit 30: the cell has ghost-point wall weights on some side
        flag = torch.zeros(grid.N, dtype=torch.bool)
        for key in nb.w1:
            flag |= (nb.w1[key] != 0) | (nb.w2[key] != 0)
        word |= flag.to(torch.int64) << 30
    word |= grid.fluid.to(torch.int64) << 31
    word[~grid.fluid] = 0
    return word
