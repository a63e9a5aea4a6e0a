"""Plain FP64 CPU oracle of the hybrid low-Mach lattice Boltzmann / finite-difference time
step (Hosseini, Darabiha, Thevenin, Section 2).

This package is TEST INFRASTRUCTURE. It is a slow, literal restatement of the method, written
for checking, not for speed: only the tests, the smoke check of the package and the CPU
baseline leg of the benchmark may import it. The GPU library never calls it and shares no code
with it (no kernels, tables, helpers or constants). Both sides read the same seeded inputs,
produced by the separate ``workloads`` module.

Every floating-point value is torch.float64 on the CPU. Functions cite the equation or section
of the paper they follow; where the paper is silent the docstring names the reading taken.

Module map
    lattice    D2Q9 / D3Q27 velocity sets and weights (Section 2.1)
    cumulant   central moments, cumulants (partition formula) and their inverses (Section 2.2)
    lb         equilibrium, source term, moments, pre-conditioning, collisions, streaming
    fd         WENO3 advection, centred diffusion, Arrhenius chemistry, thickening (Section 2.3)
    geometry   boundary links (lattice Boltzmann) and stencil ghosts (finite differences)
    units      physical -> lattice unit conversion
    step       one full hybrid time step: FD -> thermodynamic pressure -> LB
"""
