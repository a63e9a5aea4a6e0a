"""Closed forms used by the stream-collide kernel when the higher-order moments are fully relaxed:
the central moments of orders 0..2 of w_i xi_i (xi of Eq. 2 divided by w_i, in lattice units) on
D2Q9 and D3Q27, with L = rho cs2 Lambda and G = u . grad rho,
    k_0 = L + G/3, k_a = -u_a k_0, k_aa = L u_a^2 + L/3 + (G + 2 g_a u_a)/9,
    k_ab = L u_a u_b + (g_a u_b + g_b u_a)/9,
against the sums over the lattice directions (product weights 2/3, 1/6, 1/6 per axis)."""
import itertools

import numpy as np
import pytest


def _closed(D, u, g, L):
    G = float(u @ g)
    k0 = L + G / 3.0
    out = {(0,) * D: k0}
    for a in range(D):
        e = [0] * D
        e[a] = 1
        out[tuple(e)] = -u[a] * k0
        e[a] = 2
        out[tuple(e)] = L * u[a] ** 2 + L / 3.0 + (G + 2.0 * g[a] * u[a]) / 9.0
        for b in range(a + 1, D):
            e = [0] * D
            e[a] = e[b] = 1
            out[tuple(e)] = L * u[a] * u[b] + (g[a] * u[b] + g[b] * u[a]) / 9.0
    return out


def _brute(D, u, g, L):
    w1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
    usq, G = float(u @ u), float(u @ g)
    out = {}
    for n in itertools.product(range(3), repeat=D):
        if sum(n) > 2:
            continue
        tot = 0.0
        for c in itertools.product((-1, 0, 1), repeat=D):
            c = np.array(c, dtype=float)
            w = np.prod([w1[int(ci)] for ci in c])
            cu, cg = float(c @ u), float(c @ g)
            xi = (cu + 1.5 * cu * cu - 0.5 * usq) * (cg - G) + L
            tot += w * xi * np.prod((c - u) ** np.array(n))
        out[n] = tot
    return out


@pytest.mark.parametrize("D", [2, 3])
def test_low_order_source_moments_closed_form(D):
    rng = np.random.default_rng(7 + D)
    for _ in range(20):
        u = rng.normal(0.0, 0.05, D)
        g = rng.normal(0.0, 0.02, D)
        L = float(rng.normal(0.0, 1e-3))
        cf, bf = _closed(D, u, g, L), _brute(D, u, g, L)
        assert set(cf) == set(bf) and len(cf) == (6 if D == 2 else 10)
        for n in bf:
            assert abs(cf[n] - bf[n]) <= 1e-15 + 1e-12 * abs(bf[n]), (n, cf[n], bf[n])
