"""Central moments and cumulants of one discrete distribution per cell (Section 2.2: the
multiple-relaxation realisation relaxes cumulants of the pre-conditioned populations, following
the cumulant operator of Geier et al. 2015, ref. [geier_cumulant_2015]).

Everything here is written from the definitions, with no transform tricks:

* multi-index a = (a_x, a_y[, a_z]), each a_alpha in {0, 1, 2}; multi-index j of a is stored at
  position a_x + 3 a_y + 9 a_z (the same numbering as the velocity set);
* central moment   k[a] = sum_i prod_alpha (c_i,alpha - u_alpha)^a_alpha h_i;
* cumulants of the normalised distribution m = k / k[0] by the partition formula
      c[a] = sum over set partitions pi of the axis labels of a of
             (-1)^(|pi| - 1) (|pi| - 1)! prod_{B in pi} m[B];
  a partition with a singleton block contributes nothing because the first central moments
  vanish, so those are skipped. Cumulants are returned scaled by k[0] (C = k[0] c);
* inverse          m[a] = sum over partitions pi (no singletons) prod_{B in pi} c[B];
* central -> raw moments by the binomial expansion of c = (c - u) + u, then populations by
  solving the constant raw-moment system M0 h = m, M0[a, i] = prod_alpha c_i,alpha^a_alpha.
"""
import itertools
import math

import torch


def multi_indices(dim):
    """All multi-indices in storage order (position a_x + 3 a_y + 9 a_z)."""
    out = []
    for j in range(3 ** dim):
        out.append(tuple((j // 3 ** k) % 3 for k in range(dim)))
    return out


def _index_of(a):
    return sum(ak * 3 ** k for k, ak in enumerate(a))


def _set_partitions(items):
    """All set partitions of a list of distinct positions (recursive)."""
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for part in _set_partitions(rest):
        # put `first` into each existing block, or into a new block
        for b in range(len(part)):
            yield part[:b] + [[first] + part[b]] + part[b + 1:]
        yield [[first]] + part


def _partition_terms(a):
    """Partitions of the label multiset of ``a`` with no singleton block.

    Returns a list of (coefficient, [block storage indices]) where the coefficient is the
    moment->cumulant weight (-1)^(k-1) (k-1)! for k blocks.
    """
    labels = []
    for axis, count in enumerate(a):
        labels += [axis] * count
    dim = len(a)
    terms = []
    for part in _set_partitions(list(range(len(labels)))):
        if any(len(b) < 2 for b in part):
            continue
        blocks = []
        for b in part:
            bi = [0] * dim
            for pos in b:
                bi[labels[pos]] += 1
            blocks.append(_index_of(bi))
        k = len(part)
        coeff = (-1) ** (k - 1) * math.factorial(k - 1)
        terms.append((coeff, blocks))
    return terms


class CumulantSpace:
    """Precomputed index sets for one lattice."""

    def __init__(self, lat):
        self.lat = lat
        self.dim = lat.dim
        self.idx = multi_indices(lat.dim)
        self.order = torch.tensor([sum(a) for a in self.idx])
        self.terms = {j: _partition_terms(a) for j, a in enumerate(self.idx) if sum(a) >= 2}
        # raw monomial matrix M0[a, i] = prod_alpha c_i,alpha^a_alpha
        m0 = torch.ones(len(self.idx), lat.Q, dtype=torch.float64)
        for j, a in enumerate(self.idx):
            for alpha, p in enumerate(a):
                m0[j] *= lat.c[:, alpha] ** p
        self.M0 = m0
        self.M0_inv = torch.linalg.inv(m0)

    def central_moments(self, h, u):
        """k[a] for every multi-index; h [Q, N], u [dim, N] -> [Q, N]."""
        c = self.lat.c
        out = torch.empty_like(h)
        for j, a in enumerate(self.idx):
            wgt = torch.ones_like(h)
            for alpha, p in enumerate(a):
                if p:
                    wgt = wgt * (c[:, alpha, None] - u[alpha][None, :]) ** p
            out[j] = (wgt * h).sum(0)
        return out

    def cumulants_from_central(self, k):
        k0 = k[0]
        m = k / k0
        C = k.clone()
        for j, terms in self.terms.items():
            acc = torch.zeros_like(k0)
            for coeff, blocks in terms:
                prod = torch.full_like(k0, float(coeff))
                for b in blocks:
                    prod = prod * m[b]
                acc = acc + prod
            C[j] = k0 * acc
        return C

    def central_from_cumulants(self, C):
        k0 = C[0]
        c = C / k0
        k = C.clone()
        for j, terms in self.terms.items():
            acc = torch.zeros_like(k0)
            for _coeff, blocks in terms:
                prod = torch.ones_like(k0)
                for b in blocks:
                    prod = prod * c[b]
                acc = acc + prod
            k[j] = k0 * acc
        return k

    def raw_from_central(self, k, u):
        """m[a] = sum_{j <= a} prod_alpha binom(a_alpha, j_alpha) u_alpha^(a_alpha - j_alpha) k[j]."""
        m = torch.zeros_like(k)
        for ja, a in enumerate(self.idx):
            for jb in itertools.product(*[range(p + 1) for p in a]):
                coef = torch.ones_like(k[0])
                for alpha in range(self.dim):
                    coef = coef * math.comb(a[alpha], jb[alpha]) * u[alpha] ** (a[alpha] - jb[alpha])
                m[ja] = m[ja] + coef * k[_index_of(jb)]
        return m

    def populations_from_raw(self, m):
        return self.M0_inv @ m

    def populations_from_central(self, k, u):
        return self.populations_from_raw(self.raw_from_central(k, u))
