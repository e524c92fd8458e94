"""The q-state PACI model on a signed Tait graph and its Jones normalisation (Sec. II).

* t(q) = (q + sqrt(q) sqrt(q - 4) - 2) / 2 with principal square roots (Eq. potts2jones).
* Clause matrix of an edge with Tait sign eps (Eq. clause):
  T[s, s'] = 1 - (1 + t^-eps) delta(s, s'), i.e. off-diagonal 1, diagonal -t^-eps
  (equivalently e^{J_pm} = -t^{-+}).
* Z(q) = sum over all spin states sigma in {0..q-1}^{n_v} of prod_edges T[sigma_u, sigma_v].
* V = A(q) Z(q) with A(q) = (-t^{1/2} - t^{-1/2})^{-n_v-1} (-t^{3/4})^{w} t^{tau/4}
  (Eq. JonesPotts).  Fractional powers are all taken from the one principal fourth
  root s = exp(Log(t)/4), so t^{1/2} = s^2, t^{3/4} = s^3, t^{1/4} = s.
"""
from __future__ import annotations

import cmath
import itertools
import math
from decimal import Decimal, localcontext
from fractions import Fraction

from .ring import Zt
from .scaled import SC


def t_of_q(q: int) -> complex:
    q = complex(q)
    return (q + cmath.sqrt(q) * cmath.sqrt(q - 4) - 2) / 2


def clause_diag(q: int, eps: int) -> complex:
    """Diagonal entry of T for Tait sign eps: 1 - (1 + t^-eps) = -t^-eps."""
    t = t_of_q(q)
    return 1 - (1 + t ** (-eps))


def clause_matrix(q: int, eps: int):
    import numpy as np
    T = np.ones((q, q), dtype=np.complex128)
    T[np.diag_indices(q)] = clause_diag(q, eps)
    return T


def z_bruteforce(n_v: int, edges, q: int) -> complex:
    """Z(q) as the literal sum over q^n_v spin states (tiny graphs only)."""
    diag = {+1: clause_diag(q, +1), -1: clause_diag(q, -1)}
    tot = 0j
    for sigma in itertools.product(range(q), repeat=n_v):
        p = 1 + 0j
        for (u, v, eps) in edges:
            p *= diag[eps] if sigma[u] == sigma[v] else 1.0
        tot += p
    return tot


def z_bruteforce_exact(n_v: int, edges, q: int):
    """Same spin sum in Z[t]: T's diagonal is -t^-1 = t - (q-2) for eps=+1 and -t for eps=-1."""
    R = Zt(q)
    diag = {+1: (-(q - 2), 1), -1: (0, -1)}
    tot = (0, 0)
    for sigma in itertools.product(range(q), repeat=n_v):
        p = R.one
        for (u, v, eps) in edges:
            if sigma[u] == sigma[v]:
                p = R.mul(p, diag[eps])
        tot = R.add(tot, p)
    return tot


def prefactor(q: int, n_v: int, writhe: int, tau: int) -> SC:
    """A(q) of Eq. JonesPotts as a scaled complex number (principal fourth root s of t)."""
    t = t_of_q(q)
    s = cmath.exp(cmath.log(t) / 4)
    base = SC.of(-(s ** 2) - s ** -2)
    part1 = base.pow(-n_v - 1)
    part2 = SC.of(-(s ** 3)).pow(writhe)
    part3 = SC.of(s).pow(tau)
    return part1 * part2 * part3


def jones_from_z(z: SC, g, q: int) -> SC:
    return prefactor(q, g.n_v, g.writhe, g.tau) * z


def jones_from_z_exact(z, g, q: int):
    """V exactly: returns (v, den) with V = v / den, v in Z[t], den = q^(n_v+1).

    Uses the same A(q), rewritten without fractional powers: with s^4 = t,
    (-s^2 - s^-2)^(-n-1) = (-1)^(n+1) s^(2n+2) (t+1)^-(n+1), so
    A = (-1)^(w+n_v+1) t^k (t+1)^-(n_v+1), k = (3w + tau + 2 n_v + 2)/4, and
    (t+1)^-1 = (q - 1 - t)/q in Z[t][1/q].  Requires 4 | 3w + tau + 2 n_v + 2.
    """
    R = Zt(q)
    num = 3 * g.writhe + g.tau + 2 * g.n_v + 2
    if num % 4:
        raise ValueError("3w + tau + 2 n_v + 2 is not divisible by 4")
    k = num // 4
    sign = -1 if (g.writhe + g.n_v + 1) % 2 else 1
    v = R.mul(z, R.tpow(k))
    v = R.mul(v, R.pow((q - 1, -1), g.n_v + 1))
    v = (sign * v[0], sign * v[1])
    return v, q ** (g.n_v + 1)


def _dec_to_float_exp(x):
    """Decimal x -> (m, e) with x = m * 2**e and m a float (|m| ~ 1)."""
    if x == 0:
        return 0.0, 0
    n, d = x.as_integer_ratio()
    e = n.bit_length() - d.bit_length() if n > 0 else (-n).bit_length() - d.bit_length()
    fr = Fraction(n, d) / (Fraction(2) ** e)
    return float(fr), e


def exact_to_complex(v, den, q: int) -> SC:
    """Value of v/den, v = a + b t in Z[t], as a scaled complex number.

    Real and imaginary parts are formed in 80-digit decimal arithmetic:
    t = ((q - 2) + sqrt(q (q - 4))) / 2, the root being imaginary for q < 4."""
    a, b = v
    with localcontext() as ctx:
        ctx.prec = 80
        re2 = Decimal(2 * a + (q - 2) * b)
        disc = q * (q - 4)
        if disc >= 0:
            re = (re2 + Decimal(b) * Decimal(disc).sqrt()) / (2 * Decimal(den))
            im = Decimal(0)
        else:
            re = re2 / (2 * Decimal(den))
            im = Decimal(b) * Decimal(-disc).sqrt() / (2 * Decimal(den))
        mr, er = _dec_to_float_exp(re)
        mi, ei = _dec_to_float_exp(im)
    if mr == 0.0 and mi == 0.0:
        return SC(0j, 0)
    E = max(er if mr != 0.0 else -10**9, ei if mi != 0.0 else -10**9)
    return SC.of(complex(math.ldexp(mr, er - E), math.ldexp(mi, ei - E)), E)


def exact_z_to_complex(z, q: int) -> SC:
    return exact_to_complex(z, 1, q)
