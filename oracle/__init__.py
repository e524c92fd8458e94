"""CPU oracle for the PACI partition function and the Jones value (test infrastructure).

This package is TEST INFRASTRUCTURE, not part of the library.  Only `tests/`,
`__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference` legs of
`bench.py` may import it.  It shares no code with the GPU library (no headers,
helpers, tables or generators); both consume PD codes from `knotgen`.

What it computes, and where each part comes from in the paper:

* `tait`     knot diagram (PD code) -> checkerboard colouring -> signed Tait graph,
             writhe w and Tait number tau (Sec. II: twist sign, bicolouring with the
             unbounded region white, Tait-sign rule).
* `potts`    t(q) (Eq. potts2jones), the clause matrix T = 1 - (1 + t^-eps) delta
             (Eq. clause), Z(q) as the plain spin sum (Sec. II), the prefactor A(q)
             (Eq. JonesPotts) and V = A Z.
* `elim`     Z(q) by summing spins out one at a time (distributivity applied to the
             plain definition Z = sum_sigma prod_edges T); complex128 with a per-factor
             power-of-two exponent, and an exact mode in Z[t] with Python integers
             (t is a root of x^2 - (q-2) x + 1, so every clause entry lies in Z[t]).
* `kauffman` the Jones polynomial from the Kauffman bracket state sum over all
             2^n smoothings of the PD code -- independent of the Tait graph and of
             the Potts model, used to pin the rest.
* `ring`     exact arithmetic in Z[t] and Laurent-polynomial evaluation.
* `scaled`   complex numbers with a separate integer power-of-two exponent (Z and V
             overflow double precision on large knots).

Every function here is parity-pinned by tests in `tests/test_oracle_*.py`
(brute-force spin sums, the Kauffman bracket, closed-form Jones polynomials,
the values printed in the caption of Fig. 1, and knot invariants).
"""
from . import ring, scaled, tait, potts, elim, kauffman  # noqa: F401
from .tait import TaitGraph, tait_graph  # noqa: F401
from .potts import t_of_q, jones_from_z, jones_from_z_exact  # noqa: F401
from .elim import z_complex, z_exact  # noqa: F401


def jones(pd, q, outer=None, black=None):
    """V_K(t(q)) of the knot with PD code `pd` as a scaled complex number (complex128)."""
    g = tait_graph(pd, outer=outer, black=black)
    z = z_complex(g.n_v, g.edges, q)
    return jones_from_z(z, g, q)


def jones_exact(pd, q, outer=None, black=None):
    """V_K(t(q)) exactly, as (numerator in Z[t], denominator q^(n_v+1))."""
    g = tait_graph(pd, outer=outer, black=black)
    z = z_exact(g.n_v, g.edges, q)
    return jones_from_z_exact(z, g, q)
