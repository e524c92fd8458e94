"""Exact arithmetic in Z[t] with t^2 = (q-2) t - 1.

For integer q, t(q) of Eq. potts2jones satisfies t + 1/t = q - 2, i.e. it is a root
of x^2 - (q-2) x + 1.  Elements are pairs (a, b) meaning a + b t with Python ints.
The inverse of t is (q-2) - t, so every Laurent polynomial in t with integer
coefficients evaluates to an element of Z[t].  (For q = 4 the ring is
Z[x]/(x-1)^2 and evaluation at t = 1 is a + b.)
"""
from __future__ import annotations

import cmath


class Zt:
    def __init__(self, q: int):
        self.q = int(q)
        self.c = self.q - 2  # t^2 = c t - 1

    # elements are (a, b)
    def mul(self, x, y):
        a, b = x
        c, d = y
        return (a * c - b * d, a * d + b * c + self.c * b * d)

    @staticmethod
    def add(x, y):
        return (x[0] + y[0], x[1] + y[1])

    @staticmethod
    def neg(x):
        return (-x[0], -x[1])

    @property
    def one(self):
        return (1, 0)

    @property
    def t(self):
        return (0, 1)

    @property
    def tinv(self):
        return (self.c, -1)

    def pow(self, x, n: int):
        if n < 0:
            if x != self.t:
                raise ValueError("only t has a ring inverse here")
            x, n = self.tinv, -n
        r = self.one
        while n:
            if n & 1:
                r = self.mul(r, x)
            x = self.mul(x, x)
            n >>= 1
        return r

    def tpow(self, n: int):
        return self.pow(self.t, n)

    def eval_laurent(self, coeffs: dict):
        """Evaluate sum_k coeffs[k] t^k exactly."""
        acc = (0, 0)
        for k, c in coeffs.items():
            if c:
                p = self.tpow(k)
                acc = self.add(acc, (c * p[0], c * p[1]))
        return acc

    def to_complex(self, x, t: complex | None = None):
        if t is None:
            from .potts import t_of_q
            t = t_of_q(self.q)
        return complex(x[0]) + complex(x[1]) * t


def laurent_eval_complex(coeffs: dict, t: complex) -> complex:
    return sum(c * cmath.exp(k * cmath.log(t)) if t != 0 else 0 for k, c in coeffs.items())
