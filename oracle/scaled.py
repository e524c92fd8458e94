"""Complex numbers with a separate power-of-two exponent: value = m * 2**e.

Z(q) and V(t(q)) leave the double-precision range for large knots (for example
|Z| > 1e308 at q = 6 with a few hundred Tait vertices), so the oracle carries an
integer exponent beside a complex128 mantissa normalised to |m| in [0.5, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass(frozen=True)
class SC:
    m: complex
    e: int = 0

    @staticmethod
    def of(z: complex, e: int = 0) -> "SC":
        return SC(complex(z), int(e)).norm()

    def norm(self) -> "SC":
        a = abs(self.m)
        if a == 0.0 or not math.isfinite(a):
            return SC(self.m if a == 0.0 else self.m, 0 if a == 0.0 else self.e)
        _, k = math.frexp(a)
        return SC(self.m * math.ldexp(1.0, -k), self.e + k)

    def __mul__(self, o: "SC") -> "SC":
        return SC(self.m * o.m, self.e + o.e).norm()

    def __add__(self, o: "SC") -> "SC":
        if self.m == 0:
            return o
        if o.m == 0:
            return self
        e = max(self.e, o.e)
        return SC(self.m * math.ldexp(1.0, self.e - e) + o.m * math.ldexp(1.0, o.e - e), e).norm()

    def __neg__(self) -> "SC":
        return SC(-self.m, self.e)

    def inv(self) -> "SC":
        return SC(1.0 / self.m, -self.e).norm()

    def pow(self, n: int) -> "SC":
        if n < 0:
            return self.inv().pow(-n)
        r, x = SC(1.0 + 0j, 0), self
        while n:
            if n & 1:
                r = r * x
            x = x * x
            n >>= 1
        return r

    def log2abs(self) -> float:
        a = abs(self.m)
        return -math.inf if a == 0 else math.log2(a) + self.e

    def to_complex(self) -> complex:
        """Plain complex value (inf/0 if out of range)."""
        try:
            return self.m * math.ldexp(1.0, self.e)
        except OverflowError:
            return complex(math.inf, math.inf)


def rel_err(a: SC, b: SC) -> float:
    """|a - b| / |b| computed without leaving the scaled representation."""
    if b.m == 0:
        return abs(a.m) if a.m != 0 else 0.0
    d = a.e - b.e
    if d > 1000:
        return math.inf
    da = a.m * math.ldexp(1.0, d)
    return abs(da - b.m) / abs(b.m)
