// Arithmetic in F_p[t]/(t^2 - (q - 2) t + 1), p prime, q < p < 2^31: the ring in which
// Z(q) and V(t(q)) are computed exactly (t(q) is a root of x^2 - (q - 2) x + 1).  Used by
// the exact GPU kernels (exact.cu) and the host solver for V's coefficients
// (jones_exact.cpp).
#pragma once

#include <cstdint>

#include "pk_internal.h"

namespace pk {
namespace exact {

struct Ring {
  uint32_t p;    // prime modulus, q < p < 2^31
  uint32_t qm2;  // (q - 2) mod p
};
struct E {
  uint32_t a, b;  // a + b t
};

PK_HD inline uint32_t mulm(uint32_t x, uint32_t y, uint32_t p) {
  return (uint32_t)(((uint64_t)x * y) % p);
}
PK_HD inline uint32_t addm(uint32_t x, uint32_t y, uint32_t p) {
  const uint32_t s = x + y;  // x, y < 2^31: no overflow
  return s >= p ? s - p : s;
}
PK_HD inline uint32_t subm(uint32_t x, uint32_t y, uint32_t p) { return x >= y ? x - y : x + (p - y); }
PK_HD inline E emul(E x, E y, Ring r) {
  const uint32_t ac = mulm(x.a, y.a, r.p), bd = mulm(x.b, y.b, r.p);
  const uint32_t cross = addm(mulm(x.a, y.b, r.p), mulm(x.b, y.a, r.p), r.p);
  return {subm(ac, bd, r.p), addm(cross, mulm(r.qm2, bd, r.p), r.p)};
}
PK_HD inline E eadd(E x, E y, Ring r) { return {addm(x.a, y.a, r.p), addm(x.b, y.b, r.p)}; }
PK_HD inline E eneg(E x, Ring r) { return {subm(0, x.a, r.p), subm(0, x.b, r.p)}; }
// t^n for any integer n (t^-1 = (q - 2) - t)
PK_HD inline E epow_t(long long n, Ring r) {
  E base = n >= 0 ? E{0, 1} : E{r.qm2, r.p - 1};
  E res{1, 0};
  unsigned long long m = n >= 0 ? (unsigned long long)n : (unsigned long long)(-n);
  while (m) {
    if (m & 1) res = emul(res, base, r);
    base = emul(base, base, r);
    m >>= 1;
  }
  return res;
}
PK_HD inline E epow(E x, unsigned long long m, Ring r) {
  E res{1, 0};
  while (m) {
    if (m & 1) res = emul(res, x, r);
    x = emul(x, x, r);
    m >>= 1;
  }
  return res;
}
inline Ring make_ring(uint32_t prime, int32_t q) {
  return Ring{prime, (uint32_t)(((long long)q - 2 + (long long)prime) % (long long)prime)};
}

}  // namespace exact
}  // namespace pk
