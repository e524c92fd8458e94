// The Jones polynomial's coefficients from exact values at integer q (host side).
//
// The conclusions of the paper note that V_K(t)'s coefficients follow from evaluations
// at as many values of t as its degree span, by interpolation.  The tensor network has an
// integer dimension q, so the values available are V(t(q)) at integer q, and floating
// point cannot recover integer coefficients from real points t(q) ~ q - 2 (the systems are
// far too ill-conditioned).  Here every value is exact modulo a prime p:
//   * Z(q) mod p comes from the GPU (exact.cu) as a + b t in F_p[t]/(t^2 - (q-2) t + 1);
//   * V(t(q)) = (-1)^(w+n_v+1) t^k Z(q) (t+1)^-(n_v+1) with (t+1)^-1 = (q - 1 - t)/q
//     (Eq. JonesPotts in its integer-exponent form), again an element of that ring;
//   * V(t) = sum_{j=lo}^{hi} c_j t^j reduced modulo t^2 - (q-2) t + 1 must equal it: two
//     linear equations over F_p per q in the unknown integers c_j;
//   * enough q give a square-or-taller system, solved by Gaussian elimination mod p;
//   * the c_j mod several primes give the integers c_j by the Chinese remainder theorem
//     (Garner's mixed-radix form in 128-bit arithmetic), checked against one more prime.
// A link's V lies in t^(1/2) Z[t^(+-1)] when its A(q) exponent num = 3w + tau + 2 n_v + 2 is
// 2 mod 4 (h = 1 below); then W = V t^(-1/2) = (-1)^(w+n_v+1) t^((num-2)/4) Z (t+1)^-(n_v+1)
// has integer powers and is found the same way, and V's powers are W's plus 1/2.
// The exponent window [lo, hi] follows from the Kauffman bracket's extreme states: with
// |s_A|, |s_B| the loop counts of the all-A and all-B smoothings of the n crossings, the
// bracket's A-degrees lie in [-n - 2(|s_B| - 1), n + 2(|s_A| - 1)], and t = A^-4 with the
// writhe shift (-A^3)^-w; its span is at most n.
#include <algorithm>
#include <numeric>
#include <vector>

#include "exact_ring.h"
#include "pk_internal.h"

namespace pk {

namespace {

// loops of a state of the PD code: `a_state` true = A-smoothing (joins a-b and c-d)
int32_t state_loops(const Knot& k, bool a_state) {
  const int32_t two_n = 2 * (int32_t)k.pd.size();
  std::vector<int32_t> parent(two_n);
  std::iota(parent.begin(), parent.end(), 0);
  auto find = [&](int32_t u) {
    while (parent[u] != u) {
      parent[u] = parent[parent[u]];
      u = parent[u];
    }
    return u;
  };
  int32_t loops = two_n;
  for (const auto& x : k.pd) {
    const int32_t a = x[0], b = x[1], c = x[2], d = x[3];
    const int32_t pairs[2][2] = {{a, a_state ? b : d}, {c, a_state ? d : b}};
    for (const auto& pr : pairs) {
      const int32_t ra = find(pr[0]), rb = find(pr[1]);
      if (ra != rb) {
        parent[ra] = rb;
        --loops;
      }
    }
  }
  return loops;
}

long long floor_div(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

uint32_t inv_mod(uint32_t x, uint32_t p) {  // p prime, x != 0
  uint64_t r = 1, b = x % p;
  uint32_t e = p - 2;
  while (e) {
    if (e & 1) r = r * b % p;
    b = b * b % p;
    e >>= 1;
  }
  return (uint32_t)r;
}

}  // namespace

int32_t jones_half(const Knot& k) {
  const long long num = 3LL * k.writhe + k.tau + 2LL * k.n_v + 2;
  return (int32_t)(((num % 4) + 4) % 4 == 2 ? 1 : 0);
}

bool jones_window(const Knot& k, int32_t& lo, int32_t& hi) {
  if (!k.has_pd || !jones_defined(k)) return false;
  const long long n = (long long)k.pd.size();
  if (n == 0) {
    lo = hi = 0;
    return true;
  }
  const long long max_a = n + 2LL * (state_loops(k, true) - 1);
  const long long min_a = -n - 2LL * (state_loops(k, false) - 1);
  // t-exponent of A-degree a after the writhe factor: e = -(a - 3w) / 4, a multiple of 1/2
  // for a link; W = V t^(-h/2) (h = jones_half) has integer exponents e - h/2:
  // 4 (e - h/2) = 3w - a - 2h
  const long long h2 = 2LL * jones_half(k);
  lo = (int32_t)-floor_div(max_a - 3LL * k.writhe + h2, 4);
  hi = (int32_t)floor_div(3LL * k.writhe - min_a - h2, 4);
  return lo <= hi;
}

void jones_value_mod(const Knot& k, int32_t q, uint32_t p, uint32_t za, uint32_t zb, uint32_t& va,
                     uint32_t& vb) {
  using namespace exact;
  const Ring r = make_ring(p, q);
  // V t^(-h/2) = (-1)^(w+n_v+1) t^((num - 2h)/4) Z (t+1)^-(n_v+1): an integer power of t
  const long long kk = (3LL * k.writhe + k.tau + 2LL * k.n_v + 2 - 2LL * jones_half(k)) / 4;
  E v = emul(E{za, zb}, epow_t(kk, r), r);
  // (t + 1)^-(n_v+1) = ((q - 1 - t) / q)^(n_v+1)
  const uint32_t qinv = inv_mod((uint32_t)(q % p), p);
  const E f{mulm((uint32_t)((q - 1) % p), qinv, p), mulm(p - 1, qinv, p)};
  v = emul(v, epow(f, (unsigned long long)(k.n_v + 1), r), r);
  if ((k.writhe + k.n_v + 1) & 1) v = eneg(v, r);
  va = v.a;
  vb = v.b;
}

bool solve_coefficients_mod(const std::vector<int32_t>& qs, const std::vector<uint32_t>& vals, int32_t lo,
                            int32_t m, uint32_t p, std::vector<uint32_t>& c) {
  using namespace exact;
  // rows: for each q, the t^0 and t^1 parts of sum_j c_j t^(lo+j) = V(t(q))
  const size_t nq = qs.size();
  std::vector<std::vector<uint32_t>> a(2 * nq, std::vector<uint32_t>(m + 1, 0));
  for (size_t i = 0; i < nq; ++i) {
    const Ring r = make_ring(p, qs[i]);
    E tj = epow_t(lo, r);
    for (int32_t j = 0; j < m; ++j) {
      a[2 * i][j] = tj.a;
      a[2 * i + 1][j] = tj.b;
      tj = emul(tj, E{0, 1}, r);
    }
    a[2 * i][m] = vals[2 * i];
    a[2 * i + 1][m] = vals[2 * i + 1];
  }
  // Gaussian elimination to reduced row echelon form
  size_t row = 0;
  std::vector<int32_t> pivot_col;
  for (int32_t col = 0; col < m && row < a.size(); ++col) {
    size_t piv = row;
    while (piv < a.size() && a[piv][col] == 0) ++piv;
    if (piv == a.size()) return false;  // rank deficient: more q needed
    std::swap(a[piv], a[row]);
    const uint32_t inv = inv_mod(a[row][col], p);
    for (int32_t j = col; j <= m; ++j) a[row][j] = mulm(a[row][j], inv, p);
    for (size_t i = 0; i < a.size(); ++i) {
      if (i == row || a[i][col] == 0) continue;
      const uint32_t f = a[i][col];
      for (int32_t j = col; j <= m; ++j) a[i][j] = subm(a[i][j], mulm(f, a[row][j], p), p);
    }
    pivot_col.push_back(col);
    ++row;
  }
  if ((int32_t)row != m) return false;
  for (size_t i = row; i < a.size(); ++i)  // the extra equations must hold
    if (a[i][m] != 0) return false;
  c.assign(m, 0);
  for (int32_t i = 0; i < m; ++i) c[pivot_col[i]] = a[i][m];
  return true;
}

bool crt_signed(const std::vector<uint32_t>& primes, const std::vector<std::vector<uint32_t>>& res,
                std::vector<int64_t>& out) {
  // Garner on all but the last prime (128-bit), the last one checks the result
  const size_t np = primes.size();
  if (np < 2 || res.size() != np) return false;
  const size_t m = res[0].size();
  out.assign(m, 0);
  const size_t nb = np - 1;
  unsigned __int128 M = 1;
  for (size_t i = 0; i < nb; ++i) M *= primes[i];
  for (size_t j = 0; j < m; ++j) {
    std::vector<uint64_t> dig(nb);
    for (size_t i = 0; i < nb; ++i) {
      // x_i = (r_i - (d_0 + d_1 p_0 + ...)) / (p_0 ... p_{i-1}) mod p_i
      uint64_t acc = 0, prod = 1;
      for (size_t l = 0; l < i; ++l) {
        acc = (acc + dig[l] % primes[i] * prod) % primes[i];
        prod = prod * (primes[l] % primes[i]) % primes[i];
      }
      const uint64_t diff = (res[i][j] + primes[i] - acc) % primes[i];
      dig[i] = diff * inv_mod((uint32_t)prod, primes[i]) % primes[i];
    }
    unsigned __int128 x = 0, w = 1;
    for (size_t i = 0; i < nb; ++i) {
      x += (unsigned __int128)dig[i] * w;
      w *= primes[i];
    }
    __int128 s = (x > M / 2) ? (__int128)x - (__int128)M : (__int128)x;
    if (s > (__int128)INT64_MAX || s < (__int128)INT64_MIN) return false;
    // check prime
    const uint32_t pc = primes[np - 1];
    const long long sm = (long long)(s % (__int128)pc);
    const uint32_t rc = (uint32_t)((sm % (long long)pc + (long long)pc) % (long long)pc);
    if (rc != res[np - 1][j]) return false;
    out[j] = (int64_t)s;
  }
  return true;
}

}  // namespace pk
