// Contraction planning (Sec. III): the network G_T, a pairwise contraction order,
// index slicing, per-step GEMM descriptors and the device arena layout.
//
// Two equivalent forms of G_T are built from the signed Tait graph:
//  * edge network  -- one tensor per Tait vertex: its COPY tensor with the clause
//    matrices of (merged) incident edges absorbed at the lower-numbered endpoint;
//    one q-dimensional index per edge.  Contracting two tensors is contracting the
//    edge(s) between two vertices of a graph minor H; a tensor of rank d has q^d
//    entries, so the cost is O(q^Delta_H) as in Sec. III.B.
//  * spin network  -- one tensor per (merged) edge, T[s_u, s_v]; the COPY tensor of a
//    vertex is kept implicit as a spin index shared by every tensor that touches the
//    vertex (a hyperindex).  Same Z, usually far smaller intermediates.
// Parallel edges merge into one clause matrix by the entrywise product (both factors
// depend on the same two spins); a pair of opposite signs gives the all-ones matrix,
// which factorises and is dropped.  A loop is the constant factor -t^-eps.
#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <cstring>
#include <limits>
#include <map>
#include <numeric>
#include <set>

#include "pk_internal.h"

namespace pk {

using cd = std::complex<double>;

// ------------------------------------------------------------------ scaled scalars
void Scaled::norm() {
  double m = std::max(std::fabs(re), std::fabs(im));
  if (m == 0.0 || !std::isfinite(m)) {
    if (m == 0.0) e = 0;
    return;
  }
  int k;
  std::frexp(m, &k);
  re = std::ldexp(re, -k);
  im = std::ldexp(im, -k);
  e += k;
}
Scaled s_from(double re, double im) {
  Scaled s;
  s.re = re;
  s.im = im;
  s.e = 0;
  s.norm();
  return s;
}
Scaled s_mul(const Scaled& a, const Scaled& b) {
  Scaled r;
  r.re = a.re * b.re - a.im * b.im;
  r.im = a.re * b.im + a.im * b.re;
  r.e = a.e + b.e;
  r.norm();
  return r;
}
Scaled s_pow(Scaled a, int64_t n) {
  if (n < 0) {  // 1/a
    double d = a.re * a.re + a.im * a.im;
    Scaled inv;
    inv.re = a.re / d;
    inv.im = -a.im / d;
    inv.e = -a.e;
    inv.norm();
    a = inv;
    n = -n;
  }
  Scaled r = s_from(1, 0);
  while (n) {
    if (n & 1) r = s_mul(r, a);
    a = s_mul(a, a);
    n >>= 1;
  }
  return r;
}

// t(q) of Eq. potts2jones in a form that is exact at q = 2 and q = 4.
static cd t_of_q(int32_t q) {
  double qd = q;
  if (q < 4) return cd((qd - 2) / 2, std::sqrt(qd * (4 - qd)) / 2);
  return cd(((qd - 2) + std::sqrt(qd * (qd - 4))) / 2, 0);
}
void t_of_q_value(int32_t q, double& re, double& im) {
  const cd t = t_of_q(q);
  re = t.real();
  im = t.imag();
}

static cd c_pow(cd x, int64_t n) {
  if (n < 0) {
    x = 1.0 / x;
    n = -n;
  }
  cd r(1, 0);
  while (n) {
    if (n & 1) r *= x;
    x *= x;
    n >>= 1;
  }
  return r;
}

// Diagonal of the merged clause matrix of `mult` parallel edges whose Tait signs sum
// to `signsum`: prod (-t^-eps) = (-1)^mult t^-signsum (Eq. clause).
void clause_diag(int32_t q, int32_t mult, int32_t signsum, double& re, double& im) {
  cd v = c_pow(t_of_q(q), -signsum);
  if (mult & 1) v = -v;
  re = v.real();
  im = v.imag();
}

// A(q) of Eq. JonesPotts.  With s the principal fourth root of t, every fractional
// power in A is a power of s and A = (-1)^(w+n_v+1) s^num (t+1)^-(n_v+1) with
// num = 3w + tau + 2 n_v + 2: a multiple of 4 for a knot (A is then branch-free, a power
// of t), even for a link (V in Z[t^(1/2)], evaluated with the principal s).
bool jones_defined(const Knot& k) {
  const int64_t num = 3LL * k.writhe + k.tau + 2LL * k.n_v + 2;
  return k.components == 1 ? num % 4 == 0 : num % 2 == 0;
}
Scaled jones_prefactor(const Knot& k, int32_t q) {
  int64_t num = 3LL * k.writhe + k.tau + 2LL * k.n_v + 2;
  cd t = t_of_q(q);
  Scaled t1 = s_from(t.real() + 1, t.imag());
  Scaled pw;
  if (num % 4 == 0) {
    pw = s_pow(s_from(t.real(), t.imag()), num / 4);
  } else {
    const cd s4 = std::exp(std::log(t) / 4.0);   // principal fourth root of t
    pw = s_pow(s_from(s4.real(), s4.imag()), num);
  }
  Scaled r = s_mul(pw, s_pow(t1, -(int64_t)(k.n_v + 1)));
  if ((k.writhe + k.n_v + 1) & 1) {
    r.re = -r.re;
    r.im = -r.im;
  }
  return r;
}

// ------------------------------------------------------------------ network
namespace {

struct SlotSpec {
  int32_t index;     // index id
  int32_t absorbed;  // 1 = clause matrix, 0 = COPY leg
  double dre, dim;   // clause diagonal
  double ore, oim;   // clause off-diagonal
  int32_t mult = 0, signsum = 0;  // standard weights: diagonal (-1)^mult t^-signsum exactly
};
struct NetTensor {
  std::vector<int32_t> dims;  // index ids (initial layout: sorted ascending, outermost first)
  std::vector<SlotSpec> slots;
  int32_t kind = 0;           // 0 vertex sum, 1 const 1
  int32_t group = -1;         // general networks: edge group whose clause tensor this is
};
struct Merged {
  int32_t u, v, mult, signsum;
  double dre, dim, ore, oim;  // entrywise product of the members' clause matrices
  std::vector<int32_t> members;
};

struct Network {
  int32_t n_idx = 0;
  std::vector<NetTensor> t;
  Scaled factor = s_from(1, 0);
  std::array<int32_t, 2> loops{0, 0};  // folded loops: count, sum of their Tait signs
  std::vector<Merged> groups;  // spin networks: the merged edge groups, in tensor order
};

// Standard clause weights of one Tait edge: diagonal -t^-eps, off-diagonal 1 (Eq. clause).
std::array<double, 4> std_weight(int32_t q, int32_t eps) {
  double re, im;
  clause_diag(q, 1, eps, re, im);
  return {re, im, 1.0, 0.0};
}

// Parallel edges (and, in general networks, loops at one vertex) form one group whose
// clause matrix is the entrywise product of the members'.  Standard networks fold loops
// into the constant factor and drop groups whose product is the all-ones matrix; general
// networks keep every group as a tensor so that each edge weight has an adjoint.
void merge_edges(const Knot& k, int32_t q, bool general, bool std_w,
                 const std::vector<std::array<double, 4>>& w, std::vector<Merged>& out,
                 Scaled& factor, std::array<int32_t, 2>* loops = nullptr) {
  std::map<std::pair<int32_t, int32_t>, Merged> m;
  for (int32_t c = 0; c < (int32_t)k.edges.size(); ++c) {
    const auto& e = k.edges[c];
    if (e[0] == e[1] && !general) {  // loop: constant factor T[s,s] = -t^-eps
      double re, im;
      clause_diag(q, 1, e[2], re, im);
      factor = s_mul(factor, s_from(re, im));
      if (loops) {
        (*loops)[0] += 1;
        (*loops)[1] += e[2];
      }
      continue;
    }
    auto key = std::make_pair(std::min(e[0], e[1]), std::max(e[0], e[1]));
    auto it = m.find(key);
    if (it == m.end()) {
      Merged g;
      g.u = key.first;
      g.v = key.second;
      g.mult = 0;
      g.signsum = 0;
      g.dre = 1;
      g.dim = 0;
      g.ore = 1;
      g.oim = 0;
      it = m.emplace(key, g).first;
    }
    Merged& g = it->second;
    g.mult += 1;
    g.signsum += e[2];
    g.members.push_back(c);
    const double dre = g.dre * w[c][0] - g.dim * w[c][1], dim = g.dre * w[c][1] + g.dim * w[c][0];
    const double ore = g.ore * w[c][2] - g.oim * w[c][3], oim = g.ore * w[c][3] + g.oim * w[c][2];
    g.dre = dre;
    g.dim = dim;
    g.ore = ore;
    g.oim = oim;
  }
  out.clear();
  for (auto& kv : m) {
    Merged& g = kv.second;
    if (std_w) {  // exact form of the product of standard weights
      clause_diag(q, g.mult, g.signsum, g.dre, g.dim);
      g.ore = 1;
      g.oim = 0;
      if (!general && g.mult % 2 == 0 && g.signsum == 0) continue;  // all-ones: factorises
    }
    out.push_back(g);
  }
}

// Spin network.  A clause tensor T[a,b] = sum_s [s=a] M(s,b) is a COPY leg on u and an
// absorbed slot on v; a loop vector L[a] = M(a,a) is a COPY leg and an absorbed slot on
// the same spin.
void spin_network(const Knot& k, int32_t q, bool general, bool std_w,
                  const std::vector<std::array<double, 4>>& w, Network& net) {
  std::vector<Merged>& me = net.groups;
  merge_edges(k, q, general, std_w, w, me, net.factor, &net.loops);
  net.n_idx = k.n_v;
  std::vector<char> covered(k.n_v, 0);
  for (int32_t gi = 0; gi < (int32_t)me.size(); ++gi) {
    const auto& e = me[gi];
    NetTensor t;
    if (e.u == e.v)
      t.dims = {e.u};
    else
      t.dims = {e.u, e.v};
    t.slots = {{e.u, 0, 0, 0, 0, 0}, {e.v, 1, e.dre, e.dim, e.ore, e.oim, e.mult, e.signsum}};
    t.group = gi;
    covered[e.u] = covered[e.v] = 1;
    net.t.push_back(t);
  }
  for (int32_t v = 0; v < k.n_v; ++v)
    if (!covered[v]) net.t.push_back(NetTensor());  // isolated vertex: sum_s 1 = q
}

void edge_network(const Knot& k, int32_t q, Network& net) {
  std::vector<Merged> me;
  std::vector<std::array<double, 4>> w;
  for (const auto& e : k.edges) w.push_back(std_weight(q, e[2]));
  merge_edges(k, q, false, true, w, me, net.factor, &net.loops);
  net.n_idx = (int32_t)me.size();
  std::vector<NetTensor> vt(k.n_v);
  for (int32_t i = 0; i < (int32_t)me.size(); ++i) {
    const auto& e = me[i];
    vt[e.u].dims.push_back(i);
    vt[e.u].slots.push_back({i, 1, e.dre, e.dim, e.ore, e.oim, e.mult, e.signsum});
    vt[e.v].dims.push_back(i);
    vt[e.v].slots.push_back({i, 0, 0, 0, 0, 0});
  }
  net.t = std::move(vt);
}

// ------------------------------------------------------------------ orders
struct Seq {
  std::vector<std::pair<int32_t, int32_t>> pairs;  // operands of each step (tensor ids)
  std::vector<std::vector<int32_t>> sets;          // index set of every tensor (sorted)
  double cost_log = 0;                             // log2 of sum of R*K*N (unsliced)
  int32_t max_rank = 0;
};

// Result index set of contracting a and b: an index survives iff some other live
// tensor still carries it.
void result_set(const std::vector<int32_t>& a, const std::vector<int32_t>& b,
                const std::vector<int32_t>& cnt, std::vector<int32_t>& out) {
  out.clear();
  size_t i = 0, j = 0;
  while (i < a.size() || j < b.size()) {
    int32_t x;
    int c;
    if (j >= b.size() || (i < a.size() && a[i] < b[j])) {
      x = a[i++];
      c = 1;
    } else if (i >= a.size() || b[j] < a[i]) {
      x = b[j++];
      c = 1;
    } else {
      x = a[i];
      ++i;
      ++j;
      c = 2;
    }
    if (cnt[x] > c) out.push_back(x);
  }
}

size_t union_size(const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
  size_t i = 0, j = 0, n = 0;
  while (i < a.size() || j < b.size()) {
    if (j >= b.size() || (i < a.size() && a[i] < b[j]))
      ++i;
    else if (i >= a.size() || b[j] < a[i])
      ++j;
    else {
      ++i;
      ++j;
    }
    ++n;
  }
  return n;
}

// Pairwise greedy (Sec. III "greedy"): always contract the pair of tensors sharing an
// index whose result has the fewest indices; ties -> fewer indices touched, then ids.
// `restrict_var` >= 0 limits candidates to tensors holding that index (used by the
// elimination order).
struct Greedy {
  int32_t n_idx;
  std::vector<std::vector<int32_t>> sets;
  std::vector<char> live;
  std::vector<int32_t> cnt;
  std::vector<std::vector<int32_t>> occ;  // index -> tensors (may hold dead ids)
  Seq seq;

  void init(const Network& net) {
    n_idx = net.n_idx;
    cnt.assign(n_idx, 0);
    occ.assign(n_idx, {});
    for (const auto& t : net.t) {
      std::vector<int32_t> s = t.dims;
      std::sort(s.begin(), s.end());
      int32_t id = (int32_t)sets.size();
      for (int32_t x : s) {
        cnt[x]++;
        occ[x].push_back(id);
      }
      sets.push_back(s);
      live.push_back(1);
    }
    seq.sets = sets;
    for (const auto& s : sets) seq.max_rank = std::max<int32_t>(seq.max_rank, (int32_t)s.size());
  }
  // b = -1 contracts `a` with the constant 1 (sums out indices only `a` still holds)
  int32_t contract(int32_t a, int32_t b) {
    static const std::vector<int32_t> none;
    const std::vector<int32_t>& sb = b >= 0 ? sets[b] : none;
    std::vector<int32_t> r;
    result_set(sets[a], sb, cnt, r);
    for (int32_t x : sets[a]) cnt[x]--;
    for (int32_t x : sb) cnt[x]--;
    live[a] = 0;
    if (b >= 0) live[b] = 0;
    int32_t id = (int32_t)sets.size();
    for (int32_t x : r) {
      cnt[x]++;
      occ[x].push_back(id);
    }
    sets.push_back(r);
    live.push_back(1);
    seq.pairs.push_back({a, b});
    seq.sets.push_back(r);
    seq.max_rank = std::max<int32_t>(seq.max_rank, (int32_t)r.size());
    return id;
  }
  bool best_pair(int32_t restrict_var, int32_t& ba, int32_t& bb) {
    bool found = false;
    std::array<int64_t, 4> best{};
    std::vector<int32_t> r;
    auto consider = [&](int32_t a, int32_t b) {
      if (a == b || !live[a] || !live[b]) return;
      if (a > b) std::swap(a, b);
      result_set(sets[a], sets[b], cnt, r);
      std::array<int64_t, 4> key{(int64_t)r.size(),
                                 (int64_t)(sets[a].size() + sets[b].size()), a, b};
      if (!found || key < best) {
        best = key;
        found = true;
      }
    };
    if (restrict_var >= 0) {
      for (int32_t a : occ[restrict_var])
        for (int32_t b : occ[restrict_var]) consider(a, b);
    } else {
      for (int32_t a = 0; a < (int32_t)sets.size(); ++a) {
        if (!live[a]) continue;
        for (int32_t x : sets[a])
          for (int32_t b : occ[x])
            if (b > a) consider(a, b);
      }
    }
    if (found) {
      ba = (int32_t)best[2];
      bb = (int32_t)best[3];
    }
    return found;
  }
  // finish: combine disconnected pieces (outer products), smallest first; a lone
  // tensor that still has indices is summed out against the constant 1.
  void finish() {
    for (;;) {
      std::vector<int32_t> l;
      for (int32_t i = 0; i < (int32_t)sets.size(); ++i)
        if (live[i]) l.push_back(i);
      if (l.empty()) return;
      if (l.size() == 1) {
        if (!sets[l[0]].empty()) contract(l[0], -1);
        return;
      }
      std::sort(l.begin(), l.end(), [&](int32_t x, int32_t y) {
        if (sets[x].size() != sets[y].size()) return sets[x].size() < sets[y].size();
        return x < y;
      });
      contract(l[0], l[1]);
    }
  }
};

// Min-degree spin elimination order (on the spin network only).
std::vector<int32_t> min_degree_order(const Network& net) {
  std::vector<std::set<int32_t>> nb(net.n_idx);
  for (const auto& t : net.t)
    for (int32_t a : t.dims)
      for (int32_t b : t.dims)
        if (a != b) nb[a].insert(b);
  std::vector<char> done(net.n_idx, 0);
  std::vector<int32_t> order;
  for (int32_t it = 0; it < net.n_idx; ++it) {
    int32_t best = -1;
    size_t bd = 0;
    for (int32_t v = 0; v < net.n_idx; ++v)
      if (!done[v] && (best < 0 || nb[v].size() < bd)) {
        best = v;
        bd = nb[v].size();
      }
    done[best] = 1;
    order.push_back(best);
    std::vector<int32_t> N(nb[best].begin(), nb[best].end());
    for (int32_t a : N) {
      nb[a].erase(best);
      for (int32_t b : N)
        if (a != b) nb[a].insert(b);
    }
    nb[best].clear();
  }
  return order;
}

// Min-fill spin elimination order: eliminate the spin whose neighbours need the fewest
// new adjacencies to become a clique (ties: fewer neighbours, then a seeded random
// key, so different seeds give different orders).  Fill counts are cached and only
// recomputed for spins whose neighbourhood changed.
std::vector<int32_t> min_fill_order(const Network& net, uint64_t seed) {
  const int32_t n = net.n_idx;
  const int32_t W = (n + 63) / 64;
  std::vector<uint64_t> bits((size_t)n * W, 0);
  std::vector<std::vector<int32_t>> nb(n);
  auto adj = [&](int32_t a, int32_t b) { return (bits[(size_t)a * W + (b >> 6)] >> (b & 63)) & 1; };
  auto link = [&](int32_t a, int32_t b) {
    if (a == b || adj(a, b)) return;
    bits[(size_t)a * W + (b >> 6)] |= 1ull << (b & 63);
    bits[(size_t)b * W + (a >> 6)] |= 1ull << (a & 63);
    nb[a].push_back(b);
    nb[b].push_back(a);
  };
  for (const auto& t : net.t)
    for (int32_t a : t.dims)
      for (int32_t b : t.dims) link(a, b);
  uint64_t s = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  std::vector<uint64_t> key(n);
  for (int32_t v = 0; v < n; ++v) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    key[v] = seed == 0 ? (uint64_t)v : (z ^ (z >> 31));
  }
  std::vector<int64_t> fill(n, 0);
  std::vector<char> dirty(n, 1), done(n, 0);
  std::vector<int32_t> order;
  order.reserve(n);
  for (int32_t it = 0; it < n; ++it) {
    int32_t best = -1;
    for (int32_t v = 0; v < n; ++v) {
      if (done[v]) continue;
      if (dirty[v]) {
        int64_t c = 0;
        const auto& N = nb[v];
        for (size_t i = 0; i < N.size(); ++i)
          for (size_t j = i + 1; j < N.size(); ++j)
            if (!adj(N[i], N[j])) ++c;
        fill[v] = c;
        dirty[v] = 0;
      }
      if (best < 0 || fill[v] < fill[best] ||
          (fill[v] == fill[best] && (nb[v].size() < nb[best].size() ||
                                     (nb[v].size() == nb[best].size() && key[v] < key[best]))))
        best = v;
    }
    done[best] = 1;
    order.push_back(best);
    std::vector<int32_t> N = nb[best];
    for (int32_t a : N) {
      auto& L = nb[a];
      L.erase(std::remove(L.begin(), L.end(), best), L.end());
      bits[(size_t)a * W + (best >> 6)] &= ~(1ull << (best & 63));
    }
    for (size_t i = 0; i < N.size(); ++i)
      for (size_t j = i + 1; j < N.size(); ++j) link(N[i], N[j]);
    for (int32_t a : N) {
      dirty[a] = 1;
      for (int32_t b : nb[a]) dirty[b] = 1;
    }
    nb[best].clear();
  }
  return order;
}

// Separator order (Sec. III "partition" orders): recursive bisection of the network's
// tensors.  A group is split in two halves that share few indices (spins): a half grown
// breadth-first over shared indices from a seeded start, then single moves that lower the
// number of indices held on both sides while each side keeps at least 40% of the group
// (Kernighan-Lin style).  The bisections give a nested-dissection elimination order of the
// spins, contracted by the same machinery as the other elimination orders.
struct Bisection {
  const std::vector<std::vector<int32_t>>& sets;  // initial tensors' index sets
  std::vector<std::vector<int32_t>> occ;          // index -> initial tensors holding it
  uint64_t state;
  std::vector<int32_t> mark, side;
  std::vector<int32_t> c0, c1;                    // per index: holders on side 0 / 1
  Bisection(const std::vector<std::vector<int32_t>>& s, int32_t n_idx, uint64_t seed)
      : sets(s), occ(n_idx), state(seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull),
        mark(s.size(), -1), side(s.size(), 0), c0(n_idx, 0), c1(n_idx, 0) {
    for (int32_t t = 0; t < (int32_t)s.size(); ++t)
      for (int32_t x : s[t]) occ[x].push_back(t);
  }
  uint64_t next() {  // SplitMix64 step
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  void split(const std::vector<int32_t>& group, int32_t stamp, std::vector<int32_t>& g0,
             std::vector<int32_t>& g1) {
    const int32_t n = (int32_t)group.size();
    for (int32_t t : group) {
      mark[t] = stamp;
      side[t] = 0;
    }
    // breadth-first order over shared indices from a pseudo-peripheral tensor (the last
    // one reached by a search from a random start; further starts if a component runs
    // out), then the prefix of that order with the fewest shared indices among the
    // prefixes holding 40..60% of the group becomes side 1
    auto bfs = [&](int32_t start, std::vector<int32_t>& out) {
      std::vector<char> seen(sets.size(), 0);
      out.clear();
      int32_t st = start;
      while ((int32_t)out.size() < n) {
        if (seen[st]) {
          for (int32_t t : group)
            if (!seen[t]) {
              st = t;
              break;
            }
        }
        seen[st] = 1;
        size_t h = out.size();
        out.push_back(st);
        for (; h < out.size(); ++h)
          for (int32_t x : sets[out[h]])
            for (int32_t u : occ[x])
              if (mark[u] == stamp && !seen[u]) {
                seen[u] = 1;
                out.push_back(u);
              }
      }
    };
    std::vector<int32_t> order0, order1;
    bfs(group[next() % n], order0);
    bfs(order0.back(), order1);
    for (int32_t t : group)
      for (int32_t x : sets[t]) c1[x]++;  // c1: holders in the group
    int32_t cut = 0, best = -1, best_cut = 0;
    const int32_t lo = std::max<int32_t>(1, (n * 2) / 5), hi = std::max<int32_t>(lo, (n * 3) / 5);
    for (int32_t i = 0; i < n; ++i) {
      for (int32_t x : sets[order1[i]]) {
        const bool was = c0[x] > 0 && c0[x] < c1[x];
        c0[x]++;
        const bool now = c0[x] < c1[x];
        cut += (now ? 1 : 0) - (was ? 1 : 0);
      }
      if (i + 1 >= lo && i + 1 <= hi && (best < 0 || cut < best_cut)) {
        best = i + 1;
        best_cut = cut;
      }
    }
    for (int32_t t : group)
      for (int32_t x : sets[t]) c0[x] = c1[x] = 0;
    int32_t taken = best;
    for (int32_t i = 0; i < n; ++i) side[order1[i]] = i < best ? 1 : 0;
    // refinement by Fiduccia-Mattheyses passes: within a pass every tensor moves at most
    // once, always the unlocked one whose move shrinks the number of shared indices most
    // (the gain may be negative: that is how a pass leaves a local minimum) while both
    // sides keep at least 40% of the group; the pass is then undone back to the best
    // state it reached.  A pass ends after 50 moves without a new best; passes repeat
    // while they improve.
    for (int32_t t : group)
      for (int32_t x : sets[t]) (side[t] ? c1 : c0)[x]++;
    int32_t size1 = taken;
    const int32_t min_side = std::max<int32_t>(1, (n * 2) / 5);
    auto gain_of = [&](int32_t t) {
      const int32_t sd = side[t];
      int32_t gain = 0;
      for (int32_t x : sets[t]) {
        const int32_t cs = sd ? c1[x] : c0[x], co = sd ? c0[x] : c1[x];
        gain += (co > 0 ? 1 : 0) - (cs > 1 ? 1 : 0);
      }
      return gain;
    };
    auto move = [&](int32_t t) {
      const int32_t sd = side[t];
      for (int32_t x : sets[t]) {
        (sd ? c1 : c0)[x]--;
        (sd ? c0 : c1)[x]++;
      }
      side[t] = 1 - sd;
      size1 += sd ? -1 : 1;
    };
    std::vector<int32_t> locked(sets.size(), -1), moved;
    for (int32_t pass = 0; pass < 8; ++pass) {
      moved.clear();
      int32_t cur = 0, best_gain = 0, best_len = 0, since_best = 0;
      while (since_best < 50) {
        int32_t pick = -1, pick_gain = 0;
        for (int32_t t : group) {
          if (locked[t] == pass) continue;
          if ((side[t] ? size1 : n - size1) - 1 < min_side) continue;
          const int32_t g = gain_of(t);
          if (pick < 0 || g > pick_gain) {
            pick = t;
            pick_gain = g;
          }
        }
        if (pick < 0) break;
        move(pick);
        locked[pick] = pass;
        moved.push_back(pick);
        cur += pick_gain;
        if (cur > best_gain) {
          best_gain = cur;
          best_len = (int32_t)moved.size();
          since_best = 0;
        } else {
          ++since_best;
        }
      }
      for (int32_t i = (int32_t)moved.size() - 1; i >= best_len; --i) move(moved[i]);
      if (best_gain <= 0) break;
    }
    for (int32_t t : group)
      for (int32_t x : sets[t]) (side[t] ? c1 : c0)[x] = 0;
    g0.clear();
    g1.clear();
    for (int32_t t : group) (side[t] ? g1 : g0).push_back(t);
    if (g0.empty() || g1.empty()) {  // degenerate: halve by position
      g0.assign(group.begin(), group.begin() + n / 2);
      g1.assign(group.begin() + n / 2, group.end());
    }
  }
};

// Nested dissection: the spins of a group are eliminated as those held only by the first
// half (recursively), then those held only by the second half (recursively), then the
// separator (spins held by both halves) last; spins held by tensors outside the group
// belong to an enclosing separator and are ordered there.
void dissect(Bisection& bi, const std::vector<int32_t>& group, const std::vector<int32_t>& spins,
             int32_t& stamp, std::vector<char>& side_of, std::vector<int32_t>& order) {
  if (group.size() <= 2 || spins.size() <= 2) {
    order.insert(order.end(), spins.begin(), spins.end());
    return;
  }
  std::vector<int32_t> g0, g1;
  bi.split(group, stamp++, g0, g1);
  for (int32_t x : spins) side_of[x] = 0;
  for (int32_t t : g0)
    for (int32_t x : bi.sets[t]) side_of[x] |= 1;
  for (int32_t t : g1)
    for (int32_t x : bi.sets[t]) side_of[x] |= 2;
  std::vector<int32_t> s0, s1, sep;
  for (int32_t x : spins) (side_of[x] == 1 ? s0 : side_of[x] == 2 ? s1 : sep).push_back(x);
  dissect(bi, g0, s0, stamp, side_of, order);
  dissect(bi, g1, s1, stamp, side_of, order);
  order.insert(order.end(), sep.begin(), sep.end());
}

std::vector<int32_t> dissection_order(const Network& net, uint64_t seed) {
  std::vector<std::vector<int32_t>> sets;
  for (const auto& t : net.t) {
    std::vector<int32_t> d = t.dims;
    std::sort(d.begin(), d.end());
    d.erase(std::unique(d.begin(), d.end()), d.end());
    sets.push_back(d);
  }
  Bisection bi(sets, net.n_idx, seed);
  std::vector<int32_t> all(sets.size()), spins;
  std::iota(all.begin(), all.end(), 0);
  std::vector<char> held(net.n_idx, 0), side_of(net.n_idx, 0);
  for (const auto& d : sets)
    for (int32_t x : d) held[x] = 1;
  for (int32_t x = 0; x < net.n_idx; ++x)
    if (held[x]) spins.push_back(x);
  std::vector<int32_t> order;
  int32_t stamp = 0;
  dissect(bi, all, spins, stamp, side_of, order);
  return order;
}

// Contraction sequence of a spin elimination order: for each spin in turn, the tensors
// holding it are contracted pairwise (greedy among them) until at most one holds it.
void run_elimination(const Network& net, const std::vector<int32_t>& ord, Greedy& g) {
  g = Greedy();
  g.init(net);
  for (int32_t v : ord) {
    int32_t a, b;
    while (g.cnt[v] >= 2 && g.best_pair(v, a, b)) g.contract(a, b);
  }
  int32_t a, b;
  while (g.best_pair(-1, a, b)) g.contract(a, b);
  g.finish();
}

// `ord_out` (may be null) receives the spin elimination order of elimination-type orders
// (empty for the greedy orders).
bool run_order(const Network& net, int32_t order, Greedy& g, uint64_t seed = 0,
               std::vector<int32_t>* ord_out = nullptr) {
  if (ord_out) ord_out->clear();
  if (order == PK_ORDER_ELIM_SPIN || order == PK_ORDER_FILL_SPIN || order == PK_ORDER_PARTITION) {
    std::vector<int32_t> ord = order == PK_ORDER_ELIM_SPIN ? min_degree_order(net)
                               : order == PK_ORDER_FILL_SPIN ? min_fill_order(net, seed)
                                                             : dissection_order(net, seed);
    run_elimination(net, ord, g);
    if (ord_out) *ord_out = std::move(ord);
    return true;
  }
  g = Greedy();
  g.init(net);
  int32_t a, b;
  while (g.best_pair(-1, a, b)) g.contract(a, b);
  g.finish();
  return true;
}

// Index slicing: remove indices until every tensor holds at most rmax of them.  Each
// round removes the index held by the most over-size tensors (ties: the one whose
// removal shrinks them most).  `sets` loses the removed indices.
bool slice_indices(std::vector<std::vector<int32_t>>& sets, int32_t n_idx, int32_t q,
                   int32_t rmax, size_t max_count, std::vector<int32_t>& out) {
  out.clear();
  for (;;) {
    int32_t worst = 0;
    for (const auto& s : sets) worst = std::max<int32_t>(worst, (int32_t)s.size());
    if (worst <= rmax) return true;
    std::vector<int64_t> hits(n_idx, 0);
    std::vector<double> gain(n_idx, 0);
    for (const auto& s : sets)
      if ((int32_t)s.size() > rmax)
        for (int32_t x : s) {
          hits[x]++;
          gain[x] += std::pow((double)q, (double)s.size() - rmax);
        }
    int32_t bx = -1;
    for (int32_t x = 0; x < n_idx; ++x)
      if (hits[x] > 0 && (bx < 0 || hits[x] > hits[bx] || (hits[x] == hits[bx] && gain[x] > gain[bx])))
        bx = x;
    if (bx < 0 || out.size() >= max_count) return false;
    out.push_back(bx);
    for (auto& s : sets) s.erase(std::remove(s.begin(), s.end(), bx), s.end());
  }
}

// Estimated cost of a contraction sequence over index sets `sets` (one slice), in units of
// complex multiply-adds on the CUDA cores: a step of the shape the split precision runs on
// the tensor cores (M >= 64, N >= tc_min_n, K >= tc_min_k in its GEMM view) is weighted
// cost_gemm_milli / 1000 (the tensor-core GEMM does a multiply-add for a fraction of a row
// kernel's cost), and every output costs cost_out_milli / 1000 multiply-adds (its store
// and normalisation).
double sequence_cost(const Seq& seq, const std::vector<std::vector<int32_t>>& sets, int32_t q,
                     const pk_tuning& tune) {
  const double w_gemm = (double)tune.cost_gemm_milli / 1000.0, w_out = (double)tune.cost_out_milli / 1000.0;
  const double w_in = (double)tune.cost_tcin_milli / 1000.0;
  static const std::vector<int32_t> none;
  const size_t n_init = sets.size() - seq.pairs.size();
  double c = 0;
  for (size_t i = 0; i < seq.pairs.size(); ++i) {
    const auto& pr = seq.pairs[i];
    const auto& sa0 = sets[pr.first];
    const auto& sb0 = pr.second >= 0 ? sets[pr.second] : none;
    const auto& sc = sets[n_init + i];
    const bool swap = sb0.size() > sa0.size();
    const auto& sa = swap ? sb0 : sa0;
    const auto& sb = swap ? sa0 : sb0;
    auto has = [](const std::vector<int32_t>& v, int32_t x) { return std::binary_search(v.begin(), v.end(), x); };
    int m = 0, n = 0, k = 0;
    for (int32_t x : sa) {
      if (has(sc, x)) {
        if (!has(sb, x)) ++m;
      } else {
        ++k;
      }
    }
    for (int32_t x : sb)
      if (!has(sa, x)) {
        if (has(sc, x))
          ++n;
        else
          ++k;
      }
    const double macs = std::pow((double)q, (double)union_size(sa, sb));
    const double nq = std::pow((double)q, n), kq = std::pow((double)q, k);
    const bool gemm = pr.second >= 0 && std::pow((double)q, m) >= 64 && nq >= (double)tune.tc_min_n &&
                      (kq >= (double)tune.tc_min_k || (kq >= 4 && nq >= (double)tune.tc_wide_n)) &&
                      ((nq >= 32 && kq >= 16) || macs >= (double)tune.tc_min_work);
    c += macs * (gemm ? w_gemm : 1.0) + w_out * std::pow((double)q, (double)sc.size());
    if (gemm) c += w_in * (std::pow((double)q, (double)sa.size()) + std::pow((double)q, (double)sb.size()));
  }
  return c;
}

// Total estimated cost of a contraction sequence: slices x cost of one slice, or
// infinity when it needs more slices than allowed.
double sliced_cost(const Greedy& g, int32_t n_idx, int32_t q, int32_t rmax, size_t max_slices,
                   const pk_tuning& tune) {
  std::vector<std::vector<int32_t>> ss = g.seq.sets;
  std::vector<int32_t> sl;
  if (!slice_indices(ss, n_idx, q, rmax, max_slices, sl))
    return std::numeric_limits<double>::infinity();
  return std::pow((double)q, (double)sl.size()) * sequence_cost(g.seq, ss, q, tune);
}

// ---- subtree reconfiguration of a contraction tree
//
// Not in the paper (its orders are greedy and graph partitioning): a refinement of the
// chosen contraction sequence.  Every internal node r of the tree, cut a few levels down,
// is the contraction of a few subtrees F = {f_1, ..., f_k} (k <= refine); the best way to
// contract F pairwise is found exactly by dynamic programming over the subsets of F, and
// replaces the old one when it is cheaper under the planner's cost model.  An index of a
// subset S of F survives its contraction iff r's result or a member of F outside S still
// holds it (a tensor holds exactly the indices its leaves share with the rest of the
// network), so every new intermediate is what the greedy bookkeeping would produce.  Z is
// unchanged: only the bracketing of the product changes.
struct CTree {
  int32_t n_init = 0;
  std::vector<int32_t> lc, rc;  // children; leaves: -2; a one-operand step: rc = -1
  std::vector<std::vector<int32_t>> sets;
  int32_t root = -1;
};

CTree tree_of(const Seq& seq) {
  CTree t;
  t.n_init = (int32_t)(seq.sets.size() - seq.pairs.size());
  t.sets = seq.sets;
  t.lc.assign(t.n_init, -2);
  t.rc.assign(t.n_init, -2);
  for (const auto& pr : seq.pairs) {
    t.lc.push_back(pr.first);
    t.rc.push_back(pr.second);
  }
  t.root = (int32_t)t.sets.size() - 1;
  return t;
}

// The steps of the tree in post order (operands before results), renumbered.
Seq seq_of(const CTree& t) {
  Seq out;
  out.sets.assign(t.sets.begin(), t.sets.begin() + t.n_init);
  for (const auto& s : out.sets) out.max_rank = std::max<int32_t>(out.max_rank, (int32_t)s.size());
  std::vector<int32_t> id(t.sets.size(), -1);
  for (int32_t i = 0; i < t.n_init; ++i) id[i] = i;
  std::vector<std::pair<int32_t, int32_t>> st{{t.root, 0}};
  while (!st.empty()) {
    auto& top = st.back();
    const int32_t v = top.first;
    if (v < t.n_init) {
      st.pop_back();
      continue;
    }
    if (top.second == 0) {
      top.second = 1;
      st.push_back({t.lc[v], 0});
    } else if (top.second == 1) {
      top.second = 2;
      if (t.rc[v] >= 0) st.push_back({t.rc[v], 0});
    } else {
      id[v] = (int32_t)out.sets.size();
      out.pairs.push_back({id[t.lc[v]], t.rc[v] >= 0 ? id[t.rc[v]] : -1});
      out.sets.push_back(t.sets[v]);
      out.max_rank = std::max<int32_t>(out.max_rank, (int32_t)t.sets[v].size());
      st.pop_back();
    }
  }
  return out;
}

// Cost of one step in the units of sequence_cost, on bit masks of a local index numbering.
struct StepCost {
  int32_t q;
  double w_gemm, w_out, w_in, min_n, min_k, wide_n, min_work;
  double qp[65];
  StepCost(int32_t q_, const pk_tuning& tune) : q(q_) {
    w_gemm = (double)tune.cost_gemm_milli / 1000.0;
    w_out = (double)tune.cost_out_milli / 1000.0;
    w_in = (double)tune.cost_tcin_milli / 1000.0;
    min_n = (double)tune.tc_min_n;
    min_k = (double)tune.tc_min_k;
    wide_n = (double)tune.tc_wide_n;
    min_work = (double)tune.tc_min_work;
    qp[0] = 1;
    for (int i = 1; i <= 64; ++i) qp[i] = qp[i - 1] * q;
  }
  double operator()(uint64_t a, uint64_t b, uint64_t c) const {
    if (__builtin_popcountll(b) > __builtin_popcountll(a)) std::swap(a, b);
    const int m = __builtin_popcountll(a & c & ~b), n = __builtin_popcountll(b & c & ~a);
    const int k = __builtin_popcountll((a | b) & ~c);
    const bool gemm = qp[m] >= 64 && qp[n] >= min_n && (qp[k] >= min_k || (qp[k] >= 4 && qp[n] >= wide_n)) &&
                      ((qp[n] >= 32 && qp[k] >= 16) || qp[__builtin_popcountll(a | b)] >= min_work);
    return qp[__builtin_popcountll(a | b)] * (gemm ? w_gemm : 1.0) + w_out * qp[__builtin_popcountll(c)] +
           (gemm ? w_in * (qp[__builtin_popcountll(a)] + qp[__builtin_popcountll(b)]) : 0.0);
  }
};

// One pass over the tree's internal nodes (largest results first); returns whether any
// subtree changed.  `rmax` bounds the rank of new intermediates (no extra slicing).
bool reconfigure_pass(CTree& t, int32_t kmax, int32_t rmax, const StepCost& cost,
                      size_t max_nodes = SIZE_MAX) {
  std::vector<int32_t> nodes;
  for (int32_t v = t.n_init; v < (int32_t)t.sets.size(); ++v) nodes.push_back(v);
  // reachable internal binary nodes only
  std::vector<char> live(t.sets.size(), 0);
  {
    std::vector<int32_t> st{t.root};
    while (!st.empty()) {
      int32_t v = st.back();
      st.pop_back();
      live[v] = 1;
      if (v >= t.n_init) {
        st.push_back(t.lc[v]);
        if (t.rc[v] >= 0) st.push_back(t.rc[v]);
      }
    }
  }
  auto bin = [&](int32_t v) { return v >= t.n_init && t.rc[v] >= 0; };
  std::vector<int32_t> order;
  for (int32_t v : nodes)
    if (live[v] && bin(v)) order.push_back(v);
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    size_t ux = t.sets[t.lc[x]].size() + t.sets[t.rc[x]].size(), uy = t.sets[t.lc[y]].size() + t.sets[t.rc[y]].size();
    return ux > uy;
  });
  bool changed = false;
  std::vector<double> best;
  std::vector<uint64_t> keep;
  std::vector<uint32_t> split;
  if (order.size() > max_nodes) order.resize(max_nodes);
  // nodes a rebracketing of this pass has replaced (no longer in the tree)
  std::vector<char> gone(t.sets.size(), 0);
  for (int32_t r : order) {
    if (!bin(r) || gone[r]) continue;
    // frontier: expand the binary member with the most indices until kmax members
    std::vector<int32_t> F{t.lc[r], t.rc[r]};
    std::vector<int32_t> inner{r};
    while ((int32_t)F.size() < kmax) {
      int32_t bi = -1;
      for (int32_t i = 0; i < (int32_t)F.size(); ++i)
        if (bin(F[i]) && (bi < 0 || t.sets[F[i]].size() > t.sets[F[bi]].size())) bi = i;
      if (bi < 0) break;
      const int32_t v = F[bi];
      inner.push_back(v);
      F[bi] = t.lc[v];
      F.push_back(t.rc[v]);
    }
    const int32_t k = (int32_t)F.size();
    if (k < 3) continue;
    // local numbering of the indices involved
    std::vector<int32_t> U;
    for (int32_t f : F) U.insert(U.end(), t.sets[f].begin(), t.sets[f].end());
    std::sort(U.begin(), U.end());
    U.erase(std::unique(U.begin(), U.end()), U.end());
    if (U.size() > 64) continue;
    auto mask_of = [&](const std::vector<int32_t>& s) {
      uint64_t m = 0;
      for (int32_t x : s) m |= 1ull << (std::lower_bound(U.begin(), U.end(), x) - U.begin());
      return m;
    };
    std::vector<uint64_t> fm(k);
    for (int32_t i = 0; i < k; ++i) fm[i] = mask_of(t.sets[F[i]]);
    const uint64_t rm = mask_of(t.sets[r]);
    // cost of the current bracketing of F
    std::map<int32_t, uint64_t> mk;
    for (int32_t i = 0; i < k; ++i) mk[F[i]] = fm[i];
    double old_cost = 0;
    for (auto it = inner.rbegin(); it != inner.rend(); ++it) {
      const int32_t v = *it;
      const uint64_t mv = mask_of(t.sets[v]);
      old_cost += cost(mk.at(t.lc[v]), mk.at(t.rc[v]), mv);
      mk[v] = mv;
    }
    const uint32_t full = (1u << k) - 1;
    best.assign((size_t)full + 1, 0.0);
    keep.assign((size_t)full + 1, 0);
    split.assign((size_t)full + 1, 0);
    std::vector<uint64_t> uni((size_t)full + 1, 0);
    for (uint32_t S = 1; S <= full; ++S) {
      const int32_t low = __builtin_ctz(S);
      uni[S] = uni[S & (S - 1)] | fm[low];
    }
    for (uint32_t S = 1; S <= full; ++S) keep[S] = uni[S] & (rm | uni[full & ~S]);
    for (uint32_t S = 1; S <= full; ++S) {
      if ((S & (S - 1)) == 0) continue;  // a single member: no step
      double b = std::numeric_limits<double>::infinity();
      uint32_t bs = 0;
      const uint32_t lowbit = S & (~S + 1);
      if (__builtin_popcountll(keep[S]) > rmax) {
        best[S] = b;
        continue;
      }
      for (uint32_t A = (S - 1) & S; A > 0; A = (A - 1) & S) {
        if (!(A & lowbit)) continue;
        const uint32_t B = S & ~A;
        const double c = best[A] + best[B];
        if (!(c < b)) continue;
        const double cc = c + cost(keep[A], keep[B], keep[S]);
        if (cc < b) {
          b = cc;
          bs = A;
        }
      }
      best[S] = b;
      split[S] = bs;
    }
    if (!(best[full] < old_cost * (1.0 - 1e-9))) continue;
    // rebuild: r keeps its id and result; new intermediates are appended
    std::vector<int32_t> gidx;
    std::function<int32_t(uint32_t)> build = [&](uint32_t S) -> int32_t {
      if ((S & (S - 1)) == 0) return F[__builtin_ctz(S)];
      const uint32_t A = split[S], B = S & ~A;
      const int32_t a = build(A), b2 = build(B);
      if (S == full) {
        t.lc[r] = a;
        t.rc[r] = b2;
        return r;
      }
      std::vector<int32_t> set;
      for (int32_t i = 0; i < (int32_t)U.size(); ++i)
        if ((keep[S] >> i) & 1) set.push_back(U[i]);
      t.lc.push_back(a);
      t.rc.push_back(b2);
      t.sets.push_back(set);
      return (int32_t)t.sets.size() - 1;
    };
    build(full);
    for (int32_t v : inner)   // nodes appended by this pass are never visited by it
      if (v != r && v < (int32_t)gone.size()) gone[v] = 1;
    changed = true;
  }
  return changed;
}

// Reconfigures `seq` in place (at most `passes` passes); returns whether it changed.
bool reconfigure(Seq& seq, int32_t kmax, int32_t rmax, int32_t q, const pk_tuning& tune,
                 int32_t passes = 4, size_t max_nodes = SIZE_MAX) {
  if (kmax < 3 || seq.pairs.empty()) return false;
  kmax = std::min<int32_t>(kmax, 16);
  CTree t = tree_of(seq);
  const StepCost cost(q, tune);
  bool any = false;
  for (int32_t p = 0; p < passes; ++p) {
    if (!reconfigure_pass(t, kmax, rmax, cost, max_nodes)) break;
    any = true;
  }
  if (any) seq = seq_of(t);
  return any;
}

}  // namespace

// ------------------------------------------------------------------ step descriptors
bool build_step(const std::vector<int32_t>& xd, const std::vector<int32_t>* yd,
                const std::vector<int32_t>& out, int32_t q, int32_t flags, Step& st,
                bool& swapped, std::vector<int32_t>& cdims, std::string& err, int64_t tc_min_k,
                int64_t tc_min_n, int64_t tc_wide_n, int64_t tc_min_work) {
  static const std::vector<int32_t> no_dims;
  swapped = yd != nullptr && yd->size() > xd.size();
  const bool hasb = yd != nullptr;
  const auto& ad = swapped ? *yd : xd;
  const auto& bd = !hasb ? no_dims : (swapped ? xd : *yd);
  auto qpow = [&](int64_t e) {
    int64_t r = 1;
    for (int64_t i = 0; i < e; ++i) r *= q;
    return r;
  };
  auto pos_in = [](const std::vector<int32_t>& d, int32_t v) -> int32_t {
    for (size_t i = 0; i < d.size(); ++i)
      if (d[i] == v) return (int32_t)i;
    return -1;
  };
  auto in_c = [&](int32_t v) { return std::binary_search(out.begin(), out.end(), v); };
  std::memset(&st, 0, sizeof(st));
  st.b = hasb ? 0 : -1;
  const int32_t ra = (int32_t)ad.size(), rb = (int32_t)bd.size();
  auto stride_a = [&](int32_t v) -> int64_t {
    int32_t pp = pos_in(ad, v);
    return pp < 0 ? 0 : qpow(ra - 1 - pp);
  };
  auto stride_b = [&](int32_t v) -> int64_t {
    int32_t pp = pos_in(bd, v);
    return pp < 0 ? 0 : qpow(rb - 1 - pp);
  };
  // The kernel class follows from the shape alone (extents of the batch, m, n and
  // contracted indices), so it is decided before the layout: steps that run as GEMMs (the
  // tensor cores in split precision, the tiled CUDA-core GEMM otherwise) put the m indices
  // (free of B) innermost in C and the batch indices outside them, so that a tile's
  // consecutive rows are consecutive in memory and its stores coalesce; other steps keep
  // A's order.
  int32_t n_m = 0, n_n = 0, n_k = 0;
  for (int32_t v : ad) {
    if (!in_c(v))
      ++n_k;
    else if (pos_in(bd, v) < 0)
      ++n_m;
  }
  for (int32_t v : bd)
    if (pos_in(ad, v) < 0) {
      if (in_c(v))
        ++n_n;
      else
        ++n_k;
    }
  int32_t n_bat = 0;
  for (int32_t v : ad)
    if (in_c(v) && pos_in(bd, v) >= 0) ++n_bat;
  const int64_t M0 = qpow(n_m), N0 = qpow(n_n), K0 = qpow(n_k);
  const bool gemm_shape = hasb && !(flags & PK_FLAG_FORCE_ROWS) &&
                          ((flags & PK_FLAG_FORCE_GEMM) || (M0 >= 64 && N0 >= 32 && K0 >= 16) ||
                           (M0 >= 64 && N0 >= tc_min_n &&
                            (K0 >= tc_min_k || (K0 >= 4 && N0 >= tc_wide_n)) &&
                            qpow(n_m + n_n + n_k + n_bat) >= tc_min_work));
  // row indices of A in C order, inner -> outer: A's order, or its m indices then its
  // batch indices
  std::vector<int32_t> row_order;
  for (int pass = 0; pass < (gemm_shape ? 2 : 1); ++pass)
    for (int32_t i = ra - 1; i >= 0; --i) {
      const int32_t v = ad[i];
      if (!in_c(v)) continue;
      const bool batch = pos_in(bd, v) >= 0;
      if (!gemm_shape || (pass == 0) != batch) row_order.push_back(v);
    }
  std::vector<Run> rows, ks, ns;
  std::vector<int32_t> row_dims, n_dims;
  auto push = [&](std::vector<Run>& v, int64_t sa, int64_t sb) {
    if (!v.empty()) {
      Run& l = v.back();
      if (sa == l.sa * l.size && sb == l.sb * l.size) {
        l.size *= q;
        return;
      }
    }
    v.push_back({(int64_t)q, sa, sb});
  };
  for (int32_t v : row_order) {  // inner -> outer in C
    push(rows, stride_a(v), stride_b(v));
    row_dims.push_back(v);
  }
  for (int32_t i = ra - 1; i >= 0; --i) {  // inner -> outer
    const int32_t v = ad[i];
    if (!in_c(v)) push(ks, stride_a(v), stride_b(v));
  }
  for (int32_t i = rb - 1; i >= 0; --i) {
    int32_t v = bd[i];
    if (pos_in(ad, v) >= 0) continue;
    if (in_c(v)) {
      push(ns, 0, stride_b(v));
      n_dims.push_back(v);
    } else {
      push(ks, 0, stride_b(v));
    }
  }
  for (int32_t v : out)
    if (pos_in(ad, v) < 0 && pos_in(bd, v) < 0) {
      err = "internal: output index held by neither operand";
      return false;
    }
  if ((int)rows.size() > kMaxRuns || (int)ks.size() > kMaxRuns || (int)ns.size() > kMaxRuns) {
    err = "step has too many stride runs";
    return false;
  }
  st.R = st.K = st.N = 1;
  st.nrow = (int32_t)rows.size();
  st.nk = (int32_t)ks.size();
  st.nn = (int32_t)ns.size();
  for (int i = 0; i < st.nrow; ++i) {
    st.row[i] = rows[i];
    st.R *= rows[i].size;
  }
  for (int i = 0; i < st.nk; ++i) {
    st.kr[i] = ks[i];
    st.K *= ks[i].size;
  }
  for (int i = 0; i < st.nn; ++i) {
    st.nr[i] = ns[i];
    st.N *= ns[i].size;
  }
  // C layout (outermost first): N dims (B order), then the row dims (row_order reversed)
  cdims.clear();
  for (int32_t i = (int32_t)n_dims.size() - 1; i >= 0; --i) cdims.push_back(n_dims[i]);
  for (int32_t i = (int32_t)row_dims.size() - 1; i >= 0; --i) cdims.push_back(row_dims[i]);
  st.rank_c = (int32_t)cdims.size();
  // GEMM view: batch / m / n runs with their C strides (C = [n-part, row-part])
  {
    std::vector<Run4> gbv, gmv, gnv;
    auto push4 = [&](std::vector<Run4>& v, int64_t sa, int64_t sb, int64_t sc) {
      if (!v.empty()) {
        Run4& l = v.back();
        if (sa == l.sa * l.size && sb == l.sb * l.size && sc == l.sc * l.size) {
          l.size *= q;
          return;
        }
      }
      v.push_back({(int64_t)q, sa, sb, sc});
    };
    int64_t csr = 1;  // C stride of the next row dim (inner -> outer in C)
    for (int32_t v : row_order) {
      if (pos_in(bd, v) >= 0)
        push4(gbv, stride_a(v), stride_b(v), csr);
      else
        push4(gmv, stride_a(v), 0, csr);
      csr *= q;
    }
    int64_t csn = st.R;
    for (int32_t i = rb - 1; i >= 0; --i) {
      int32_t v = bd[i];
      if (pos_in(ad, v) >= 0 || !in_c(v)) continue;
      push4(gnv, 0, stride_b(v), csn);
      csn *= q;
    }
    if ((int)gbv.size() > kMaxRuns || (int)gmv.size() > kMaxRuns || (int)gnv.size() > kMaxRuns) {
      err = "step has too many stride runs";
      return false;
    }
    st.ngb = (int32_t)gbv.size();
    st.ngm = (int32_t)gmv.size();
    st.ngn = (int32_t)gnv.size();
    st.Bsz = st.M = 1;
    for (int i = 0; i < st.ngb; ++i) {
      st.gb[i] = gbv[i];
      st.Bsz *= gbv[i].size;
    }
    for (int i = 0; i < st.ngm; ++i) {
      st.gm[i] = gmv[i];
      st.M *= gmv[i].size;
    }
    for (int i = 0; i < st.ngn; ++i) st.gn[i] = gnv[i];
    st.a_kinner = (ra > 0 && !in_c(ad[ra - 1])) ? 1 : 0;
    st.b_kinner = (rb > 0 && pos_in(ad, bd[rb - 1]) >= 0 && !in_c(bd[rb - 1])) ? 1 : 0;
  }
  const int64_t outs = st.R * st.N;
  if (hasb && (flags & PK_FLAG_FORCE_GEMM))
    st.kernel = KGEMM;
  else if (flags & PK_FLAG_FORCE_ROWS)
    st.kernel = KROWS;
  else if (hasb && st.M >= 64 && st.N >= 32 && st.K >= 16)
    st.kernel = KGEMM;
  else if ((outs <= 4096 && st.K >= 4096) || (outs <= 1024 && st.K >= 256))
    st.kernel = KSPLITK;
  else
    st.kernel = KROWS;
  st.chunks = st.kernel == KSPLITK ? (int32_t)std::min<int64_t>(64, (st.K + 2047) / 2048) : 0;
  // split precision on the tensor cores: every GEMM step, and row steps of GEMM shape with
  // a short K (tc_min_k <= K < 16: one zero-padded chunk), whose outputs can cost the row
  // kernel more float-float work than the tensor cores' epilogue (complex64 and complex128
  // keep the row kernel for them)
  const bool short_k = hasb && st.kernel == KROWS && !(flags & PK_FLAG_FORCE_ROWS) && st.M >= 64 &&
                       st.N >= tc_min_n && (st.K >= tc_min_k || (st.K >= 4 && st.N >= tc_wide_n)) &&
                       st.R * st.K * st.N >= tc_min_work;
  st.tc = ((st.kernel == KGEMM || short_k) && !(flags & PK_FLAG_NO_TC))
              ? ((flags & PK_FLAG_TC_DIGITS4) ? 4 : 5)
              : 0;
  return true;
}

// ------------------------------------------------------------------ plan assembly
bool valid_tuning(const pk_tuning& t) {
  return (t.batch_threads == 128 || t.batch_threads == 256 || t.batch_threads == 512) &&
         t.batch_ktab >= 256 && t.batch_ktab <= 2048 && t.seq_outs >= 1 && t.seq_outs <= 65536 &&
         t.seq_work >= 1 && t.seq_work <= (1 << 24) && t.seq_k >= 1 && t.seq_k <= kTinyK &&
         t.tc_min_k >= 4 && t.tc_min_k <= 16 && t.tc_db_groups >= 0 && t.tc_db_groups <= 4096 &&
         t.tc_min_n >= 8 && t.tc_min_n <= 32 && t.cost_gemm_milli >= 10 &&
         t.cost_gemm_milli <= 1000 && t.cost_out_milli >= 0 && t.cost_out_milli <= 1000000 &&
         t.tc_wide_n >= 16 && t.tc_wide_n <= ((int64_t)1 << 30) && t.cost_tcin_milli >= 0 &&
         t.cost_tcin_milli <= 1000000 && t.tc_min_work >= 0 && t.tc_min_work <= ((int64_t)1 << 40);
}

void build_segments(const std::vector<Step>& steps, const pk_tuning& tune,
                    std::vector<Segment>& segments, std::vector<TinyStep>& tiny) {
  segments.clear();
  tiny.clear();
  const int64_t max_k = std::min<int64_t>(tune.seq_k, kTinyK);
  auto small = [&](const Step& st) {
    return st.kernel == KROWS && !st.tc && st.R * st.N <= tune.seq_outs && st.K <= max_k &&
           st.R * st.N * st.K <= tune.seq_work;
  };
  const int32_t n_steps = (int32_t)steps.size();
  int32_t s0 = 0;
  while (s0 < n_steps) {
    if (!small(steps[s0])) {
      ++s0;
      continue;
    }
    int32_t s1 = s0;
    while (s1 < n_steps && small(steps[s1])) ++s1;
    if (s1 - s0 >= 2) {
      Segment sg;
      sg.first = s0;
      sg.count = s1 - s0;
      sg.tiny0 = (int32_t)tiny.size();
      for (int32_t i = s0; i < s1; ++i) {
        const Step& st = steps[i];
        TinyStep ts;
        std::memset(&ts, 0, sizeof(ts));
        ts.a = st.a;
        ts.b = st.b;
        ts.c = st.c;
        ts.nrow = st.nrow;
        ts.nk = st.nk;
        ts.nn = st.nn;
        ts.off_a = st.off_a;
        ts.off_b = st.off_b;
        ts.off_c = st.off_c;
        ts.R = st.R;
        ts.K = st.K;
        ts.N = st.N;
        std::memcpy(ts.row, st.row, sizeof(ts.row));
        std::memcpy(ts.kr, st.kr, sizeof(ts.kr));
        std::memcpy(ts.nr, st.nr, sizeof(ts.nr));
        tiny.push_back(ts);
      }
      segments.push_back(sg);
    }
    s0 = s1;
  }
}

uint64_t Plan::ws_bytes(int32_t precision) const {
  if (precision == PK_C64) {
    if (tail.empty()) return off_arena + (uint64_t)arena_elems * 8ull;
    return off_tail + (uint64_t)tail_elems * 16ull;  // complex128 tail region after the arena
  }
  if (precision == PK_SPLIT && tc_bytes > 0)   // float-float pairs, then the digit scratch
    return off_arena + tc_offset() + (uint64_t)tc_bytes;
  return off_arena + (uint64_t)arena_elems * 16ull;  // complex128 and float-float pairs
}

static uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

bool order_stats(const Knot& k, int32_t q, int32_t order, int32_t restarts, double* out) {
  if (q < 1 || q > 64) return false;
  std::vector<std::pair<int32_t, uint64_t>> cands;
  const int32_t r = restarts > 0 ? restarts : 8;
  if (order == PK_ORDER_GREEDY_EDGE || order == PK_ORDER_GREEDY_SPIN || order == PK_ORDER_ELIM_SPIN)
    cands = {{order, 0}};
  else if (order == PK_ORDER_FILL_SPIN || order == PK_ORDER_PARTITION)
    for (int32_t i = 0; i < r; ++i) cands.push_back({order, (uint64_t)i});
  else
    return false;
  std::vector<std::array<double, 4>> w;
  for (const auto& e : k.edges) w.push_back(std_weight(q, e[2]));
  bool have = false;
  for (const auto& cand : cands) {
    Network net;
    if (cand.first == PK_ORDER_GREEDY_EDGE)
      edge_network(k, q, net);
    else
      spin_network(k, q, false, true, w, net);
    Greedy g;
    run_order(net, cand.first, g, cand.second);
    const double rank = g.seq.max_rank;
    double macs = 0;   // complex multiply-adds: q^(indices of A and B together) per step
    static const std::vector<int32_t> none;
    for (size_t i = 0; i < g.seq.pairs.size(); ++i) {
      const auto& pr = g.seq.pairs[i];
      macs += std::pow((double)q, (double)union_size(g.seq.sets[pr.first],
                                                     pr.second >= 0 ? g.seq.sets[pr.second] : none));
    }
    const double cost = std::log2(std::max(1.0, macs));
    if (!have || rank < out[0] || (rank == out[0] && cost < out[1])) {
      out[0] = rank;
      out[1] = cost;
      out[2] = (double)net.t.size();
      out[3] = (double)net.n_idx;
      have = true;
    }
  }
  return have;
}

bool make_plan(const Knot& k, int32_t q, const pk_plan_opts& opts, const pk_tuning& tune, Plan& p,
               std::string& err) {
  p = Plan();
  p.tuning = tune;
  if (q < 1 || q > 64) {
    err = "q out of range";
    return false;
  }
  p.q = q;
  p.knot = k;
  const double lq = std::log2((double)q);
  double max_log2 = opts.max_log2_elems > 0 ? opts.max_log2_elems : 31.0;
  if (max_log2 > 31.0) max_log2 = 31.0;  // 32-bit row indexing in the kernels
  double max_log2_slices = opts.max_log2_slices > 0 ? opts.max_log2_slices : 40.0;
  int32_t rmax = q == 1 ? 1 << 20 : (int32_t)std::floor(max_log2 / lq + 1e-9);
  const size_t max_slice_idx = q == 1 ? 0 : (size_t)std::floor(max_log2_slices / lq + 1e-9);

  // clause weights: standard (-t^-eps, 1) or given per Tait edge
  const bool grad = (opts.flags & PK_FLAG_GRAD) != 0;
  p.general = grad || opts.edge_weights != nullptr;
  p.std_weights = opts.edge_weights == nullptr;
  p.weights.clear();
  for (int32_t c = 0; c < (int32_t)k.edges.size(); ++c) {
    if (opts.edge_weights) {
      const double* w = opts.edge_weights + 4 * c;
      for (int j = 0; j < 4; ++j)
        if (!std::isfinite(w[j])) {
          err = "edge weights must be finite";
          return false;
        }
      p.weights.push_back({w[0], w[1], w[2], w[3]});
    } else {
      p.weights.push_back(std_weight(q, k.edges[c][2]));
    }
  }

  // candidate orders: (order, seed); min-fill restarts differ by their tie-break seed
  const int32_t restarts = opts.restarts > 0 ? opts.restarts : 8;
  std::vector<std::pair<int32_t, uint64_t>> cands;
  if (p.general && opts.order == PK_ORDER_GREEDY_EDGE) {
    err = "the edge network is not available for gradient or weighted plans";
    return false;
  }
  if (opts.order == PK_ORDER_AUTO) {
    cands = {{PK_ORDER_GREEDY_SPIN, 0}, {PK_ORDER_ELIM_SPIN, 0}};
    if (!p.general) cands.push_back({PK_ORDER_GREEDY_EDGE, 0});
    for (int32_t r = 0; r < restarts; ++r) cands.push_back({PK_ORDER_FILL_SPIN, (uint64_t)r});
  } else if (opts.order >= 1 && opts.order <= 3) {
    cands = {{opts.order, 0}};
  } else if (opts.order == PK_ORDER_FILL_SPIN) {
    for (int32_t r = 0; r < restarts; ++r) cands.push_back({PK_ORDER_FILL_SPIN, (uint64_t)r});
  } else if (opts.order == PK_ORDER_PARTITION) {
    for (int32_t r = 0; r < restarts; ++r) cands.push_back({PK_ORDER_PARTITION, (uint64_t)r});
  } else {
    err = "unknown order";
    return false;
  }
  // the cheapest candidates (by estimated cost after slicing), best first; with
  // opts.refine the kRefineTop cheapest are kept for the reconfiguration below
  constexpr size_t kRefineTop = 16;
  const size_t keep_top = opts.refine > 0 ? kRefineTop : 1;
  struct Cand {
    double cost;
    int32_t order;
    Network net;
    Greedy g;
  };
  std::vector<Cand> top_c;
  for (const auto& cand : cands) {
    const int32_t o = cand.first;
    Network net;
    if (o == PK_ORDER_GREEDY_EDGE)
      edge_network(k, q, net);
    else
      spin_network(k, q, p.general, p.std_weights, p.weights, net);
    Greedy g;
    run_order(net, o, g, cand.second);
    // cost in complex MACs at this q after slicing: slices x work per slice
    const double c = sliced_cost(g, net.n_idx, q, rmax, max_slice_idx, tune);
    if (!std::isfinite(c)) continue;
    if (top_c.size() == keep_top && !(c < top_c.back().cost)) continue;
    auto at = std::upper_bound(top_c.begin(), top_c.end(), c,
                               [](double x, const Cand& y) { return x < y.cost; });
    top_c.insert(at, Cand{c, o, std::move(net), std::move(g)});
    if (top_c.size() > keep_top) top_c.pop_back();
  }
  if (top_c.empty()) {
    err = "plan needs more slices than allowed";
    return false;
  }
  size_t best_i = 0;
  if (opts.refine > 0) {
    // subtree reconfiguration of each kept candidate with frontiers of 4, 6, ... up to
    // opts.refine subtrees in turn, then frontiers of opts.refine + 2 at the kWideNodes
    // nodes with the widest operands; the cheapest result wins
    constexpr size_t kWideNodes = 12;
    const int32_t kmax = std::max<int32_t>(4, std::min<int32_t>(opts.refine, 10));
    for (size_t i = 0; i < top_c.size(); ++i) {
      Cand& cd = top_c[i];
      Greedy rg = cd.g;
      bool changed = false;
      for (int32_t kk = 4; kk <= kmax; kk += 2) changed |= reconfigure(rg.seq, kk, rmax, q, tune);
      changed |= reconfigure(rg.seq, kmax + 2, rmax, q, tune, 2, kWideNodes);
      if (changed) {
        const double c = sliced_cost(rg, cd.net.n_idx, q, rmax, max_slice_idx, tune);
        if (c < cd.cost) {
          cd.cost = c;
          cd.g = std::move(rg);
        }
      }
      if (cd.cost < top_c[best_i].cost) best_i = i;
    }
  }
  Network best_net = std::move(top_c[best_i].net);
  Greedy best_g = std::move(top_c[best_i].g);
  const int32_t best_order = top_c[best_i].order;
  p.order_used = best_order;
  p.est_cost = top_c[best_i].cost;
  Network& net = best_net;
  Greedy& g = best_g;
  p.factor = net.factor;
  p.loop_count = net.loops[0];
  p.loop_signsum = net.loops[1];
  p.n_idx = net.n_idx;
  p.n_init = (int32_t)net.t.size();
  const int32_t n_tens = (int32_t)g.seq.sets.size();
  const int32_t n_steps = (int32_t)g.seq.pairs.size();
  if (n_tens != p.n_init + n_steps) {
    err = "internal: tensor count mismatch";
    return false;
  }

  // ---- slicing: remove indices until every tensor has rank <= rmax
  std::vector<std::vector<int32_t>> sets = g.seq.sets;
  std::vector<char> sliced(net.n_idx, 0);
  if (!slice_indices(sets, net.n_idx, q, rmax, max_slice_idx, p.sliced)) {
    err = "plan needs more slices than allowed";
    return false;
  }
  for (int32_t x : p.sliced) sliced[x] = 1;
  p.n_slices = 1;
  for (size_t i = 0; i < p.sliced.size(); ++i) p.n_slices *= q;
  std::vector<int32_t> slice_ord(net.n_idx, -1);
  for (size_t i = 0; i < p.sliced.size(); ++i) slice_ord[p.sliced[i]] = (int32_t)i;

  // ---- tensors and layouts
  p.tensors.resize(n_tens);
  for (int32_t i = 0; i < p.n_init; ++i) {
    TensorInfo& ti = p.tensors[i];
    for (int32_t x : net.t[i].dims)
      if (!sliced[x]) ti.dims.push_back(x);  // initial layout: network order
  }
  auto qpow = [&](int64_t e) {
    int64_t r = 1;
    for (int64_t i = 0; i < e; ++i) r *= q;
    return r;
  };
  p.steps.resize(n_steps);
  for (int32_t s = 0; s < n_steps; ++s) {
    int32_t x = g.seq.pairs[s].first, y = g.seq.pairs[s].second;
    int32_t cid = p.n_init + s;
    Step st;
    bool sw = false;
    if (!build_step(p.tensors[x].dims, y >= 0 ? &p.tensors[y].dims : nullptr, sets[cid], q,
                    opts.flags, st, sw, p.tensors[cid].dims, err, tune.tc_min_k, tune.tc_min_n,
                    tune.tc_wide_n, tune.tc_min_work))
      return false;
    st.a = sw ? y : x;
    st.b = sw ? x : y;
    st.c = cid;
    p.steps[s] = st;
  }
  p.final_tensor = n_tens - 1;
  p.tc_bytes = 0;
  p.n_tc = 0;
  for (const Step& st : p.steps)
    if (st.tc) {
      p.n_tc++;
      p.tc_bytes = std::max<int64_t>(p.tc_bytes, tc_scratch(st.Bsz, st.M, st.N, st.K, st.tc).bytes);
    }

  // ---- sizes, lifetimes, stats
  p.max_rank = 0;
  for (int32_t i = 0; i < n_tens; ++i) {
    TensorInfo& ti = p.tensors[i];
    ti.elems = qpow((int64_t)ti.dims.size());
    p.max_rank = std::max<int32_t>(p.max_rank, (int32_t)ti.dims.size());
    ti.born = i < p.n_init ? -1 : i - p.n_init;
    ti.dies = ti.born;
  }
  p.tensors[p.final_tensor].dies = n_steps;
  double cm = 0, by = 0;
  int64_t partials = 0;
  for (int32_t s = 0; s < n_steps; ++s) {
    const Step& st = p.steps[s];
    p.tensors[st.a].dies = std::max(p.tensors[st.a].dies, s);
    if (st.b >= 0) p.tensors[st.b].dies = std::max(p.tensors[st.b].dies, s);
    cm += (double)st.R * (double)st.K * (double)st.N;
    by += 8.0 * (double)(p.tensors[st.a].elems + (st.b >= 0 ? p.tensors[st.b].elems : 0) +
                         p.tensors[st.c].elems);
    if (st.kernel == KSPLITK) partials = std::max<int64_t>(partials, st.R * st.N * st.chunks);
  }
  p.cmacs = cm * (double)p.n_slices;
  p.bytes_c64 = by * (double)p.n_slices;
  p.log2_max_elems = p.max_rank * lq;
  p.splitk_partials = partials;

  // ---- arena: first fit by decreasing size over lifetime intervals
  std::vector<int32_t> ord(n_tens);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) {
    if (p.tensors[x].elems != p.tensors[y].elems) return p.tensors[x].elems > p.tensors[y].elems;
    return x < y;
  });
  struct Placed {
    int64_t off, len;
    int32_t born, dies;
  };
  std::vector<Placed> placed;
  int64_t top = 0;
  for (int32_t id : ord) {
    TensorInfo& ti = p.tensors[id];
    int64_t len = (ti.elems + 63) / 64 * 64;
    std::vector<std::pair<int64_t, int64_t>> busy;
    for (const auto& pl : placed)
      if (!(pl.dies < ti.born || ti.dies < pl.born)) busy.push_back({pl.off, pl.off + pl.len});
    std::sort(busy.begin(), busy.end());
    int64_t off = 0;
    for (const auto& iv : busy) {
      if (off + len <= iv.first) break;
      off = std::max(off, iv.second);
    }
    ti.offset = off;
    placed.push_back({off, len, ti.born, ti.dies});
    top = std::max(top, off + len);
  }
  p.arena_elems = top;
  for (auto& st : p.steps) {
    st.off_a = p.tensors[st.a].offset;
    st.off_b = st.b >= 0 ? p.tensors[st.b].offset : 0;
    st.off_c = p.tensors[st.c].offset;
  }

  // ---- recipes
  p.recipes.clear();
  p.slots.clear();
  for (int32_t i = 0; i < p.n_init; ++i) {
    const NetTensor& nt = net.t[i];
    const TensorInfo& ti = p.tensors[i];
    Recipe r;
    std::memset(&r, 0, sizeof(r));
    r.kind = nt.kind;
    r.rank = (int32_t)ti.dims.size();
    r.slot0 = (int32_t)p.slots.size();
    r.nslot = (int32_t)nt.slots.size();
    r.elems = ti.elems;
    r.offset = ti.offset;
    r.meta = i;
    for (const auto& ss : nt.slots) {
      Slot sl;
      std::memset(&sl, 0, sizeof(sl));
      int32_t pp = -1;
      for (size_t j = 0; j < ti.dims.size(); ++j)
        if (ti.dims[j] == ss.index) pp = (int32_t)(ti.dims.size() - 1 - j);
      sl.dimpos = pp;
      sl.slice_ord = pp < 0 ? slice_ord[ss.index] : -1;
      sl.absorbed = ss.absorbed;
      sl.dre = ss.dre;
      sl.dim = ss.dim;
      sl.ore = ss.ore;
      sl.oim = ss.oim;
      if (ss.absorbed) sl.pad = slot_exact_pack(ss.mult, ss.signsum);
      p.slots.push_back(sl);
    }
    p.recipes.push_back(r);
  }

  // ---- edge groups of general networks (for weights and the reverse pass)
  p.groups.clear();
  p.leaf_dims.clear();
  for (int32_t i = 0; i < p.n_init; ++i) p.leaf_dims.push_back(net.t[i].dims);
  if (p.general) {
    for (int32_t i = 0; i < p.n_init; ++i) {
      const NetTensor& nt = net.t[i];
      if (nt.group < 0) continue;
      const Merged& mg = net.groups[nt.group];
      EdgeGroup eg;
      eg.u = mg.u;
      eg.v = mg.v;
      eg.leaf = i;
      eg.slot = p.recipes[i].slot0 + 1;  // the absorbed slot
      eg.members = mg.members;
      p.groups.push_back(eg);
    }
  }

  // ---- split precision: the last `tail` steps in complex128
  {
    int32_t T = opts.tail_steps > 0 ? opts.tail_steps : 0;
    T = std::min<int32_t>(T, n_steps);
    p.tail_first = n_steps - T;
    std::vector<int64_t> tail_off(n_tens, -1);
    std::vector<int32_t> tail_meta(n_tens, -1);
    int64_t top2 = 0;
    auto place = [&](int64_t elems) {
      int64_t o = top2;
      top2 += (elems + 63) / 64 * 64;
      return o;
    };
    p.conv.clear();
    p.tail.clear();
    auto operand = [&](int32_t x) {  // tail offset and meta slot of an operand
      if (tail_off[x] < 0) {
        ConvRec cr;
        cr.src_off = p.tensors[x].offset;
        cr.dst_off = place(p.tensors[x].elems);
        cr.elems = p.tensors[x].elems;
        cr.src_meta = x;
        cr.dst_meta = n_tens + (int32_t)p.conv.size();
        p.conv.push_back(cr);
        tail_off[x] = cr.dst_off;
        tail_meta[x] = cr.dst_meta;
      }
    };
    for (int32_t s2 = p.tail_first; s2 < n_steps; ++s2) {
      const Step& st = p.steps[s2];
      operand(st.a);
      if (st.b >= 0) operand(st.b);
      TailStep ts;
      std::memset(&ts, 0, sizeof(ts));
      ts.step = s2;
      ts.meta_a = tail_meta[st.a];
      ts.meta_b = st.b >= 0 ? tail_meta[st.b] : -1;
      ts.off_a = tail_off[st.a];
      ts.off_b = st.b >= 0 ? tail_off[st.b] : 0;
      ts.off_c = place(p.tensors[st.c].elems);
      tail_off[st.c] = ts.off_c;
      tail_meta[st.c] = st.c;
      p.tail.push_back(ts);
    }
    p.tail_elems = top2;
    p.final_tail_off = tail_off[p.final_tensor];
    p.n_meta = n_tens + (int32_t)p.conv.size();
  }

  // ---- segments: maximal runs (>= 2) of consecutive small row-kernel steps
  build_segments(p.steps, tune, p.segments, p.tiny);

  // ---- workspace layout
  uint64_t off = 0;
  p.off_recipe = off;
  off = align256(off + sizeof(Recipe) * p.recipes.size());
  p.off_slots = off;
  off = align256(off + sizeof(Slot) * std::max<size_t>(1, p.slots.size()));
  p.off_conv = off;
  off = align256(off + sizeof(ConvRec) * std::max<size_t>(1, p.conv.size()));
  p.off_tiny = off;
  off = align256(off + sizeof(TinyStep) * p.tiny.size());
  p.off_meta = off;
  off = align256(off + 16ull * p.n_meta);
  p.off_counter = off;
  off = align256(off + 4ull * std::max<int32_t>(1, n_steps));
  p.off_result = off;
  off = align256(off + 32ull * (uint64_t)p.n_slices + 32);
  p.off_scratch = off;
  off = align256(off + 16ull * (uint64_t)std::max<int64_t>(1, partials));
  p.off_arena = off;
  p.off_tail = align256(p.off_arena + 8ull * (uint64_t)p.arena_elems);
  p.program.assign(p.off_meta, 0);
  if (!p.recipes.empty())
    std::memcpy(p.program.data() + p.off_recipe, p.recipes.data(), sizeof(Recipe) * p.recipes.size());
  if (!p.slots.empty())
    std::memcpy(p.program.data() + p.off_slots, p.slots.data(), sizeof(Slot) * p.slots.size());
  if (!p.conv.empty())
    std::memcpy(p.program.data() + p.off_conv, p.conv.data(), sizeof(ConvRec) * p.conv.size());
  if (!p.tiny.empty())
    std::memcpy(p.program.data() + p.off_tiny, p.tiny.data(), sizeof(TinyStep) * p.tiny.size());
  if (grad && !make_grad_program(p, opts.checkpoint_stride, opts.flags, tune, err)) return false;
  // clause values of general networks, stored scaled by powers of two (Recipe::exp2)
  if (p.general) apply_weights(p);
  return true;
}

bool set_weights(Plan& p, const double* w) {
  std::vector<std::array<double, 4>> nw;
  for (int32_t c = 0; c < (int32_t)p.knot.edges.size(); ++c) {
    if (!w) {
      nw.push_back(std_weight(p.q, p.knot.edges[c][2]));
      continue;
    }
    for (int j = 0; j < 4; ++j)
      if (!std::isfinite(w[4 * c + j])) return false;
    nw.push_back({w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]});
  }
  p.weights = nw;
  p.std_weights = w == nullptr;
  apply_weights(p);
  return true;
}

// Binary exponent of max(|x|) over the four values (frexp convention), 0 when all are 0.
static int32_t max_exp4(double a, double b, double c, double d) {
  const double m = std::max(std::max(std::fabs(a), std::fabs(b)), std::max(std::fabs(c), std::fabs(d)));
  if (!(m > 0)) return 0;
  int e;
  std::frexp(m, &e);
  return e;
}

void apply_weights(Plan& p) {
  p.slot_exp.assign(p.slots.size(), 0);
  for (const EdgeGroup& g : p.groups) {
    double dre = 1, dim = 0, ore = 1, oim = 0;
    int64_t x = 0;   // the clause entries are (dre, dim, ore, oim) * 2^x
    if (p.std_weights) {
      int32_t ss = 0;
      for (int32_t c : g.members) ss += p.knot.edges[c][2];
      clause_diag(p.q, (int32_t)g.members.size(), ss, dre, dim);
    } else {
      // entrywise product of the members' matrices, renormalised by exact powers of two
      // after every factor so that no partial product overflows or underflows
      for (int32_t c : g.members) {
        const auto& w = p.weights[c];
        const double a = dre * w[0] - dim * w[1], b = dre * w[1] + dim * w[0];
        const double c2 = ore * w[2] - oim * w[3], d = ore * w[3] + oim * w[2];
        const int32_t e = max_exp4(a, b, c2, d);
        dre = std::ldexp(a, -e);
        dim = std::ldexp(b, -e);
        ore = std::ldexp(c2, -e);
        oim = std::ldexp(d, -e);
        x += e;
      }
    }
    Slot& sl = p.slots[g.slot];
    sl.dre = dre;
    sl.dim = dim;
    sl.ore = ore;
    sl.oim = oim;
    p.slot_exp[g.slot] = (int32_t)std::max<int64_t>(INT32_MIN / 2, std::min<int64_t>(INT32_MAX / 2, x));
  }
  // each initial tensor's entries carry the powers of two of its absorbed slots
  auto set_exp = [&](std::vector<Recipe>& recs) {
    for (Recipe& r : recs) {
      int64_t x = 0;
      for (int32_t j = r.slot0; j < r.slot0 + r.nslot; ++j)
        if (p.slots[j].absorbed) x += p.slot_exp[j];
      r.exp2 = (int32_t)std::max<int64_t>(INT32_MIN / 2, std::min<int64_t>(INT32_MAX / 2, x));
    }
  };
  set_exp(p.recipes);
  if (!p.recipes.empty())
    std::memcpy(p.program.data() + p.off_recipe, p.recipes.data(), sizeof(Recipe) * p.recipes.size());
  if (p.grad.built) {
    set_exp(p.grad.recipes);
    if (!p.grad.recipes.empty())
      std::memcpy(p.grad.program.data() + p.grad.off_recipe, p.grad.recipes.data(),
                  sizeof(Recipe) * p.grad.recipes.size());
  }
  if (!p.slots.empty()) {
    std::memcpy(p.program.data() + p.off_slots, p.slots.data(), sizeof(Slot) * p.slots.size());
    if (p.grad.built)
      std::memcpy(p.grad.program.data() + p.grad.off_slots, p.slots.data(),
                  sizeof(Slot) * p.slots.size());
  }
}

}  // namespace pk
