// Knot input: PD codes, signed graphs and random grid walks -> signed Tait graph (Sec. II).
//
// Faces are traced with the corner permutation of the 4-valent planar map: corner
// (X, i) lies between arm i and arm i+1 (counter-clockwise) of crossing X; walking
// away from X along arm i+1 with that region on the right leads to the arc's other
// end (Y, j), where the same region is the corner (Y, j).  Cycles of this map are the
// regions of the diagram.
#include <algorithm>
#include <cstring>
#include <map>

#include "pk_internal.h"

namespace pk {
namespace {

// For each crossing: true if the over-strand leaves through arm b (index 1).
bool over_leaves_b(const std::array<int32_t, 4>& x, int32_t two_n) {
  if (two_n == 2) return x[1] == x[0];  // one crossing: over enters on c, leaves on a
  return x[1] == (x[3] + 1) % two_n;
}

}  // namespace

// `signs` (NULL for a knot labelled along its orientation): the twist sign of every
// crossing, +1 when the over-strand leaves through arm b; it fixes the orientation of a
// link, whose labels cannot run 0..2n-1 along one strand.
bool knot_from_pd(const int32_t* pd, int32_t n, int32_t outer_arc, int32_t outer_side, Knot& k,
                  std::string& err, const int32_t* signs) {
  k = Knot();
  k.has_pd = true;
  if (n < 0 || (n > 0 && pd == nullptr)) {
    err = "bad PD size";
    return false;
  }
  if (n == 0) {  // crossingless circle: one black region inside, white outside
    k.n_v = 1;
    return true;
  }
  const int32_t two_n = 2 * n;
  k.pd.resize(n);
  std::vector<int32_t> seen(two_n, 0);
  for (int32_t i = 0; i < n; ++i) {
    for (int j = 0; j < 4; ++j) {
      int32_t a = pd[4 * i + j];
      if (a < 0 || a >= two_n) {
        err = "arc label out of range";
        return false;
      }
      k.pd[i][j] = a;
      seen[a]++;
    }
    if (!signs && k.pd[i][2] != (k.pd[i][0] + 1) % two_n) {
      err = "under-strand must run a -> a+1";
      return false;
    }
    if (signs && signs[i] != 1 && signs[i] != -1) {
      err = "twist signs must be +-1";
      return false;
    }
  }
  for (int32_t a = 0; a < two_n; ++a)
    if (seen[a] != 2) {
      err = "each arc label must occur exactly twice";
      return false;
    }
  // arc ends: (crossing, arm) pairs; outgoing flag per arm
  std::vector<int32_t> ob(n);
  std::vector<std::array<int32_t, 2>> ends(two_n, {-1, -1});  // encoded 4*X+arm
  std::vector<int32_t> tail_end(two_n, -1), head_end(two_n, -1);
  for (int32_t x = 0; x < n; ++x) {
    ob[x] = signs ? (signs[x] > 0 ? 1 : 0) : (over_leaves_b(k.pd[x], two_n) ? 1 : 0);
    for (int arm = 0; arm < 4; ++arm) {
      int32_t a = k.pd[x][arm];
      bool out = (arm == 2) || (arm == 1 && ob[x]) || (arm == 3 && !ob[x]);
      int32_t code = 4 * x + arm;
      if (ends[a][0] < 0)
        ends[a][0] = code;
      else
        ends[a][1] = code;
      if (out) {
        if (tail_end[a] >= 0) {
          err = "arc leaves two crossings";
          return false;
        }
        tail_end[a] = code;
      } else {
        if (head_end[a] >= 0) {
          err = "arc enters two crossings";
          return false;
        }
        head_end[a] = code;
      }
    }
  }
  // components: arc -> next arc through its head crossing
  {
    std::vector<int32_t> nxt(two_n);
    for (int32_t x = 0; x < n; ++x) {
      const auto& c = k.pd[x];
      nxt[c[0]] = c[2];
      if (ob[x])
        nxt[c[3]] = c[1];
      else
        nxt[c[1]] = c[3];
    }
    std::vector<char> vis(two_n, 0);
    int comps = 0;
    for (int32_t s = 0; s < two_n; ++s) {
      if (vis[s]) continue;
      ++comps;
      for (int32_t u = s; !vis[u]; u = nxt[u]) vis[u] = 1;
    }
    k.components = comps;
  }
  // faces by the corner permutation
  const int32_t nc = 4 * n;
  std::vector<int32_t> next_corner(nc), face(nc, -1);
  for (int32_t x = 0; x < n; ++x)
    for (int i = 0; i < 4; ++i) {
      int32_t code = 4 * x + ((i + 1) & 3);
      int32_t a = k.pd[x][(i + 1) & 3];
      int32_t other = (ends[a][0] == code) ? ends[a][1] : ends[a][0];
      if (ends[a][0] == code && ends[a][1] == code) other = code;
      next_corner[4 * x + i] = other;  // corner (Y, j) with j the arrival arm
    }
  int32_t nf = 0;
  for (int32_t c = 0; c < nc; ++c) {
    if (face[c] >= 0) continue;
    for (int32_t u = c; face[u] < 0; u = next_corner[u]) face[u] = nf;
    ++nf;
  }
  if (nf != n + 2) {
    err = "diagram is not planar (face count != crossings + 2)";
    return false;
  }
  // 2-colouring: corners i and i+1 of a crossing are different regions
  std::vector<std::vector<int32_t>> adj(nf);
  for (int32_t x = 0; x < n; ++x)
    for (int i = 0; i < 4; ++i) {
      int32_t f = face[4 * x + i], g = face[4 * x + ((i + 1) & 3)];
      adj[f].push_back(g);
    }
  std::vector<int32_t> col(nf, -1);
  col[0] = 0;
  std::vector<int32_t> st{0};
  while (!st.empty()) {
    int32_t f = st.back();
    st.pop_back();
    for (int32_t g : adj[f]) {
      if (col[g] < 0) {
        col[g] = 1 - col[f];
        st.push_back(g);
      } else if (col[g] == col[f]) {
        err = "regions cannot be 2-coloured";
        return false;
      }
    }
  }
  // region left of an arc = corner (tail crossing, tail arm); right = corner before it
  auto side_face = [&](int32_t arc, int32_t side) {
    int32_t code = tail_end[arc];
    int32_t x = code >> 2, arm = code & 3;
    return side == 0 ? face[4 * x + arm] : face[4 * x + ((arm + 3) & 3)];
  };
  int32_t black;
  if (outer_arc >= 0) {
    if (outer_arc >= two_n || (outer_side != 0 && outer_side != 1)) {
      err = "bad outer region";
      return false;
    }
    black = 1 - col[side_face(outer_arc, outer_side)];
  } else {
    black = col[side_face(0, 1)];
  }
  std::vector<int32_t> vid(nf, -1);
  int32_t nv = 0;
  for (int32_t f = 0; f < nf; ++f)
    if (col[f] == black) vid[f] = nv++;
  k.n_v = nv;
  k.n_c = n;
  k.edges.resize(n);
  int32_t w = 0, tau = 0;
  for (int32_t x = 0; x < n; ++x) {
    int32_t f0 = face[4 * x + 0], f1 = face[4 * x + 1], f2 = face[4 * x + 2],
            f3 = face[4 * x + 3];
    int32_t u, v;
    if (col[f0] == black) {
      u = vid[f0];
      v = vid[f2];
    } else {
      u = vid[f1];
      v = vid[f3];
    }
    // Tait sign: region on the left of the over-strand as it leaves (Sec. II)
    int32_t out_arm = ob[x] ? 1 : 3;
    int32_t eps = (col[face[4 * x + out_arm]] == black) ? 1 : -1;
    int32_t twist = ob[x] ? 1 : -1;  // right-hand rule
    k.edges[x] = {u, v, eps};
    w += twist;
    tau += eps;
  }
  k.writhe = w;
  k.tau = tau;
  return true;
}

bool knot_from_graph(int32_t n_v, int32_t n_e, const int32_t* uve, int32_t writhe, Knot& k,
                     std::string& err) {
  k = Knot();
  if (n_v < 1 || n_e < 0 || (n_e > 0 && uve == nullptr)) {
    err = "bad graph size";
    return false;
  }
  k.n_v = n_v;
  k.n_c = n_e;
  k.writhe = writhe;
  k.edges.resize(n_e);
  int32_t tau = 0;
  for (int32_t e = 0; e < n_e; ++e) {
    int32_t u = uve[3 * e], v = uve[3 * e + 1], s = uve[3 * e + 2];
    if (u < 0 || u >= n_v || v < 0 || v >= n_v || (s != 1 && s != -1)) {
      err = "bad edge";
      return false;
    }
    k.edges[e] = {u, v, s};
    tau += s;
  }
  k.tau = tau;
  k.components = 1;
  return true;
}

// ------------------------------------------------------------------ simplification (Sec. III.A)
// Reidemeister moves on the signed Tait graph, repeated until none applies:
//  * R-I on a loop (u, u, eps): the kink's crossing goes; tau -= eps, w -= eps;
//  * R-I on a spike (a vertex v of degree 1, edge (u, v, eps)): the crossing and the black
//    region v go; n_v -= 1, tau -= eps, w += eps;
//  * R-II unpoke of two parallel edges of opposite Tait signs: both crossings go (their
//    twist signs are opposite too), w and tau are unchanged.
// The diagram changes but not the knot, so V is unchanged: A(q) Z is evaluated with the new
// (n_v, w, tau).
bool simplify_knot(const Knot& in, Knot& out) {
  std::vector<std::array<int32_t, 3>> E = in.edges;
  int32_t w = in.writhe, tau = in.tau;
  std::vector<char> alive_v(in.n_v, 1);
  bool changed = true;
  while (changed) {
    changed = false;
    std::vector<std::array<int32_t, 3>> keep;
    for (const auto& e : E) {   // loops
      if (e[0] == e[1]) {
        tau -= e[2];
        w -= e[2];
        changed = true;
      } else {
        keep.push_back(e);
      }
    }
    E.swap(keep);
    // opposite-sign parallel pairs
    std::map<std::pair<int32_t, int32_t>, std::vector<int32_t>> pos, neg;
    for (int32_t i = 0; i < (int32_t)E.size(); ++i) {
      const auto key = std::make_pair(std::min(E[i][0], E[i][1]), std::max(E[i][0], E[i][1]));
      (E[i][2] > 0 ? pos : neg)[key].push_back(i);
    }
    std::vector<char> drop(E.size(), 0);
    for (auto& kv : pos) {
      auto it = neg.find(kv.first);
      if (it == neg.end()) continue;
      const size_t m = std::min(kv.second.size(), it->second.size());
      for (size_t j = 0; j < m; ++j) drop[kv.second[j]] = drop[it->second[j]] = 1;
      if (m) changed = true;
    }
    keep.clear();
    for (size_t i = 0; i < E.size(); ++i)
      if (!drop[i]) keep.push_back(E[i]);
    E.swap(keep);
    // spikes, one at a time (a removal can make another)
    std::vector<int32_t> deg(in.n_v, 0);
    for (const auto& e : E) {
      deg[e[0]]++;
      deg[e[1]]++;
    }
    for (int32_t i = 0; i < (int32_t)E.size(); ++i) {
      const int32_t u = E[i][0], v = E[i][1];
      const int32_t leaf = deg[v] == 1 ? v : deg[u] == 1 ? u : -1;
      if (leaf < 0) continue;
      alive_v[leaf] = 0;
      tau -= E[i][2];
      w += E[i][2];
      deg[u]--;
      deg[v]--;
      E.erase(E.begin() + i);
      changed = true;
      break;
    }
  }
  std::vector<int32_t> id(in.n_v, -1);
  int32_t n = 0;
  for (int32_t v = 0; v < in.n_v; ++v)
    if (alive_v[v]) id[v] = n++;
  out = Knot();
  out.n_v = n;
  out.n_c = (int32_t)E.size();
  out.writhe = w;
  out.tau = tau;
  out.components = in.components;
  for (const auto& e : E) out.edges.push_back({id[e[0]], id[e[1]], e[2]});
  return true;
}

// ------------------------------------------------------------------ grid walk (Sec. III.A)
namespace {
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  uint64_t below(uint64_t n) { return (uint64_t)(((unsigned __int128)next() * n) >> 64); }
  void perm(std::vector<int32_t>& a, int32_t n) {
    a.resize(n);
    for (int32_t i = 0; i < n; ++i) a[i] = i;
    for (int32_t i = n - 1; i > 0; --i) std::swap(a[i], a[below((uint64_t)i + 1)]);
  }
};

void crossings_of(const std::vector<int32_t>& xs, const std::vector<int32_t>& ys,
                  std::vector<std::array<int32_t, 2>>& cr) {
  const int32_t L = (int32_t)xs.size();
  cr.clear();
  for (int32_t i = 0; i < L; ++i) {
    int32_t x = xs[i];
    int32_t ylo = std::min(ys[i], ys[(i + 1) % L]), yhi = std::max(ys[i], ys[(i + 1) % L]);
    for (int32_t j = 0; j < L; ++j) {
      int32_t yj = ys[(j + 1) % L];
      int32_t xlo = std::min(xs[j], xs[(j + 1) % L]), xhi = std::max(xs[j], xs[(j + 1) % L]);
      if (xlo < x && x < xhi && ylo < yj && yj < yhi) cr.push_back({i, j});
    }
  }
}
}  // namespace

bool grid_walk_pd(int32_t L, uint64_t seed, bool random_over_under, int32_t nmin, int32_t nmax,
                  std::vector<std::array<int32_t, 4>>& pd, int32_t& outer_arc,
                  int32_t& outer_side, std::string& err) {
  if (L < 2 || L > 4096) {
    err = "grid side out of range";
    return false;
  }
  SplitMix64 rng{seed};
  std::vector<int32_t> xs, ys;
  std::vector<std::array<int32_t, 2>> cr;
  bool ok = false;
  for (int32_t draw = 0; draw < 200000; ++draw) {
    rng.perm(xs, L);
    rng.perm(ys, L);
    crossings_of(xs, ys, cr);
    int32_t n = (int32_t)cr.size();
    if (n >= nmin && n <= nmax) {
      ok = true;
      break;
    }
  }
  if (!ok) {
    err = "no grid walk in the crossing range";
    return false;
  }
  const int32_t n = (int32_t)cr.size();
  std::vector<int32_t> bits(n, 1);
  if (random_over_under)
    for (int32_t c = 0; c < n; ++c) bits[c] = (int32_t)(rng.next() >> 63);
  pd.clear();
  outer_arc = -1;
  outer_side = 0;
  if (n == 0) return true;
  // events along the curve V_0, H_0, V_1, H_1, ... : (segment, distance, crossing, vertical)
  struct Ev {
    int32_t seg, dist, c, vert;
  };
  std::vector<Ev> ev;
  for (int32_t c = 0; c < n; ++c) {
    int32_t i = cr[c][0], j = cr[c][1];
    ev.push_back({2 * i, std::abs(ys[(j + 1) % L] - ys[i]), c, 1});
    ev.push_back({2 * j + 1, std::abs(xs[i] - xs[j]), c, 0});
  }
  std::sort(ev.begin(), ev.end(), [](const Ev& a, const Ev& b) {
    if (a.seg != b.seg) return a.seg < b.seg;
    if (a.dist != b.dist) return a.dist < b.dist;
    if (a.c != b.c) return a.c < b.c;
    return a.vert < b.vert;
  });
  std::vector<int32_t> vpos(n), hpos(n);
  for (int32_t m = 0; m < 2 * n; ++m) (ev[m].vert ? vpos : hpos)[ev[m].c] = m;
  const int32_t two_n = 2 * n;
  pd.resize(n);
  for (int32_t c = 0; c < n; ++c) {
    int32_t i = cr[c][0], j = cr[c][1];
    int32_t dv[2] = {0, ys[(i + 1) % L] > ys[i] ? 1 : -1};
    int32_t dh[2] = {xs[(j + 1) % L] > xs[j] ? 1 : -1, 0};
    int32_t v_in = (vpos[c] - 1 + two_n) % two_n, v_out = vpos[c];
    int32_t h_in = (hpos[c] - 1 + two_n) % two_n, h_out = hpos[c];
    const int32_t *du, *dov;
    int32_t a, cc, o_in, o_out;
    if (bits[c]) {  // vertical over
      du = dh;
      dov = dv;
      a = h_in;
      cc = h_out;
      o_in = v_in;
      o_out = v_out;
    } else {
      du = dv;
      dov = dh;
      a = v_in;
      cc = v_out;
      o_in = h_in;
      o_out = h_out;
    }
    // arm b (counter-clockwise after the incoming under-arm) points along R(-du)
    int32_t bx = du[1], by = -du[0];
    if (dov[0] == bx && dov[1] == by)
      pd[c] = {a, o_out, cc, o_in};
    else
      pd[c] = {a, o_in, cc, o_out};
  }
  // unbounded region: west of the vertical segment at x = 0
  int32_t i0 = (int32_t)(std::find(xs.begin(), xs.end(), 0) - xs.begin());
  int32_t seg = 2 * i0;
  int32_t len2 = std::abs(ys[(i0 + 1) % L] - ys[i0]);  // compare 2*dist with len
  int32_t m_last = -1;
  for (int32_t m = 0; m < two_n; ++m)
    if (ev[m].seg < seg || (ev[m].seg == seg && 2 * ev[m].dist <= len2)) m_last = m;
  outer_arc = ((m_last % two_n) + two_n) % two_n;
  outer_side = ys[(i0 + 1) % L] > ys[i0] ? 0 : 1;
  return true;
}

}  // namespace pk
