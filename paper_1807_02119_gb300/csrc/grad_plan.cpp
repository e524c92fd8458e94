// Reverse pass over the contraction tree (adjoint contraction) for plans made with
// PK_FLAG_GRAD.
//
// Z is linear in every tensor of the tree.  For a step C = sum A B (sum over the indices
// of A and B that C does not keep) the adjoints are
//     dZ/dA = sum C' B   and   dZ/dB = sum A C'      (C' = dZ/dC, holomorphic: no conjugate)
// where each sum runs over the indices of C' and of the other operand that the target
// does not hold.  An index of the target that neither C' nor the other operand holds is
// one that the forward step summed away (or that C' is constant along): the adjoint is
// constant along it, so it is left out of the stored adjoint and read back with stride 0.
// Each adjoint is therefore one more pairwise contraction of the same form as a forward
// step and runs on the same kernels; a step whose second operand is the constant 1 (a
// plain sum) passes C' down unchanged.  The root's adjoint is the constant 1.
//
// Memory: forward intermediates whose tree level (leaves 0, a step's result 1 + the
// larger level of its operands) is a multiple of the checkpoint stride are kept for the
// reverse pass; the others are recomputed.  A region is a checkpointed tensor (or the
// root) with the steps below it down to the next checkpoints; regions are processed from
// the root down, each one recomputing its intermediates (in forward order) and then
// running its adjoint steps (in reverse order), so every intermediate is computed at
// most twice.  All tensors of the program share one arena laid out by first fit over
// their lifetimes.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <numeric>

#include "pk_internal.h"

namespace pk {
namespace {

struct Inst {
  std::vector<int32_t> dims;
  int64_t elems = 1;
  int32_t born = -1, dies = -1;
  int32_t meta = -1;
  int64_t off = 0;
};

struct Op {
  Step st;
  int32_t in_a, in_b, out;  // instance ids (in_b = -1: the constant 1)
  int8_t phase;             // 0 forward, 1 recompute, 2 adjoint
};

uint64_t a256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

bool holds(const std::vector<int32_t>& d, int32_t x) {
  return std::find(d.begin(), d.end(), x) != d.end();
}

}  // namespace

bool make_grad_program(Plan& p, int32_t stride, int32_t flags, const pk_tuning& tune, std::string& err) {
  GradProgram& G = p.grad;
  G = GradProgram();
  G.stride = stride > 1 ? stride : 1;
  const int32_t q = p.q;
  const int32_t n_tens = (int32_t)p.tensors.size();
  const int32_t S = (int32_t)p.steps.size();
  const int32_t root = p.final_tensor;
  auto qpow = [&](int64_t e) {
    int64_t r = 1;
    for (int64_t i = 0; i < e; ++i) r *= q;
    return r;
  };

  // tree levels, consumers, which tensors lead to a clause tensor, checkpoints
  std::vector<int32_t> level(n_tens, 0), cons(n_tens, -1);
  std::vector<char> need(n_tens, 0), ckpt(n_tens, 0);
  for (const EdgeGroup& g : p.groups) need[g.leaf] = 1;
  for (int32_t s = 0; s < S; ++s) {
    const Step& st = p.steps[s];
    int32_t l = level[st.a];
    if (st.b >= 0) l = std::max(l, level[st.b]);
    level[st.c] = l + 1;
    cons[st.a] = s;
    if (st.b >= 0) cons[st.b] = s;
    need[st.c] = need[st.a] || (st.b >= 0 && need[st.b]);
  }
  for (int32_t i = p.n_init; i < n_tens; ++i)
    ckpt[i] = (i == root || G.stride <= 1 || level[i] % G.stride == 0) ? 1 : 0;
  std::vector<int32_t> owner(S, -1);
  for (int32_t s = S - 1; s >= 0; --s) {  // a consumer comes after its operands
    const int32_t X = p.n_init + s;
    if (ckpt[X]) {
      owner[s] = X;
    } else {
      if (cons[X] < 0) {
        err = "internal: intermediate without a consumer";
        return false;
      }
      owner[s] = owner[cons[X]];
    }
  }
  std::vector<std::vector<int32_t>> region(n_tens);
  for (int32_t s = 0; s < S; ++s) region[owner[s]].push_back(s);

  std::vector<Inst> inst(n_tens);
  for (int32_t i = 0; i < n_tens; ++i) {
    inst[i].dims = p.tensors[i].dims;
    inst[i].elems = p.tensors[i].elems;
    inst[i].meta = i;
  }
  int32_t next_meta = n_tens;
  auto new_inst = [&](const std::vector<int32_t>& dims, int32_t t) {
    Inst x;
    x.dims = dims;
    x.elems = qpow((int64_t)dims.size());
    x.born = x.dies = t;
    x.meta = next_meta++;
    inst.push_back(x);
    return (int32_t)inst.size() - 1;
  };
  auto use = [&](int32_t id, int32_t t) {
    if (id >= 0) inst[id].dies = std::max(inst[id].dies, t);
  };
  std::vector<Op> ops;

  // forward pass
  for (int32_t s = 0; s < S; ++s) {
    const Step& st = p.steps[s];
    const int32_t t = (int32_t)ops.size();
    inst[st.c].born = inst[st.c].dies = t;
    use(st.a, t);
    use(st.b, t);
    ops.push_back({st, st.a, st.b, st.c, 0});
  }

  // reverse pass, region by region from the root down
  std::vector<int32_t> cur(n_tens), adj(n_tens, -2);  // adj: -1 constant 1, -2 not yet formed
  std::iota(cur.begin(), cur.end(), 0);
  adj[root] = -1;
  std::vector<int32_t> heads;
  for (int32_t X = p.n_init; X < n_tens; ++X)
    if (!region[X].empty()) heads.push_back(X);
  std::sort(heads.rbegin(), heads.rend());
  for (int32_t X : heads) {
    if (!need[X]) continue;
    const std::vector<int32_t>& R = region[X];
    for (int32_t s : R) {  // recompute the region's intermediates
      if (p.n_init + s == X) continue;
      Step st = p.steps[s];
      const int32_t A = st.a, B = st.b, C = st.c;
      const int32_t t = (int32_t)ops.size();
      const int32_t id = new_inst(p.tensors[C].dims, t);
      st.a = inst[cur[A]].meta;
      st.b = B >= 0 ? inst[cur[B]].meta : -1;
      st.c = inst[id].meta;
      use(cur[A], t);
      if (B >= 0) use(cur[B], t);
      ops.push_back({st, cur[A], B >= 0 ? cur[B] : -1, id, 1});
      cur[C] = id;
    }
    for (auto it = R.rbegin(); it != R.rend(); ++it) {  // adjoint steps
      const Step& fs = p.steps[*it];
      const int32_t A = fs.a, B = fs.b, C = fs.c;
      if (!need[C]) continue;
      const int32_t Xb = adj[C];
      if (Xb == -2) {
        err = "internal: adjoint needed before it is formed";
        return false;
      }
      if (B < 0) {  // C = sum A: the adjoint of A is C' (constant along the summed indices)
        adj[A] = Xb;
        continue;
      }
      for (int side = 0; side < 2; ++side) {
        const int32_t T = side == 0 ? A : B, O = side == 0 ? B : A;
        if (!need[T]) continue;
        const std::vector<int32_t> xd = Xb >= 0 ? inst[Xb].dims : std::vector<int32_t>();
        const std::vector<int32_t> od = inst[cur[O]].dims;
        std::vector<int32_t> out;
        for (int32_t x : p.tensors[T].dims)
          if (holds(xd, x) || holds(od, x)) out.push_back(x);
        std::sort(out.begin(), out.end());
        Step st;
        bool sw = false;
        std::vector<int32_t> cd;
        int32_t ia, ib;
        if (Xb >= 0) {
          if (!build_step(xd, &od, out, q, flags, st, sw, cd, err)) return false;
          ia = sw ? cur[O] : Xb;
          ib = sw ? Xb : cur[O];
        } else {
          if (!build_step(od, nullptr, out, q, flags, st, sw, cd, err)) return false;
          ia = cur[O];
          ib = -1;
        }
        const int32_t t = (int32_t)ops.size();
        const int32_t id = new_inst(cd, t);
        st.a = inst[ia].meta;
        st.b = ib >= 0 ? inst[ib].meta : -1;
        st.c = inst[id].meta;
        use(ia, t);
        use(ib, t);
        ops.push_back({st, ia, ib, id, 2});
        adj[T] = id;
      }
    }
  }
  const int32_t END = (int32_t)ops.size();
  use(root, END);  // the slice result reads the root
  for (const EdgeGroup& g : p.groups) {
    if (adj[g.leaf] == -2) {
      err = "internal: clause tensor without an adjoint";
      return false;
    }
    use(adj[g.leaf], END);
  }

  // arena: first fit by decreasing size over lifetime intervals
  std::vector<int32_t> ord(inst.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) {
    if (inst[x].elems != inst[y].elems) return inst[x].elems > inst[y].elems;
    return x < y;
  });
  struct Placed {
    int64_t off, len;
    int32_t born, dies;
  };
  std::vector<Placed> placed;
  int64_t top = 0;
  for (int32_t id : ord) {
    Inst& in = inst[id];
    const int64_t len = (in.elems + 63) / 64 * 64;
    std::vector<std::pair<int64_t, int64_t>> busy;
    for (const auto& pl : placed)
      if (!(pl.dies < in.born || in.dies < pl.born)) busy.push_back({pl.off, pl.off + pl.len});
    std::sort(busy.begin(), busy.end());
    int64_t off = 0;
    for (const auto& iv : busy) {
      if (off + len <= iv.first) break;
      off = std::max(off, iv.second);
    }
    in.off = off;
    placed.push_back({off, len, in.born, in.dies});
    top = std::max(top, off + len);
  }
  G.arena_elems = top;
  G.n_meta = next_meta;

  // steps with their offsets
  for (Op& op : ops) {
    op.st.tc = 0;  // the reverse program keeps its GEMM steps on the CUDA cores
    op.st.off_a = inst[op.in_a].off;
    op.st.off_b = op.in_b >= 0 ? inst[op.in_b].off : 0;
    op.st.off_c = inst[op.out].off;
    G.steps.push_back(op.st);
    G.phase.push_back(op.phase);
    G.cmacs[op.phase] += (double)op.st.R * (double)op.st.K * (double)op.st.N;
    if (op.st.kernel == KSPLITK)
      G.partials = std::max<int64_t>(G.partials, op.st.R * op.st.N * op.st.chunks);
  }
  for (int32_t i = p.n_init; i < n_tens; ++i) G.n_checkpoints += ckpt[i];
  G.recipes = p.recipes;
  for (int32_t i = 0; i < p.n_init; ++i) G.recipes[i].offset = inst[i].off;
  G.root_offset = inst[root].off;
  G.root_meta = root;
  for (const EdgeGroup& g : p.groups) {
    const int32_t a = adj[g.leaf];
    GradLeaf L;
    std::memset(&L, 0, sizeof(L));
    L.meta = a >= 0 ? inst[a].meta : -1;
    L.offset = a >= 0 ? inst[a].off : 0;
    const std::vector<int32_t>& full = p.leaf_dims[g.leaf];
    L.rank = (int32_t)full.size();
    for (int j = 0; j < 2; ++j) {
      L.slice_ord[j] = -1;
      L.stride[j] = 0;
    }
    for (int32_t j = 0; j < L.rank && j < 2; ++j) {
      const int32_t x = full[j];
      auto it = std::find(p.sliced.begin(), p.sliced.end(), x);
      if (it != p.sliced.end()) {
        L.slice_ord[j] = (int32_t)(it - p.sliced.begin());
        continue;
      }
      if (a < 0) continue;
      const std::vector<int32_t>& ad = inst[a].dims;
      for (size_t k = 0; k < ad.size(); ++k)
        if (ad[k] == x) L.stride[j] = qpow((int64_t)(ad.size() - 1 - k));
    }
    G.leaves.push_back(L);
  }

  // runs of small steps as sequence launches
  build_segments(G.steps, tune, G.segments, G.tiny);

  // workspace layout
  const uint64_t nl = std::max<size_t>(1, G.leaves.size());
  uint64_t off = 0;
  G.off_recipe = off;
  off = a256(off + sizeof(Recipe) * G.recipes.size());
  G.off_slots = off;
  off = a256(off + sizeof(Slot) * std::max<size_t>(1, p.slots.size()));
  G.off_leaves = off;
  off = a256(off + sizeof(GradLeaf) * nl);
  G.off_tiny = off;
  off = a256(off + sizeof(TinyStep) * G.tiny.size());
  G.off_meta = off;
  off = a256(off + 16ull * (uint64_t)G.n_meta);
  G.off_counter = off;
  off = a256(off + 4ull * std::max<size_t>(1, G.steps.size()));
  G.off_result = off;
  off = a256(off + 32ull * (uint64_t)p.n_slices + 32);
  G.off_scratch = off;
  off = a256(off + 16ull * (uint64_t)std::max<int64_t>(1, G.partials));
  G.off_acc = off;
  off = a256(off + 16ull * (uint64_t)q * (uint64_t)q * nl + 8ull * nl);
  G.off_arena = off;
  G.program.assign(G.off_meta, 0);
  if (!G.recipes.empty())
    std::memcpy(G.program.data() + G.off_recipe, G.recipes.data(), sizeof(Recipe) * G.recipes.size());
  if (!p.slots.empty())
    std::memcpy(G.program.data() + G.off_slots, p.slots.data(), sizeof(Slot) * p.slots.size());
  if (!G.leaves.empty())
    std::memcpy(G.program.data() + G.off_leaves, G.leaves.data(), sizeof(GradLeaf) * G.leaves.size());
  if (!G.tiny.empty())
    std::memcpy(G.program.data() + G.off_tiny, G.tiny.data(), sizeof(TinyStep) * G.tiny.size());
  G.built = true;
  return true;
}

bool grad_finalize(const Plan& p, const double* acc, const int64_t* acc_exp, const Scaled& z,
                   double* dlogz, double* dlogv_dt) {
  typedef std::complex<double> cd;
  const int32_t q = p.q;
  const cd zm(z.re, z.im);
  if (zm == cd(0, 0)) return false;
  const size_t n_e = p.knot.edges.size();
  std::vector<cd> dl((size_t)n_e * q * q, cd(0, 0));
  for (size_t gi = 0; gi < p.groups.size(); ++gi) {
    const EdgeGroup& g = p.groups[gi];
    const double* base = acc + 2ull * q * q * gi;
    const int64_t de = acc_exp[gi] - z.e;
    const double scale = std::ldexp(1.0, (int)std::max<int64_t>(-2000, std::min<int64_t>(2000, de)));
    const bool loop = g.u == g.v;
    for (int32_t c : g.members) {
      const bool flip = p.knot.edges[c][0] != g.u;
      for (int32_t a = 0; a < q; ++a)
        for (int32_t b = 0; b < q; ++b) {
          if (loop && a != b) continue;
          const int32_t idx = loop ? a : (flip ? b * q + a : a * q + b);
          cd v(base[2 * idx], base[2 * idx + 1]);
          for (int32_t c2 : g.members) {  // the other members' entries at (a, b)
            if (c2 == c) continue;
            const auto& w = p.weights[c2];
            v *= (a == b) ? cd(w[0], w[1]) : cd(w[2], w[3]);
          }
          dl[((size_t)c * q + a) * q + b] = v * scale / zm;
        }
    }
  }
  if (dlogz)
    for (size_t i = 0; i < dl.size(); ++i) {
      dlogz[2 * i] = dl[i].real();
      dlogz[2 * i + 1] = dl[i].imag();
    }
  if (dlogv_dt) {
    if (!p.std_weights) {
      dlogv_dt[0] = dlogv_dt[1] = std::nan("");
    } else {
      double tre, tim;
      t_of_q_value(q, tre, tim);
      const cd t(tre, tim);
      const Knot& k = p.knot;
      // d/dt log of s^num (s^4 = t) is (num / 4) / t: an integer k for a knot, a multiple
      // of 1/2 for a link
      const double kk = (double)(3LL * k.writhe + k.tau + 2LL * k.n_v + 2) / 4.0;
      cd r = kk / t - (double)(k.n_v + 1) / (t + 1.0);
      for (size_t c = 0; c < n_e; ++c) {
        cd s(0, 0);
        for (int32_t a = 0; a < q; ++a) s += dl[((size_t)c * q + a) * q + a];
        const int32_t eps = k.edges[c][2];
        r += (eps > 0 ? 1.0 / (t * t) : cd(-1.0, 0.0)) * s;  // d(-t^-eps)/dt = eps t^(-eps-1)
      }
      dlogv_dt[0] = r.real();
      dlogv_dt[1] = r.imag();
    }
  }
  return true;
}

}  // namespace pk
