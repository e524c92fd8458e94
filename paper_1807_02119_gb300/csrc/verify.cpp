// Host-side verification of a plan's index maps and memory layout (pk_plan_verify).
//
// Every gathered or scattered index map of a step is affine: a list of stride runs per
// index class (rows, contracted, columns; in the GEMM view batch, m and n runs with their
// C strides), fixed when the plan is made.  Because the maps are affine their bounds can be
// checked exhaustively once per plan instead of per access inside the kernels: an
// operand's runs must enumerate its dense row-major tensor exactly once (sorted by
// stride, each stride equals the product of the extents below it and the extents multiply
// to the tensor's size), the result must be the step's own new tensor, and every tensor
// must lie inside the arena without overlapping another tensor that is live at the same
// step.  The records the kernels read (the sequence kernel's copies of small steps, the
// complex128 tail steps, the digit scratch of the tensor-core steps, the reverse program)
// are checked against the same rules.
#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "pk_internal.h"

namespace pk {
namespace {

using Map = std::vector<std::pair<int64_t, int64_t>>;  // (extent, stride)

// True when the runs with a nonzero stride enumerate offsets 0 .. total-1 exactly once.
// Runs of stride 0 are indices the operand does not have (it is broadcast over them: a
// contracted spin present in one operand only, or a free index of the other operand).
bool dense(const Map& runs, int64_t total) {
  std::vector<std::pair<int64_t, int64_t>> r;  // (stride, extent) of runs longer than 1
  for (const auto& x : runs) {
    if (x.first < 1 || x.second < 0) return false;
    if (x.first > 1 && x.second != 0) r.push_back({x.second, x.first});
  }
  std::sort(r.begin(), r.end());
  int64_t expect = 1;
  for (const auto& x : r) {
    if (x.first != expect) return false;
    if (expect > ((int64_t)1 << 62) / x.second) return false;
    expect *= x.second;
  }
  return expect == total;
}

// True when no run longer than 1 has stride 0 (the operand has every index of the class).
bool present(const Map& runs) {
  for (const auto& x : runs)
    if (x.first > 1 && x.second == 0) return false;
  return true;
}

int64_t extent(const Map& runs) {
  int64_t e = 1;
  for (const auto& x : runs) e *= x.first;
  return e;
}

struct Checker {
  std::string err;
  bool fail(const std::string& where, const std::string& what) {
    if (err.empty()) err = where + ": " + what;
    return false;
  }
};

// The row view and the GEMM view of one step.  ea/eb/ec: the operands' element counts
// (eb = 0 when B is the constant 1).
bool check_step(const Step& s, int64_t ea, int64_t eb, int64_t ec, const std::string& where,
                Checker& ck) {
  if (s.nrow < 0 || s.nrow > kMaxRuns || s.nk < 0 || s.nk > kMaxRuns || s.nn < 0 ||
      s.nn > kMaxRuns || s.ngb < 0 || s.ngb > kMaxRuns || s.ngm < 0 || s.ngm > kMaxRuns ||
      s.ngn < 0 || s.ngn > kMaxRuns)
    return ck.fail(where, "run count out of range");
  Map row_a, row_b, k_a, k_b, n_b;
  for (int i = 0; i < s.nrow; ++i) {
    row_a.push_back({s.row[i].size, s.row[i].sa});
    if (s.row[i].sb != 0) row_b.push_back({s.row[i].size, s.row[i].sb});
  }
  for (int i = 0; i < s.nk; ++i) {
    k_a.push_back({s.kr[i].size, s.kr[i].sa});
    k_b.push_back({s.kr[i].size, s.kr[i].sb});
  }
  for (int i = 0; i < s.nn; ++i) n_b.push_back({s.nr[i].size, s.nr[i].sb});
  if (extent(row_a) != s.R || extent(k_a) != s.K || extent(n_b) != s.N)
    return ck.fail(where, "run extents do not multiply to R, K, N");
  if (s.R * s.N != ec) return ck.fail(where, "R N differs from the result's size");
  Map a = row_a;
  a.insert(a.end(), k_a.begin(), k_a.end());
  if (!present(row_a)) return ck.fail(where, "a row index absent from A");
  if (!dense(a, ea)) return ck.fail(where, "A's row and contracted runs do not cover A once");
  if (eb > 0) {
    Map b = row_b;
    b.insert(b.end(), k_b.begin(), k_b.end());
    b.insert(b.end(), n_b.begin(), n_b.end());
    if (!present(n_b)) return ck.fail(where, "a column index absent from B");
    if (!dense(b, eb)) return ck.fail(where, "B's batch, contracted and column runs do not cover B once");
  } else if (s.N != 1 || s.b >= 0) {
    return ck.fail(where, "a step without B (a sum over A's contracted indices) has N = 1");
  }
  // GEMM view
  Map ga, gbm, gc;
  int64_t bsz = 1, m = 1, n = 1;
  for (int i = 0; i < s.ngb; ++i) {
    ga.push_back({s.gb[i].size, s.gb[i].sa});
    gbm.push_back({s.gb[i].size, s.gb[i].sb});
    gc.push_back({s.gb[i].size, s.gb[i].sc});
    bsz *= s.gb[i].size;
  }
  for (int i = 0; i < s.ngm; ++i) {
    ga.push_back({s.gm[i].size, s.gm[i].sa});
    gc.push_back({s.gm[i].size, s.gm[i].sc});
    m *= s.gm[i].size;
  }
  for (int i = 0; i < s.ngn; ++i) {
    gbm.push_back({s.gn[i].size, s.gn[i].sb});
    gc.push_back({s.gn[i].size, s.gn[i].sc});
    n *= s.gn[i].size;
  }
  if (bsz != s.Bsz || m != s.M || bsz * m != s.R || n != s.N)
    return ck.fail(where, "GEMM view extents do not match Bsz, M, R, N");
  if (!present(ga) || (eb > 0 && !present(gbm)) || !present(gc))
    return ck.fail(where, "GEMM view: a batch, m or n index absent from its operand");
  ga.insert(ga.end(), k_a.begin(), k_a.end());
  gbm.insert(gbm.end(), k_b.begin(), k_b.end());
  if (!dense(ga, ea)) return ck.fail(where, "GEMM view: A's runs do not cover A once");
  if (eb > 0 && !dense(gbm, eb)) return ck.fail(where, "GEMM view: B's runs do not cover B once");
  if (!dense(gc, ec)) return ck.fail(where, "GEMM view: C's runs do not cover C once");
  if (s.tc != 0 && s.tc != 4 && s.tc != 5) return ck.fail(where, "tensor-core digits must be 4 or 5");
  if (s.kernel == KSPLITK && (s.chunks < 1 || s.chunks > 64))
    return ck.fail(where, "split-K chunk count out of range");
  return true;
}

bool same_runs(const Run* x, const Run* y, int n) {
  for (int i = 0; i < n; ++i)
    if (x[i].size != y[i].size || x[i].sa != y[i].sa || x[i].sb != y[i].sb) return false;
  return true;
}

// [off, off + len) intervals that are live together must not overlap.
struct Live {
  int64_t off, len;
  int32_t born, dies;
  int32_t id;
};
bool disjoint(std::vector<Live> v, const std::string& what, Checker& ck) {
  std::sort(v.begin(), v.end(), [](const Live& x, const Live& y) { return x.off < y.off; });
  for (size_t i = 0; i < v.size(); ++i)
    for (size_t j = i + 1; j < v.size() && v[j].off < v[i].off + v[i].len; ++j)
      if (!(v[i].dies < v[j].born || v[j].dies < v[i].born) && v[i].len > 0 && v[j].len > 0)
        return ck.fail(what, "tensors " + std::to_string(v[i].id) + " and " +
                                 std::to_string(v[j].id) + " overlap while both are live");
  return true;
}

bool check_forward(const Plan& p, int32_t precision, Checker& ck) {
  const int32_t nt = (int32_t)p.tensors.size();
  const int32_t ns = (int32_t)p.steps.size();
  if (p.n_init < 0 || p.n_init > nt || nt != p.n_init + ns)
    return ck.fail("plan", "tensor count differs from initial tensors + steps");
  if (p.final_tensor < 0 || p.final_tensor >= nt) return ck.fail("plan", "bad final tensor");
  if ((int32_t)p.recipes.size() != p.n_init) return ck.fail("plan", "one recipe per initial tensor");
  std::vector<Live> live;
  for (int32_t t = 0; t < nt; ++t) {
    const TensorInfo& ti = p.tensors[t];
    const std::string w = "tensor " + std::to_string(t);
    if (ti.offset < 0 || ti.elems < 1 || ti.offset + ti.elems > p.arena_elems)
      return ck.fail(w, "outside the arena");
    if (ti.offset % 64 != 0) return ck.fail(w, "not on a 512-byte boundary");
    if (ti.elems > ((int64_t)1 << 31))   // the kernels decode indices with 32-bit division
      return ck.fail(w, "more than 2^31 entries");
    live.push_back({ti.offset, ti.elems, ti.born, ti.dies, t});
  }
  if (!disjoint(live, "arena", ck)) return false;
  for (int32_t i = 0; i < p.n_init; ++i) {
    const Recipe& r = p.recipes[i];
    if (r.offset != p.tensors[i].offset || r.elems != p.tensors[i].elems || r.meta != i)
      return ck.fail("recipe " + std::to_string(i), "differs from its tensor");
    if (r.slot0 < 0 || r.nslot < 0 || r.slot0 + r.nslot > (int32_t)p.slots.size())
      return ck.fail("recipe " + std::to_string(i), "slot range outside the slot table");
  }
  for (int32_t i = 0; i < ns; ++i) {
    const Step& s = p.steps[i];
    const std::string w = "step " + std::to_string(i);
    if (s.a < 0 || s.a >= nt || s.b < -1 || s.b >= nt || s.c != p.n_init + i)
      return ck.fail(w, "operand or result id out of range");
    if (p.tensors[s.a].born >= i || p.tensors[s.a].dies < i ||
        (s.b >= 0 && (p.tensors[s.b].born >= i || p.tensors[s.b].dies < i)))
      return ck.fail(w, "reads a tensor that is not live");
    if (s.off_a != p.tensors[s.a].offset || (s.b >= 0 && s.off_b != p.tensors[s.b].offset) ||
        s.off_c != p.tensors[s.c].offset)
      return ck.fail(w, "offsets differ from the tensors' arena offsets");
    if (!check_step(s, p.tensors[s.a].elems, s.b >= 0 ? p.tensors[s.b].elems : 0,
                    p.tensors[s.c].elems, w, ck))
      return false;
    if (precision == PK_SPLIT && s.tc) {
      const TcScratch x = tc_scratch(s.Bsz, s.M, s.N, s.K, s.tc);
      if (x.bytes > p.tc_bytes) return ck.fail(w, "digit scratch larger than the plan reserves");
    }
  }
  // sequence-kernel records: exact copies of their steps' row views
  for (const Segment& g : p.segments) {
    const std::string w = "sequence run at step " + std::to_string(g.first);
    if (g.count < 2 || g.first < 0 || g.first + g.count > ns || g.tiny0 < 0 ||
        g.tiny0 + g.count > (int32_t)p.tiny.size())
      return ck.fail(w, "range outside the steps or records");
    for (int32_t j = 0; j < g.count; ++j) {
      const Step& s = p.steps[g.first + j];
      const TinyStep& t = p.tiny[g.tiny0 + j];
      if (s.kernel != KROWS || s.tc || t.a != s.a || t.b != s.b || t.c != s.c ||
          t.off_a != s.off_a || t.off_b != s.off_b || t.off_c != s.off_c || t.R != s.R ||
          t.K != s.K || t.N != s.N || t.nrow != s.nrow || t.nk != s.nk || t.nn != s.nn ||
          !same_runs(t.row, s.row, s.nrow) || !same_runs(t.kr, s.kr, s.nk) ||
          !same_runs(t.nr, s.nr, s.nn) || s.K > kTinyK)
        return ck.fail(w, "record differs from step " + std::to_string(g.first + j));
    }
  }
  // complex128 tail of the complex64 precision
  if (precision == PK_C64 && !p.tail.empty()) {
    std::vector<Live> tl;
    for (const ConvRec& c : p.conv) {
      if (c.src_meta < 0 || c.src_meta >= nt || c.src_off != p.tensors[c.src_meta].offset ||
          c.elems != p.tensors[c.src_meta].elems || c.dst_off < 0 || c.dst_off + c.elems > p.tail_elems)
        return ck.fail("widening record", "outside its tensor or the tail region");
      tl.push_back({c.dst_off, c.elems, 0, (int32_t)p.tail.size(), c.dst_meta});
    }
    for (size_t j = 0; j < p.tail.size(); ++j) {
      const TailStep& t = p.tail[j];
      const Step& s = p.steps[t.step];
      if (t.step != p.tail_first + (int32_t)j) return ck.fail("tail", "steps not consecutive");
      const std::string w = "tail step " + std::to_string(t.step);
      const int64_t eb = s.b >= 0 ? p.tensors[s.b].elems : 0;
      if (t.off_a < 0 || t.off_a + p.tensors[s.a].elems > p.tail_elems || t.off_b < 0 ||
          t.off_b + eb > p.tail_elems || t.off_c < 0 || t.off_c + p.tensors[s.c].elems > p.tail_elems)
        return ck.fail(w, "outside the tail region");
      tl.push_back({t.off_c, p.tensors[s.c].elems, (int32_t)j, (int32_t)p.tail.size(), s.c});
    }
    if (!disjoint(tl, "tail region", ck)) return false;
  }
  // workspace layout: state records in order, the arena (and the split digit scratch or the
  // tail region) inside the workspace
  if (!(p.off_recipe <= p.off_slots && p.off_slots <= p.off_conv && p.off_conv <= p.off_tiny &&
        p.off_tiny <= p.off_meta && p.off_meta + 16ull * p.n_meta <= p.off_counter &&
        p.off_counter + 4ull * (uint64_t)ns <= p.off_result &&
        p.off_result + 32ull * (uint64_t)(p.n_slices + 1) <= p.off_scratch &&
        p.off_scratch + 16ull * (uint64_t)p.splitk_partials <= p.off_arena))
    return ck.fail("workspace", "state records overlap");
  const uint64_t esz = precision == PK_C64 ? 8 : 16;
  uint64_t end = p.off_arena + esz * (uint64_t)p.arena_elems;
  if (precision == PK_SPLIT && p.tc_bytes > 0) end = p.off_arena + p.tc_offset() + (uint64_t)p.tc_bytes;
  if (precision == PK_C64 && !p.tail.empty()) {
    if (p.off_tail < p.off_arena + 8ull * (uint64_t)p.arena_elems)
      return ck.fail("workspace", "tail region overlaps the arena");
    end = p.off_tail + 16ull * (uint64_t)p.tail_elems;
  }
  if (end > p.ws_bytes(precision)) return ck.fail("workspace", "extends past pk_plan_workspace_bytes");
  return true;
}

// The reverse program: every step inside its arena with dense maps.
bool check_grad(const Plan& p, Checker& ck) {
  const GradProgram& G = p.grad;
  for (size_t i = 0; i < G.steps.size(); ++i) {
    const Step& s = G.steps[i];
    const std::string w = "reverse step " + std::to_string(i);
    // operand sizes: the extents of the indices each operand has (nonzero strides)
    int64_t ea = 1, eb = s.b >= 0 ? s.N : 0;
    for (int j = 0; j < s.nrow; ++j) {
      if (s.row[j].sa != 0) ea *= s.row[j].size;
      if (s.row[j].sb != 0) eb *= s.row[j].size;
    }
    for (int j = 0; j < s.nk; ++j) {
      if (s.kr[j].sa != 0) ea *= s.kr[j].size;
      if (s.kr[j].sb != 0) eb *= s.kr[j].size;
    }
    const int64_t ec = s.R * s.N;
    if (s.off_a < 0 || s.off_a + ea > G.arena_elems || s.off_c < 0 || s.off_c + ec > G.arena_elems ||
        (s.b >= 0 && (s.off_b < 0 || s.off_b + eb > G.arena_elems)))
      return ck.fail(w, "outside the reverse program's arena");
    if (s.a < 0 || s.a >= G.n_meta || s.c < 0 || s.c >= G.n_meta || s.b >= G.n_meta)
      return ck.fail(w, "bookkeeping slot out of range");
    if (!check_step(s, ea, eb, ec, w, ck)) return false;
  }
  for (const Recipe& r : G.recipes)
    if (r.offset < 0 || r.offset + r.elems > G.arena_elems)
      return ck.fail("reverse program", "initial tensor outside the arena");
  return true;
}

}  // namespace

bool verify_plan(const Plan& p, int32_t precision, std::string& err) {
  Checker ck;
  if (!check_forward(p, precision, ck) || (p.grad.built && !check_grad(p, ck))) {
    err = ck.err;
    return false;
  }
  return true;
}

}  // namespace pk
