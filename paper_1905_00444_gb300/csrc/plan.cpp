// Contraction planner: order, open sites, cuts, fold program, workspace layout.
//
// Order (Sec. III.D: few large, high-arithmetic-intensity contractions): the grid is
// swept line by line along its shorter dimension, one site per step.  With the
// boundary kept as [x-legs][h'_0..h'_{r-1}][v][h_r..h_{L-1}] ("kink" layout), the
// site at position r contracts the adjacent pair (v, h_r) and leaves (h'_r, v') in the
// same place, so every step is C[nh][p][nl][s] = sum_k S[k][nh*NL+nl] B[p][k][s]: a
// strided batched GEMM that needs no tensor transpose (the T's of TTGT are elided).
// New open output legs (fast sampling, Sec. III.B) go outermost.
//
// Cuts (Sec. III.A): a cut slices one bond into pieces; the slice id is mixed-radix
// over the cuts (first cut most significant).  When the largest intermediate exceeds
// the cap, the planner halves bonds greedily (fewest tensors at the peak, then the
// least total work) until it fits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>

#include "qfx_internal.h"

namespace {

uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

struct Geometry {
  int rows, cols;
  bool transposed;
  int W, L;  // lines, positions per line
  int qubit(int line, int pos) const {
    return transposed ? line * cols + pos : pos * cols + line;
  }
};

struct Leg {
  int id;       // edge id >= 0, or -(1 + qubit) for an open output leg
  int64_t dim;
};

// Tensor sizes are products of bond dimensions of up to 2^40 each, so they are formed with
// a product that saturates at 2^62 instead of overflowing; a plan whose largest tensor
// exceeds kMaxPlanElements is refused.
constexpr int64_t kSat = int64_t(1) << 62;
constexpr int64_t kMaxPlanElements = int64_t(1) << 50;
int64_t smul(int64_t a, int64_t b) {   // a, b >= 1
  return a > kSat / b ? kSat : std::min(a * b, kSat);
}

struct SimResult {
  bool ok = true;
  std::string err;
  std::vector<qfx::Step> steps;
  int64_t peak = 1;          // largest intermediate in elements (buffers and sites)
  int peak_count = 0;
  double flops = 0, bytes = 0;
  std::vector<int> intro;    // open sites in order of introduction
};

// slot edge ids per site: up, left, right, down
using Slots = std::vector<std::array<int, 4>>;

SimResult simulate(const Geometry& geo, const std::vector<int>& order, const Slots& slots,
                   const std::vector<int64_t>& edim, const std::vector<char>& is_open) {
  SimResult r;
  std::vector<Leg> bnd;
  auto d = [&](int e) -> int64_t { return e < 0 ? 1 : edim[e]; };
  for (size_t si = 0; si < order.size(); ++si) {
    int q = order[si];
    const auto& s = slots[q];
    int64_t xd = is_open[q] ? 2 : 1;
    int64_t site_size = smul(smul(smul(smul(d(s[0]), d(s[1])), xd), d(s[2])), d(s[3]));
    r.peak = std::max(r.peak, site_size);
    std::vector<Leg> nlegs;
    if (is_open[q]) { nlegs.push_back({-(1 + q), 2}); r.intro.push_back(q); }
    std::vector<Leg> rd;
    if (s[2] >= 0) rd.push_back({s[2], d(s[2])});
    if (s[3] >= 0) rd.push_back({s[3], d(s[3])});
    qfx::Step st{};
    st.site = q;
    st.N = smul(smul(xd, d(s[2])), d(s[3]));
    st.NL = smul(d(s[2]), d(s[3]));
    if (si == 0) {
      if (s[0] >= 0 || s[1] >= 0) { r.ok = false; r.err = "first site has contracted bonds"; return r; }
      st.P = st.K = st.Sd = 1;
      st.flops = 0;
      st.bytes = 0;
      bnd = nlegs;
      bnd.insert(bnd.end(), rd.begin(), rd.end());
      r.steps.push_back(st);
      continue;
    }
    std::vector<int> kids;
    if (s[0] >= 0) kids.push_back(s[0]);
    if (s[1] >= 0) kids.push_back(s[1]);
    if (kids.empty()) { r.ok = false; r.err = "site without contracted bond"; return r; }
    size_t pos = bnd.size();
    for (size_t i = 0; i < bnd.size(); ++i)
      if (bnd[i].id == kids[0]) { pos = i; break; }
    if (pos == bnd.size() || pos + kids.size() > bnd.size()) { r.ok = false; r.err = "kink leg missing"; return r; }
    for (size_t j = 0; j < kids.size(); ++j)
      if (bnd[pos + j].id != kids[j]) { r.ok = false; r.err = "kink legs not adjacent"; return r; }
    int64_t P = 1, K = 1, Sd = 1;
    for (size_t i = 0; i < pos; ++i) P = smul(P, bnd[i].dim);
    for (size_t j = 0; j < kids.size(); ++j) K = smul(K, bnd[pos + j].dim);
    for (size_t i = pos + kids.size(); i < bnd.size(); ++i) Sd = smul(Sd, bnd[i].dim);
    st.P = P; st.K = K; st.Sd = Sd;
    st.flops = 8.0 * (double)P * (double)K * (double)st.N * (double)Sd;
    st.bytes = 8.0 * ((double)P * K * Sd + (double)K * st.N + (double)P * st.N * Sd);
    std::vector<Leg> nb = nlegs;
    nb.insert(nb.end(), bnd.begin(), bnd.begin() + pos);
    nb.insert(nb.end(), rd.begin(), rd.end());
    nb.insert(nb.end(), bnd.begin() + pos + kids.size(), bnd.end());
    bnd.swap(nb);
    int64_t out_el = smul(smul(P, st.N), Sd);
    if (out_el > r.peak) { r.peak = out_el; r.peak_count = 0; }
    if (out_el == r.peak) r.peak_count++;
    r.flops += st.flops;
    r.bytes += st.bytes;
    r.steps.push_back(st);
  }
  // all bonds must be closed at the end
  for (const auto& l : bnd)
    if (l.id >= 0 && l.dim != 1) { r.ok = false; r.err = "bond left open"; return r; }
  return r;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" qfx_status qfx_plan_create(const qfx_circuit* c, const qfx_plan_opts* o,
                                      qfx_plan** out) {
  if (!c || !o || !out) return qfx::fail(QFX_EINVAL, "qfx_plan_create: NULL argument");
  *out = nullptr;
  try {
    if (o->plan_family != 0 && o->plan_family != 1)
      return qfx::fail(QFX_EINVAL, "plan_family: 0 (line sweep) or 1 (contraction tree)");

    if (o->precision < QFX_PREC_FP32_SIMT || o->precision > QFX_PREC_C3M_BF16X2)
      return qfx::fail(QFX_EINVAL, "unknown precision");
    const int n = c->rows * c->cols;
    Geometry geo{c->rows, c->cols, c->rows > c->cols, 0, 0};
    geo.W = geo.transposed ? c->rows : c->cols;
    geo.L = geo.transposed ? c->cols : c->rows;

    auto p = new qfx_plan;
    std::unique_ptr<qfx_plan> guard(p);
    p->rows = c->rows; p->cols = c->cols; p->n = n;
    p->x1_words = (n + 63) / 64;
    p->n_gates = (int)c->gates.size();
    p->lines = geo.W;
    p->line_len = geo.L;
    p->precision = o->precision;
    if (o->tc_flags & ~(QFX_TC_FAST_ACCUMULATION | QFX_TC_REGISTER_ROWS)) return qfx::fail(QFX_EINVAL, "unknown tc_flags bits");
    p->tc_flags = o->tc_flags;
    if (o->adjoint_store_bytes) p->adjoint_store_bytes = o->adjoint_store_bytes;
    p->transposed = geo.transposed;
    for (int line = 0; line < geo.W; ++line)
      for (int pos = 0; pos < geo.L; ++pos) p->order.push_back(geo.qubit(line, pos));

    // edges of the grid and the legs on them (two-qubit gates in time order)
    std::map<std::pair<int, int>, int> eid;
    for (int r = 0; r < c->rows; ++r)
      for (int cc = 0; cc < c->cols; ++cc) {
        int q = r * c->cols + cc;
        if (cc + 1 < c->cols) { eid[{q, q + 1}] = (int)p->edges.size(); p->edges.push_back({q, q + 1}); }
        if (r + 1 < c->rows) { eid[{q, q + c->cols}] = (int)p->edges.size(); p->edges.push_back({q, q + c->cols}); }
      }
    const int E = (int)p->edges.size();
    std::vector<std::vector<int>> legs(E);
    for (size_t gi = 0; gi < c->gates.size(); ++gi) {
      const auto& g = c->gates[gi];
      if (g.q1 < 0) continue;
      legs[eid.at({std::min(g.q0, g.q1), std::max(g.q0, g.q1)})].push_back((int)gi);
    }
    // a diagonal gate's leg is one bit of its bond, a general gate's two (its operator
    // Schmidt split has four terms); the earliest gate holds the most significant bits
    auto leg_bits = [&](int gi) { return c->gates[gi].kind == QFX_GATE_U4 ? 2 : 1; };
    p->edge_legs.resize(E);
    std::vector<int64_t> full(E), edim(E);
    for (int e = 0; e < E; ++e) {
      int bits = 0;
      for (int gi : legs[e]) bits += leg_bits(gi);
      p->edge_legs[e] = bits;
      if (bits > 40) return qfx::fail(QFX_EINVAL, "more than 40 bond bits on one edge");
      full[e] = int64_t(1) << bits;
      edim[e] = full[e];
    }
    auto edge_of = [&](int a, int b) -> int {
      if (a < 0 || b < 0) return -1;
      auto it = eid.find({std::min(a, b), std::max(a, b)});
      return it == eid.end() ? -1 : it->second;
    };
    Slots slots(n);
    for (int line = 0; line < geo.W; ++line)
      for (int pos = 0; pos < geo.L; ++pos) {
        int q = geo.qubit(line, pos);
        int up = pos > 0 ? geo.qubit(line, pos - 1) : -1;
        int left = line > 0 ? geo.qubit(line - 1, pos) : -1;
        int right = line + 1 < geo.W ? geo.qubit(line + 1, pos) : -1;
        int down = pos + 1 < geo.L ? geo.qubit(line, pos + 1) : -1;
        slots[q] = {edge_of(q, up), edge_of(q, left), edge_of(q, right), edge_of(q, down)};
      }

    // open sites
    if (o->n_open < 0 || o->n_open > qfx::kMaxOpen || o->n_open > n)
      return qfx::fail(QFX_EINVAL, "n_open must be in [0, min(24, n)]");
    std::vector<char> is_open(n, 0);
    if (o->open_sites) {
      for (int i = 0; i < o->n_open; ++i) {
        int q = o->open_sites[i];
        if (q < 0 || q >= n || is_open[q]) return qfx::fail(QFX_EINVAL, "bad or repeated open site");
        is_open[q] = 1;
        p->open_sites.push_back(q);
      }
    } else {
      for (int i = n - o->n_open; i < n; ++i) {
        is_open[p->order[i]] = 1;
        p->open_sites.push_back(p->order[i]);
      }
    }

    // forced cuts
    if (o->n_forced_cuts < 0 || (o->n_forced_cuts > 0 && !o->forced_cuts))
      return qfx::fail(QFX_EINVAL, "bad forced cut array");
    std::vector<int> cut_edges;
    for (int i = 0; i < o->n_forced_cuts; ++i) {
      const qfx_cut& k = o->forced_cuts[i];
      if (k.qa < 0 || k.qa >= n || k.qb < 0 || k.qb >= n) return qfx::fail(QFX_EINVAL, "cut qubit out of range");
      int e = edge_of(k.qa, k.qb);
      if (e < 0) return qfx::fail(QFX_EINVAL, "cut between non-neighbours");
      if (std::find(cut_edges.begin(), cut_edges.end(), e) != cut_edges.end())
        return qfx::fail(QFX_EINVAL, "edge cut twice");
      if (!is_pow2(k.size) || k.size > full[e]) return qfx::fail(QFX_EINVAL, "cut size must be a power of two <= bond dimension");
      cut_edges.push_back(e);
      edim[e] = k.size;
    }

    const bool tree = o->plan_family == 1;
    p->family = tree ? 1 : 0;
    // the tree family's site legs, in the fold's layout [up][left][x][right][down]
    std::vector<std::vector<int>> site_legs(n);
    for (int q = 0; q < n; ++q) {
      auto add_edge = [&](int e) { if (e >= 0 && full[e] > 1) site_legs[q].push_back(e); };
      add_edge(slots[q][0]);
      add_edge(slots[q][1]);
      if (is_open[q]) site_legs[q].push_back(-(1 + q));
      add_edge(slots[q][2]);
      add_edge(slots[q][3]);
    }
    SimResult sim = simulate(geo, p->order, slots, edim, is_open);
    if (!sim.ok) return qfx::fail(QFX_EPLAN, "planner: " + sim.err);
    const uint64_t cap = o->max_intermediate_bytes;
    int tree_base = 0;   // seed base of the tree planner's chosen order
    if (tree) {
      std::string terr;
      if (!qfx::tree_cut_search(site_legs, E, edim, cut_edges, cap / 8, full, &tree_base, &terr))
        return qfx::fail(QFX_EPLAN, terr);
      sim = simulate(geo, p->order, slots, edim, is_open);   // intro order of the open sites
      if (!sim.ok) return qfx::fail(QFX_EPLAN, "planner: " + sim.err);
    }
    auto slices_of = [&](const std::vector<int64_t>& dims) {
      double s = 1;
      for (int e : cut_edges) s *= (double)full[e] / (double)dims[e];
      return s;
    };
    while (!tree && cap > 0 && (uint64_t)sim.peak > cap / 8) {
      int best = -1;
      SimResult best_sim;
      double best_work = 0;
      for (int e = 0; e < E; ++e) {
        if (edim[e] < 2) continue;
        std::vector<int64_t> trial = edim;
        trial[e] /= 2;
        std::vector<int> ce = cut_edges;
        if (std::find(ce.begin(), ce.end(), e) == ce.end()) ce.push_back(e);
        double sl = 1;
        for (int x : ce) sl *= (double)full[x] / (double)trial[x];
        SimResult t = simulate(geo, p->order, slots, trial, is_open);
        if (!t.ok) continue;
        double work = t.flops * sl;
        bool better = best < 0 || t.peak < best_sim.peak ||
                      (t.peak == best_sim.peak && t.peak_count < best_sim.peak_count) ||
                      (t.peak == best_sim.peak && t.peak_count == best_sim.peak_count && work < best_work);
        if (better) { best = e; best_sim = t; best_work = work; }
      }
      if (best < 0 || (int)cut_edges.size() >= qfx::kMaxCuts)
        return qfx::fail(QFX_EPLAN, "no cut set meets max_intermediate_bytes");
      edim[best] /= 2;
      if (std::find(cut_edges.begin(), cut_edges.end(), best) == cut_edges.end()) cut_edges.push_back(best);
      sim = best_sim;
    }
    if (!tree && sim.peak > kMaxPlanElements)
      return qfx::fail(QFX_EPLAN, "largest intermediate above 2^50 elements: cut bonds or set "
                                  "max_intermediate_bytes");
    for (int e = 0; e < E; ++e)
      if (edim[e] > (int64_t(1) << 30))
        return qfx::fail(QFX_EPLAN, "a bond keeps more than 2^30 values after its cuts: cut it");
    double nsl = slices_of(edim);
    if (nsl > 4.0e18) return qfx::fail(QFX_EPLAN, "too many slices");

    // cuts in digit order
    int64_t suffix = 1;
    p->cut_dev.resize(cut_edges.size());
    for (int i = (int)cut_edges.size() - 1; i >= 0; --i) {
      int e = cut_edges[i];
      qfx::CutDev cd{};
      cd.edge = e;
      cd.size = (int32_t)edim[e];
      cd.radix = full[e] / edim[e];
      cd.suffix = suffix;
      suffix *= cd.radix;
      p->cut_dev[i] = cd;
    }
    p->n_slices = suffix;
    for (int e : cut_edges) p->cuts.push_back({p->edges[e].first, p->edges[e].second, (int32_t)edim[e]});

    // steps
    p->steps = sim.steps;
    for (auto& st : p->steps) {
      st.variant = qfx::pick_variant(st.N, st.Sd);
      // Steps with fewer than 32 columns n stay on the FP32 tiles (unless the autotuner
      // measured otherwise): the tensor-core tile splits every row of B into term planes
      // for only N outputs, and at N = 16 that split bounds it below the FP32 tiles
      // (measured ~22 against ~30 TFLOP/s).
      if (&st != &p->steps[0] && st.N >= 32 &&
          qfx::tc_eligible(p->precision, st.K, st.N, st.P * st.Sd, p->tc_flags))
        st.variant = qfx::tc_variant_of(p->precision);
    }
    if (o->autotune_cache) qfx::apply_autotune_cache(p, o->autotune_cache);
    uint64_t simage = 0;   // site image of the tensor-core steps, after the cache's choices
    for (auto& st : p->steps)
      if (st.variant >= qfx::kVariantTcBf16)
        simage = std::max(simage, qfx::tc_scratch_bytes(p->precision, st.K, st.N));
    p->max_elements = 1;
    p->flops_per_item = sim.flops;
    p->bytes_per_item = sim.bytes;
    p->largest_step = 0;
    for (size_t i = 1; i < p->steps.size(); ++i) {
      const auto& st = p->steps[i];
      p->max_elements = std::max(p->max_elements, st.P * st.N * st.Sd);
      if (st.flops > p->steps[p->largest_step].flops) p->largest_step = (int)i;
    }

    // output bit i (open_sites[i]) -> bit of the final tensor (introduction order)
    for (int q : p->open_sites) {
      auto it = std::find(sim.intro.begin(), sim.intro.end(), q);
      p->open_perm.push_back((int32_t)(it - sim.intro.begin()));
    }

    // fold program
    std::vector<int> gate_leg_bit(c->gates.size(), -1);   // lowest bit of each leg
    for (int e = 0; e < E; ++e) {
      int top = p->edge_legs[e];
      for (int gi : legs[e]) {   // time order: earliest = most significant
        top -= leg_bits(gi);
        gate_leg_bit[gi] = top;
      }
    }
    p->sites.resize(n);
    int64_t offset = 0;
    for (int q = 0; q < n; ++q) {
      qfx::FoldSite fs{};
      fs.qubit = q;
      fs.ev_begin = (int32_t)p->events.size();
      for (int k = 0; k < 4; ++k) fs.edge[k] = slots[q][k];
      auto dd = [&](int e) -> int32_t { return e < 0 ? 1 : (int32_t)edim[e]; };
      fs.dim[0] = dd(slots[q][0]);
      fs.dim[1] = dd(slots[q][1]);
      fs.dim[2] = is_open[q] ? 2 : 1;
      fs.dim[3] = dd(slots[q][2]);
      fs.dim[4] = dd(slots[q][3]);
      fs.x_open = is_open[q];
      fs.size = (int64_t)fs.dim[0] * fs.dim[1] * fs.dim[2] * fs.dim[3] * fs.dim[4];
      fs.offset = offset;
      offset += (fs.size + 63) & ~int64_t(63);
      for (size_t gi = 0; gi < c->gates.size(); ++gi) {
        const auto& g = c->gates[gi];
        if (g.q0 != q && g.q1 != q) continue;
        qfx::FoldEvent ev{};
        ev.gate = g.index;
        ev.mat = (int32_t)(p->mats.size() / 8);
        const bool general = g.kind == QFX_GATE_U4;
        if (general && q == g.q1) {
          // B_k[o1][i1] = G[2*o0 + o1][2*i0 + i1], k = 2*o0 + i0: four 2x2 matrices in a row
          for (int k = 0; k < 4; ++k)
            for (int o1 = 0; o1 < 2; ++o1)
              for (int i1 = 0; i1 < 2; ++i1) {
                const int r = 2 * (k >> 1) + o1, col = 2 * (k & 1) + i1;
                p->mats.push_back(g.m[2 * (4 * r + col)]);
                p->mats.push_back(g.m[2 * (4 * r + col) + 1]);
              }
        } else {
          p->mats.insert(p->mats.end(), g.m, g.m + 8);
        }
        if (g.q1 < 0) {
          ev.kind = qfx::EV_GATE;
        } else {
          int e = edge_of(g.q0, g.q1);
          int slot = -1;
          for (int k = 0; k < 4; ++k)
            if (slots[q][k] == e) slot = k;
          if (slot < 0) return qfx::fail(QFX_EPLAN, "planner: gate edge not a site slot");
          if (general) ev.kind = (q == g.q0) ? qfx::EV_ELEM : qfx::EV_BLOCK;
          else         ev.kind = (q == g.q0) ? qfx::EV_PROJ : qfx::EV_DIAG;
          ev.slot = slot;
          ev.bit = gate_leg_bit[gi];
        }
        p->events.push_back(ev);
      }
      fs.ev_end = (int32_t)p->events.size();
      p->sites[q] = fs;
    }
    p->site_total = offset;
    p->gate_ev.assign(2 * c->gates.size(), -1);
    for (size_t e = 0; e < p->events.size(); ++e) {
      const int g = p->events[e].gate;
      if (p->gate_ev[2 * g] < 0) p->gate_ev[2 * g] = (int32_t)e;
      else p->gate_ev[2 * g + 1] = (int32_t)e;
    }

    // workspace layout
    qfx::Layout& L = p->layout;
    L.header_per_item = align256((uint64_t)n * 8);
    if (tree) {
      // item block: the site tensors, then an arena for the tree's intermediates and the
      // permuted copies of its operands
      L.buf0 = L.buf1 = 0;
      L.sites = 0;
      const uint64_t arena = align256((uint64_t)p->site_total * 8);
      std::vector<uint64_t> site_off(n);
      for (int q = 0; q < n; ++q) site_off[q] = L.sites + (uint64_t)p->sites[q].offset * 8;
      std::vector<int> root;
      uint64_t arena_bytes = 0;
      int64_t max_el = 1;
      std::string terr;
      if (!qfx::build_tree_nodes(site_legs, edim, tree_base, site_off, arena, p->tree, &arena_bytes, &root,
                                 &max_el, &terr))
        return qfx::fail(QFX_EPLAN, terr);
      if (max_el > kMaxPlanElements)
        return qfx::fail(QFX_EPLAN, "largest intermediate above 2^50 elements: cut bonds or set "
                                    "max_intermediate_bytes");
      p->tree_final_off = p->tree.empty() ? site_off[0] : p->tree.back().offC;
      // one reported step per tree node
      p->steps.clear();
      p->flops_per_item = 0;
      p->bytes_per_item = 0;
      p->largest_step = 0;
      uint64_t tc_scratch = 0;
      for (auto& nd : p->tree) {
        nd.variant = qfx::pick_variant(nd.N, nd.Sd);
        // split-precision plans run every node the tensor-core tiles take (N >= 32, as for
        // the line sweep) on them, chunk by chunk
        if (nd.N >= 32 && qfx::tc_eligible(p->precision, nd.chunk, nd.N, nd.P * nd.Sd, p->tc_flags)) {
          nd.variant = qfx::tc_variant_of(p->precision);
          tc_scratch = std::max(tc_scratch, qfx::tc_scratch_bytes(p->precision, nd.chunk, nd.N));
        }
        // a chunked contraction with a small result: its chunks side by side in one FP32
        // launch, partial products in the item's scratch, then their sum
        nd.parts = 0;
        const int64_t out_el = nd.P * nd.N * nd.Sd, parts = nd.K / nd.chunk;
        if (nd.chunk < nd.K && nd.K % nd.chunk == 0 && nd.P == 1 && out_el <= qfx::kTreeSplitOut &&
            parts <= 65535 && (uint64_t)parts * (uint64_t)out_el * 8 <= qfx::kTreeSplitBytes) {
          nd.variant = qfx::pick_variant(nd.N, nd.Sd);
          nd.parts = (int32_t)parts;
          tc_scratch = std::max(tc_scratch, (uint64_t)parts * (uint64_t)out_el * 8);
        }
        qfx::Step st{};
        st.site = nd.out;
        st.variant = nd.variant;
        st.P = nd.P; st.K = nd.K; st.N = nd.N; st.NL = nd.NL; st.Sd = nd.Sd;
        st.flops = nd.flops;
        st.bytes = nd.bytes;
        st.parts = nd.parts;
        p->flops_per_item += nd.flops;
        p->bytes_per_item += nd.bytes;
        p->steps.push_back(st);
        if (st.flops > p->steps[p->largest_step].flops) p->largest_step = (int)p->steps.size() - 1;
      }
      p->max_elements = max_el;
      // output bit i -> bit of the root tensor's index (its last leg is the lowest bit)
      p->open_perm.clear();
      for (int q : p->open_sites) {
        const auto it = std::find(root.begin(), root.end(), -(1 + q));
        if (it == root.end()) return qfx::fail(QFX_EPLAN, "tree planner: open site missing from the result");
        p->open_perm.push_back((int32_t)(root.size() - 1 - (it - root.begin())));
      }
      if (root.size() != p->open_sites.size()) return qfx::fail(QFX_EPLAN, "tree planner: bond left open");
      L.simage = arena + arena_bytes;
      L.item_bytes = L.simage + align256(tc_scratch);
    } else {
      L.buf0 = 0;
      L.buf1 = align256((uint64_t)p->max_elements * 8);
      L.sites = L.buf1 + align256((uint64_t)p->max_elements * 8);
      L.simage = L.sites + align256((uint64_t)p->site_total * 8);
      L.item_bytes = L.simage + align256(simage);
    }
    qfx::build_table_image(p);
    *out = guard.release();
    return QFX_OK;
  } catch (const std::exception& e) {
    return qfx::fail(QFX_EINVAL, std::string("qfx_plan_create: ") + e.what());
  }
}

extern "C" qfx_status qfx_plan_info(const qfx_plan* p, qfx_plan_stats* s) {
  if (!p || !s) return qfx::fail(QFX_EINVAL, "qfx_plan_info: NULL argument");
  std::memset(s, 0, sizeof(*s));
  s->n_slices = p->n_slices;
  s->n_steps = (int32_t)p->steps.size();
  s->n_open = (int32_t)p->open_sites.size();
  s->n_cuts = (int32_t)p->cuts.size();
  s->n_sites = p->n;
  s->flops_per_item = p->flops_per_item;
  s->bytes_per_item = p->bytes_per_item;
  s->max_elements = p->max_elements;
  s->item_bytes = p->layout.item_bytes;
  s->workspace_min = qfx_workspace_bytes(p, 1);
  s->largest_step = p->largest_step;
  s->precision = p->precision;
  s->x1_words = p->x1_words;
  return QFX_OK;
}

extern "C" uint64_t qfx_workspace_bytes(const qfx_plan* p, int64_t n_concurrent) {
  if (!p || n_concurrent < 1) return 0;
  return qfx::table_bytes(p) + align256((uint64_t)n_concurrent * p->layout.header_per_item) +
         (uint64_t)n_concurrent * p->layout.item_bytes;
}

extern "C" qfx_status qfx_plan_step(const qfx_plan* p, int32_t i, qfx_step_info* out) {
  if (!p || !out || i < 0 || i >= (int32_t)p->steps.size())
    return qfx::fail(QFX_EINVAL, "qfx_plan_step: bad argument");
  const auto& s = p->steps[i];
  out->site = s.site;
  out->variant = s.variant;
  out->P = s.P; out->K = s.K; out->N = s.N; out->NL = s.NL; out->Sd = s.Sd;
  out->flops = s.flops;
  out->bytes = s.bytes;
  out->parts = s.parts;
  out->reserved = 0;
  return QFX_OK;
}

extern "C" qfx_status qfx_plan_cut(const qfx_plan* p, int32_t i, qfx_cut* out) {
  if (!p || !out || i < 0 || i >= (int32_t)p->cuts.size())
    return qfx::fail(QFX_EINVAL, "qfx_plan_cut: bad argument");
  *out = p->cuts[i];
  return QFX_OK;
}

extern "C" qfx_status qfx_plan_open_sites(const qfx_plan* p, int32_t* out) {
  if (!p || (!out && !p->open_sites.empty())) return qfx::fail(QFX_EINVAL, "qfx_plan_open_sites: NULL argument");
  for (size_t i = 0; i < p->open_sites.size(); ++i) out[i] = p->open_sites[i];
  return QFX_OK;
}

extern "C" void qfx_plan_destroy(qfx_plan* p) {
  if (!p) return;
  qfx::free_table_image(p);
  delete p;
}
