// Contraction-tree plans ("region" plans, plan family 1).
//
// The line sweep absorbs one site per step, so every column's boundary is a separator of
// the grid and a memory cap needs cut bits in every one of them (2^59 slices for
// 7x7x(1+40+1) at 8 GiB).  Sec. III (Fig. 3) instead contracts regions into tensors of
// bounded rank, combines the region tensors with few high-arithmetic-intensity
// contractions and absorbs the rest site by site; the cuts (Sec. III.A) are chosen so that
// every intermediate fits.  This planner builds such a tree greedily:
//   - order: repeatedly contract the connected pair whose result grows least over its
//     larger operand (log2 sizes; ties: the smaller result, then the lower tensor ids);
//     when no pair shares a bond (everything cut apart) the two smallest tensors are
//     multiplied;
//   - cuts: while the largest intermediate exceeds the cap, halve the bond of the largest
//     intermediates whose halving gives the lowest largest intermediate, then the least
//     total work (slices x flops per slice), rebuilding the order for each trial; then
//     double back, one at a time, the halvings that the later ones made unnecessary, as
//     long as the total work drops;
//   - every order is the best of greedy runs with small and with larger random
//     perturbations of the score (the larger ones only where they keep the largest tensor);
//   - the whole search runs from several seed bases and keeps the least total work.
// Each tree node is one TTGT contraction (Sec. III.E) run by the same GEMM kernel as the
// line sweep, C[nh][p][nl][s] = sum_k S[k][nh*NL + nl] B[p][k][s] with NL = N: the larger
// operand is B; when its shared legs are adjacent it is used in place (P = legs before,
// Sd = legs after, the result keeps its leg order with the shared legs replaced by the
// other operand's free legs); otherwise it is permuted to [shared][free] first.  The
// smaller operand is permuted to [shared, in B's order][free] unless it already is.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>

#include "qfx_internal.h"

namespace qfx {
namespace {

constexpr int64_t kSatT = int64_t(1) << 62;
int64_t tmul(int64_t a, int64_t b) { return a > kSatT / b ? kSatT : std::min(a * b, kSatT); }
uint64_t a256t(uint64_t x) { return (x + 255) & ~uint64_t(255); }

struct Pair { int a, b; };

}  // namespace

// Greedy contraction order of the network given each site's legs and the leg dims.
// Fills `pairs` (tensor ids; intermediates numbered from n in creation order) and returns
// the largest tensor (elements, saturating) and the Eq. 1 flops of the tree.  Every bond
// joins two tensors, so the candidate pairs of a step are found through the bonds of the
// live tensors (owner[x] = its two endpoints), not among all pairs.
static void greedy_tree_seed(const std::vector<std::vector<int>>& site_legs,
                             const std::function<int64_t(int)>& dim, uint64_t seed,
                             std::vector<Pair>& pairs, int64_t* peak, double* flops,
                             double noise = 0.02) {
  const int n = (int)site_legs.size();
  std::vector<std::vector<int>> legs(site_legs);
  legs.reserve(2 * (size_t)n);
  int maxleg = -1;
  for (const auto& l : site_legs)
    for (int x : l) maxleg = std::max(maxleg, x);
  std::vector<double> ld(maxleg + 1);   // log2 dim per bond (open legs: 1)
  std::vector<int> own0(maxleg + 1, -1), own1(maxleg + 1, -1);
  for (int x = 0; x <= maxleg; ++x) ld[x] = std::log2((double)dim(x));
  auto ldim = [&](int x) { return x < 0 ? 1.0 : ld[x]; };
  for (int t = 0; t < n; ++t)
    for (int x : legs[t])
      if (x >= 0) (own0[x] < 0 ? own0[x] : own1[x]) = t;
  auto other = [&](int x, int t) { return own0[x] == t ? own1[x] : own0[x]; };
  std::vector<double> lsz;   // log2 size per tensor
  for (auto& l : legs) {
    double sz = 0;
    for (int x : l) sz += ldim(x);
    lsz.push_back(sz);
  }
  std::vector<char> alive(n, 1);
  int n_alive = n;
  *peak = 1;
  for (auto& l : legs) {
    int64_t e = 1;
    for (int x : l) e = tmul(e, dim(x));
    *peak = std::max(*peak, e);
  }
  *flops = 0;
  pairs.clear();
  while (n_alive > 1) {
    int ta = -1, tb = -1;
    double best = 0, best_out = 0;
    for (int t = 0; t < (int)legs.size(); ++t) {
      if (!alive[t]) continue;
      for (int x : legs[t]) {
        if (x < 0) continue;
        const int u = other(x, t);
        if (u < t || !alive[u]) continue;   // each pair from its lower id
        double shared = 0;
        bool seen = false, first = true;   // evaluate the pair once: at its first shared bond
        for (int y : legs[t]) {
          if (y < 0 || other(y, t) != u) continue;
          if (!seen && y != x) { first = false; break; }
          seen = true;
          shared += ldim(y);
        }
        if (!first) continue;
        const double out = lsz[t] + lsz[u] - 2 * shared;
        double score = out - std::max(lsz[t], lsz[u]);
        if (seed) {   // a deterministic perturbation per seed
          uint64_t h = seed * 0x9E3779B97F4A7C15ull ^ ((uint64_t)t << 32 ^ (uint64_t)u);
          h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29;
          score += noise * (double)(h >> 11) / 9007199254740992.0;
        }
        if (ta < 0 || score < best - 1e-9 || (std::fabs(score - best) <= 1e-9 && out < best_out - 1e-9)) {
          ta = t; tb = u; best = score; best_out = out;
        }
      }
    }
    if (ta < 0) {   // nothing shares a bond: multiply the two smallest
      for (int t = 0; t < (int)legs.size(); ++t) {
        if (!alive[t]) continue;
        if (ta < 0 || lsz[t] < lsz[ta]) { tb = ta; ta = t; }
        else if (tb < 0 || lsz[t] < lsz[tb]) tb = t;
      }
      if (ta > tb) std::swap(ta, tb);
    }
    std::vector<int> out;
    int64_t k = 1, eo = 1;
    for (int x : legs[ta]) {
      if (x >= 0 && other(x, ta) == tb) k = tmul(k, dim(x));
      else out.push_back(x);
    }
    for (int x : legs[tb])
      if (!(x >= 0 && other(x, tb) == ta)) out.push_back(x);
    for (int x : out) eo = tmul(eo, dim(x));
    *peak = std::max(*peak, eo);
    *flops += 8.0 * (double)eo * (double)k;
    pairs.push_back({ta, tb});
    const int c = (int)legs.size();
    for (int x : out)
      if (x >= 0) {
        if (own0[x] == ta || own0[x] == tb) own0[x] = c;
        else own1[x] = c;
      }
    double sz = 0;
    for (int x : out) sz += ldim(x);
    legs.push_back(std::move(out));
    lsz.push_back(sz);
    alive[ta] = alive[tb] = 0;
    alive.push_back(1);
    --n_alive;
  }
}

// The order used: the best, by largest tensor then flops, of the plain greedy order and
// kTreeSeeds perturbed ones (deterministic).
constexpr int kTreeSeeds = 8;
static void greedy_tree(const std::vector<std::vector<int>>& site_legs,
                        const std::function<int64_t(int)>& dim, std::vector<Pair>& pairs,
                        int64_t* peak, double* flops, uint64_t base) {
  greedy_tree_seed(site_legs, dim, 0, pairs, peak, flops);
  for (int sd = 1; sd <= kTreeSeeds; ++sd) {
    std::vector<Pair> pp;
    int64_t pk;
    double fl;
    greedy_tree_seed(site_legs, dim, (uint64_t)sd + 16 * base, pp, &pk, &fl);
    if (pk < *peak || (pk == *peak && fl < *flops)) { pairs.swap(pp); *peak = pk; *flops = fl; }
  }
}

// Polish of an order: greedy orders with larger perturbations of the score (up to 0.25,
// 0.5 or 1 in log2 units, `seeds` of them, deterministic) may find fewer flops for the
// same cuts; one is kept when its largest tensor is no larger than the order's.
constexpr int kPolishSeeds = 48;
static void polish_tree(const std::vector<std::vector<int>>& site_legs, const std::function<int64_t(int)>& dim,
                        std::vector<Pair>& pairs, int64_t* peak, double* flops, uint64_t base) {
  static const double amp[3] = {0.25, 0.5, 1.0};
  for (int sd = 0; sd < kPolishSeeds; ++sd) {
    std::vector<Pair> pp;
    int64_t pk;
    double fl;
    greedy_tree_seed(site_legs, dim, (uint64_t)(1000 + sd) + 64 * base, pp, &pk, &fl, amp[sd % 3]);
    if (pk <= *peak && fl < *flops) { pairs.swap(pp); *peak = pk; *flops = fl; }
  }
}

// One cut search from the caller's dims with the orders of seed base `base`; *work_out is
// the total work (flops per slice x slices) of the final polished order.
static bool cut_search_once(const std::vector<std::vector<int>>& site_legs, int n_edges,
                            std::vector<int64_t>& edim, std::vector<int>& cut_edges, uint64_t cap_elems,
                            const std::vector<int64_t>& full, uint64_t base, std::string* err,
                            double* work_out) {
  auto dimf = [&](int x) -> int64_t { return x < 0 ? 2 : edim[x]; };
  const std::vector<int64_t> entry = edim;          // the caller's (forced) cuts stay
  const size_t n_entry = cut_edges.size();
  std::vector<Pair> pairs;
  int64_t peak;
  double flops;
  greedy_tree(site_legs, dimf, pairs, &peak, &flops, base);
  int guard = 0;
  while (cap_elems > 0 && (uint64_t)peak > cap_elems) {
    if (++guard > 400) { *err = "tree planner: no cut set found"; return false; }
    // candidate bonds: those of the largest intermediates
    std::vector<std::vector<int>> legs(site_legs);
    std::vector<int> cand;
    for (const auto& pr : pairs) {
      std::vector<int> out;
      for (int x : legs[pr.a])
        if (std::find(legs[pr.b].begin(), legs[pr.b].end(), x) == legs[pr.b].end()) out.push_back(x);
      for (int x : legs[pr.b])
        if (std::find(legs[pr.a].begin(), legs[pr.a].end(), x) == legs[pr.a].end()) out.push_back(x);
      int64_t e = 1;
      for (int x : out) e = tmul(e, dimf(x));
      if (e == peak)
        for (int x : out)
          if (x >= 0 && edim[x] >= 2 && std::find(cand.begin(), cand.end(), x) == cand.end()) cand.push_back(x);
      legs.push_back(out);
    }
    for (const auto& l : site_legs) {   // a site tensor itself can be the largest
      int64_t e = 1;
      for (int x : l) e = tmul(e, dimf(x));
      if (e == peak)
        for (int x : l)
          if (x >= 0 && edim[x] >= 2 && std::find(cand.begin(), cand.end(), x) == cand.end()) cand.push_back(x);
    }
    if (cand.empty()) { *err = "tree planner: the largest tensor has no bond left to cut"; return false; }
    int best = -1;
    int64_t best_peak = 0;
    double best_work = 0;
    for (int x : cand) {
      edim[x] /= 2;
      std::vector<Pair> pp;
      int64_t pk;
      double fl;
      greedy_tree(site_legs, dimf, pp, &pk, &fl, base);
      polish_tree(site_legs, dimf, pp, &pk, &fl, base);
      double slices = 1;
      for (int e = 0; e < n_edges; ++e) slices *= (double)full[e] / (double)edim[e];
      const double work = fl * slices;
      if (best < 0 || pk < best_peak || (pk == best_peak && work < best_work)) {
        best = x; best_peak = pk; best_work = work;
      }
      edim[x] *= 2;
    }
    edim[best] /= 2;
    if (std::find(cut_edges.begin(), cut_edges.end(), best) == cut_edges.end()) cut_edges.push_back(best);
    greedy_tree(site_legs, dimf, pairs, &peak, &flops, base);
    polish_tree(site_legs, dimf, pairs, &peak, &flops, base);
  }
  // undo halvings that later ones made unnecessary: double a bond this search cut back
  // while some order still fits the cap with less total work, the largest gain first
  auto total_work = [&](double fl) {
    double slices = 1;
    for (int e = 0; e < n_edges; ++e) slices *= (double)full[e] / (double)edim[e];
    return fl * slices;
  };
  if (cap_elems > 0) {
    double work = total_work(flops);
    for (int pass = 0; pass < 64; ++pass) {
      int best = -1;
      double best_work = work;
      for (int x : cut_edges) {
        if (edim[x] >= entry[x]) continue;
        edim[x] *= 2;
        std::vector<Pair> pp;
        int64_t pk;
        double fl;
        greedy_tree(site_legs, dimf, pp, &pk, &fl, base);
        polish_tree(site_legs, dimf, pp, &pk, &fl, base);
        const double w = total_work(fl);
        if ((uint64_t)pk <= cap_elems && w < best_work) { best = x; best_work = w; }
        edim[x] /= 2;
      }
      if (best < 0) break;
      edim[best] *= 2;
      work = best_work;
    }
    cut_edges.erase(std::remove_if(cut_edges.begin() + (std::ptrdiff_t)n_entry, cut_edges.end(),
                                   [&](int x) { return edim[x] >= entry[x]; }),
                    cut_edges.end());
  }
  greedy_tree(site_legs, dimf, pairs, &peak, &flops, base);   // the order build_tree_nodes makes
  polish_tree(site_legs, dimf, pairs, &peak, &flops, base);
  *work_out = total_work(flops);
  return true;
}

// The cut search from kStarts seed bases (each a different family of perturbed orders: the
// searches diverge after their first different choice); the one with the least total work
// is kept, and its base, which build_tree_nodes needs to rebuild the same order.
constexpr int kStarts = 8;
bool tree_cut_search(const std::vector<std::vector<int>>& site_legs, int n_edges,
                     std::vector<int64_t>& edim, std::vector<int>& cut_edges, uint64_t cap_elems,
                     const std::vector<int64_t>& full, int* base_out, std::string* err) {
  bool found = false;
  double best_work = 0;
  std::vector<int64_t> best_dim;
  std::vector<int> best_cuts;
  std::string last_err;
  for (int b = 0; b < kStarts; ++b) {
    std::vector<int64_t> d = edim;
    std::vector<int> c = cut_edges;
    double w = 0;
    std::string e;
    if (!cut_search_once(site_legs, n_edges, d, c, cap_elems, full, (uint64_t)b, &e, &w)) {
      last_err = e;
      continue;
    }
    if (!found || w < best_work) {
      found = true;
      best_work = w;
      best_dim = d;
      best_cuts = c;
      *base_out = b;
    }
  }
  if (!found) {
    *err = last_err;
    return false;
  }
  edim = best_dim;
  cut_edges = best_cuts;
  return true;
}

// Leg orders, kernel shapes, permutes and the arena layout of the tree for the final dims.
// Fuses a permute (input shape, out axis a = input axis ord[a]): axes of extent 1 are
// dropped and output axes that are consecutive input axes in order are merged.  Returns
// false when more than kTreeMaxRank axes remain.
static bool fuse_perm(const std::vector<int64_t>& shape, const std::vector<int>& ord, int* rank,
                      int64_t* fshape, int32_t* ford) {
  std::vector<int> keep;                       // input axes of extent > 1, kept in output order
  for (int a : ord)
    if (shape[a] > 1) keep.push_back(a);
  // runs of consecutive input axes in the output order
  std::vector<std::pair<int, int>> runs;       // [first input axis, last input axis]
  for (int a : keep) {
    if (!runs.empty() && runs.back().second + 1 == a) {
      // the next kept input axis after runs.back().second must be `a` (skip extent-1 axes)
      runs.back().second = a;
    } else {
      runs.push_back({a, a});
    }
  }
  // extent-1 input axes between fused ones do not matter; re-index the runs by input order
  std::vector<int> firsts;
  for (auto& r : runs) firsts.push_back(r.first);
  std::vector<int> sorted = firsts;
  std::sort(sorted.begin(), sorted.end());
  const int R = (int)runs.size();
  if (R > kTreeMaxRank) return false;
  if (R == 0) { *rank = 1; fshape[0] = 1; ford[0] = 0; return true; }
  for (int j = 0; j < R; ++j) {      // input shape of the fused tensor, in input order
    const int i = (int)(std::find(firsts.begin(), firsts.end(), sorted[j]) - firsts.begin());
    int64_t e = 1;
    for (int a = runs[i].first; a <= runs[i].second; ++a) e *= shape[a];
    fshape[j] = e;
  }
  for (int i = 0; i < R; ++i)        // output axis i is fused input axis rank-of(runs[i])
    ford[i] = (int32_t)(std::find(sorted.begin(), sorted.end(), runs[i].first) - sorted.begin());
  *rank = R;
  return true;
}

bool build_tree_nodes(const std::vector<std::vector<int>>& site_legs, const std::vector<int64_t>& edim,
                      int base, const std::vector<uint64_t>& site_off, uint64_t arena_base,
                      std::vector<TreeNode>& nodes, uint64_t* arena_bytes,
                      std::vector<int>* root_legs, int64_t* max_el, std::string* err) {
  auto dimf = [&](int x) -> int64_t { return x < 0 ? 2 : edim[x]; };
  const int n = (int)site_legs.size();
  std::vector<Pair> pairs;
  int64_t peak;
  double flops;
  greedy_tree(site_legs, dimf, pairs, &peak, &flops, (uint64_t)base);
  polish_tree(site_legs, dimf, pairs, &peak, &flops, (uint64_t)base);
  *max_el = peak;
  std::vector<std::vector<int>> legs(site_legs);
  auto elems = [&](const std::vector<int>& l) {
    int64_t e = 1;
    for (int x : l) e = tmul(e, dimf(x));
    return e;
  };
  // arena: first-fit over [offset, size) blocks
  struct Blk { uint64_t off, size; };
  std::vector<Blk> used;
  uint64_t top = 0;
  auto alloc = [&](uint64_t size) -> uint64_t {
    size = a256t(std::max<uint64_t>(size, 256));
    std::sort(used.begin(), used.end(), [](const Blk& x, const Blk& y) { return x.off < y.off; });
    uint64_t cur = 0;
    for (const auto& b : used) {
      if (b.off >= cur + size) break;
      cur = std::max(cur, b.off + b.size);
    }
    used.push_back({cur, size});
    top = std::max(top, cur + size);
    return cur;
  };
  auto release = [&](uint64_t off) {
    for (size_t i = 0; i < used.size(); ++i)
      if (used[i].off == off) { used.erase(used.begin() + i); return; }
  };
  std::vector<uint64_t> where(site_off);   // byte offset per tensor; sites: in the site region
  std::vector<char> in_arena(n, 0);
  nodes.clear();
  for (const auto& pr : pairs) {
    int ta = pr.a, tb = pr.b;
    if (elems(legs[ta]) > elems(legs[tb])) std::swap(ta, tb);   // B is the larger operand
    const auto& la = legs[ta];
    const auto& lb = legs[tb];
    std::vector<int> shared, afree, bpos;
    for (size_t i = 0; i < lb.size(); ++i)
      if (std::find(la.begin(), la.end(), lb[i]) != la.end()) { shared.push_back(lb[i]); bpos.push_back((int)i); }
    for (int x : la)
      if (std::find(lb.begin(), lb.end(), x) == lb.end()) afree.push_back(x);
    TreeNode nd{};
    nd.a = ta;
    nd.b = tb;
    // a chunked contraction needs B as [shared][free] (P = 1): its chunks are row ranges
    const bool chunked = [&] {
      int64_t k = 1;
      for (int x : shared) k = tmul(k, dimf(x));
      return k > kTreeChunk;
    }();
    const bool adjacent = shared.empty() ||
                          (bpos.back() - bpos.front() + 1 == (int)bpos.size() && (!chunked || bpos.front() == 0));
    std::vector<int> outl;
    int64_t P = 1, Sd = 1;
    if (adjacent) {
      const int lo = shared.empty() ? 0 : bpos.front(), hi = shared.empty() ? 0 : bpos.back() + 1;
      for (int i = 0; i < lo; ++i) { P = tmul(P, dimf(lb[i])); outl.push_back(lb[i]); }
      for (int x : afree) outl.push_back(x);
      for (int i = hi; i < (int)lb.size(); ++i) { Sd = tmul(Sd, dimf(lb[i])); outl.push_back(lb[i]); }
      nd.permB = 0;
    } else {
      // B -> [shared][free]
      std::vector<int> bord;   // new order as indices into lb
      for (int p : bpos) bord.push_back(p);
      for (int i = 0; i < (int)lb.size(); ++i)
        if (std::find(bpos.begin(), bpos.end(), i) == bpos.end()) { bord.push_back(i); Sd = tmul(Sd, dimf(lb[i])); }
      nd.permB = 1;
      std::vector<int64_t> shp;
      for (int x : lb) shp.push_back(dimf(x));
      if (!fuse_perm(shp, bord, &nd.rankB, nd.shapeB, nd.ordB)) {
        *err = "tree planner: a permute needs more than 10 fused axes";
        return false;
      }
      for (int x : afree) outl.push_back(x);
      for (int i = (int)shared.size(); i < (int)bord.size(); ++i) outl.push_back(lb[bord[i]]);
    }
    // A -> [shared in B's order][free in A's order]
    std::vector<int> aord;
    for (int x : shared) aord.push_back((int)(std::find(la.begin(), la.end(), x) - la.begin()));
    for (int i = 0; i < (int)la.size(); ++i)
      if (std::find(shared.begin(), shared.end(), la[i]) == shared.end()) aord.push_back(i);
    bool ident = true;
    for (int i = 0; i < (int)aord.size(); ++i) ident = ident && aord[i] == i;
    nd.permA = 0;
    if (!ident) {
      std::vector<int64_t> shp;
      for (int x : la) shp.push_back(dimf(x));
      if (!fuse_perm(shp, aord, &nd.rankA, nd.shapeA, nd.ordA)) {
        *err = "tree planner: a permute needs more than 10 fused axes";
        return false;
      }
      bool fid = true;   // fused to the identity (only extent-1 axes moved)
      for (int i = 0; i < nd.rankA; ++i) fid = fid && nd.ordA[i] == i;
      nd.permA = fid ? 0 : 1;
    }
    int64_t K = 1, N = 1;
    for (int x : shared) K = tmul(K, dimf(x));
    for (int x : afree) N = tmul(N, dimf(x));
    nd.P = P; nd.K = K; nd.N = N; nd.NL = N; nd.Sd = Sd;
    nd.chunk = K;
    if (K > kTreeChunk) {
      if (P != 1 || K % kTreeChunk) { *err = "tree planner: a chunked contraction is not in [shared][free] form"; return false; }
      nd.chunk = kTreeChunk;
    }
    nd.flops = 8.0 * (double)P * (double)K * (double)N * (double)Sd;
    nd.bytes = 8.0 * ((double)P * K * Sd + (double)K * N + (double)P * N * Sd);
    // memory: scratch copies, then the result; operands released afterwards
    nd.offA = where[ta];
    nd.offB = where[tb];
    const uint64_t sa = nd.permA ? alloc((uint64_t)elems(la) * 8) : 0;
    const uint64_t sb = nd.permB ? alloc((uint64_t)elems(lb) * 8) : 0;
    const uint64_t oc = alloc((uint64_t)elems(outl) * 8);
    nd.offA2 = nd.permA ? arena_base + sa : nd.offA;
    nd.offB2 = nd.permB ? arena_base + sb : nd.offB;
    nd.offC = arena_base + oc;
    if (nd.permA) release(sa);
    if (nd.permB) release(sb);
    if (ta >= n && in_arena[ta]) release(where[ta] - arena_base);
    if (tb >= n && in_arena[tb]) release(where[tb] - arena_base);
    // every access of the node stays inside its tensors (checked here, before any launch)
    const int64_t ea = elems(la), eb = elems(lb), ec = elems(outl);
    if (tmul(K, N) != ea || tmul(tmul(P, K), Sd) != eb || tmul(tmul(P, N), Sd) != ec) {
      *err = "tree planner: inconsistent step shape";
      return false;
    }
    legs.push_back(outl);
    where.push_back(arena_base + oc);
    in_arena.push_back(1);
    nd.out = (int)legs.size() - 1;
    nodes.push_back(nd);
  }
  *arena_bytes = a256t(top);
  // operand, scratch and result regions inside the site region or the arena
  for (const auto& nd : nodes) {
    const uint64_t end = arena_base + *arena_bytes;
    const uint64_t ra = (uint64_t)tmul(nd.K, nd.N) * 8, rb = (uint64_t)tmul(tmul(nd.P, nd.K), nd.Sd) * 8;
    const uint64_t rc = (uint64_t)tmul(tmul(nd.P, nd.N), nd.Sd) * 8;
    if (nd.offA + ra > end || nd.offA2 + ra > end || nd.offB + rb > end || nd.offB2 + rb > end ||
        nd.offC < arena_base || nd.offC + rc > end) {
      *err = "tree planner: a tensor leaves the work item's block";
      return false;
    }
  }
  *root_legs = legs.back();
  if (pairs.empty()) *root_legs = site_legs[0];
  return true;
}

}  // namespace qfx
