// Host side of the method: the tensor network of the QAOA ansatz, its line
// graph, greedy elimination orders and the step-dependent slicing search.
//
//  * Network: Sec. III.A (ansatz), Sec. IV.A (gates as tensors, Table I),
//    Sec. IV.B (line graph with diagonal gates, Fig. 2).
//  * Greedy order and width: Sec. IV.B (elimination, c = max N_G(v)), Sec. V.A.1.
//  * Slicing: Sec. VI.C (late parallelisation), Sec. VI.D (step-dependent
//    slicing, Fig. 8), Alg. 1 (max-degree vertices removed one at a time).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "qt_internal.h"

namespace qt {

// ------------------------------- BitGraph ----------------------------------
void BitGraph::init(int nv) {
  n = nv;
  W = (nv + 63) / 64;
  if (W == 0) W = 1;
  rows.assign((size_t)n * W, 0ull);
  alive.assign(n, 1);
}

void BitGraph::add_edge(int a, int b) {
  if (a == b) return;
  row(a)[b >> 6] |= 1ull << (b & 63);
  row(b)[a >> 6] |= 1ull << (a & 63);
}

int BitGraph::degree(int v) const {
  const uint64_t* r = row(v);
  int d = 0;
  for (int w = 0; w < W; ++w) d += __builtin_popcountll(r[w]);
  return d;
}

int BitGraph::eliminate(int v) {
  uint64_t* rv = row(v);
  int d = 0;
  for (int w = 0; w < W; ++w) {
    uint64_t bits = rv[w];
    while (bits) {
      int a = w * 64 + __builtin_ctzll(bits);
      bits &= bits - 1;
      ++d;
      uint64_t* ra = row(a);
      for (int x = 0; x < W; ++x) ra[x] |= rv[x];
      ra[a >> 6] &= ~(1ull << (a & 63));
      ra[v >> 6] &= ~(1ull << (v & 63));
    }
  }
  std::memset(rv, 0, sizeof(uint64_t) * W);
  alive[v] = 0;
  return d;
}

void BitGraph::remove(int v) {
  uint64_t* rv = row(v);
  for (int w = 0; w < W; ++w) {
    uint64_t bits = rv[w];
    while (bits) {
      int a = w * 64 + __builtin_ctzll(bits);
      bits &= bits - 1;
      row(a)[v >> 6] &= ~(1ull << (v & 63));
    }
  }
  std::memset(rv, 0, sizeof(uint64_t) * W);
  alive[v] = 0;
}

BitGraph line_graph(const std::vector<Tensor>& tensors, int n_vars) {
  BitGraph g;
  g.init(n_vars);
  for (const Tensor& t : tensors)
    for (size_t i = 0; i < t.labels.size(); ++i)
      for (size_t j = i + 1; j < t.labels.size(); ++j) g.add_edge(t.labels[i], t.labels[j]);
  return g;
}

BitGraph network_graph(const qt_net* net) {
  BitGraph g = line_graph(net->tensors, net->n_vars);
  const int a = (int)net->open.size();
  if (a > 0) {
    const int first = net->n_vars - a;
    g.keep.assign(g.n, 0);
    for (int j = 0; j < a; ++j) {
      g.keep[first + j] = 1;
      for (int t = j + 1; t < a; ++t) g.add_edge(first + j, first + t);
    }
  }
  return g;
}

// ------------------------------- greedy ------------------------------------
// Number of missing edges among v's neighbours (the fill-in of eliminating v).
static int64_t fill_in(const BitGraph& g, int v, int deg) {
  const uint64_t* rv = g.row(v);
  int64_t twice_edges = 0;
  for (int w = 0; w < g.W; ++w) {
    uint64_t bits = rv[w];
    while (bits) {
      int a = w * 64 + __builtin_ctzll(bits);
      bits &= bits - 1;
      const uint64_t* ra = g.row(a);
      for (int x = 0; x < g.W; ++x) twice_edges += __builtin_popcountll(ra[x] & rv[x]);
    }
  }
  return (int64_t)deg * (deg - 1) / 2 - twice_edges / 2;
}

OrderResult greedy_order(const BitGraph& g0, int algo) {
  BitGraph g = g0;
  OrderResult res;
  const int n = g.n;
  std::vector<int64_t> deg(n, 0), fill(n, 0);
  int remaining = 0;
  for (int v = 0; v < n; ++v) {
    if (!g.alive[v]) continue;
    remaining += g.takeable(v);
    deg[v] = g.degree(v);
    if (algo == QT_GREEDY_MINFILL) fill[v] = fill_in(g, v, (int)deg[v]);
  }
  res.order.reserve(remaining);
  res.widths.reserve(remaining);
  std::vector<uint64_t> dirty(g.W);
  std::vector<int> nb;
  while (remaining > 0) {
    int best = -1;
    for (int v = 0; v < n; ++v) {
      if (!g.takeable(v)) continue;
      if (best < 0) { best = v; continue; }
      bool better;
      if (algo == QT_GREEDY_MINFILL)
        better = fill[v] < fill[best] || (fill[v] == fill[best] && deg[v] < deg[best]);
      else
        better = deg[v] < deg[best];
      if (better) best = v;  // ties keep the smaller id (scan is ascending)
    }
    // neighbours of best before elimination
    nb.clear();
    const uint64_t* rb = g.row(best);
    for (int w = 0; w < g.W; ++w) {
      uint64_t bits = rb[w];
      while (bits) {
        nb.push_back(w * 64 + __builtin_ctzll(bits));
        bits &= bits - 1;
      }
    }
    res.order.push_back(best);
    res.widths.push_back((int32_t)nb.size());
    g.eliminate(best);
    --remaining;
    if (algo == QT_GREEDY_MINFILL) {
      std::fill(dirty.begin(), dirty.end(), 0ull);
      for (int a : nb) {
        dirty[a >> 6] |= 1ull << (a & 63);
        const uint64_t* ra = g.row(a);
        for (int x = 0; x < g.W; ++x) dirty[x] |= ra[x];
      }
      for (int w = 0; w < g.W; ++w) {
        uint64_t bits = dirty[w];
        while (bits) {
          int a = w * 64 + __builtin_ctzll(bits);
          bits &= bits - 1;
          if (!g.alive[a]) continue;
          deg[a] = g.degree(a);
          fill[a] = fill_in(g, a, (int)deg[a]);
        }
      }
    } else {
      for (int a : nb) deg[a] = g.degree(a);
    }
  }
  return res;
}

// ------------------------- randomised greedy --------------------------------
// rgreedy (Sec. V.A.2): every step draws the next vertex with probability
// proportional to exp(-N_G(v)/tau); best of q runs. Weights are shifted by the
// step's smallest degree, r^(d - d_min) with r = exp(-1/tau), the power taken
// by repeated multiplication; one uniform draw per step from a SplitMix64
// stream (Steele, Lea, Flood, OOPSLA 2014) seeded with `seed`; the vertex taken
// is the first, in ascending id, whose running weight sum exceeds u * total.
namespace {
struct SplitMix64 {
  uint64_t s;
  double uniform() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  }
};

OrderResult rgreedy_run(const BitGraph& g0, const std::vector<double>& pw, SplitMix64& rng) {
  BitGraph g = g0;
  OrderResult res;
  const int n = g.n;
  std::vector<int> deg(n, 0), cand;
  std::vector<double> w;
  int remaining = 0;
  for (int v = 0; v < n; ++v)
    if (g.alive[v]) {
      deg[v] = g.degree(v);
      remaining += g.takeable(v);
    }
  std::vector<int> nb;
  while (remaining > 0) {
    cand.clear();
    int dmin = 1 << 30;
    for (int v = 0; v < n; ++v)
      if (g.takeable(v)) {
        cand.push_back(v);
        dmin = std::min(dmin, deg[v]);
      }
    w.resize(cand.size());
    double total = 0.0;
    for (size_t c = 0; c < cand.size(); ++c) {
      w[c] = pw[deg[cand[c]] - dmin];
      total += w[c];
    }
    const double target = rng.uniform() * total;
    int pick = cand.back();
    double run = 0.0;
    for (size_t c = 0; c < cand.size(); ++c) {
      run += w[c];
      if (run > target) {
        pick = cand[c];
        break;
      }
    }
    nb.clear();
    const uint64_t* rp = g.row(pick);
    for (int x = 0; x < g.W; ++x) {
      uint64_t bits = rp[x];
      while (bits) {
        nb.push_back(x * 64 + __builtin_ctzll(bits));
        bits &= bits - 1;
      }
    }
    res.order.push_back(pick);
    res.widths.push_back((int32_t)nb.size());
    g.eliminate(pick);
    --remaining;
    for (int a : nb) deg[a] = g.degree(a);
  }
  return res;
}
}  // namespace

OrderResult rgreedy_order(const BitGraph& g, double tau, int q, uint64_t seed) {
  SplitMix64 rng{seed};
  const double r = std::exp(-1.0 / tau);
  std::vector<double> pw((size_t)g.n + 1, 1.0);
  for (size_t k = 1; k < pw.size(); ++k) pw[k] = pw[k - 1] * r;
  OrderResult best;
  int32_t best_w = 0;
  double best_cost = 0.0;
  for (int run = 0; run < q; ++run) {
    OrderResult o = rgreedy_run(g, pw, rng);
    int32_t w = 0;
    double cost = 0.0;
    for (int32_t x : o.widths) {
      w = std::max(w, x);
      cost += std::ldexp(1.0, x);
    }
    if (run == 0 || w < best_w || (w == best_w && cost < best_cost)) {
      best = std::move(o);
      best_w = w;
      best_cost = cost;
    }
  }
  return best;
}

// ---------------------------- slicing search --------------------------------
static double plan_cost(const std::vector<int32_t>& a, const std::vector<int32_t>& b, int nb,
                        const std::vector<int32_t>& c) {
  double total = 0.0;
  for (int32_t w : a) total += std::ldexp(1.0, w);
  for (int i = 0; i < nb; ++i) total += std::ldexp(1.0, b[i]);
  for (int32_t w : c) total += std::ldexp(1.0, w);
  return total;
}

SlicePlan step_dependent_slicing(const BitGraph& g0, int algo, int width_limit, int max_vars,
                                 int r) {
  BitGraph g = g0;
  OrderResult cur = greedy_order(g, algo);
  int64_t runs = 1;
  std::vector<int32_t> done_order, done_widths, sliced;
  int32_t first_step = -1;
  auto maxw = [](const std::vector<int32_t>& v, int32_t init) {
    int32_t m = init;
    for (int32_t x : v) m = std::max(m, x);
    return m;
  };
  int32_t width = maxw(cur.widths, 0);
  int alive_count = 0;
  for (int v = 0; v < g.n; ++v) alive_count += g.takeable(v);
  while (width > width_limit && (int)sliced.size() < max_vars && alive_count > 0) {
    int rr = std::min<int>(r, max_vars - (int)sliced.size());
    int peak = 0;
    for (size_t i = 0; i < cur.widths.size(); ++i)
      if (cur.widths[i] > cur.widths[peak]) peak = (int)i;
    bool have = false;
    int32_t best_w = 0;
    double best_cost = 0.0;
    int best_s = 0;
    BitGraph best_g;
    OrderResult best_o;
    std::vector<int32_t> best_removed;
    BitGraph h = g;  // h = g with the first s vertices of cur eliminated
    int32_t done_max = maxw(done_widths, 0);
    int32_t prefix_max = 0;
    for (int s = 0; s <= peak; ++s) {
      if (s > 0) {
        h.eliminate(cur.order[s - 1]);
        prefix_max = std::max(prefix_max, cur.widths[s - 1]);
      }
      BitGraph b = h;
      std::vector<int32_t> removed;
      for (int t = 0; t < rr; ++t) {
        int bestv = -1, bestd = -1;
        for (int v = 0; v < b.n; ++v) {
          if (!b.takeable(v)) continue;
          int d = b.degree(v);
          if (d > bestd) { bestd = d; bestv = v; }
        }
        if (bestv < 0) break;
        b.remove(bestv);
        removed.push_back(bestv);
      }
      OrderResult o2 = greedy_order(b, algo);
      ++runs;
      int32_t w = std::max(std::max(done_max, prefix_max), maxw(o2.widths, 0));
      double cost = plan_cost(done_widths, cur.widths, s, o2.widths);
      bool better = !have || w < best_w || (w == best_w && cost < best_cost);
      if (better) {
        have = true;
        best_w = w;
        best_cost = cost;
        best_s = s;
        best_g = b;
        best_o = std::move(o2);
        best_removed = removed;
      }
    }
    if (first_step < 0) first_step = (int32_t)done_order.size() + best_s;
    for (int i = 0; i < best_s; ++i) {
      done_order.push_back(cur.order[i]);
      done_widths.push_back(cur.widths[i]);
    }
    for (int32_t v : best_removed) sliced.push_back(v);
    alive_count -= best_s + (int)best_removed.size();
    g = std::move(best_g);
    cur = std::move(best_o);
    width = best_w;
  }
  SlicePlan plan;
  plan.order = done_order;
  plan.order.insert(plan.order.end(), cur.order.begin(), cur.order.end());
  plan.widths = done_widths;
  plan.widths.insert(plan.widths.end(), cur.widths.begin(), cur.widths.end());
  plan.sliced = sliced;
  plan.slice_step = first_step < 0 ? 0 : first_step;
  plan.width = maxw(plan.widths, 0);
  plan.greedy_runs = runs;
  return plan;
}

}  // namespace qt
