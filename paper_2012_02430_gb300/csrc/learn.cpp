// Learned proposals for step-dependent slicing (host side).
//
// The slicing search of Sec. VI.C-D scans every step s up to the peak of the
// current order and re-orders the graph greedily for each (Fig. 8: the costly
// part, n/(2r) N ordering runs). Here a candidate is a pair (s, v): the step s
// and the first vertex v sliced there, v among the `topv` vertices of largest
// degree at that step (topv = 1 is the paper's max-degree rule). Each candidate
// gets a feature vector read off the graph at step s without any ordering run;
// a small MLP (trained on the GPU by the kernels in mlp.cu, on candidates whose
// true width this code measured) predicts the plan width, and only the `topm`
// best-scored candidates are re-ordered greedily. Greedy ordering decides: the
// chosen candidate is the best verified one by (width, sum of 2^w, s, rank).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "qt_internal.h"

namespace qt {

constexpr int kFeatures = kProposalFeatures;

struct Candidate {
  int s = 0, v = -1, rank = 0;
  float f[kFeatures];
  float score = 0.f;
};

static int count_fill(const BitGraph& g, int v, int deg) {
  const uint64_t* rv = g.row(v);
  int64_t twice = 0;
  for (int w = 0; w < g.W; ++w) {
    uint64_t bits = rv[w];
    while (bits) {
      const int a = w * 64 + __builtin_ctzll(bits);
      bits &= bits - 1;
      const uint64_t* ra = g.row(a);
      for (int x = 0; x < g.W; ++x) twice += __builtin_popcountll(ra[x] & rv[x]);
    }
  }
  return (int)((int64_t)deg * (deg - 1) / 2 - twice / 2);
}

// Candidates (and their features) of one slicing round on graph g with greedy
// order `order` / `widths`; n0 = vertices of the whole network.
static std::vector<Candidate> round_candidates(const BitGraph& g, const std::vector<int32_t>& order,
                                               const std::vector<int32_t>& widths, int n0,
                                               int topv) {
  std::vector<Candidate> out;
  if (widths.empty()) return out;
  int peak = 0;
  for (size_t i = 0; i < widths.size(); ++i)
    if (widths[i] > widths[peak]) peak = (int)i;
  const double W = std::max(1, widths[peak]);
  BitGraph h = g;
  double prefix_cost = 0.0;
  int prefix_max = 0;
  const int pv = order[peak];
  for (int s = 0; s <= peak; ++s) {
    if (s > 0) {
      h.eliminate(order[s - 1]);
      prefix_cost += std::ldexp(1.0, widths[s - 1]);
      prefix_max = std::max(prefix_max, widths[s - 1]);
    }
    // degrees of the alive vertices, ranked by (-degree, id)
    std::vector<std::pair<int, int>> ranked;
    int64_t deg_sum = 0;
    int alive = 0;
    for (int x = 0; x < h.n; ++x) {
      if (!h.takeable(x)) continue;
      const int d = h.degree(x);
      ranked.push_back({-d, x});
      deg_sum += d;
      ++alive;
    }
    if (alive == 0) break;
    std::sort(ranked.begin(), ranked.end());
    const int dmax = -ranked[0].first;
    int nmax = 0;
    for (auto& pr : ranked) nmax += (-pr.first == dmax);
    const double edges = (double)deg_sum / 2.0;
    const int dpeak = h.alive[pv] ? h.degree(pv) : 0;
    const int kv = std::min<int>(topv, (int)ranked.size());
    for (int j = 0; j < kv; ++j) {
      Candidate c;
      c.s = s;
      c.v = ranked[j].second;
      c.rank = j;
      const int dv = -ranked[j].first;
      const int fill = count_fill(h, c.v, dv);
      const bool near_peak = c.v == pv || (h.alive[pv] && h.has(c.v, pv));
      c.f[0] = (float)(s / (double)(peak + 1));
      c.f[1] = (float)(widths[s] / W);
      c.f[2] = (float)(dv / W);
      c.f[3] = (float)(dmax / W);
      c.f[4] = (float)(j / (double)topv);
      c.f[5] = (float)(alive / (double)n0);
      c.f[6] = (float)((2.0 * edges / alive) / W);
      c.f[7] = (float)(prefix_max / W);
      c.f[8] = (float)(std::log2(1.0 + prefix_cost) / W);
      c.f[9] = (float)(fill / std::max(1.0, dv * (dv - 1) / 2.0));
      c.f[10] = (float)(nmax / (double)alive);
      c.f[11] = (float)(dpeak / W);
      c.f[12] = near_peak ? 1.f : 0.f;
      c.f[13] = (float)((peak - s) / (double)(peak + 1));
      c.f[14] = (float)(s > 0 ? widths[s - 1] / W : 0.0);
      c.f[15] = (float)(edges / std::max(1.0, alive * (alive - 1) / 2.0));
      out.push_back(c);
    }
  }
  return out;
}

struct Eval {
  int32_t width = 0;
  double cost = 0.0;
  BitGraph g;
  OrderResult o;
  std::vector<int32_t> removed;
};

// Plan of one candidate: eliminate order[:s], slice v, then r-1 more vertices of
// largest degree, re-order greedily (the deciding ordering run).
static Eval evaluate(const BitGraph& g, const std::vector<int32_t>& order,
                     const std::vector<int32_t>& widths, const std::vector<int32_t>& done_widths,
                     int s, int v, int r, int algo) {
  Eval e;
  e.g = g;
  for (int i = 0; i < s; ++i) e.g.eliminate(order[i]);
  e.g.remove(v);
  e.removed.push_back(v);
  for (int t = 1; t < r; ++t) {
    int best = -1, bestd = -1;
    for (int x = 0; x < e.g.n; ++x) {
      if (!e.g.takeable(x)) continue;
      const int d = e.g.degree(x);
      if (d > bestd) {
        bestd = d;
        best = x;
      }
    }
    if (best < 0) break;
    e.g.remove(best);
    e.removed.push_back(best);
  }
  e.o = greedy_order(e.g, algo);
  int32_t w = 0;
  for (int32_t x : done_widths) w = std::max(w, x);
  for (int i = 0; i < s; ++i) w = std::max(w, widths[i]);
  for (int32_t x : e.o.widths) w = std::max(w, x);
  double cost = 0.0;
  for (int32_t x : done_widths) cost += std::ldexp(1.0, x);
  for (int i = 0; i < s; ++i) cost += std::ldexp(1.0, widths[i]);
  for (int32_t x : e.o.widths) cost += std::ldexp(1.0, x);
  e.width = w;
  e.cost = cost;
  return e;
}

// MLP forward on the host (same layout and arithmetic order as the GPU kernels):
// params = W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
int mlp_param_count(int nf, int hidden) { return hidden * nf + hidden + hidden * hidden + hidden + hidden + 1; }

void mlp_forward_host(const float* params, int nf, int hidden, const float* x, int batch, float* y) {
  const float* W1 = params;
  const float* b1 = W1 + hidden * nf;
  const float* W2 = b1 + hidden;
  const float* b2 = W2 + hidden * hidden;
  const float* w3 = b2 + hidden;
  const float* b3 = w3 + hidden;
  std::vector<float> h1(hidden), h2(hidden);
  for (int b = 0; b < batch; ++b) {
    const float* xb = x + (size_t)b * nf;
    for (int j = 0; j < hidden; ++j) {
      float a = b1[j];
      for (int i = 0; i < nf; ++i) a += W1[j * nf + i] * xb[i];
      h1[j] = a > 0.f ? a : 0.f;
    }
    for (int j = 0; j < hidden; ++j) {
      float a = b2[j];
      for (int i = 0; i < hidden; ++i) a += W2[j * hidden + i] * h1[i];
      h2[j] = a > 0.f ? a : 0.f;
    }
    float a = b3[0];
    for (int i = 0; i < hidden; ++i) a += w3[i] * h2[i];
    y[b] = a;
  }
}

bool slice_dataset(const qt_net* net, int topv, std::vector<float>& feats,
                   std::vector<float>& labels, std::vector<int32_t>& meta) {
  BitGraph g = network_graph(net);
  OrderResult cur = greedy_order(g, net->algo);
  std::vector<Candidate> cands = round_candidates(g, cur.order, cur.widths, net->n_vars, topv);
  int W = 0;
  for (int x : cur.widths) W = std::max(W, x);
  const std::vector<int32_t> none;
  for (const Candidate& c : cands) {
    Eval e = evaluate(g, cur.order, cur.widths, none, c.s, c.v, 1, net->algo);
    feats.insert(feats.end(), c.f, c.f + kFeatures);
    labels.push_back((float)(e.width / (double)std::max(1, W)));
    meta.push_back(c.s);
    meta.push_back(c.v);
    meta.push_back(e.width);
  }
  return true;
}

// Step-dependent slicing with learned proposals (see the verified set below).
SlicePlan learned_slicing(const qt_net* net, const float* params, int hidden, int width_limit,
                          int max_vars, int r, int topv, int topm, int spread,
                          int64_t& greedy_runs) {
  BitGraph g = network_graph(net);
  const int algo = net->algo;
  OrderResult cur = greedy_order(g, algo);
  greedy_runs = 1;
  std::vector<int32_t> done_order, done_widths, sliced;
  int32_t first_step = -1;
  int32_t width = 0;
  for (int32_t x : cur.widths) width = std::max(width, x);
  int alive = 0;
  for (int v = 0; v < g.n; ++v) alive += g.takeable(v);
  while (width > width_limit && (int)sliced.size() < max_vars && alive > 0) {
    const int rr = std::min<int>(r, max_vars - (int)sliced.size());
    std::vector<Candidate> cands = round_candidates(g, cur.order, cur.widths, net->n_vars, topv);
    if (cands.empty()) break;
    // verified set: the model's topm best scores (kept `gap` steps apart while
    // enough candidates remain) plus `spread` candidates evenly spaced in (s, rank)
    // order; spread >= the number of candidates verifies all of them
    const int C = (int)cands.size();
    std::vector<char> chosen(C, 0);
    if (spread >= C) {
      std::fill(chosen.begin(), chosen.end(), 1);
    } else if (params && topm == 0) {
      // one candidate per step: the best-scored of its topv vertices
      std::vector<float> x((size_t)C * kFeatures), y(C);
      for (int i = 0; i < C; ++i)
        std::memcpy(&x[(size_t)i * kFeatures], cands[i].f, sizeof(float) * kFeatures);
      mlp_forward_host(params, kFeatures, hidden, x.data(), C, y.data());
      for (int i = 0; i < C;) {
        int j = i, best = i;
        while (j < C && cands[j].s == cands[i].s) {
          if (y[j] < y[best]) best = j;
          ++j;
        }
        chosen[best] = 1;
        i = j;
      }
    } else {
      for (int i = 0; i < spread; ++i)
        chosen[spread == 1 ? 0 : (int)((int64_t)i * (C - 1) / (spread - 1))] = 1;
      if (params && topm > 0) {
        std::vector<float> x((size_t)C * kFeatures), y(C);
        for (int i = 0; i < C; ++i)
          std::memcpy(&x[(size_t)i * kFeatures], cands[i].f, sizeof(float) * kFeatures);
        mlp_forward_host(params, kFeatures, hidden, x.data(), C, y.data());
        int peak_s = 0;
        for (const Candidate& c : cands) peak_s = std::max(peak_s, c.s);
        std::vector<int> idx(C);
        for (int i = 0; i < C; ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return y[a] < y[b]; });
        const int gap = std::max(1, (peak_s + 1) / (4 * topm));
        std::vector<int> pick;
        for (int i : idx) {
          if ((int)pick.size() >= topm) break;
          bool near = false;
          for (int q : pick) near = near || std::abs(cands[q].s - cands[i].s) < gap;
          if (!near) pick.push_back(i);
        }
        for (int i : idx) {
          if ((int)pick.size() >= topm) break;
          if (std::find(pick.begin(), pick.end(), i) == pick.end()) pick.push_back(i);
        }
        for (int i : pick) chosen[i] = 1;
      }
    }
    std::vector<Candidate> verify;
    for (int i = 0; i < C; ++i)
      if (chosen[i]) verify.push_back(cands[i]);
    cands.swap(verify);
    bool have = false;
    Eval best;
    int best_s = 0, best_rank = 0;
    for (const Candidate& c : cands) {
      Eval e = evaluate(g, cur.order, cur.widths, done_widths, c.s, c.v, rr, algo);
      ++greedy_runs;
      const bool better =
          !have || e.width < best.width || (e.width == best.width && e.cost < best.cost) ||
          (e.width == best.width && e.cost == best.cost &&
           (c.s < best_s || (c.s == best_s && c.rank < best_rank)));
      if (better) {
        have = true;
        best = std::move(e);
        best_s = c.s;
        best_rank = c.rank;
      }
    }
    if (first_step < 0) first_step = (int32_t)done_order.size() + best_s;
    for (int i = 0; i < best_s; ++i) {
      done_order.push_back(cur.order[i]);
      done_widths.push_back(cur.widths[i]);
    }
    for (int32_t v : best.removed) sliced.push_back(v);
    alive -= best_s + (int)best.removed.size();
    g = std::move(best.g);
    cur = std::move(best.o);
    width = best.width;
  }
  SlicePlan plan;
  plan.order = done_order;
  plan.order.insert(plan.order.end(), cur.order.begin(), cur.order.end());
  plan.widths = done_widths;
  plan.widths.insert(plan.widths.end(), cur.widths.begin(), cur.widths.end());
  plan.sliced = sliced;
  plan.slice_step = first_step < 0 ? 0 : first_step;
  plan.width = 0;
  for (int32_t x : plan.widths) plan.width = std::max(plan.width, x);
  plan.greedy_runs = greedy_runs;
  return plan;
}

// ---------------------------------------------------------------------------
// Learned elimination steps (the other half of the proposals). At every step of a
// greedy ordering the candidates are the `topc` alive vertices best by the greedy
// key (min-fill: fill, degree, id; min-degree: degree, id); rank 0 is the vertex
// greedy itself takes. Each gets 16 features read off the current graph; a model
// trained on rollouts (the candidate eliminated, then greedy to the end, labelled
// by log2 of the plan cost sum 2^w) picks one. Greedy stays the judge: the learned
// order is kept only if its (width, cost) is below the plain greedy order's.
// ---------------------------------------------------------------------------
struct StepCand {
  int v, deg, fill;
};

static std::vector<StepCand> step_candidates(const BitGraph& h, int algo, int topc) {
  std::vector<StepCand> all;
  for (int x = 0; x < h.n; ++x) {
    if (!h.takeable(x)) continue;
    const int d = h.degree(x);
    all.push_back({x, d, algo == QT_GREEDY_MINFILL ? count_fill(h, x, d) : 0});
  }
  const int k = std::min<int>(topc, (int)all.size());
  std::partial_sort(all.begin(), all.begin() + k, all.end(), [&](const StepCand& a, const StepCand& b) {
    if (algo == QT_GREEDY_MINFILL && a.fill != b.fill) return a.fill < b.fill;
    if (a.deg != b.deg) return a.deg < b.deg;
    return a.v < b.v;
  });
  all.resize(k);
  return all;
}

// features of candidate j at step t (W0: the plain greedy width of the whole graph,
// n0: vertices of the network, maxw: the largest width of the steps taken so far)
static void step_features(const BitGraph& h, const std::vector<StepCand>& c, int j, int t, int n0,
                          int W0, int maxw, int alive, int64_t deg_sum, int dmax, float* f) {
  const StepCand& x = c[j];
  const double W = std::max(1, W0);
  int nmin = 1 << 30, nmax = 0;
  int64_t nsum = 0;
  std::vector<uint64_t> two(h.W, 0);
  const uint64_t* rv = h.row(x.v);
  for (int w = 0; w < h.W; ++w) {
    uint64_t bits = rv[w];
    while (bits) {
      const int a = w * 64 + __builtin_ctzll(bits);
      bits &= bits - 1;
      const int da = h.degree(a);
      nmin = std::min(nmin, da);
      nmax = std::max(nmax, da);
      nsum += da;
      const uint64_t* ra = h.row(a);
      for (int q = 0; q < h.W; ++q) two[q] |= ra[q];
    }
  }
  int hop2 = 0;
  for (int q = 0; q < h.W; ++q) hop2 += __builtin_popcountll(two[q] | rv[q]);
  int common = 0;  // neighbours shared with the greedy choice (rank 0)
  const uint64_t* r0 = h.row(c[0].v);
  for (int q = 0; q < h.W; ++q) common += __builtin_popcountll(rv[q] & r0[q]);
  const double edges = deg_sum / 2.0;
  f[0] = (float)(x.deg / W);
  f[1] = (float)(x.fill / std::max(1.0, x.deg * (x.deg - 1) / 2.0));
  f[2] = (float)(j / (double)std::max<size_t>(1, c.size()));
  f[3] = (float)((x.fill - c[0].fill) / W);
  f[4] = (float)((x.deg - c[0].deg) / W);
  f[5] = (float)(x.deg ? (nsum / (double)x.deg) / W : 0.0);
  f[6] = (float)(nmax / W);
  f[7] = (float)(x.deg ? nmin / W : 0.0);
  f[8] = (float)(alive / (double)n0);
  f[9] = (float)(t / (double)n0);
  f[10] = (float)(maxw / W);
  f[11] = (float)((alive ? 2.0 * edges / alive : 0.0) / W);
  f[12] = (float)(edges / std::max(1.0, alive * (alive - 1) / 2.0));
  f[13] = (float)(j == 0 ? 1.0 : common / std::max(1.0, (double)x.deg));
  f[14] = (float)(x.deg / std::max(1.0, (double)dmax));
  f[15] = (float)(hop2 / std::max(1.0, (double)alive));
}

static void graph_stats(const BitGraph& h, int& alive, int64_t& deg_sum, int& dmax) {
  alive = 0;
  deg_sum = 0;
  dmax = 0;
  for (int x = 0; x < h.n; ++x) {
    if (!h.takeable(x)) continue;
    const int d = h.degree(x);
    ++alive;
    deg_sum += d;
    dmax = std::max(dmax, d);
  }
}

static double log2_cost(const std::vector<int32_t>& widths) {
  double c = 0.0;
  for (int32_t w : widths) c += std::ldexp(1.0, w);
  return std::log2(std::max(1.0, c));
}

bool order_dataset(const qt_net* net, int topc, int stride, std::vector<float>& feats,
                   std::vector<float>& labels, std::vector<int32_t>& meta) {
  const BitGraph g = network_graph(net);
  const int algo = net->algo;
  const OrderResult gr = greedy_order(g, algo);
  int W0 = 0;
  for (int32_t w : gr.widths) W0 = std::max(W0, w);
  BitGraph h = g;
  std::vector<int32_t> prefix;
  int maxw = 0;
  for (size_t t = 0; t < gr.order.size(); ++t) {
    if (t % (size_t)std::max(1, stride) == 0) {
      const std::vector<StepCand> c = step_candidates(h, algo, topc);
      if (c.size() >= 2) {
        int alive, dmax;
        int64_t deg_sum;
        graph_stats(h, alive, deg_sum, dmax);
        for (size_t j = 0; j < c.size(); ++j) {
          float f[kFeatures];
          step_features(h, c, (int)j, (int)t, net->n_vars, W0, maxw, alive, deg_sum, dmax, f);
          BitGraph r = h;
          const int d = r.eliminate(c[j].v);
          const OrderResult rest = greedy_order(r, algo);
          std::vector<int32_t> ws = prefix;
          ws.push_back(d);
          ws.insert(ws.end(), rest.widths.begin(), rest.widths.end());
          int width = 0;
          for (int32_t w : ws) width = std::max(width, w);
          feats.insert(feats.end(), f, f + kFeatures);
          labels.push_back((float)log2_cost(ws));
          meta.push_back((int32_t)t);
          meta.push_back(c[j].v);
          meta.push_back(width);
        }
      }
    }
    prefix.push_back(gr.widths[t]);
    maxw = std::max(maxw, gr.widths[t]);
    h.eliminate(gr.order[t]);
  }
  return true;
}

OrderResult learned_order(const BitGraph& g, int algo, const float* params, int hidden, int topc,
                          int n0, int W0) {
  BitGraph h = g;
  OrderResult res;
  int maxw = 0;
  std::vector<float> x, y;
  for (int t = 0;; ++t) {
    const std::vector<StepCand> c = step_candidates(h, algo, topc);
    if (c.empty()) break;
    int pick = 0;
    if (c.size() >= 2) {
      int alive, dmax;
      int64_t deg_sum;
      graph_stats(h, alive, deg_sum, dmax);
      x.assign(c.size() * kFeatures, 0.f);
      y.assign(c.size(), 0.f);
      for (size_t j = 0; j < c.size(); ++j)
        step_features(h, c, (int)j, t, n0, W0, maxw, alive, deg_sum, dmax, &x[j * kFeatures]);
      mlp_forward_host(params, kFeatures, hidden, x.data(), (int)c.size(), y.data());
      for (size_t j = 1; j < c.size(); ++j)
        if (y[j] < y[pick]) pick = (int)j;
    }
    const int d = h.eliminate(c[pick].v);
    res.order.push_back(c[pick].v);
    res.widths.push_back(d);
    maxw = std::max(maxw, d);
  }
  return res;
}

}  // namespace qt

