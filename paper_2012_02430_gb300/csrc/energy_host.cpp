// Host side of the batched energy: one lightcone tensor network per edge
// (the energy as a duplicated bra-ket expression, Sec. III.B, restricted to the
// backward lightcone of Z_u Z_v, Sec. III.A), each ordered greedily (Sec. V.A.1)
// and compiled with the bucket-elimination schedule compiler (Alg. 1), then
// packed into flat device tables for one persistent kernel launch.
//
// Lightcone reading: with d(w) the graph distance from w to {u, v}, the layer-k
// cost gate on edge (a, b) stays iff min(d(a), d(b)) <= p - k, the layer-k
// mixer on w stays iff d(w) <= p - k, and |+> stays on every w with d(w) <= p.
// Qubit w with L(w) = max(0, p - d(w)) mixers has ket variables (w, 0..L-1),
// bra variables likewise, and one final variable shared by ket and bra; the
// observable is (1, -1) on the final variables of u and v; <Z_u Z_v> is
// 2^(-|S|) times the contraction, S = {w : d(w) <= p}.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <tuple>

#include "energy_internal.h"

namespace qt {

static void lightcone(const qt_energy* E, const double* gammas, const double* betas, int u,
                      int v, std::vector<Tensor>& T, std::vector<int32_t>& tags, int& n_vars,
                      double& norm) {
  const int n = E->n, p = E->p;
  // distances to {u, v}
  std::vector<int> d(n, -1);
  std::deque<int> q;
  d[u] = d[v] = 0;
  q.push_back(u);
  q.push_back(v);
  while (!q.empty()) {
    int a = q.front();
    q.pop_front();
    for (int b : E->adj[a])
      if (d[b] < 0) {
        d[b] = d[a] + 1;
        q.push_back(b);
      }
  }
  std::vector<int> qubits;
  for (int w = 0; w < n; ++w)
    if (d[w] >= 0 && d[w] <= p) qubits.push_back(w);
  std::vector<int> nmix(n, 0);
  for (int w : qubits) nmix[w] = std::max(0, p - d[w]);
  // variable ids in order of first use: kind 0 final, 1 ket, 2 bra
  std::map<std::tuple<int, int, int>, int> ids;
  auto var = [&](int kind, int w, int t) {
    auto key = std::make_tuple(kind, w, t);
    auto it = ids.find(key);
    if (it != ids.end()) return it->second;
    int id = (int)ids.size();
    ids.emplace(key, id);
    return id;
  };
  auto idx = [&](int side, int w, int t) {
    return t >= nmix[w] ? var(0, w, 0) : var(side, w, t);
  };
  T.clear();
  tags.clear();
  for (int side = 1; side <= 2; ++side) {
    const double sgn = side == 1 ? 1.0 : -1.0;  // bra: complex conjugate
    for (int w : qubits) {
      T.push_back({{idx(side, w, 0)}, {1.0, 0.0, 1.0, 0.0}});
      tags.push_back(0);
    }
    for (int k = 1; k <= p; ++k) {
      const double g = gammas[k - 1], b = betas[k - 1];
      const double er = std::cos(g), ei = -std::sin(g) * sgn;
      const double c = std::cos(b), s = std::sin(b) * sgn;
      for (size_t e = 0; e < E->edges.size() / 2; ++e) {
        const int a = E->edges[2 * e], bb = E->edges[2 * e + 1];
        if (d[a] >= 0 && d[bb] >= 0 && std::min(d[a], d[bb]) <= p - k) {
          T.push_back({{idx(side, a, k - 1), idx(side, bb, k - 1)},
                       {1.0, 0.0, er, ei, er, ei, 1.0, 0.0}});
          tags.push_back(1 | (k << 4) | (side << 12));
        }
      }
      for (int w : qubits)
        if (d[w] <= p - k) {
          T.push_back({{idx(side, w, k - 1), idx(side, w, k)}, {c, 0.0, 0.0, -s, 0.0, -s, c, 0.0}});
          tags.push_back(2 | (k << 4) | (side << 12));
        }
    }
  }
  T.push_back({{var(0, u, 0)}, {1.0, 0.0, -1.0, 0.0}});
  T.push_back({{var(0, v, 0)}, {1.0, 0.0, -1.0, 0.0}});
  tags.push_back(0);
  tags.push_back(0);
  n_vars = (int)ids.size();
  norm = std::ldexp(1.0, -(int)qubits.size());
}

bool energy_build_networks(qt_energy* E, std::string& err) {
  const int ne = (int)E->edges.size() / 2;
  E->nets.assign(ne, EnergyNet{});
  for (int e = 0; e < ne; ++e) {
    EnergyNet& N = E->nets[e];
    lightcone(E, E->gammas.data(), E->betas.data(), E->edges[2 * e], E->edges[2 * e + 1],
              N.tensors, N.tags, N.n_vars, N.norm);
    BitGraph g = line_graph(N.tensors, N.n_vars);
    OrderResult o = greedy_order(g, E->algo);
    N.plan = SlicePlan();
    N.plan.order = o.order;
    N.plan.widths = o.widths;
    N.plan.width = 0;
    for (int w : o.widths) N.plan.width = std::max(N.plan.width, w);
  }
  (void)err;
  return true;
}

bool energy_compile(qt_energy* E, int precision, std::string& err) {
  E->sw_template.clear();  // the sweep's template follows the compiled layout
  E->sw_tmpl_ws = nullptr;
  const int ne = (int)E->nets.size();
  E->precision = precision;
  E->elem_bytes = precision == QT_FP64 ? 16 : 8;
  E->h_ops.clear();
  E->h_steps.clear();
  E->h_nets.assign(ne, ENet{});
  E->h_scalars.clear();
  E->gate_elems = 0;
  E->arena_elems = 64;
  E->total_flops = 0;
  E->total_bytes = 0;
  E->max_width = 0;
  E->hist_width.assign(64, 0);
  std::vector<int64_t> gate_base(ne, 0);
  for (int e = 0; e < ne; ++e) {
    EnergyNet& N = E->nets[e];
    if (!compile_schedule(N.tensors, N.n_vars, N.plan, precision, 1, E->fuse, N.sched, err))
      return false;
    gate_base[e] = E->gate_elems;
    E->gate_elems += N.sched.gate_elems;
    E->arena_elems = std::max<int64_t>(E->arena_elems, N.sched.slice_elems);
    E->max_width = std::max(E->max_width, N.plan.width);
    E->hist_width[std::min(N.plan.width, 63)]++;
  }
  if (E->gate_elems >= (int64_t(1) << 31) || E->arena_elems >= (int64_t(1) << 31)) {
    err = "energy tables exceed 2^31 elements";
    return false;
  }
  // networks in descending cost for the work queue
  std::vector<int> byc(ne);
  for (int e = 0; e < ne; ++e) byc[e] = e;
  auto cost = [&](int e) {
    const Schedule& S = E->nets[e].sched;
    return S.slice_flops + S.slice_bytes;
  };
  std::stable_sort(byc.begin(), byc.end(), [&](int a, int b) { return cost(a) > cost(b); });
  for (int slot = 0; slot < ne; ++slot) {
    const int e = byc[slot];
    EnergyNet& N = E->nets[e];
    const Schedule& S = N.sched;
    ENet nd{};
    nd.first_step = (uint32_t)E->h_steps.size();
    nd.edge = (uint32_t)e;
    nd.norm = N.norm;
    for (const SGroup& g : S.groups) {
      EStep sd{};
      sd.m = (uint16_t)g.ops.size();
      sd.u = (uint16_t)g.u;
      sd.nsum = (uint16_t)g.nsum;
      sd.first_op = (uint32_t)E->h_ops.size();
      sd.out = (uint32_t)S.tensors[g.out].offset;
      for (size_t j = 0; j < g.ops.size(); ++j) {
        const STensor& t = S.tensors[g.ops[j]];
        EOp od{};
        unsigned int um = 0;
        for (int b = 0; b < g.u; ++b)
          if (std::find(t.labels.begin(), t.labels.end(), g.ulabels[b]) != t.labels.end())
            um |= 1u << b;
        od.umask = um;
        od.level = (uint16_t)g.levels[j];
        od.in_arena = t.kind == TK_GATE ? 0 : 1;
        od.off = (uint32_t)(t.kind == TK_GATE ? gate_base[e] + t.offset : t.offset);
        E->h_ops.push_back(od);
      }
      E->h_steps.push_back(sd);
      if (g.u > 24) {
        err = "a lightcone step exceeds rank 24";
        return false;
      }
    }
    nd.nsteps = (uint32_t)(E->h_steps.size() - nd.first_step);
    nd.first_scalar = (uint32_t)E->h_scalars.size();
    for (int32_t tid : S.scalars) E->h_scalars.push_back((uint32_t)S.tensors[tid].offset);
    nd.nscalars = (uint32_t)(E->h_scalars.size() - nd.first_scalar);
    E->h_nets[slot] = nd;
    E->total_flops += S.slice_flops;
    E->total_bytes += S.slice_launch_bytes;
  }
  // gate data in the precision, canonical layout per network
  const size_t eb = (size_t)E->elem_bytes;
  E->h_gates.assign((size_t)E->gate_elems * eb, 0);
  for (int e = 0; e < ne; ++e) {
    const Schedule& S = E->nets[e].sched;
    for (const STensor& t : S.tensors) {
      if (t.kind != TK_GATE) continue;
      std::vector<double> dd = canonical_data(E->nets[e].tensors[t.gate], t.labels);
      for (size_t k = 0; k < dd.size(); ++k) {
        const size_t at = (size_t)(gate_base[e] + t.offset) * 2 + k;
        if (precision == QT_FP64) {
          double x = dd[k];
          std::memcpy(E->h_gates.data() + at * sizeof(double), &x, sizeof(double));
        } else {
          float x = (float)dd[k];
          std::memcpy(E->h_gates.data() + at * sizeof(float), &x, sizeof(float));
        }
      }
    }
  }
  E->compiled = true;
  return true;
}

void energy_gate_image(const qt_energy* E, const double* gammas, const double* betas,
                       unsigned char* dst) {
  // the phase and mixer matrices are symmetric, so their canonical layout is their
  // own element order whatever the label order; constant tensors are copied
  const int p = E->p;
  std::vector<double> ph(4 * (size_t)p), mx(4 * (size_t)p);  // [k][side]: (re, im) pairs
  for (int k = 0; k < p; ++k)
    for (int side = 1; side <= 2; ++side) {
      const double sgn = side == 1 ? 1.0 : -1.0;
      ph[4 * k + 2 * (side - 1)] = std::cos(gammas[k]);
      ph[4 * k + 2 * (side - 1) + 1] = -std::sin(gammas[k]) * sgn;
      mx[4 * k + 2 * (side - 1)] = std::cos(betas[k]);
      mx[4 * k + 2 * (side - 1) + 1] = std::sin(betas[k]) * sgn;
    }
  const bool f64 = E->precision == QT_FP64;
  auto put = [&](size_t at, double v) {
    if (f64) std::memcpy(dst + at * sizeof(double), &v, sizeof(double));
    else {
      const float x = (float)v;
      std::memcpy(dst + at * sizeof(float), &x, sizeof(float));
    }
  };
  int64_t base = 0;
  for (const EnergyNet& N : E->nets) {
    const Schedule& S = N.sched;
    for (const STensor& t : S.tensors) {
      if (t.kind != TK_GATE) continue;
      const int tag = N.tags[t.gate];
      const int kind = tag & 15, k = (tag >> 4) & 255, side = tag >> 12;
      const size_t at = (size_t)(base + t.offset) * 2;
      if (kind == 0) {
        const std::vector<double> dd = canonical_data(N.tensors[t.gate], t.labels);
        for (size_t q = 0; q < dd.size(); ++q) put(at + q, dd[q]);
      } else if (kind == 1) {
        const double er = ph[4 * (k - 1) + 2 * (side - 1)], ei = ph[4 * (k - 1) + 2 * (side - 1) + 1];
        const double v[8] = {1.0, 0.0, er, ei, er, ei, 1.0, 0.0};
        for (int q = 0; q < 8; ++q) put(at + q, v[q]);
      } else {
        const double c = mx[4 * (k - 1) + 2 * (side - 1)], sn = mx[4 * (k - 1) + 2 * (side - 1) + 1];
        const double v[8] = {c, 0.0, 0.0, -sn, 0.0, -sn, c, 0.0};
        for (int q = 0; q < 8; ++q) put(at + q, v[q]);
      }
    }
    base += S.gate_elems;
  }
}

void energy_sweep_template(qt_energy* E) {
  const bool f64 = E->precision == QT_FP64;
  const size_t eb = f64 ? sizeof(double) : sizeof(float);
  E->sw_template.assign((size_t)E->gate_elems * 2 * eb, 0);
  E->sw_slots.clear();
  E->sw_codes.clear();
  unsigned char* dst = E->sw_template.data();
  auto put = [&](size_t at, double v) {
    if (f64) std::memcpy(dst + at * sizeof(double), &v, sizeof(double));
    else {
      const float x = (float)v;
      std::memcpy(dst + at * sizeof(float), &x, sizeof(float));
    }
  };
  int64_t base = 0;
  for (const EnergyNet& N : E->nets) {
    const Schedule& S = N.sched;
    for (const STensor& t : S.tensors) {
      if (t.kind != TK_GATE) continue;
      const int tag = N.tags[t.gate];
      const int kind = tag & 15;
      if (kind == 0) {
        const std::vector<double> dd = canonical_data(N.tensors[t.gate], t.labels);
        const size_t at = (size_t)(base + t.offset) * 2;
        for (size_t q = 0; q < dd.size(); ++q) put(at + q, dd[q]);
      } else {
        // (the phase and mixer matrices are symmetric: their element order is canonical)
        E->sw_slots.push_back((uint32_t)(base + t.offset));
        E->sw_codes.push_back((uint32_t)tag);
      }
    }
    base += S.gate_elems;
  }
}

void energy_sweep_table(qt_energy* E, int n_sets, const double* gammas, const double* betas) {
  const bool f64 = E->precision == QT_FP64;
  const size_t eb = f64 ? sizeof(double) : sizeof(float);
  const int p = E->p;
  E->sw_table.assign((size_t)n_sets * p * 8 * eb, 0);
  unsigned char* dst = E->sw_table.data();
  for (int q = 0; q < n_sets; ++q)
    for (int k = 0; k < p; ++k) {
      const double g = gammas[(size_t)q * p + k], b = betas[(size_t)q * p + k];
      // [kind 1 phase, kind 2 mixer][side 1, 2][2]: exp(-i g) / its conjugate; cos, sin b
      const double v[8] = {std::cos(g), -std::sin(g), std::cos(g), std::sin(g),
                           std::cos(b), std::sin(b),  std::cos(b), -std::sin(b)};
      for (int e = 0; e < 8; ++e) {
        const size_t at = (((size_t)q * p + k) * 8 + e) * eb;
        if (f64) std::memcpy(dst + at, &v[e], sizeof(double));
        else {
          const float x = (float)v[e];
          std::memcpy(dst + at, &x, sizeof(float));
        }
      }
    }
}

}  // namespace qt
