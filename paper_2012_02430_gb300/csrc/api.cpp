// The C ABI (include/qtensor.h): argument checks, state checks, error strings,
// and the network builder of Sec. III.A / Sec. IV.A-B.
#include <cmath>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <utility>

#include "qt_internal.h"

namespace qt {
// engine.cu
void build_stage(qt_net* net);
qt_status upload(qt_net* net, void* ws, size_t bytes, void* stream, std::string& err);
qt_status run(qt_net* net, long long first, long long count, void* ws, void* stream,
              double* d_out, std::string& err);
size_t stage_image_bytes(const qt_net* net);
qt_status launch_plan(qt_net* net, std::string& out, std::string& err);
qt_status sweep_run(qt_net* net, void* ws, void* stream, int n_sets, const void* images,
                    size_t staging_off, size_t stride, size_t results_off, std::string& err);
qt_status download_result(const double* d_out, double* host, int64_t n_doubles, void* stream,
                          std::string& err);
qt_status read_status(const qt_net* net, const void* ws, void* stream, int* status,
                      std::string& err);
// the result and the status word, copied back with one stream synchronisation
qt_status download_result_status(const qt_net* net, const void* ws, const double* d_out,
                                 double* host, int64_t n_doubles, int* status, void* stream,
                                 std::string& err);
void prof_clear(qt_net* net);
qt_status autotune(qt_net* net, void* ws, void* stream, std::string& report, std::string& err);
qt_status prof_read(qt_net* net, std::string& out, std::string& err);
}  // namespace qt

namespace {

thread_local std::string g_err;

qt_status fail(qt_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

qt_status ok() {
  g_err.clear();
  return QT_OK;
}

// Gate tensors of the ansatz, FP64, axis t of the labels = bit t of the index.
void make_tensors(qt_net* net) {
  const int n = net->n, p = net->p;
  auto var = [n](int v, int k) { return k * n + v; };
  std::vector<qt::Tensor>& T = net->tensors;
  // the tensors are rewritten in place (new angles keep every label and size, so a call
  // after the first allocates nothing); the list ends where this call's tensors end
  size_t idx = 0;
  auto emit = [&](std::initializer_list<int32_t> lab, std::initializer_list<double> dat) {
    if (idx < T.size()) {
      T[idx].labels.assign(lab);
      T[idx].data.assign(dat);
    } else {
      T.push_back({std::vector<int32_t>(lab), std::vector<double>(dat)});
    }
    ++idx;
  };
  for (int v = 0; v < n; ++v) emit({var(v, 0)}, {1.0, 0.0, 1.0, 0.0});
  for (int k = 1; k <= p; ++k) {
    const double g = net->gammas[k - 1], b = net->betas[k - 1];
    // D(a, b) = exp(-i gamma [a != b]); M(a, a') = cos(beta) or -i sin(beta)
    const double er = std::cos(g), ei = -std::sin(g);
    const double c = std::cos(b), s = std::sin(b);
    for (int e = 0; e < net->n_edges; ++e) {
      const int u = net->edges[2 * e], w = net->edges[2 * e + 1];
      emit({var(u, k - 1), var(w, k - 1)}, {1.0, 0.0, er, ei, er, ei, 1.0, 0.0});
    }
    for (int v = 0; v < n; ++v) {
      int j = -1;  // open qubit number, Sec. VII
      if (k == p)
        for (size_t t = 0; t < net->open.size(); ++t)
          if (net->open[t] == v) j = (int)t;
      if (k < p) {
        emit({var(v, k - 1), var(v, k)}, {c, 0.0, 0.0, -s, 0.0, -s, c, 0.0});
      } else if (j >= 0) {
        // the whole mixer, its output index left open as variable n*p + j
        emit({var(v, p - 1), n * p + j}, {c, 0.0, 0.0, -s, 0.0, -s, c, 0.0});
      } else {
        // row a' = z_v of M, as a function of a
        if (net->z[v] == 0) emit({var(v, p - 1)}, {c, 0.0, 0.0, -s});
        else emit({var(v, p - 1)}, {0.0, -s, c, 0.0});
      }
    }
  }
  T.resize(idx);
}

bool check_net(const qt_net* net) { return net != nullptr; }

}  // namespace

extern "C" qt_status qt_prepare(qt_net* net, int32_t precision, int32_t batch,
                                size_t* workspace_bytes);

namespace qt {
void set_last_error(const std::string& msg) { g_err = msg; }

qt_status prepare_fitting(qt_net* net, int32_t precision, size_t budget,
                          size_t (*room)(const qt_net*, const void*), const void* room_arg,
                          std::string& err) {
  size_t need = 0;
  qt_status s = qt_prepare(net, precision, 1, &need);
  if (s != QT_OK) {
    err = g_err;
    return s;
  }
  const size_t extra = room ? room(net, room_arg) : 0;
  if (need + extra > budget) {
    err = "one slice needs " + std::to_string(need + extra) + " bytes of workspace; " +
          std::to_string(budget) + " are available";
    return QT_ENOMEM;
  }
  // the batch-1 schedule fits; the workspace grows with the batch
  int64_t lo = 1, hi = net->sched.nslices;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    s = qt_prepare(net, precision, (int32_t)std::min<int64_t>(mid, 1 << 30), &need);
    if (s != QT_OK) {
      err = g_err;
      return s;
    }
    if (need + extra <= budget) lo = mid;
    else hi = mid - 1;
  }
  s = qt_prepare(net, precision, (int32_t)lo, &need);
  if (s != QT_OK) err = g_err;
  return s;
}
bool slice_dataset(const qt_net* net, int topv, std::vector<float>& feats,
                   std::vector<float>& labels, std::vector<int32_t>& meta);
SlicePlan learned_slicing(const qt_net* net, const float* params, int hidden, int width_limit,
                          int max_vars, int r, int topv, int topm, int spread,
                          int64_t& greedy_runs);
bool order_dataset(const qt_net* net, int topc, int stride, std::vector<float>& feats,
                   std::vector<float>& labels, std::vector<int32_t>& meta);
OrderResult learned_order(const BitGraph& g, int algo, const float* params, int hidden, int topc,
                          int n0, int W0);
}  // namespace qt

extern "C" {

const char* qt_last_error(void) { return g_err.c_str(); }

const char* qt_version(void) { return "qtensor-gb300 0.1 (sm_103a)"; }

qt_status qt_build_network(const int32_t* edges, int32_t n_vertices, int32_t n_edges, int32_t p,
                           const double* gammas, const double* betas, const uint8_t* bitstring,
                           qt_net** out) {
  if (!out) return fail(QT_EINVAL, "qt_build_network: out is NULL");
  *out = nullptr;
  if (!gammas || !betas || !bitstring || (n_edges > 0 && !edges))
    return fail(QT_EINVAL, "qt_build_network: null input array");
  if (n_vertices < 1 || p < 1 || n_edges < 0)
    return fail(QT_EINVAL, "qt_build_network: need n_vertices >= 1, p >= 1, n_edges >= 0");
  if ((int64_t)n_vertices * p > (1 << 20))
    return fail(QT_EINVAL, "qt_build_network: more than 2^20 variables");
  std::set<std::pair<int, int>> seen;
  for (int e = 0; e < n_edges; ++e) {
    int a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || b < 0 || a >= n_vertices || b >= n_vertices)
      return fail(QT_EINVAL, "qt_build_network: edge id out of range");
    if (a == b) return fail(QT_EINVAL, "qt_build_network: self-loop");
    if (!seen.insert({std::min(a, b), std::max(a, b)}).second)
      return fail(QT_EINVAL, "qt_build_network: repeated edge");
  }
  for (int v = 0; v < n_vertices; ++v)
    if (bitstring[v] > 1) return fail(QT_EINVAL, "qt_build_network: bit not 0/1");
  for (int k = 0; k < p; ++k)
    if (!std::isfinite(gammas[k]) || !std::isfinite(betas[k]))
      return fail(QT_EINVAL, "qt_build_network: angle not finite");
  qt_net* net = new (std::nothrow) qt_net();
  if (!net) return fail(QT_ENOMEM, "qt_build_network: out of host memory");
  try {
    net->n = n_vertices;
    net->p = p;
    net->n_edges = n_edges;
    net->n_vars = n_vertices * p;
    net->edges.assign(edges, edges + 2 * (size_t)n_edges);
    net->gammas.assign(gammas, gammas + p);
    net->betas.assign(betas, betas + p);
    net->z.assign(bitstring, bitstring + n_vertices);
    make_tensors(net);
  } catch (const std::bad_alloc&) {
    delete net;
    return fail(QT_ENOMEM, "qt_build_network: out of host memory");
  }
  *out = net;
  return ok();
}

qt_status qt_set_angles(qt_net* net, const double* gammas, const double* betas) {
  if (!check_net(net) || !gammas || !betas) return fail(QT_EINVAL, "qt_set_angles: null argument");
  for (int k = 0; k < net->p; ++k)
    if (!std::isfinite(gammas[k]) || !std::isfinite(betas[k]))
      return fail(QT_EINVAL, "qt_set_angles: angle not finite");
  net->gammas.assign(gammas, gammas + net->p);
  net->betas.assign(betas, betas + net->p);
  make_tensors(net);
  net->stage_dirty = true;
  net->data_version++;
  return ok();
}

qt_status qt_set_bitstring(qt_net* net, const uint8_t* bitstring) {
  if (!check_net(net) || !bitstring) return fail(QT_EINVAL, "qt_set_bitstring: null argument");
  for (int v = 0; v < net->n; ++v)
    if (bitstring[v] > 1) return fail(QT_EINVAL, "qt_set_bitstring: bit not 0/1");
  net->z.assign(bitstring, bitstring + net->n);
  make_tensors(net);
  net->stage_dirty = true;
  net->data_version++;
  return ok();
}

qt_status qt_set_open(qt_net* net, const int32_t* qubits, int32_t a) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_set_open: null network");
  if (a < 0 || a > QT_MAX_OPEN || (a > 0 && !qubits))
    return fail(QT_EINVAL, "qt_set_open: need 0 <= a <= QT_MAX_OPEN and a qubit list");
  std::set<int32_t> seen;
  for (int j = 0; j < a; ++j)
    if (qubits[j] < 0 || qubits[j] >= net->n || !seen.insert(qubits[j]).second)
      return fail(QT_EINVAL, "qt_set_open: qubit repeated or out of range");
  try {
    net->open.assign(qubits, qubits + a);
    net->n_vars = net->n * net->p + a;
    make_tensors(net);
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_set_open: out of host memory");
  }
  net->plan = qt::SlicePlan();
  net->ordered = false;
  net->sched = qt::Schedule();
  net->stage_dirty = true;
  return ok();
}

qt_status qt_order(qt_net* net, int32_t algo, uint64_t seed, int32_t* width_out) {
  (void)seed;
  if (!check_net(net)) return fail(QT_EINVAL, "qt_order: null network");
  if (algo != QT_GREEDY_MINFILL && algo != QT_GREEDY_MINDEG)
    return fail(QT_EINVAL, "qt_order: unknown ordering rule");
  try {
    qt::BitGraph g = qt::network_graph(net);
    qt::OrderResult r = qt::greedy_order(g, algo);
    net->plan = qt::SlicePlan();
    net->plan.order = r.order;
    net->plan.widths = r.widths;
    int w = 0;
    for (int x : r.widths) w = std::max(w, x);
    net->plan.width = w;
    net->algo = algo;
    net->ordered = true;
    net->sched = qt::Schedule();
    net->stage_dirty = true;
    if (width_out) *width_out = w;
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_order: out of host memory");
  }
  return ok();
}

qt_status qt_order_rgreedy(qt_net* net, double tau, int32_t q, uint64_t seed, int32_t* width_out) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_order_rgreedy: null network");
  if (!(tau > 0.0) || !std::isfinite(tau) || q < 1)
    return fail(QT_EINVAL, "qt_order_rgreedy: need a finite tau > 0 and q >= 1");
  try {
    qt::BitGraph g = qt::network_graph(net);
    qt::OrderResult r = qt::rgreedy_order(g, tau, q, seed);
    net->plan = qt::SlicePlan();
    net->plan.order = r.order;
    net->plan.widths = r.widths;
    net->plan.greedy_runs = q;
    int w = 0;
    for (int x : r.widths) w = std::max(w, x);
    net->plan.width = w;
    net->algo = QT_GREEDY_MINDEG;  // the rule rgreedy randomises, for later slicing
    net->ordered = true;
    net->sched = qt::Schedule();
    net->stage_dirty = true;
    if (width_out) *width_out = w;
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_order_rgreedy: out of host memory");
  }
  return ok();
}

qt_status qt_slice(qt_net* net, int32_t width_limit, int32_t max_vars, int32_t r, int32_t* k_out,
                   int32_t* width_out) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_slice: null network");
  if (!net->ordered) return fail(QT_ESTATE, "qt_slice: call qt_order first");
  if (width_limit < 1 || r < 1 || max_vars < 0 || max_vars > 62)
    return fail(QT_EINVAL, "qt_slice: need width_limit >= 1, r >= 1, 0 <= max_vars <= 62");
  try {
    qt::BitGraph g = qt::network_graph(net);
    net->plan = qt::step_dependent_slicing(g, net->algo, width_limit, max_vars, r);
    net->sched = qt::Schedule();
    net->stage_dirty = true;
    if (k_out) *k_out = (int32_t)net->plan.sliced.size();
    if (width_out) *width_out = net->plan.width;
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_slice: out of host memory");
  }
  return ok();
}

static qt_status copy_out(const std::vector<int32_t>& v, int32_t* dst, int32_t cap, int32_t* len) {
  if (!len) return fail(QT_EINVAL, "null length pointer");
  *len = (int32_t)v.size();
  if (dst)
    for (int32_t i = 0; i < cap && i < (int32_t)v.size(); ++i) dst[i] = v[i];
  return ok();
}

qt_status qt_get_order(const qt_net* net, int32_t* order, int32_t cap, int32_t* len) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_get_order: null network");
  if (!net->ordered) return fail(QT_ESTATE, "qt_get_order: call qt_order first");
  return copy_out(net->plan.order, order, cap, len);
}

qt_status qt_get_widths(const qt_net* net, int32_t* widths, int32_t cap, int32_t* len) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_get_widths: null network");
  if (!net->ordered) return fail(QT_ESTATE, "qt_get_widths: call qt_order first");
  return copy_out(net->plan.widths, widths, cap, len);
}

qt_status qt_get_slices(const qt_net* net, int32_t* vars, int32_t cap, int32_t* len,
                        int32_t* slice_step) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_get_slices: null network");
  if (!net->ordered) return fail(QT_ESTATE, "qt_get_slices: call qt_order first");
  if (slice_step) *slice_step = net->plan.slice_step;
  return copy_out(net->plan.sliced, vars, cap, len);
}

qt_status qt_num_tensors(const qt_net* net, int32_t* count, int32_t* n_vars) {
  if (!check_net(net) || !count) return fail(QT_EINVAL, "qt_num_tensors: null argument");
  *count = (int32_t)net->tensors.size();
  if (n_vars) *n_vars = net->n_vars;
  return ok();
}

qt_status qt_get_tensor(const qt_net* net, int32_t t, int32_t* labels, int32_t* rank,
                        double* data) {
  if (!check_net(net) || !rank) return fail(QT_EINVAL, "qt_get_tensor: null argument");
  if (t < 0 || t >= (int32_t)net->tensors.size())
    return fail(QT_EINVAL, "qt_get_tensor: tensor index out of range");
  const qt::Tensor& T = net->tensors[t];
  *rank = (int32_t)T.labels.size();
  if (labels)
    for (size_t i = 0; i < T.labels.size(); ++i) labels[i] = T.labels[i];
  if (data) std::memcpy(data, T.data.data(), T.data.size() * sizeof(double));
  return ok();
}

qt_status qt_prepare(qt_net* net, int32_t precision, int32_t batch, size_t* workspace_bytes) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_prepare: null network");
  if (!net->ordered) return fail(QT_ESTATE, "qt_prepare: call qt_order first");
  if (precision < QT_FP32_SIMT || precision > QT_FP64)
    return fail(QT_EINVAL, "qt_prepare: unknown precision");
  if (batch < 1) return fail(QT_EINVAL, "qt_prepare: batch must be >= 1");
  std::string err;
  try {
    if (!qt::compile_schedule(net->tensors, net->n_vars, net->plan, precision, batch, net->fuse,
                              net->sched, err, (int)net->open.size())) {
      net->sched = qt::Schedule();
      return fail(err.find("rank") != std::string::npos ? QT_ERANGE : QT_EINVAL,
                  "qt_prepare: " + err);
    }
    net->sched.force_gemm = net->force_gemm;
    net->sched.force_stream = net->force_stream;
    net->sched.force_tri = net->force_tri;
    net->sched.tma_block = net->tma_block;
    net->sched.tcgen05 = net->tcgen05;
    net->sched.force_scaled = net->force_scaled;
  } catch (const std::bad_alloc&) {
    net->sched = qt::Schedule();
    return fail(QT_ENOMEM, "qt_prepare: out of host memory");
  }
  net->stage_dirty = true;
  if (workspace_bytes) *workspace_bytes = net->sched.total_bytes;
  return ok();
}

qt_status qt_stats(const qt_net* net, char* buf, size_t cap, size_t* needed) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_stats: null network");
  if (!net->sched.valid) return fail(QT_ESTATE, "qt_stats: call qt_prepare first");
  std::string s = qt::schedule_json(net->sched, net->plan);
  s.pop_back();
  s += ",\"launches\":" + std::to_string(net->launches) +
       ",\"tma_gemm_launches\":" + std::to_string(net->tma_launches) +
       ",\"stream_gemm_launches\":" + std::to_string(net->stream_launches) +
       ",\"tcgen05_gemm_launches\":" + std::to_string(net->umma_launches) + "}";
  if (needed) *needed = s.size() + 1;
  if (buf && cap > 0) {
    size_t n = std::min(cap - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = '\0';
  }
  return ok();
}

static qt_status check_ws(const qt_net* net, void* ws, size_t bytes, const char* who) {
  if (!ws) return fail(QT_EINVAL, std::string(who) + ": null workspace");
  if (((uintptr_t)ws) % 256 != 0)
    return fail(QT_EINVAL, std::string(who) + ": workspace not 256-byte aligned");
  if (bytes < net->sched.total_bytes)
    return fail(QT_ENOMEM, std::string(who) + ": workspace smaller than qt_prepare's size");
  return QT_OK;
}

qt_status qt_upload(qt_net* net, void* workspace, size_t workspace_bytes, void* stream) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_upload: null network");
  if (!net->sched.valid) return fail(QT_ESTATE, "qt_upload: call qt_prepare first");
  qt_status s = check_ws(net, workspace, workspace_bytes, "qt_upload");
  if (s != QT_OK) return s;
  std::string err;
  s = qt::upload(net, workspace, workspace_bytes, stream, err);
  if (s != QT_OK) return fail(s, "qt_upload: " + err);
  return ok();
}

qt_status qt_run(qt_net* net, int64_t first, int64_t count, void* workspace, size_t workspace_bytes,
                 void* stream, double* d_out) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_run: null network");
  if (!net->sched.valid) return fail(QT_ESTATE, "qt_run: call qt_prepare first");
  if (!d_out) return fail(QT_EINVAL, "qt_run: null output pointer");
  if (first < 0 || count < 1 || first + count > net->sched.nslices)
    return fail(QT_EINVAL, "qt_run: slice range outside [0, 2^k)");
  qt_status s = check_ws(net, workspace, workspace_bytes, "qt_run");
  if (s != QT_OK) return s;
  if (net->uploaded_gen != net->sched.generation || net->uploaded_ws != workspace)
    return fail(QT_ESTATE, "qt_run: this workspace does not hold the prepared schedule's upload; "
                           "call qt_upload after qt_prepare");
  if (net->uploaded_data != net->data_version)
    return fail(QT_ESTATE, "qt_run: angles or bitstring changed since qt_upload; call qt_upload");
  std::string err;
  s = qt::run(net, first, count, workspace, stream, d_out, err);
  if (s != QT_OK) return fail(s, "qt_run: " + err);
  return ok();
}

static qt_status contract_impl(qt_net* net, int32_t precision, void* workspace,
                               size_t workspace_bytes, void* stream, double* host_out,
                               const char* who) {
  if (!net->ordered) return fail(QT_ESTATE, std::string(who) + ": call qt_order first");
  std::string err;
  if (!net->sched.valid || net->sched.precision != precision) {
    // the largest batch whose workspace fits
    qt_status s = qt::prepare_fitting(net, precision, workspace_bytes, nullptr, nullptr, err);
    if (s != QT_OK) return fail(s, std::string(who) + ": " + err);
  }
  qt_status s = check_ws(net, workspace, workspace_bytes, who);
  if (s != QT_OK) return s;
  s = qt::upload(net, workspace, workspace_bytes, stream, err);
  if (s != QT_OK) return fail(s, std::string(who) + ": " + err);
  const int64_t A = net->sched.n_amps;
  double* d_out = reinterpret_cast<double*>((char*)workspace + net->sched.off_acc + 16 * A);
  s = qt::run(net, 0, net->sched.nslices, workspace, stream, d_out, err);
  if (s != QT_OK) return fail(s, std::string(who) + ": " + err);
  // the amplitudes and the status word read back together, one stream synchronisation
  int status = 0;
  s = qt::download_result_status(net, workspace, d_out, host_out, 2 * A, &status, stream, err);
  if (s != QT_OK) return fail(s, std::string(who) + ": " + err);
  if (status) return fail(QT_ETIMEOUT, std::string(who) + ": a bounded device wait gave up");
  return ok();
}

qt_status qt_contract(qt_net* net, int32_t precision, void* workspace, size_t workspace_bytes,
                      void* stream, double* amp_re, double* amp_im) {
  if (!check_net(net) || !amp_re || !amp_im) return fail(QT_EINVAL, "qt_contract: null argument");
  if (!net->open.empty())
    return fail(QT_ESTATE, "qt_contract: the network has open qubits; use qt_contract_batch");
  double h[2];
  qt_status s = contract_impl(net, precision, workspace, workspace_bytes, stream, h, "qt_contract");
  if (s != QT_OK) return s;
  *amp_re = h[0];
  *amp_im = h[1];
  return ok();
}

qt_status qt_contract_batch(qt_net* net, int32_t precision, void* workspace,
                            size_t workspace_bytes, void* stream, double* amps) {
  if (!check_net(net) || !amps) return fail(QT_EINVAL, "qt_contract_batch: null argument");
  return contract_impl(net, precision, workspace, workspace_bytes, stream, amps,
                       "qt_contract_batch");
}

qt_status qt_contract_sweep(qt_net* net, int32_t precision, int32_t n_sets, const double* gammas,
                            const double* betas, void* workspace, size_t workspace_bytes,
                            void* stream, double* amps) {
  const char* who = "qt_contract_sweep";
  if (!check_net(net) || !gammas || !betas || !amps)
    return fail(QT_EINVAL, std::string(who) + ": null argument");
  if (n_sets < 1) return fail(QT_EINVAL, std::string(who) + ": need n_sets >= 1");
  if (!net->ordered) return fail(QT_ESTATE, std::string(who) + ": call qt_order first");
  if (!net->open.empty())
    return fail(QT_ESTATE, std::string(who) + ": the network has open qubits");
  for (int64_t e = 0; e < (int64_t)n_sets * net->p; ++e)
    if (!std::isfinite(gammas[e]) || !std::isfinite(betas[e]))
      return fail(QT_EINVAL, std::string(who) + ": angle not finite");
  auto align256 = [](size_t x) { return (x + 255) / 256 * 256; };
  // room after the schedule's workspace: one gate + gate-meta image per set, the amplitudes
  // (the gate image does not depend on the batch)
  auto room = [](const qt_net* nt, const void* arg) {
    const size_t sets = (size_t)*static_cast<const int32_t*>(arg);
    return (qt::stage_image_bytes(nt) + 255) / 256 * 256 * sets + (16 * sets + 255) / 256 * 256;
  };
  auto reserve = [&]() { return room(net, &n_sets); };
  if (!net->sched.valid || net->sched.precision != precision ||
      net->sched.total_bytes + reserve() > workspace_bytes) {
    std::string perr;
    qt_status s = qt::prepare_fitting(net, precision, workspace_bytes, room, &n_sets, perr);
    if (s != QT_OK) return fail(s, std::string(who) + ": " + perr);
  }
  qt_status s = check_ws(net, workspace, workspace_bytes - reserve(), who);
  if (s != QT_OK) return s;
  const qt::Schedule& S = net->sched;
  const size_t img = qt::stage_image_bytes(net);
  const size_t stride = align256(img);
  const size_t staging_off = align256(S.total_bytes);
  const size_t results_off = staging_off + stride * (size_t)n_sets;
  // host: every set's gate and gate-meta image (the order, slices and schedule are reused)
  std::vector<unsigned char> images(stride * (size_t)n_sets);
  for (int k = 0; k < n_sets; ++k) {
    s = qt_set_angles(net, gammas + (size_t)k * net->p, betas + (size_t)k * net->p);
    if (s != QT_OK) return s;
    qt::build_stage(net);
    net->stage_dirty = false;
    std::memcpy(images.data() + (size_t)k * stride, net->gate_stage.data(), img);
  }
  std::string err;
  s = qt::upload(net, workspace, workspace_bytes, stream, err);  // scalar table, last set's gates
  if (s != QT_OK) return fail(s, std::string(who) + ": " + err);
  s = qt::sweep_run(net, workspace, stream, n_sets, images.data(), staging_off, stride,
                    results_off, err);
  if (s != QT_OK) return fail(s, std::string(who) + ": " + err);
  s = qt::download_result(reinterpret_cast<const double*>((char*)workspace + results_off), amps,
                          2 * (int64_t)n_sets, stream, err);
  if (s != QT_OK) return fail(s, std::string(who) + ": " + err);
  int status = 0;
  s = qt::read_status(net, workspace, stream, &status, err);
  if (s != QT_OK) return fail(s, std::string(who) + ": " + err);
  if (status) return fail(QT_ETIMEOUT, std::string(who) + ": a bounded device wait gave up");
  return ok();
}

qt_status qt_launch_plan(qt_net* net, char* buf, size_t cap, size_t* needed) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_launch_plan: null network");
  if (!net->sched.valid) return fail(QT_ESTATE, "qt_launch_plan: call qt_prepare first");
  std::string s, err;
  qt_status r = qt::launch_plan(net, s, err);
  if (r != QT_OK) return fail(r, "qt_launch_plan: " + err);
  if (needed) *needed = s.size() + 1;
  if (buf && cap > 0) {
    size_t n = std::min(cap - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return ok();
}

qt_status qt_profile(qt_net* net, int32_t enable) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_profile: null network");
  qt::prof_clear(net);
  net->prof = enable != 0;
  return ok();
}

qt_status qt_profile_read(qt_net* net, char* buf, size_t cap, size_t* needed) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_profile_read: null network");
  std::string out, err;
  qt_status s = qt::prof_read(net, out, err);
  if (s != QT_OK) return fail(s, "qt_profile_read: " + err);
  if (needed) *needed = out.size() + 1;
  if (buf && cap > 0) {
    size_t n = std::min(cap - 1, out.size());
    std::memcpy(buf, out.data(), n);
    buf[n] = '\0';
  }
  return ok();
}

qt_status qt_plan_info(const qt_net* net, int64_t* greedy_runs, double* plan_cost) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_plan_info: null network");
  if (!net->ordered) return fail(QT_ESTATE, "qt_plan_info: call qt_order first");
  if (greedy_runs) *greedy_runs = net->plan.greedy_runs;
  if (plan_cost) {
    double c = 0.0;
    for (int32_t w : net->plan.widths) c += std::ldexp(1.0, w);
    *plan_cost = c;
  }
  return ok();
}

qt_status qt_slice_dataset(const qt_net* net, int32_t topv, float* features, float* labels,
                           int32_t* meta, int32_t cap, int32_t* count) {
  if (!check_net(net) || !count) return fail(QT_EINVAL, "qt_slice_dataset: null argument");
  if (!net->ordered) return fail(QT_ESTATE, "qt_slice_dataset: call qt_order first");
  if (topv < 1) return fail(QT_EINVAL, "qt_slice_dataset: topv must be >= 1");
  std::vector<float> f, l;
  std::vector<int32_t> m;
  try {
    qt::slice_dataset(net, topv, f, l, m);
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_slice_dataset: out of host memory");
  }
  *count = (int32_t)l.size();
  const int32_t n = std::min<int32_t>(cap, (int32_t)l.size());
  if (features && n > 0) std::memcpy(features, f.data(), sizeof(float) * n * qt::kProposalFeatures);
  if (labels && n > 0) std::memcpy(labels, l.data(), sizeof(float) * n);
  if (meta && n > 0) std::memcpy(meta, m.data(), sizeof(int32_t) * n * 3);
  return ok();
}

qt_status qt_slice_learned(qt_net* net, const float* params, int32_t hidden, int32_t width_limit,
                           int32_t max_vars, int32_t r, int32_t topv, int32_t topm, int32_t spread,
                           int32_t* k_out, int32_t* width_out) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_slice_learned: null network");
  if (!net->ordered) return fail(QT_ESTATE, "qt_slice_learned: call qt_order first");
  if (width_limit < 1 || r < 1 || max_vars < 0 || max_vars > 62 || topv < 1 || topm < 0 ||
      spread < 0 || (!params && spread < 1) ||
      (params && (hidden < 1 || hidden > 1024)))
    return fail(QT_EINVAL, "qt_slice_learned: argument out of range");
  try {
    int64_t runs = 0;
    net->plan =
        qt::learned_slicing(net, params, hidden, width_limit, max_vars, r, topv, topm, spread, runs);
    net->sched = qt::Schedule();
    net->stage_dirty = true;
    if (k_out) *k_out = (int32_t)net->plan.sliced.size();
    if (width_out) *width_out = net->plan.width;
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_slice_learned: out of host memory");
  }
  return ok();
}

qt_status qt_order_dataset(const qt_net* net, int32_t topc, int32_t stride, float* features,
                           float* labels, int32_t* meta, int32_t cap, int32_t* count) {
  if (!check_net(net) || !count) return fail(QT_EINVAL, "qt_order_dataset: null argument");
  if (!net->ordered) return fail(QT_ESTATE, "qt_order_dataset: call qt_order first");
  if (topc < 2 || stride < 1) return fail(QT_EINVAL, "qt_order_dataset: need topc >= 2, stride >= 1");
  std::vector<float> f, l;
  std::vector<int32_t> m;
  try {
    qt::order_dataset(net, topc, stride, f, l, m);
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_order_dataset: out of host memory");
  }
  *count = (int32_t)l.size();
  const int32_t n = std::min<int32_t>(cap, (int32_t)l.size());
  if (features && n > 0) std::memcpy(features, f.data(), sizeof(float) * n * qt::kProposalFeatures);
  if (labels && n > 0) std::memcpy(labels, l.data(), sizeof(float) * n);
  if (meta && n > 0) std::memcpy(meta, m.data(), sizeof(int32_t) * n * 3);
  return ok();
}

qt_status qt_order_learned(qt_net* net, const float* params, int32_t hidden, int32_t topc,
                           int32_t judge, int32_t* width_out, int32_t* learned_kept) {
  if (!check_net(net) || !params) return fail(QT_EINVAL, "qt_order_learned: null argument");
  if (hidden < 1 || hidden > 1024 || topc < 1)
    return fail(QT_EINVAL, "qt_order_learned: need 1 <= hidden <= 1024 and topc >= 1");
  try {
    const qt::BitGraph g = qt::network_graph(net);
    const int algo = net->algo;
    const qt::OrderResult gr = qt::greedy_order(g, algo);
    int W0 = 0;
    for (int32_t w : gr.widths) W0 = std::max(W0, w);
    qt::OrderResult lr = qt::learned_order(g, algo, params, hidden, topc, net->n_vars, W0);
    auto key = [](const qt::OrderResult& o) {
      int w = 0;
      double c = 0.0;
      for (int32_t x : o.widths) {
        w = std::max(w, x);
        c += std::ldexp(1.0, x);
      }
      return std::make_pair(w, c);
    };
    const bool keep = !judge || key(lr) < key(gr);
    const qt::OrderResult& r = keep ? lr : gr;
    net->plan = qt::SlicePlan();
    net->plan.order = r.order;
    net->plan.widths = r.widths;
    net->plan.greedy_runs = judge ? 2 : 1;
    int w = 0;
    for (int x : r.widths) w = std::max(w, x);
    net->plan.width = w;
    net->ordered = true;
    net->sched = qt::Schedule();
    net->stage_dirty = true;
    if (width_out) *width_out = w;
    if (learned_kept) *learned_kept = keep ? 1 : 0;
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_order_learned: out of host memory");
  }
  return ok();
}

qt_status qt_mlp_forward_host(const float* params, int32_t n_features, int32_t hidden,
                              const float* x, int32_t batch, float* y) {
  if (!params || !x || !y || n_features < 1 || hidden < 1 || batch < 0)
    return fail(QT_EINVAL, "qt_mlp_forward_host: bad argument");
  qt::mlp_forward_host(params, n_features, hidden, x, batch, y);
  return ok();
}

qt_status qt_set_option(qt_net* net, int32_t option, int64_t value) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_set_option: null network");
  switch (option) {
    case QT_OPT_FUSION:
      net->fuse = value != 0;
      net->sched = qt::Schedule();  // prepare again
      break;
    case QT_OPT_GRAPHS:
      net->graphs = value != 0;
      break;
    case QT_OPT_GEMM:
      if (value < 0 || value > 2) return fail(QT_EINVAL, "qt_set_option: QT_OPT_GEMM takes 0..2");
      net->force_gemm = value != 0;
      net->force_stream = value == 2;
      net->sched = qt::Schedule();  // prepare again
      break;
    case QT_OPT_SEGMENTS:
      if (value < 0 || value > 13) return fail(QT_EINVAL, "qt_set_option: QT_OPT_SEGMENTS takes 0..13");
      net->segments = value != 0;
      net->seg_max_u = value >= 2 ? (int)value : 12;
      net->sched = qt::Schedule();  // prepare again
      break;
    case QT_OPT_CONCURRENT:
      net->concurrent = value != 0;
      net->sched = qt::Schedule();  // prepare again
      break;
    case QT_OPT_TRIANGLE:
      net->force_tri = value != 0;
      net->sched = qt::Schedule();  // prepare again
      break;
    case QT_OPT_TMA:
      if (value < 0 || value > 4) return fail(QT_EINVAL, "qt_set_option: QT_OPT_TMA takes 0..4");
      net->tma = value != 0;
      net->tma_block = value >= 2 ? (int)value - 1 : 0;
      net->sched = qt::Schedule();  // prepare again
      break;
    case QT_OPT_SCALED:
      net->force_scaled = value != 0;
      net->sched = qt::Schedule();  // prepare again
      break;
    case QT_OPT_SEG_CLUSTER:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
        return fail(QT_EINVAL, "qt_set_option: QT_OPT_SEG_CLUSTER takes 0, 1, 2, 4 or 8");
      net->seg_cluster = (int)value;
      net->sched = qt::Schedule();  // prepare again
      break;
    case QT_OPT_TCGEN05:
      if (value < 0 || value > 4) return fail(QT_EINVAL, "qt_set_option: QT_OPT_TCGEN05 takes 0..4");
      net->tcgen05 = (int)value;
      net->sched = qt::Schedule();  // prepare again
      break;
    default:
      return fail(QT_EINVAL, "qt_set_option: unknown option");
  }
  return ok();
}

qt_status qt_autotune(qt_net* net, void* workspace, size_t workspace_bytes, void* stream, char* buf,
                      size_t cap, size_t* needed) {
  if (!check_net(net)) return fail(QT_EINVAL, "qt_autotune: null network");
  if (!net->sched.valid) return fail(QT_ESTATE, "qt_autotune: call qt_prepare first");
  qt_status s = check_ws(net, workspace, workspace_bytes, "qt_autotune");
  if (s != QT_OK) return s;
  if (net->uploaded_gen != net->sched.generation || net->uploaded_ws != workspace ||
      net->uploaded_data != net->data_version)
    return fail(QT_ESTATE, "qt_autotune: call qt_upload after qt_prepare or new angles");
  std::string report, err;
  s = qt::autotune(net, workspace, stream, report, err);
  if (s != QT_OK) return fail(s, "qt_autotune: " + err);
  if (needed) *needed = report.size() + 1;
  if (buf && cap > 0) {
    size_t n = std::min(cap - 1, report.size());
    std::memcpy(buf, report.data(), n);
    buf[n] = '\0';
  }
  return ok();
}

void qt_free(qt_net* net) { delete net; }

}  // extern "C"
