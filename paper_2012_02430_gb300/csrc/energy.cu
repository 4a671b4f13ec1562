// Batched lightcone energy on the GPU: one persistent kernel launch contracts
// every edge's lightcone network (Sec. III.A-B), replayed from a captured CUDA
// graph. Blocks take networks from an atomic work counter (largest first) and
// run each network's bucket steps (Alg. 1, fused where indices die together)
// cooperatively in a per-block scratch arena; the per-edge <Z_u Z_v> and the
// energy sum_E (1 - <Z_u Z_v>) / 2 are written in FP64.
//
// Magnitudes stay bounded here (a lightcone network has a few dozen binary
// indices and gate entries of modulus <= 1), so no exponent tracking is used.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>
#include <sstream>
#include <string>

#include "energy_internal.h"

namespace qt {
void set_last_error(const std::string& msg);
}

namespace {

using qt::ENet;
using qt::EOp;
using qt::EStep;

template <typename R> struct C2T;
template <> struct C2T<float> { using t = float2; };
template <> struct C2T<double> { using t = double2; };

__device__ __forceinline__ unsigned int pext32(unsigned int x, unsigned int m) {
  unsigned int r = 0;
  int k = 0;
  while (m) {
    const int b = __ffs(m) - 1;
    r |= ((x >> b) & 1u) << k;
    ++k;
    m &= m - 1;
  }
  return r;
}

template <typename R>
__device__ __forceinline__ void cmul(R& ar, R& ai, R br, R bi) {
  const R r = ar * br - ai * bi;
  const R i = ar * bi + ai * br;
  ar = r;
  ai = i;
}

// one bucket step (or fused group) of a network, by the whole block
template <typename R>
__device__ void block_step(const EStep& st, const EOp* ops, const R* gates, R* arena) {
  using C2 = typename C2T<R>::t;
  const int lane = threadIdx.x & 31;
  const unsigned int npairs = 1u << (st.u - 1);
  const int grp = 1 << (st.nsum - 1);
  for (unsigned int base = 0; base < npairs; base += blockDim.x) {
    const unsigned int g = base + threadIdx.x;
    const bool active = g < npairs;
    const unsigned int I = g << 1;
    R p0r = 1, p0i = 0, p1r = 1, p1i = 0;
    if (active) {
      for (int j = 0; j < st.m; ++j) {
        const EOp o = ops[j];
        if (o.level != 0) continue;
        const R* src = o.in_arena ? arena : gates;
        const unsigned int off = o.off + pext32(I, o.umask);
        R r0, i0, r1, i1;
        if (o.umask & 1u) {
          const C2 a = reinterpret_cast<const C2*>(src)[off];
          const C2 b = reinterpret_cast<const C2*>(src)[off + 1];
          r0 = a.x; i0 = a.y; r1 = b.x; i1 = b.y;
        } else {
          const C2 a = reinterpret_cast<const C2*>(src)[off];
          r0 = r1 = a.x; i0 = i1 = a.y;
        }
        cmul<R>(p0r, p0i, r0, i0);
        cmul<R>(p1r, p1i, r1, i1);
      }
    }
    R sr = active ? p0r + p1r : R(0), si = active ? p0i + p1i : R(0);
    for (int l = 1; l < st.nsum; ++l) {
      if (active) {
        for (int j = 0; j < st.m; ++j) {
          const EOp o = ops[j];
          if (o.level != l) continue;
          const R* src = o.in_arena ? arena : gates;
          const C2 a = reinterpret_cast<const C2*>(src)[o.off + pext32(I, o.umask)];
          cmul<R>(sr, si, a.x, a.y);
        }
      }
      sr += __shfl_xor_sync(0xffffffffu, sr, 1 << (l - 1));
      si += __shfl_xor_sync(0xffffffffu, si, 1 << (l - 1));
    }
    if (active && (lane & (grp - 1)) == 0) {
      C2 w;
      w.x = sr;
      w.y = si;
      reinterpret_cast<C2*>(arena)[st.out + (I >> st.nsum)] = w;
    }
  }
}

// Persistent kernel: each block repeatedly takes the next network index from
// the counter (no waiting: an atomic add) until none is left.
// With an angle sweep, work item w is network w % nnets of angle set w / nnets: the
// set's gate image starts gate_stride elements after the previous one, and its
// <Z_u Z_v> go to zz[set * nnets + edge].
template <typename R>
__global__ void k_energy(const ENet* nets, int nnets, int nsets, long long gate_stride,
                         const EStep* steps, const EOp* ops, const uint32_t* scalars,
                         const R* gates, R* arenas, long long arena_elems, int* counter,
                         double* zz) {
  using C2 = typename C2T<R>::t;
  R* arena = arenas + 2 * arena_elems * (long long)blockIdx.x;
  __shared__ int cur;
  const int nwork = nnets * nsets;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int w = cur;
    __syncthreads();
    if (w >= nwork) break;
    const int set = w / nnets, ni = w - set * nnets;
    const ENet nd = nets[ni];
    const R* g = gates + 2 * gate_stride * (long long)set;
    for (uint32_t s = 0; s < nd.nsteps; ++s) {
      const EStep st = steps[nd.first_step + s];
      block_step<R>(st, ops + st.first_op, g, arena);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double pr = 1.0, pi = 0.0;
      for (uint32_t k = 0; k < nd.nscalars; ++k) {
        const C2 v = reinterpret_cast<const C2*>(arena)[scalars[nd.first_scalar + k]];
        const double vr = (double)v.x, vi = (double)v.y;
        const double nr = pr * vr - pi * vi, nim = pr * vi + pi * vr;
        pr = nr;
        pi = nim;
      }
      zz[(long long)set * nnets + nd.edge] = pr * nd.norm;
    }
    __syncthreads();
  }
}

// energy = sum over edges of (1 - zz_e) / 2, fixed order; block b: angle set b
__global__ void __launch_bounds__(1024) k_energy_sum(const double* zz, int n, double* out) {
  __shared__ double sh[1024];
  zz += (long long)blockIdx.x * n;
  out += blockIdx.x;
  double acc = 0.0;
  for (int e = threadIdx.x; e < n; e += 1024) acc += 0.5 * (1.0 - zz[e]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

struct EGraph {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;
  void* ws = nullptr;
  double* zz = nullptr;
  double* energy = nullptr;
  int threads = 0, blocks = 0;
  ~EGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (capture) cudaStreamDestroy(capture);
  }
};

thread_local std::string g_msg;

qt_status fail(qt_status s, const std::string& m) {
  qt::set_last_error(m);
  return s;
}

bool cuda_ok(cudaError_t e, const char* what, std::string& err) {
  if (e == cudaSuccess) return true;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
    n = 148;
  return n;
}

template <typename R>
int blocks_for(int threads) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_energy<R>, threads, 0) != cudaSuccess ||
      per < 1)
    per = 1;
  return per * sm_count();
}

void layout(qt_energy* E) {
  const size_t eb = (size_t)E->elem_bytes;
  size_t off = 0;
  E->off_gates = off;
  off = a256(off + (size_t)E->gate_elems * eb);
  E->off_ops = off;
  off = a256(off + E->h_ops.size() * sizeof(EOp));
  E->off_steps = off;
  off = a256(off + E->h_steps.size() * sizeof(EStep));
  E->off_nets = off;
  off = a256(off + E->h_nets.size() * sizeof(ENet));
  E->off_scalars = off;
  off = a256(off + E->h_scalars.size() * sizeof(uint32_t) + 4);
  E->off_zz = off;
  off = a256(off + (E->h_nets.size() + 1) * sizeof(double));
  E->off_counter = off;
  off = a256(off + 64);
  E->off_arenas = off;
  off = a256(off + (size_t)E->blocks * (size_t)E->arena_elems * eb);
  E->total_bytes_ws = off;
}

void layout_sweep(qt_energy* E, int nsets) {
  const size_t eb = (size_t)E->elem_bytes;
  size_t off = 0;
  E->sw_off_gates = off;
  off = a256(off + (size_t)nsets * (size_t)E->gate_elems * eb);
  E->sw_off_ops = off;
  off = a256(off + E->h_ops.size() * sizeof(EOp));
  E->sw_off_steps = off;
  off = a256(off + E->h_steps.size() * sizeof(EStep));
  E->sw_off_nets = off;
  off = a256(off + E->h_nets.size() * sizeof(ENet));
  E->sw_off_scalars = off;
  off = a256(off + E->h_scalars.size() * sizeof(uint32_t) + 4);
  E->sw_off_zz = off;
  off = a256(off + (size_t)nsets * E->h_nets.size() * sizeof(double));
  E->sw_off_energy = off;
  off = a256(off + (size_t)nsets * sizeof(double));
  E->sw_off_counter = off;
  off = a256(off + 64);
  E->sw_off_arenas = off;
  off = a256(off + (size_t)E->blocks * (size_t)E->arena_elems * eb);
  // device assembly of the gate images: template, slots, codes, per-set table
  if (E->sw_template.empty()) qt::energy_sweep_template(E);
  E->sw_off_tmpl = off;
  off = a256(off + E->sw_template.size());
  E->sw_off_slots = off;
  off = a256(off + E->sw_slots.size() * sizeof(uint32_t) + 4);
  E->sw_off_codes = off;
  off = a256(off + E->sw_codes.size() * sizeof(uint32_t) + 4);
  E->sw_off_table = off;
  off = a256(off + (size_t)nsets * E->p * 8 * eb);
  E->sw_total = off;
  E->sweep_sets = nsets;
  E->sw_tmpl_ws = nullptr;
}

// Every set's gate image: the template copied, then the angle-dependent gates written
// from the set's table (phase {1, e, e, 1} with e = exp(-i g) or its conjugate; mixer
// {c, -i s, -i s, c}). One thread per complex element of the images, then one per gate.
template <typename R>
__global__ void k_sweep_copy(const R* __restrict__ tmpl, long long img_c, int nsets, R* images) {
  using C2 = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
  const C2* src = reinterpret_cast<const C2*>(tmpl);
  C2* dst = reinterpret_cast<C2*>(images);
  const long long total = img_c * nsets;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = src[e % img_c];
}

template <typename R>
__global__ void k_sweep_gates(const uint32_t* __restrict__ slots, const uint32_t* __restrict__ codes,
                              int nslots, const R* __restrict__ table, int p, int nsets,
                              long long img_c, R* images) {
  const long long total = (long long)nslots * nsets;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e / nslots), j = (int)(e - (long long)q * nslots);
    const uint32_t code = codes[j];
    const int kind = code & 15, k = (code >> 4) & 255, side = code >> 12;
    const R* t = table + ((size_t)q * p + (k - 1)) * 8 + (kind - 1) * 4 + (side - 1) * 2;
    const R a = t[0], b = t[1];
    R* g = images + 2 * ((long long)q * img_c + slots[j]);
    if (kind == 1) {
      g[0] = R(1); g[1] = R(0); g[2] = a; g[3] = b; g[4] = a; g[5] = b; g[6] = R(1); g[7] = R(0);
    } else {
      g[0] = a; g[1] = R(0); g[2] = R(0); g[3] = -b; g[4] = R(0); g[5] = -b; g[6] = a; g[7] = R(0);
    }
  }
}

template <typename R>
qt_status enqueue_sweep(qt_energy* E, int nsets, char* base, cudaStream_t s, double* zz,
                        double* energy, std::string& err) {
  if (!cuda_ok(cudaMemsetAsync(base + E->sw_off_counter, 0, sizeof(int), s), "reset counter", err))
    return QT_ECUDA;
  k_energy<R><<<E->blocks, E->block_threads, 0, s>>>(
      reinterpret_cast<const ENet*>(base + E->sw_off_nets), (int)E->h_nets.size(), nsets,
      (long long)E->gate_elems, reinterpret_cast<const EStep*>(base + E->sw_off_steps),
      reinterpret_cast<const EOp*>(base + E->sw_off_ops),
      reinterpret_cast<const uint32_t*>(base + E->sw_off_scalars),
      reinterpret_cast<const R*>(base + E->sw_off_gates),
      reinterpret_cast<R*>(base + E->sw_off_arenas), (long long)E->arena_elems,
      reinterpret_cast<int*>(base + E->sw_off_counter), zz);
  k_energy_sum<<<nsets, 1024, 0, s>>>(zz, (int)E->h_nets.size(), energy);
  if (!cuda_ok(cudaGetLastError(), "energy sweep launch", err)) return QT_ECUDA;
  return QT_OK;
}

template <typename R>
qt_status enqueue(qt_energy* E, char* base, cudaStream_t s, double* zz, double* energy,
                  std::string& err) {
  if (!cuda_ok(cudaMemsetAsync(base + E->off_counter, 0, sizeof(int), s), "reset counter", err))
    return QT_ECUDA;
  k_energy<R><<<E->blocks, E->block_threads, 0, s>>>(
      reinterpret_cast<const ENet*>(base + E->off_nets), (int)E->h_nets.size(), 1, 0ll,
      reinterpret_cast<const EStep*>(base + E->off_steps),
      reinterpret_cast<const EOp*>(base + E->off_ops),
      reinterpret_cast<const uint32_t*>(base + E->off_scalars),
      reinterpret_cast<const R*>(base + E->off_gates), reinterpret_cast<R*>(base + E->off_arenas),
      (long long)E->arena_elems, reinterpret_cast<int*>(base + E->off_counter), zz);
  k_energy_sum<<<1, 1024, 0, s>>>(zz, (int)E->h_nets.size(), energy);
  if (!cuda_ok(cudaGetLastError(), "energy launch", err)) return QT_ECUDA;
  return QT_OK;
}

qt_status run_energy(qt_energy* E, char* base, cudaStream_t s, double* zz, double* energy,
                     bool use_graph, std::string& err) {
  const bool f64 = E->precision == QT_FP64;
  if (!use_graph)
    return f64 ? enqueue<double>(E, base, s, zz, energy, err)
               : enqueue<float>(E, base, s, zz, energy, err);
  if (!E->engine) E->engine = new EGraph();
  EGraph& g = *static_cast<EGraph*>(E->engine);
  if (!(g.exec && g.ws == base && g.zz == zz && g.energy == energy &&
        g.threads == E->block_threads && g.blocks == E->blocks)) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    if (!g.capture &&
        !cuda_ok(cudaStreamCreateWithFlags(&g.capture, cudaStreamNonBlocking), "capture stream", err))
      return QT_ECUDA;
    if (!cuda_ok(cudaStreamBeginCapture(g.capture, cudaStreamCaptureModeThreadLocal), "capture", err))
      return QT_ECUDA;
    qt_status r = f64 ? enqueue<double>(E, base, g.capture, zz, energy, err)
                      : enqueue<float>(E, base, g.capture, zz, energy, err);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(g.capture, &gr);
    if (r != QT_OK) {
      if (gr) cudaGraphDestroy(gr);
      return r;
    }
    if (!cuda_ok(e, "end capture", err)) return QT_ECUDA;
    e = cudaGraphInstantiate(&g.exec, gr, 0);
    cudaGraphDestroy(gr);
    if (!cuda_ok(e, "instantiate", err)) {
      g.exec = nullptr;
      return QT_ECUDA;
    }
    g.ws = base;
    g.zz = zz;
    g.energy = energy;
    g.threads = E->block_threads;
    g.blocks = E->blocks;
  }
  if (!cuda_ok(cudaGraphLaunch(g.exec, s), "graph launch", err)) return QT_ECUDA;
  return QT_OK;
}

qt_status check_ws(qt_energy* E, void* ws, size_t bytes, const char* who) {
  if (!E) return fail(QT_EINVAL, std::string(who) + ": null handle");
  if (!E->compiled) return fail(QT_ESTATE, std::string(who) + ": call qt_energy_prepare first");
  if (!ws) return fail(QT_EINVAL, std::string(who) + ": null workspace");
  if ((uintptr_t)ws % 256) return fail(QT_EINVAL, std::string(who) + ": workspace not 256-byte aligned");
  if (bytes < E->total_bytes_ws)
    return fail(QT_ENOMEM, std::string(who) + ": workspace smaller than qt_energy_prepare's size");
  return QT_OK;
}

}  // namespace

qt_energy::~qt_energy() { delete static_cast<EGraph*>(engine); }

extern "C" {

qt_status qt_energy_build(const int32_t* edges, int32_t n_vertices, int32_t n_edges, int32_t p,
                          const double* gammas, const double* betas, int32_t algo,
                          qt_energy** out) {
  if (!out) return fail(QT_EINVAL, "qt_energy_build: out is NULL");
  *out = nullptr;
  if (!gammas || !betas || (n_edges > 0 && !edges))
    return fail(QT_EINVAL, "qt_energy_build: null input array");
  if (n_vertices < 2 || p < 1 || n_edges < 1)
    return fail(QT_EINVAL, "qt_energy_build: need n_vertices >= 2, p >= 1, n_edges >= 1");
  if (algo != QT_GREEDY_MINFILL && algo != QT_GREEDY_MINDEG)
    return fail(QT_EINVAL, "qt_energy_build: unknown ordering rule");
  std::set<std::pair<int, int>> seen;
  for (int e = 0; e < n_edges; ++e) {
    const int a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || b < 0 || a >= n_vertices || b >= n_vertices)
      return fail(QT_EINVAL, "qt_energy_build: edge id out of range");
    if (a == b) return fail(QT_EINVAL, "qt_energy_build: self-loop");
    if (!seen.insert({std::min(a, b), std::max(a, b)}).second)
      return fail(QT_EINVAL, "qt_energy_build: repeated edge");
  }
  for (int k = 0; k < p; ++k)
    if (!std::isfinite(gammas[k]) || !std::isfinite(betas[k]))
      return fail(QT_EINVAL, "qt_energy_build: angle not finite");
  qt_energy* E = new (std::nothrow) qt_energy();
  if (!E) return fail(QT_ENOMEM, "qt_energy_build: out of host memory");
  try {
    E->n = n_vertices;
    E->p = p;
    E->algo = algo;
    E->edges.assign(edges, edges + 2 * (size_t)n_edges);
    E->gammas.assign(gammas, gammas + p);
    E->betas.assign(betas, betas + p);
    E->adj.assign(n_vertices, {});
    for (int e = 0; e < n_edges; ++e) {
      E->adj[edges[2 * e]].push_back(edges[2 * e + 1]);
      E->adj[edges[2 * e + 1]].push_back(edges[2 * e]);
    }
    std::string err;
    if (!qt::energy_build_networks(E, err)) {
      delete E;
      return fail(QT_EINVAL, "qt_energy_build: " + err);
    }
  } catch (const std::bad_alloc&) {
    delete E;
    return fail(QT_ENOMEM, "qt_energy_build: out of host memory");
  }
  *out = E;
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_set_angles(qt_energy* E, const double* gammas, const double* betas) {
  if (!E || !gammas || !betas) return fail(QT_EINVAL, "qt_energy_set_angles: null argument");
  for (int k = 0; k < E->p; ++k)
    if (!std::isfinite(gammas[k]) || !std::isfinite(betas[k]))
      return fail(QT_EINVAL, "qt_energy_set_angles: angle not finite");
  E->gammas.assign(gammas, gammas + E->p);
  E->betas.assign(betas, betas + E->p);
  // same structure: keep every order, rebuild the tensors' data
  std::vector<qt::SlicePlan> plans;
  for (auto& N : E->nets) plans.push_back(N.plan);
  std::string err;
  qt::energy_build_networks(E, err);
  for (size_t i = 0; i < E->nets.size(); ++i) E->nets[i].plan = plans[i];
  if (E->compiled) {
    const int threads = E->block_threads, blocks = E->blocks;
    if (!qt::energy_compile(E, E->precision, err)) return fail(QT_EINVAL, "qt_energy_set_angles: " + err);
    E->block_threads = threads;
    E->blocks = blocks;
    layout(E);
  }
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_prepare(qt_energy* E, int32_t precision, size_t* workspace_bytes) {
  if (!E) return fail(QT_EINVAL, "qt_energy_prepare: null handle");
  if (precision != QT_FP32_SIMT && precision != QT_FP64)
    return fail(QT_EINVAL, "qt_energy_prepare: unknown precision");
  std::string err;
  try {
    if (!qt::energy_compile(E, precision, err)) return fail(QT_ERANGE, "qt_energy_prepare: " + err);
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_energy_prepare: out of host memory");
  }
  if (E->blocks <= 0)
    E->blocks = precision == QT_FP64 ? blocks_for<double>(E->block_threads)
                                     : blocks_for<float>(E->block_threads);
  layout(E);
  if (workspace_bytes) *workspace_bytes = E->total_bytes_ws;
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_upload(qt_energy* E, void* ws, size_t bytes, void* stream) {
  qt_status s = check_ws(E, ws, bytes, "qt_energy_upload");
  if (s != QT_OK) return s;
  std::string err;
  char* base = (char*)ws;
  cudaStream_t st = (cudaStream_t)stream;
  struct Part { size_t off; const void* src; size_t n; };
  const Part parts[] = {
      {E->off_gates, E->h_gates.data(), E->h_gates.size()},
      {E->off_ops, E->h_ops.data(), E->h_ops.size() * sizeof(qt::EOp)},
      {E->off_steps, E->h_steps.data(), E->h_steps.size() * sizeof(qt::EStep)},
      {E->off_nets, E->h_nets.data(), E->h_nets.size() * sizeof(qt::ENet)},
      {E->off_scalars, E->h_scalars.data(), E->h_scalars.size() * sizeof(uint32_t)}};
  for (const Part& p : parts)
    if (p.n && !cuda_ok(cudaMemcpyAsync(base + p.off, p.src, p.n, cudaMemcpyHostToDevice, st),
                        "energy upload", err))
      return fail(QT_ECUDA, "qt_energy_upload: " + err);
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_run(qt_energy* E, void* ws, size_t bytes, void* stream, double* d_zz,
                        double* d_energy) {
  qt_status s = check_ws(E, ws, bytes, "qt_energy_run");
  if (s != QT_OK) return s;
  if (!d_zz || !d_energy) return fail(QT_EINVAL, "qt_energy_run: null output");
  std::string err;
  s = run_energy(E, (char*)ws, (cudaStream_t)stream, d_zz, d_energy, true, err);
  if (s != QT_OK) return fail(s, "qt_energy_run: " + err);
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_autotune(qt_energy* E, void* ws, size_t bytes, void* stream,
                             int32_t* threads_out) {
  qt_status s = check_ws(E, ws, bytes, "qt_energy_autotune");
  if (s != QT_OK) return s;
  std::string err;
  char* base = (char*)ws;
  cudaStream_t st = (cudaStream_t)stream;
  double* zz = reinterpret_cast<double*>(base + E->off_zz);
  double* en = zz + E->h_nets.size();
  const int saved_blocks = E->blocks;
  float best = 1e30f;
  int best_t = E->block_threads;
  const int cands[] = {32, 64, 128, 256};
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int t : cands) {
    E->block_threads = t;
    E->blocks = E->precision == QT_FP64 ? blocks_for<double>(t) : blocks_for<float>(t);
    if (E->blocks > saved_blocks) E->blocks = saved_blocks;  // arenas were laid out for saved_blocks
    float tot = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(a, st);
      s = run_energy(E, base, st, zz, en, false, err);
      cudaEventRecord(b, st);
      if (s != QT_OK) break;
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep) tot += ms;
    }
    if (s != QT_OK) break;
    if (tot < best) {
      best = tot;
      best_t = t;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  E->block_threads = best_t;
  E->blocks = E->precision == QT_FP64 ? blocks_for<double>(best_t) : blocks_for<float>(best_t);
  if (E->blocks > saved_blocks) E->blocks = saved_blocks;
  if (s != QT_OK) return fail(s, "qt_energy_autotune: " + err);
  if (threads_out) *threads_out = best_t;
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_compute(qt_energy* E, int32_t precision, void* ws, size_t bytes, void* stream,
                            double* zz_host, double* energy_host) {
  if (!E || !energy_host) return fail(QT_EINVAL, "qt_energy_compute: null argument");
  if (!E->compiled || E->precision != precision) {
    size_t need = 0;
    qt_status s = qt_energy_prepare(E, precision, &need);
    if (s != QT_OK) return s;
  }
  qt_status s = qt_energy_upload(E, ws, bytes, stream);
  if (s != QT_OK) return s;
  char* base = (char*)ws;
  double* zz = reinterpret_cast<double*>(base + E->off_zz);
  double* en = zz + E->h_nets.size();
  s = qt_energy_run(E, ws, bytes, stream, zz, en);
  if (s != QT_OK) return s;
  std::string err;
  cudaStream_t st = (cudaStream_t)stream;
  if (zz_host &&
      !cuda_ok(cudaMemcpyAsync(zz_host, zz, E->h_nets.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, st),
               "download zz", err))
    return fail(QT_ECUDA, "qt_energy_compute: " + err);
  if (!cuda_ok(cudaMemcpyAsync(energy_host, en, sizeof(double), cudaMemcpyDeviceToHost, st),
               "download energy", err) ||
      !cuda_ok(cudaStreamSynchronize(st), "synchronize", err))
    return fail(QT_ECUDA, "qt_energy_compute: " + err);
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_get_order(const qt_energy* E, int32_t edge, int32_t* order, int32_t cap,
                              int32_t* len, int32_t* n_vars, int32_t* width) {
  if (!E || !len) return fail(QT_EINVAL, "qt_energy_get_order: null argument");
  if (edge < 0 || edge >= (int32_t)E->nets.size())
    return fail(QT_EINVAL, "qt_energy_get_order: edge out of range");
  const qt::EnergyNet& N = E->nets[edge];
  *len = (int32_t)N.plan.order.size();
  if (order)
    for (int32_t i = 0; i < cap && i < *len; ++i) order[i] = N.plan.order[i];
  if (n_vars) *n_vars = N.n_vars;
  if (width) *width = N.plan.width;
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_stats(const qt_energy* E, char* buf, size_t cap, size_t* needed) {
  if (!E) return fail(QT_EINVAL, "qt_energy_stats: null handle");
  if (!E->compiled) return fail(QT_ESTATE, "qt_energy_stats: call qt_energy_prepare first");
  std::ostringstream o;
  o << "{\"edges\":" << E->nets.size() << ",\"steps\":" << E->h_steps.size()
    << ",\"ops\":" << E->h_ops.size() << ",\"max_width\":" << E->max_width
    << ",\"flops\":" << E->total_flops << ",\"bytes\":" << E->total_bytes
    << ",\"gate_elems\":" << E->gate_elems << ",\"arena_elems\":" << E->arena_elems
    << ",\"block_threads\":" << E->block_threads << ",\"blocks\":" << E->blocks
    << ",\"workspace_bytes\":" << E->total_bytes_ws << ",\"upload_bytes\":"
    << E->h_gates.size() + E->h_ops.size() * sizeof(qt::EOp) +
           E->h_steps.size() * sizeof(qt::EStep) + E->h_nets.size() * sizeof(qt::ENet) +
           E->h_scalars.size() * sizeof(uint32_t)
    << ",\"width_hist\":[";
  bool first = true;
  for (size_t w = 0; w < E->hist_width.size(); ++w)
    if (E->hist_width[w]) {
      o << (first ? "" : ",") << "[" << w << "," << E->hist_width[w] << "]";
      first = false;
    }
  o << "]}";
  const std::string s = o.str();
  if (needed) *needed = s.size() + 1;
  if (buf && cap > 0) {
    const size_t n = std::min(cap - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = '\0';
  }
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_sweep_prepare(qt_energy* E, int32_t n_sets, size_t* workspace_bytes) {
  if (!E) return fail(QT_EINVAL, "qt_energy_sweep_prepare: null handle");
  if (!E->compiled) return fail(QT_ESTATE, "qt_energy_sweep_prepare: call qt_energy_prepare first");
  if (n_sets < 1 || (int64_t)n_sets * (int64_t)E->h_nets.size() >= (int64_t(1) << 31))
    return fail(QT_EINVAL, "qt_energy_sweep_prepare: n_sets out of range");
  layout_sweep(E, n_sets);
  if (workspace_bytes) *workspace_bytes = E->sw_total;
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_sweep_upload(qt_energy* E, int32_t n_sets, const double* gammas,
                                 const double* betas, void* ws, size_t bytes, void* stream) {
  if (!E || !gammas || !betas) return fail(QT_EINVAL, "qt_energy_sweep_upload: null argument");
  if (!E->compiled) return fail(QT_ESTATE, "qt_energy_sweep_upload: call qt_energy_prepare first");
  if (n_sets < 1 || n_sets > E->sweep_sets)
    return fail(QT_EINVAL, "qt_energy_sweep_upload: n_sets outside [1, the prepared sweep size]");
  if (!ws || (uintptr_t)ws % 256) return fail(QT_EINVAL, "qt_energy_sweep_upload: bad workspace");
  if (bytes < E->sw_total) return fail(QT_ENOMEM, "qt_energy_sweep_upload: workspace too small");
  for (int64_t q = 0; q < (int64_t)n_sets * E->p; ++q)
    if (!std::isfinite(gammas[q]) || !std::isfinite(betas[q]))
      return fail(QT_EINVAL, "qt_energy_sweep_upload: angle not finite");
  try {
    if (E->sw_template.empty()) {  // recompiled since qt_energy_sweep_prepare: lay out again
      layout_sweep(E, E->sweep_sets);
      if (bytes < E->sw_total) return fail(QT_ENOMEM, "qt_energy_sweep_upload: workspace too small");
    }
    qt::energy_sweep_table(E, n_sets, gammas, betas);
  } catch (const std::bad_alloc&) {
    return fail(QT_ENOMEM, "qt_energy_sweep_upload: out of host memory");
  }
  std::string err;
  char* base = (char*)ws;
  cudaStream_t st = (cudaStream_t)stream;
  struct Part { size_t off; const void* src; size_t n; };
  // structure tables and the template once per workspace; the angle table every call
  const bool fresh = E->sw_tmpl_ws != ws;
  const Part parts[] = {
      {E->sw_off_ops, E->h_ops.data(), fresh ? E->h_ops.size() * sizeof(qt::EOp) : 0},
      {E->sw_off_steps, E->h_steps.data(), fresh ? E->h_steps.size() * sizeof(qt::EStep) : 0},
      {E->sw_off_nets, E->h_nets.data(), fresh ? E->h_nets.size() * sizeof(qt::ENet) : 0},
      {E->sw_off_scalars, E->h_scalars.data(),
       fresh ? E->h_scalars.size() * sizeof(uint32_t) : 0},
      {E->sw_off_tmpl, E->sw_template.data(), fresh ? E->sw_template.size() : 0},
      {E->sw_off_slots, E->sw_slots.data(), fresh ? E->sw_slots.size() * sizeof(uint32_t) : 0},
      {E->sw_off_codes, E->sw_codes.data(), fresh ? E->sw_codes.size() * sizeof(uint32_t) : 0},
      {E->sw_off_table, E->sw_table.data(), E->sw_table.size()}};
  for (const Part& p : parts)
    if (p.n && !cuda_ok(cudaMemcpyAsync(base + p.off, p.src, p.n, cudaMemcpyHostToDevice, st),
                        "sweep upload", err))
      return fail(QT_ECUDA, "qt_energy_sweep_upload: " + err);
  E->sw_tmpl_ws = ws;
  const long long img_c = (long long)E->gate_elems;
  const int nslots = (int)E->sw_slots.size();
  const unsigned gcopy = (unsigned)std::max<long long>(
      1, std::min<long long>((img_c * n_sets + 255) / 256, 152ll * 16));
  const unsigned ggate = (unsigned)std::max<long long>(
      1, std::min<long long>(((long long)nslots * n_sets + 255) / 256, 152ll * 16));
  if (E->precision == QT_FP64) {
    double* img = reinterpret_cast<double*>(base + E->sw_off_gates);
    k_sweep_copy<double><<<gcopy, 256, 0, st>>>(
        reinterpret_cast<const double*>(base + E->sw_off_tmpl), img_c, n_sets, img);
    if (nslots)
      k_sweep_gates<double><<<ggate, 256, 0, st>>>(
          reinterpret_cast<const uint32_t*>(base + E->sw_off_slots),
          reinterpret_cast<const uint32_t*>(base + E->sw_off_codes), nslots,
          reinterpret_cast<const double*>(base + E->sw_off_table), E->p, n_sets, img_c, img);
  } else {
    float* img = reinterpret_cast<float*>(base + E->sw_off_gates);
    k_sweep_copy<float><<<gcopy, 256, 0, st>>>(
        reinterpret_cast<const float*>(base + E->sw_off_tmpl), img_c, n_sets, img);
    if (nslots)
      k_sweep_gates<float><<<ggate, 256, 0, st>>>(
          reinterpret_cast<const uint32_t*>(base + E->sw_off_slots),
          reinterpret_cast<const uint32_t*>(base + E->sw_off_codes), nslots,
          reinterpret_cast<const float*>(base + E->sw_off_table), E->p, n_sets, img_c, img);
  }
  if (!cuda_ok(cudaGetLastError(), "sweep image kernels", err))
    return fail(QT_ECUDA, "qt_energy_sweep_upload: " + err);
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_sweep_run(qt_energy* E, int32_t n_sets, void* ws, size_t bytes, void* stream,
                              double* d_energy, double* d_zz) {
  if (!E || !d_energy) return fail(QT_EINVAL, "qt_energy_sweep_run: null argument");
  if (!E->compiled) return fail(QT_ESTATE, "qt_energy_sweep_run: call qt_energy_prepare first");
  if (n_sets < 1 || n_sets > E->sweep_sets)
    return fail(QT_EINVAL, "qt_energy_sweep_run: n_sets outside [1, the prepared sweep size]");
  if (!ws || (uintptr_t)ws % 256) return fail(QT_EINVAL, "qt_energy_sweep_run: bad workspace");
  if (bytes < E->sw_total) return fail(QT_ENOMEM, "qt_energy_sweep_run: workspace too small");
  std::string err;
  char* base = (char*)ws;
  double* zz = d_zz ? d_zz : reinterpret_cast<double*>(base + E->sw_off_zz);
  qt_status s = E->precision == QT_FP64
                    ? enqueue_sweep<double>(E, n_sets, base, (cudaStream_t)stream, zz, d_energy, err)
                    : enqueue_sweep<float>(E, n_sets, base, (cudaStream_t)stream, zz, d_energy, err);
  if (s != QT_OK) return fail(s, "qt_energy_sweep_run: " + err);
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_energy_sweep(qt_energy* E, int32_t n_sets, const double* gammas, const double* betas,
                          void* ws, size_t bytes, void* stream, double* d_energy, double* d_zz) {
  if (!d_energy) return fail(QT_EINVAL, "qt_energy_sweep: null output");
  qt_status s = qt_energy_sweep_upload(E, n_sets, gammas, betas, ws, bytes, stream);
  if (s != QT_OK) return s;
  return qt_energy_sweep_run(E, n_sets, ws, bytes, stream, d_energy, d_zz);
}

void qt_energy_free(qt_energy* E) { delete E; }

}  // extern "C"
