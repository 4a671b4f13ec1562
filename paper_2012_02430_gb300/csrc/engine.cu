// Device side: the bucket-step kernels, the per-slice finalisation and the
// FP64 slice reduction, plus the host driver that launches them.
//
// One bucket step of Alg. 1 is  R(out) = sum_{v} prod_j T_j  over the union U
// of the operands' indices, out = U minus the bucket vertex v. In canonical
// layout v is bit 0 of every operand, so the two terms of the sum are one
// adjacent value pair: a thread owns a pair of U elements, loads one 16-byte
// vector per operand (8 bytes when the operand lacks v... which cannot happen
// for bucket operands, but fused groups allow it), multiplies, adds the two
// products and writes one output. An operand's element index is the bit
// extract of the U index by the operand's membership mask ("pext"); slicing
// adds the fixed slice values as a block offset (sliced indices sit above all
// others in a shared tensor).
//
// Range control: every tensor carries a power-of-two exponent E (true value =
// stored * 2^E) and the max-abs of its stored values. A consumer scales
// operand j by 2^-s_j with s_j the binary exponent of its max-abs, so stored
// values stay near 1; the result's exponent is sum_j (E_j + s_j). The slice
// result is rebuilt in FP64 with ldexp and the slices are summed in FP64
// (the reduce-sum of Alg. 1) in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "qt_internal.h"

namespace qt {

constexpr int MAXOP = 12;
constexpr int TILED_MAXOP = 6;
constexpr int PAIR_TILE_BITS = 13;  // pairs per tile of the tiled kernel: 8192
constexpr int TILE_THREADS = 256;
constexpr int Q_PER_THREAD = (1 << PAIR_TILE_BITS) / TILE_THREADS;  // 32

struct KOp {
  long long base;          // element offset from the workspace base
  long long slice_stride;  // elements between slice-local copies (0 for shared tensors)
  long long meta;          // meta slot (shared) or first slot (per slice)
  unsigned int umask;      // U bits present in the operand
  unsigned int smask;      // slice-id bits fixed into the operand
  int sshift;              // position of the slice block (unsliced rank)
  int meta_per_slice;
};

struct KStep {
  int m, u, nsum, pad0;
  long long nslices, slice_first;
  long long out_base, out_slice_stride, out_meta;
  int out_meta_per_slice, pad1;
  KOp op[MAXOP];
};

struct Meta {
  unsigned int maxabs;  // float bits of max(|re|, |im|) over the stored values
  int E;                // exponent: true value = stored * 2^E
};

struct ScalarTerm {
  long long base, slice_stride, meta;
  unsigned int smask;
  int per_slice;
};
static_assert(sizeof(ScalarTerm) == kScalarTermBytes, "scalar table record size");

template <typename R> struct CT;
template <> struct CT<float> { using c2 = float2; using c4 = float4; };
template <> struct CT<double> { using c2 = double2; struct c4 { double2 a, b; }; };

__device__ __forceinline__ unsigned long long pext64(unsigned long long x, unsigned int m) {
  unsigned long long r = 0;
  int k = 0;
  while (m) {
    int b = __ffs(m) - 1;
    r |= ((x >> b) & 1ull) << k;
    ++k;
    m &= m - 1;
  }
  return r;
}

// binary exponent s with maxabs * 2^-s in [0.5, 1); 0 for a zero tensor
__device__ __forceinline__ int scale_exp(unsigned int maxabs_bits) {
  if (maxabs_bits == 0u) return 0;
  int e = (int)((maxabs_bits >> 23) & 0xffu);
  int s = e - 126;
  return max(-125, min(125, s));
}

template <typename R> __device__ __forceinline__ R pow2_neg(int s);
template <> __device__ __forceinline__ float pow2_neg<float>(int s) {
  return __int_as_float((127 - s) << 23);
}
template <> __device__ __forceinline__ double pow2_neg<double>(int s) {
  return __longlong_as_double((long long)(1023 - s) << 52);
}

__device__ __forceinline__ float absmax(float re, float im) { return fmaxf(fabsf(re), fabsf(im)); }
__device__ __forceinline__ float absmax(double re, double im) {
  return (float)fmax(fabs(re), fabs(im));
}

template <typename R>
__device__ __forceinline__ void cmul(R& ar, R& ai, R br, R bi) {
  R r = ar * br - ai * bi;
  R i = ar * bi + ai * br;
  ar = r;
  ai = i;
}

// loads the value pair (U bit 0 = 0 and 1) of an operand at element offset off
template <typename R>
__device__ __forceinline__ void load_pair(const R* data, long long off, bool has_bit0, R& r0,
                                          R& i0, R& r1, R& i1) {
  using C2 = typename CT<R>::c2;
  if (has_bit0) {
    if constexpr (sizeof(R) == 4) {
      float4 v = __ldg(reinterpret_cast<const float4*>(data + 2 * off));
      r0 = v.x; i0 = v.y; r1 = v.z; i1 = v.w;
    } else {
      C2 a = __ldg(reinterpret_cast<const C2*>(data + 2 * off));
      C2 b = __ldg(reinterpret_cast<const C2*>(data + 2 * off + 2));
      r0 = a.x; i0 = a.y; r1 = b.x; i1 = b.y;
    }
  } else {
    C2 a = __ldg(reinterpret_cast<const C2*>(data + 2 * off));
    r0 = r1 = a.x;
    i0 = i1 = a.y;
  }
}

template <typename R>
__device__ __forceinline__ void store_out(R* data, long long off, R re, R im) {
  using C2 = typename CT<R>::c2;
  C2 v;
  v.x = re;
  v.y = im;
  *reinterpret_cast<C2*>(data + 2 * off) = v;
}

// Flat kernel: one U-element pair per thread, offsets from bit extracts.
// For steps whose per-slice U space is small (the common case).
template <typename R>
__global__ void __launch_bounds__(256) k_bucket_flat(const KStep st, R* data, Meta* meta) {
  const long long npairs = 1ll << (st.u - 1);
  const long long total = st.nslices * npairs;
  const int lane = threadIdx.x & 31;
  const int grp = 1 << (st.nsum - 1);
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total;
       base += (long long)gridDim.x * blockDim.x) {
    const long long g = base + threadIdx.x;
    const bool active = g < total;
    long long i = active ? g >> (st.u - 1) : 0;
    const unsigned long long I = (unsigned long long)(g & (npairs - 1)) << 1;
    R p0r = 1, p0i = 0, p1r = 1, p1i = 0;
    int Eout = 0;
    if (active) {
      const unsigned long long sid = (unsigned long long)(st.slice_first + i);
      for (int j = 0; j < st.m; ++j) {
        const KOp& o = st.op[j];
        long long off = o.base + i * o.slice_stride + (long long)pext64(I, o.umask);
        if (o.smask) off += (long long)(pext64(sid, o.smask) << o.sshift);
        const Meta mt = meta[o.meta + (o.meta_per_slice ? i : 0)];
        const int s = scale_exp(mt.maxabs);
        Eout += mt.E + s;
        const R sc = pow2_neg<R>(s);
        R r0, i0, r1, i1;
        load_pair<R>(data, off, o.umask & 1u, r0, i0, r1, i1);
        cmul<R>(p0r, p0i, r0 * sc, i0 * sc);
        cmul<R>(p1r, p1i, r1 * sc, i1 * sc);
      }
    }
    R sr = active ? p0r + p1r : R(0), si = active ? p0i + p1i : R(0);
    for (int w = 1; w < grp; w <<= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, w);
      si += __shfl_xor_sync(0xffffffffu, si, w);
    }
    const bool writer = active && (lane & (grp - 1)) == 0;
    float mx = 0.f;
    if (writer) {
      const long long oo = st.out_base + i * st.out_slice_stride + (long long)(I >> st.nsum);
      store_out<R>(data, oo, sr, si);
      mx = absmax(sr, si);
      if ((g & (npairs - 1)) == 0) meta[st.out_meta + (st.out_meta_per_slice ? i : 0)].E = Eout;
    }
    const int key = active ? (int)i : -1;
    const unsigned int peers = __match_any_sync(0xffffffffu, key);
    const unsigned int red = __reduce_max_sync(peers, __float_as_uint(mx));
    if (active && lane == __ffs(peers) - 1 && red != 0u)
      atomicMax(&meta[st.out_meta + (st.out_meta_per_slice ? i : 0)].maxabs, red);
  }
}

// Tiled kernel: a tile is 2^PAIR_TILE_BITS pairs of one slice; a thread owns
// 32 of them (thread bits = U bits 1..8, loop bits = U bits 9..13). Operand
// offsets = tile part (one warp, per tile) + thread part (registers) + loop
// part (shared-memory table), so the inner loop is loads and complex FMAs.
template <typename R, int M>
__global__ void __launch_bounds__(TILE_THREADS) k_bucket_tiled(const KStep st, R* data,
                                                               Meta* meta) {
  __shared__ int qoff[M][Q_PER_THREAD];
  __shared__ long long toff[M];
  __shared__ R tsc[M];
  __shared__ long long tout;
  __shared__ unsigned int blkmax;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int grp = 1 << (st.nsum - 1);
  for (int e = tid; e < M * Q_PER_THREAD; e += TILE_THREADS) {
    const int j = e / Q_PER_THREAD, q = e % Q_PER_THREAD;
    qoff[j][q] = (int)pext64((unsigned long long)q << 9, st.op[j].umask);
  }
  if (tid == 0) blkmax = 0u;
  int thr[M];
  bool has0[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    thr[j] = (int)pext64((unsigned long long)tid << 1, st.op[j].umask);
    has0[j] = st.op[j].umask & 1u;
  }
  const long long tiles_per_slice = 1ll << (st.u - 1 - PAIR_TILE_BITS);
  const long long ntiles = st.nslices * tiles_per_slice;
  long long cur_slice = -1;
  float mx = 0.f;
  for (long long T = blockIdx.x; T < ntiles; T += gridDim.x) {
    const long long i = T / tiles_per_slice;
    const long long Tl = T - i * tiles_per_slice;
    __syncthreads();  // previous tile done with toff/tsc; qoff/blkmax initialised
    if (i != cur_slice) {
      if (cur_slice >= 0) {  // flush the running max of the previous slice
        unsigned int v = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
        if (lane == 0) atomicMax(&blkmax, v);
        __syncthreads();
        if (tid == 0 && blkmax)
          atomicMax(&meta[st.out_meta + (st.out_meta_per_slice ? cur_slice : 0)].maxabs, blkmax);
        __syncthreads();
        if (tid == 0) blkmax = 0u;
      }
      cur_slice = i;
      mx = 0.f;
    }
    if (tid < 32) {
      const unsigned long long sid = (unsigned long long)(st.slice_first + i);
      const unsigned long long Ihi = (unsigned long long)Tl << (PAIR_TILE_BITS + 1);
      int Eout = 0;
      if (lane < M) {
        const KOp& o = st.op[lane];
        long long off = o.base + i * o.slice_stride + (long long)pext64(Ihi, o.umask);
        if (o.smask) off += (long long)(pext64(sid, o.smask) << o.sshift);
        toff[lane] = off;
        const Meta mt = meta[o.meta + (o.meta_per_slice ? i : 0)];
        const int s = scale_exp(mt.maxabs);
        tsc[lane] = pow2_neg<R>(s);
        Eout = mt.E + s;
      }
      Eout = __reduce_add_sync(0xffffffffu, Eout);
      if (lane == 0) {
        tout = st.out_base + i * st.out_slice_stride + (long long)(Ihi >> st.nsum);
        if (Tl == 0) meta[st.out_meta + (st.out_meta_per_slice ? i : 0)].E = Eout;
      }
    }
    __syncthreads();
    long long base[M];
    R sc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      base[j] = toff[j] + thr[j];
      sc[j] = tsc[j];
    }
    const long long obase = tout;
#pragma unroll 4
    for (int q = 0; q < Q_PER_THREAD; ++q) {
      R p0r = 1, p0i = 0, p1r = 1, p1i = 0;
#pragma unroll
      for (int j = 0; j < M; ++j) {
        R r0, i0, r1, i1;
        load_pair<R>(data, base[j] + qoff[j][q], has0[j], r0, i0, r1, i1);
        cmul<R>(p0r, p0i, r0 * sc[j], i0 * sc[j]);
        cmul<R>(p1r, p1i, r1 * sc[j], i1 * sc[j]);
      }
      R sr = p0r + p1r, si = p0i + p1i;
      for (int w = 1; w < grp; w <<= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, w);
        si += __shfl_xor_sync(0xffffffffu, si, w);
      }
      if ((lane & (grp - 1)) == 0) {
        const unsigned long long pl = ((unsigned long long)q << 8) | (unsigned)tid;
        store_out<R>(data, obase + (long long)((pl << 1) >> st.nsum), sr, si);
        mx = fmaxf(mx, absmax(sr, si));
      }
    }
  }
  // final flush
  __syncthreads();
  unsigned int v = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
  if (lane == 0) atomicMax(&blkmax, v);
  __syncthreads();
  if (tid == 0 && cur_slice >= 0 && blkmax)
    atomicMax(&meta[st.out_meta + (st.out_meta_per_slice ? cur_slice : 0)].maxabs, blkmax);
}

// Per slice: product of the scalar factors in FP64, exponent applied.
template <typename R>
__global__ void k_finalize(const ScalarTerm* terms, int nterms, const R* data, const Meta* meta,
                           long long nslices, long long slice_first, double2* partials) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nslices) return;
  const unsigned long long sid = (unsigned long long)(slice_first + i);
  double pr = 1.0, pi = 0.0;
  long long E = 0;
  for (int t = 0; t < nterms; ++t) {
    const ScalarTerm& s = terms[t];
    long long off = s.base + (s.per_slice ? i * s.slice_stride : 0);
    if (s.smask) off += (long long)pext64(sid, s.smask);
    const double vr = (double)data[2 * off], vi = (double)data[2 * off + 1];
    const double nr = pr * vr - pi * vi, ni = pr * vi + pi * vr;
    pr = nr;
    pi = ni;
    E += meta[s.meta + (s.per_slice ? i : 0)].E;
  }
  const int e = (int)max(-100000ll, min(100000ll, E));
  partials[i] = make_double2(ldexp(pr, e), ldexp(pi, e));
}

// Fixed-order FP64 sum of a batch's slice results into the accumulator:
// thread t adds partials t, t+1024, ... in order, then a fixed tree.
__global__ void __launch_bounds__(1024) k_reduce(const double2* partials, long long n,
                                                 double2* acc, int first_batch) {
  __shared__ double sr[1024], si[1024];
  double r = 0.0, im = 0.0;
  for (long long j = threadIdx.x; j < n; j += 1024) {
    r += partials[j].x;
    im += partials[j].y;
  }
  sr[threadIdx.x] = r;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sr[threadIdx.x] += sr[threadIdx.x + w];
      si[threadIdx.x] += si[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (first_batch) {
      acc->x = sr[0];
      acc->y = si[0];
    } else {
      acc->x += sr[0];
      acc->y += si[0];
    }
  }
}

__global__ void k_write_out(const double2* acc, double norm, double* out) {
  out[0] = acc->x * norm;
  out[1] = acc->y * norm;
}

// ------------------------------ host driver ---------------------------------
static thread_local std::string g_cuda_err;

static bool cuda_ok(cudaError_t e, const char* what, std::string& err) {
  if (e == cudaSuccess) return true;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

static int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
      sms = 148;
  }
  return sms;
}

static void* prof_event(qt_net* net) {
  if (!net->prof_pool.empty()) {
    void* e = net->prof_pool.back();
    net->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return (void*)e;
}

static void prof_begin(qt_net* net, cudaStream_t s, ProfRec& r) {
  r.ev0 = prof_event(net);
  r.ev1 = prof_event(net);
  if (r.ev0) cudaEventRecord((cudaEvent_t)r.ev0, s);
}

static void prof_end(qt_net* net, cudaStream_t s, ProfRec& r) {
  if (r.ev1) cudaEventRecord((cudaEvent_t)r.ev1, s);
  net->prof_recs.push_back(r);
}

void prof_clear(qt_net* net) {
  for (ProfRec& r : net->prof_recs) {
    if (r.ev0) net->prof_pool.push_back(r.ev0);
    if (r.ev1) net->prof_pool.push_back(r.ev1);
  }
  net->prof_recs.clear();
}

// JSON array of the recorded launches with their durations (waits for them).
qt_status prof_read(qt_net* net, std::string& out, std::string& err) {
  out = "[";
  bool first = true;
  for (const ProfRec& r : net->prof_recs) {
    float ms = -1.f;
    if (r.ev0 && r.ev1) {
      if (!cuda_ok(cudaEventSynchronize((cudaEvent_t)r.ev1), "profile event", err)) return QT_ECUDA;
      if (!cuda_ok(cudaEventElapsedTime(&ms, (cudaEvent_t)r.ev0, (cudaEvent_t)r.ev1),
                   "profile elapsed", err))
        return QT_ECUDA;
    }
    char buf[256];
    std::snprintf(buf, sizeof buf,
                  "%s{\"step\":%d,\"kernel\":%d,\"slices\":%lld,\"bytes\":%lld,"
                  "\"flops\":%lld,\"ms\":%.6f}",
                  first ? "" : ",", r.step, r.kernel, (long long)r.slices, (long long)r.bytes,
                  (long long)r.flops, ms);
    out += buf;
    first = false;
  }
  out += "]";
  return QT_OK;
}

// builds the host copies uploaded by qt_upload: gate data, gate meta, scalar table
void build_stage(qt_net* net) {
  const Schedule& S = net->sched;
  const size_t eb = (size_t)S.elem_bytes;
  const size_t gate_bytes = (size_t)S.gate_elems * eb;
  const size_t meta_bytes = (size_t)S.n_shared_meta * sizeof(Meta);
  std::vector<ScalarTerm> terms;
  for (int32_t tid : S.scalars) {
    const STensor& t = S.tensors[tid];
    ScalarTerm st{};
    if (t.kind == TK_GATE) st.base = (long long)(S.off_gates / eb) + t.offset;
    else if (t.kind == TK_PREFIX) st.base = (long long)(S.off_prefix / eb) + t.offset;
    else st.base = (long long)(S.off_slices / eb) + t.offset;
    st.slice_stride = t.kind == TK_SLICE ? S.slice_elems : 0;
    st.per_slice = t.kind == TK_SLICE;
    st.smask = t.kind == TK_SLICE ? 0u : t.smask;
    st.meta = t.meta;
    terms.push_back(st);
  }
  net->gate_stage.assign(gate_bytes + meta_bytes + terms.size() * sizeof(ScalarTerm), 0);
  unsigned char* g = net->gate_stage.data();
  Meta* gm = reinterpret_cast<Meta*>(g + gate_bytes);
  for (int64_t m = 0; m < S.n_shared_meta; ++m) gm[m] = Meta{0u, 0};
  for (const STensor& t : S.tensors) {
    if (t.kind != TK_GATE) continue;
    std::vector<double> d = canonical_data(net->tensors[t.gate], t.labels);
    float mx = 0.f;
    for (size_t e = 0; e < d.size(); ++e) {
      if (S.precision == QT_FP64) {
        double v = d[e];
        std::memcpy(g + (t.offset * 2 + e) * sizeof(double), &v, sizeof(double));
      } else {
        float v = (float)d[e];
        std::memcpy(g + (t.offset * 2 + e) * sizeof(float), &v, sizeof(float));
      }
      mx = std::max(mx, (float)std::fabs(d[e]));
    }
    unsigned int bits;
    std::memcpy(&bits, &mx, 4);
    gm[t.meta] = Meta{bits, 0};
  }
  if (!terms.empty())
    std::memcpy(g + gate_bytes + meta_bytes, terms.data(), terms.size() * sizeof(ScalarTerm));
  net->stage_dirty = false;
}

static size_t n_gate_meta(const Schedule& S) {
  size_t n = 0;
  for (const STensor& t : S.tensors) n += t.kind == TK_GATE;
  return n;
}

qt_status upload(qt_net* net, void* ws, size_t bytes, void* stream, std::string& err) {
  const Schedule& S = net->sched;
  if (net->stage_dirty) build_stage(net);
  const size_t eb = (size_t)S.elem_bytes;
  const size_t gate_bytes = (size_t)S.gate_elems * eb;
  const size_t meta_bytes = (size_t)S.n_shared_meta * sizeof(Meta);
  const size_t term_bytes = net->gate_stage.size() - gate_bytes - meta_bytes;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  const unsigned char* g = net->gate_stage.data();
  if (gate_bytes && !cuda_ok(cudaMemcpyAsync(base + S.off_gates, g, gate_bytes,
                                             cudaMemcpyHostToDevice, s),
                             "upload gates", err))
    return QT_ECUDA;
  if (meta_bytes && !cuda_ok(cudaMemcpyAsync(base + S.off_meta, g + gate_bytes, meta_bytes,
                                             cudaMemcpyHostToDevice, s),
                             "upload meta", err))
    return QT_ECUDA;
  if (term_bytes && !cuda_ok(cudaMemcpyAsync(base + S.off_terms, g + gate_bytes + meta_bytes,
                                             term_bytes, cudaMemcpyHostToDevice, s),
                             "upload scalar table", err))
    return QT_ECUDA;
  (void)bytes;
  return QT_OK;
}

static void fill_op(const Schedule& S, const SStep& st, int j, KOp& o) {
  const STensor& t = S.tensors[st.ops[j]];
  const long long eb = S.elem_bytes;
  o = KOp{};
  unsigned int um = 0;
  for (int b = 0; b < st.u; ++b)
    if (std::find(t.labels.begin(), t.labels.end(), st.ulabels[b]) != t.labels.end())
      um |= 1u << b;
  o.umask = um;
  if (t.kind == TK_SLICE) {
    o.base = (long long)S.off_slices / eb + t.offset;
    o.slice_stride = S.slice_elems;
    o.meta = t.meta;
    o.meta_per_slice = 1;
  } else {
    o.base = (long long)(t.kind == TK_GATE ? S.off_gates : S.off_prefix) / eb + t.offset;
    o.slice_stride = 0;
    o.meta = t.meta;
    o.meta_per_slice = 0;
    if (st.region == 1 && t.nsliced) {
      o.smask = t.smask;
      o.sshift = t.rank - t.nsliced;
    }
  }
}

template <typename R>
static qt_status launch_step(qt_net* net, int step_index, const SStep& st, long long nslices,
                             long long slice_first, char* base, cudaStream_t s,
                             std::string& err) {
  const Schedule& S = net->sched;
  KStep k{};
  k.m = (int)st.ops.size();
  k.u = st.u;
  k.nsum = st.nsum;
  k.nslices = nslices;
  k.slice_first = slice_first;
  const STensor& out = S.tensors[st.out];
  const long long eb = S.elem_bytes;
  if (out.kind == TK_SLICE) {
    k.out_base = (long long)S.off_slices / eb + out.offset;
    k.out_slice_stride = S.slice_elems;
    k.out_meta_per_slice = 1;
  } else {
    k.out_base = (long long)S.off_prefix / eb + out.offset;
    k.out_slice_stride = 0;
    k.out_meta_per_slice = 0;
  }
  k.out_meta = out.meta;
  if (k.m > MAXOP) {
    err = "bucket with more operands than the kernels take";
    return QT_ERANGE;
  }
  for (int j = 0; j < k.m; ++j) fill_op(S, st, j, k.op[j]);
  R* data = reinterpret_cast<R*>(base);
  Meta* meta = reinterpret_cast<Meta*>(base + S.off_meta);
  const bool tiled = st.u - 1 >= PAIR_TILE_BITS + 1 && k.m <= TILED_MAXOP;
  ProfRec pr{step_index, tiled ? 1 : 0, nslices, st.bytes * (S.elem_bytes / 8) * nslices,
             st.flops * nslices, nullptr, nullptr};
  if (net->prof) prof_begin(net, s, pr);
  net->launches++;
  if (tiled) {
    const long long ntiles = nslices << (st.u - 1 - PAIR_TILE_BITS);
    const long long grid = std::min<long long>(ntiles, (long long)num_sms() * 4);
    switch (k.m) {
#define QT_CASE(MM)                                                                  \
  case MM:                                                                           \
    k_bucket_tiled<R, MM><<<(unsigned)grid, TILE_THREADS, 0, s>>>(k, data, meta);    \
    break;
      QT_CASE(1) QT_CASE(2) QT_CASE(3) QT_CASE(4) QT_CASE(5) QT_CASE(6)
#undef QT_CASE
      default: break;
    }
  } else {
    const long long total = nslices << (st.u - 1);
    const long long blocks = (total + 255) / 256;
    const long long grid = std::max<long long>(1, std::min<long long>(blocks, (long long)num_sms() * 16));
    k_bucket_flat<R><<<(unsigned)grid, 256, 0, s>>>(k, data, meta);
  }
  if (net->prof) prof_end(net, s, pr);
  if (!cuda_ok(cudaGetLastError(), "bucket kernel launch", err)) return QT_ECUDA;
  return QT_OK;
}

template <typename R>
static qt_status run_impl(qt_net* net, long long first, long long count, char* base,
                          cudaStream_t s, double* d_out, std::string& err) {
  const Schedule& S = net->sched;
  const size_t ngm = n_gate_meta(S);
  Meta* meta = reinterpret_cast<Meta*>(base + S.off_meta);
  // prefix (contract_first): once, unsliced
  if (S.n_shared_meta > (int64_t)ngm &&
      !cuda_ok(cudaMemsetAsync(meta + ngm, 0, (S.n_shared_meta - ngm) * sizeof(Meta), s),
               "reset prefix meta", err))
    return QT_ECUDA;
  for (size_t si = 0; si < S.steps.size(); ++si) {
    const SStep& st = S.steps[si];
    if (st.region != 0) continue;
    qt_status r = launch_step<R>(net, (int)si, st, 1, 0, base, s, err);
    if (r != QT_OK) return r;
  }
  const ScalarTerm* terms = reinterpret_cast<const ScalarTerm*>(base + S.off_terms);
  const int nterms = (int)S.scalars.size();
  double2* partials = reinterpret_cast<double2*>(base + S.off_partials);
  double2* acc = reinterpret_cast<double2*>(base + S.off_acc);
  bool first_batch = true;
  for (long long b0 = first; b0 < first + count; b0 += S.batch) {
    const long long nb = std::min<long long>(S.batch, first + count - b0);
    if (S.n_slice_meta_tensors &&
        !cuda_ok(cudaMemsetAsync(meta + S.n_shared_meta, 0,
                                 (size_t)(S.n_slice_meta_tensors * S.batch) * sizeof(Meta), s),
                 "reset slice meta", err))
      return QT_ECUDA;
    for (size_t si = 0; si < S.steps.size(); ++si) {
      const SStep& st = S.steps[si];
      if (st.region != 1) continue;
      qt_status r = launch_step<R>(net, (int)si, st, nb, b0, base, s, err);
      if (r != QT_OK) return r;
    }
    ProfRec pr{-1, 2, nb, 0, 0, nullptr, nullptr};
    if (net->prof) prof_begin(net, s, pr);
    net->launches += 2;
    k_finalize<R><<<(unsigned)((nb + 127) / 128), 128, 0, s>>>(
        terms, nterms, reinterpret_cast<const R*>(base), meta, nb, b0, partials);
    k_reduce<<<1, 1024, 0, s>>>(partials, nb, acc, first_batch ? 1 : 0);
    if (net->prof) prof_end(net, s, pr);
    if (!cuda_ok(cudaGetLastError(), "finalize/reduce launch", err)) return QT_ECUDA;
    first_batch = false;
  }
  net->launches++;
  k_write_out<<<1, 1, 0, s>>>(acc, std::pow(2.0, -0.5 * net->n), d_out);
  if (!cuda_ok(cudaGetLastError(), "write_out launch", err)) return QT_ECUDA;
  return QT_OK;
}

qt_status run(qt_net* net, long long first, long long count, void* ws, void* stream,
              double* d_out, std::string& err) {
  char* base = (char*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  if (net->sched.precision == QT_FP64) return run_impl<double>(net, first, count, base, s, d_out, err);
  return run_impl<float>(net, first, count, base, s, d_out, err);
}

qt_status download_result(const double* d_out, double* host, void* stream, std::string& err) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!cuda_ok(cudaMemcpyAsync(host, d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s),
               "download result", err))
    return QT_ECUDA;
  if (!cuda_ok(cudaStreamSynchronize(s), "stream synchronize", err)) return QT_ECUDA;
  return QT_OK;
}

}  // namespace qt

qt_net::~qt_net() {
  qt::prof_clear(this);
  for (void* e : prof_pool) cudaEventDestroy((cudaEvent_t)e);
}
