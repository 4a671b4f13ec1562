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
#include <sstream>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "gemm.h"
#include "qt_internal.h"

namespace qt {

constexpr int MAXOP = 12;

struct KOp {
  long long base;          // element offset from the workspace base
  long long slice_stride;  // elements between slice-local copies (0 for shared tensors)
  long long meta;          // meta slot (shared) or first slot (per slice)
  unsigned long long smask;  // slice-id bits fixed into the operand
  unsigned int umask;      // U bits present in the operand
  int sshift;              // position of the slice block (unsliced rank)
  int meta_per_slice;
  int level;               // nested-sum level at which the operand is multiplied in
  int soff;                // segment launch: element offset in the block's shared arena (-1: global)
  int tid;                 // schedule tensor id
  int mslot;               // segment launch: slot of its metadata in the block's cache
};

struct KStep {
  int m, u, nsum, ms;  // ms: streaming operands (tiled kernel), placed first
  long long nslices, slice_first;
  long long out_base, out_slice_stride, out_meta;
  int out_meta_per_slice;
  int out_soff;        // segment launch: shared-arena offset of the result (-1: none)
  int out_global;      // segment launch: the result is also stored to global memory
  int out_mslot;       // segment launch: slot of the result's metadata in the block's cache
  int flags;           // bit 0: the tiled kernel takes its scaled path in every slice
  int item0;           // segment launch: the step's first work item within its level
  KOp op[MAXOP];
};

// A tensor a segment launch reads but does not produce, staged into the block's
// shared arena at the start of the launch (its block for the block's slice).
struct SegStage {
  long long base, slice_stride;
  unsigned long long smask;
  int sshift;
  int n;     // elements
  int soff;  // arena offset
  int cum;   // elements staged by the records before this one
};

// One dependency level of a segment launch: its steps read only results of
// earlier levels. Steps [first, first + nwarp) are small (at most 32 value
// pairs), the next nblock larger. Every step is cut into work items of 32 value
// pairs (one warp each); the level's `items` items run concurrently over all warps
// of the slice's block or cluster.
struct SegLevel {
  int first, nwarp, nblock, items;
};

struct Meta {
  unsigned int maxabs;  // float bits of max(|re|, |im|) over the stored values
  int E;                // exponent: true value = stored * 2^E
};

// A factor of the slice result: a tensor over open (omask, bit j = open index j)
// and sliced (smask) indices only, stored (open bits, slice bits) from bit 0 up.
struct ScalarTerm {
  long long base, slice_stride, meta;
  unsigned long long smask;
  unsigned int omask;
  int per_slice;
};
static_assert(sizeof(ScalarTerm) == kScalarTermBytes, "scalar table record size");

template <typename R> struct CT;
template <> struct CT<float> { using c2 = float2; using c4 = float4; };
template <> struct CT<double> { using c2 = double2; struct c4 { double2 a, b; }; };

__device__ __forceinline__ unsigned long long pext64(unsigned long long x, unsigned long long m) {
  unsigned long long r = 0;
  int k = 0;
  while (m) {
    int b = __ffsll((long long)m) - 1;
    r |= ((x >> b) & 1ull) << k;
    ++k;
    m &= m - 1;
  }
  return r;
}

// pext over a 32-bit mask for 32-bit x, one run of adjacent mask bits at a time (the
// union index of the flat and segment kernels fits 32 bits)
__device__ __forceinline__ unsigned int pext32r(unsigned int x, unsigned int m) {
  unsigned int r = 0;
  int k = 0;
  while (m) {
    const int b = __ffs(m) - 1;
    const unsigned int next = m + (m & (0u - m));  // the lowest run cleared, a carry above it
    const int len = __popc(m & ~next);
    r |= ((x >> b) & (0xffffffffu >> (32 - len))) << k;
    k += len;
    m &= next;
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

// Flat kernel: one U-element pair (U bit 0) per thread, lanes cover U bits 1-5;
// offsets from bit extracts. For launches whose per-slice U space is small.
// Level-0 operands multiply both values of the pair, the pair is summed, then
// for level l = 1 .. nsum-1 the level-l operands multiply each lane's partial
// sum before the lanes that differ in U bit l are added (a shuffle).
// MO: operands the kernel is compiled for (st.m <= MO); every operand's metadata and
// values are loaded first, all loads in flight at once, then multiplied in operand order
template <typename R, int MO>
__global__ void __launch_bounds__(256) k_bucket_flat(const KStep st, R* data, Meta* meta) {
  using C2 = typename CT<R>::c2;
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
    const unsigned long long sid = (unsigned long long)(st.slice_first + i);
    R p0r = 1, p0i = 0, p1r = 1, p1i = 0;
    int Eout = 0;
    R vr0[MO], vi0[MO], vr1[MO], vi1[MO];
    unsigned int mxb[MO];
    if (active) {
#pragma unroll
      for (int j = 0; j < MO; ++j) {
        if (j >= st.m) break;
        const KOp& o = st.op[j];
        const Meta mt = meta[o.meta + (o.meta_per_slice ? i : 0)];
        mxb[j] = mt.maxabs;
        Eout += mt.E;
        long long off = o.base + i * o.slice_stride + (long long)pext32r((unsigned int)I, o.umask);
        if (o.smask) off += (long long)(pext64(sid, o.smask) << o.sshift);
        if (o.level == 0) {
          load_pair<R>(data, off, o.umask & 1u, vr0[j], vi0[j], vr1[j], vi1[j]);
        } else {
          const C2 v = __ldg(reinterpret_cast<const C2*>(data + 2 * off));
          vr0[j] = v.x;
          vi0[j] = v.y;
        }
      }
#pragma unroll
      for (int j = 0; j < MO; ++j) {
        if (j >= st.m) break;
        const int s = scale_exp(mxb[j]);
        Eout += s;
        if (st.op[j].level != 0) continue;
        const R sc = pow2_neg<R>(s);
        cmul<R>(p0r, p0i, vr0[j] * sc, vi0[j] * sc);
        cmul<R>(p1r, p1i, vr1[j] * sc, vi1[j] * sc);
      }
    }
    R sr = active ? p0r + p1r : R(0), si = active ? p0i + p1i : R(0);
    for (int l = 1; l < st.nsum; ++l) {
      if (active) {
#pragma unroll
        for (int j = 0; j < MO; ++j) {
          if (j >= st.m) break;
          if (st.op[j].level != l) continue;
          const R sc = pow2_neg<R>(scale_exp(mxb[j]));
          cmul<R>(sr, si, vr0[j] * sc, vi0[j] * sc);
        }
      }
      sr += __shfl_xor_sync(0xffffffffu, sr, 1 << (l - 1));
      si += __shfl_xor_sync(0xffffffffu, si, 1 << (l - 1));
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

static_assert(sizeof(KStep) <= kStepRecordBytes, "step record size");
// a segment block's shared layout keeps every part 8-byte aligned (16 at part starts):
// the cluster path stores metadata words and complex values remotely
static_assert(sizeof(KStep) % 16 == 0 && sizeof(SegStage) % 8 == 0 && sizeof(SegLevel) % 8 == 0 &&
                  sizeof(Meta) == 8,
              "segment shared layout alignment");

// Segment kernel: a run of consecutive small launches as one launch. Block b
// handles slice b of the batch and runs the run's steps one after another with
// a block barrier between them (a step's operands are earlier results of the
// same slice, gates or prefix tensors, so no other block is waited for). Each
// step is the flat kernel's arithmetic restricted to one slice. The run's step
// records are staged in shared memory once. Tensors written earlier in the same
// launch (and their metadata, updated by L2 atomics) are read through L2 only
// (ld.global.cg): neither the read-only path nor L1 may hold a stale copy of an
// arena slot that an earlier step of the launch rewrote.
template <typename R>
constexpr int seg_threads() { return sizeof(R) == 4 ? 512 : 256; }
constexpr int SEG_MAX_U = 13;
constexpr int SEG_MAX_STEPS = 64;  // step records per segment launch (shared memory)
constexpr int SEG_SMEM_MAX = 220 * 1024;  // dynamic shared memory of a segment block

template <typename R>
__device__ __forceinline__ void load_pair_cg(const R* data, long long off, bool has_bit0, R& r0,
                                             R& i0, R& r1, R& i1) {
  using C2 = typename CT<R>::c2;
  if (has_bit0) {
    if constexpr (sizeof(R) == 4) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(data + 2 * off));
      r0 = v.x; i0 = v.y; r1 = v.z; i1 = v.w;
    } else {
      const C2 a = __ldcg(reinterpret_cast<const C2*>(data + 2 * off));
      const C2 b = __ldcg(reinterpret_cast<const C2*>(data + 2 * off + 2));
      r0 = a.x; i0 = a.y; r1 = b.x; i1 = b.y;
    }
  } else {
    const C2 a = __ldcg(reinterpret_cast<const C2*>(data + 2 * off));
    r0 = r1 = a.x;
    i0 = i1 = a.y;
  }
}

__device__ __forceinline__ Meta ld_meta_cg(const Meta* m) {
  const uint2 v = __ldcg(reinterpret_cast<const uint2*>(m));
  return Meta{v.x, (int)v.y};
}

// The block's metadata (every shared slot and this slice's per-slice slots) is
// cached in shared memory for the whole launch: operand scales are read there,
// and each step's result metadata is reduced in the block and written to both
// the cache and global memory (no global atomics, no metadata round trip
// through L2 between steps). Per-slice slot t of slice i is global slot
// n_shared + t * batch + i and cache slot n_shared + t.
constexpr int SEG_META_MAX = 6144;  // cached metadata slots (48 KB)
constexpr size_t SEG_ARENA_BYTES = 96 * 1024;  // shared arena for results that stay in the launch

// Results read only by later steps of the same launch live in a per-block shared
// arena (offsets planned on the host by dependency level); inputs produced before
// the launch are staged into the arena once; results read after the launch are
// also stored to global memory. The steps run level by level (a level's steps
// read only earlier levels): small steps one per warp, concurrently, larger ones
// with the whole block; one block barrier per level.

// One value pair of a step inside a segment work item. The pair index is
// I = 2 (32 chunk + lane): an operand's element offset pext(I, umask) is its arena
// offset plus the chunk's high bits (obase[j], computed once per item by lane j)
// plus the lane's six low bits, looked up in the block's table lt[umask & 63][lane].
// Loads every operand, multiplies level by level (levels >= 1 summed across lanes by
// shuffles over the lanes that share the pair's higher bits), returns the lane's
// partial result.
template <typename R>
__device__ __forceinline__ void seg_pair(const KStep& st, const R* sc, const int* obase,
                                         const unsigned char* lt, bool active, int lane,
                                         const R* arena, R& sr, R& si) {
  const int m = st.m;
  R vr0[MAXOP], vi0[MAXOP], vr1[MAXOP], vi1[MAXOP];
#pragma unroll
  for (int j = 0; j < MAXOP; ++j) {
    if (j >= m) break;
    vr0[j] = vi0[j] = vr1[j] = vi1[j] = R(0);
    if (active) {
      using C2 = typename CT<R>::c2;
      const KOp& o = st.op[j];
      const unsigned int um = o.umask;
      // the element and, for a level-0 operand holding U bit 0, its neighbour (the
      // offset is then even: one 16-byte load for complex64)
      const R* p = arena + 2 * (obase[j] + lt[((um & 63u) << 5) | (unsigned int)lane]);
      if constexpr (sizeof(R) == 4) {
        if (o.level == 0 && (um & 1u)) {
          const float4 v = *reinterpret_cast<const float4*>(p);
          vr0[j] = v.x; vi0[j] = v.y; vr1[j] = v.z; vi1[j] = v.w;
        } else {
          const float2 v = *reinterpret_cast<const float2*>(p);
          vr0[j] = vr1[j] = v.x;
          vi0[j] = vi1[j] = v.y;
        }
      } else {
        const C2 a = *reinterpret_cast<const C2*>(p);
        vr0[j] = vr1[j] = a.x;
        vi0[j] = vi1[j] = a.y;
        if (o.level == 0 && (um & 1u)) {
          const C2 b = *reinterpret_cast<const C2*>(p + 2);
          vr1[j] = b.x;
          vi1[j] = b.y;
        }
      }
    }
  }
  R p0r = 1, p0i = 0, p1r = 1, p1i = 0;
#pragma unroll
  for (int j = 0; j < MAXOP; ++j) {
    if (j >= m) break;
    if (st.op[j].level == 0) {
      cmul<R>(p0r, p0i, vr0[j] * sc[j], vi0[j] * sc[j]);
      cmul<R>(p1r, p1i, vr1[j] * sc[j], vi1[j] * sc[j]);
    }
  }
  sr = active ? p0r + p1r : R(0);
  si = active ? p0i + p1i : R(0);
  for (int l = 1; l < st.nsum; ++l) {
#pragma unroll
    for (int j = 0; j < MAXOP; ++j) {
      if (j >= m) break;
      if (st.op[j].level == l) cmul<R>(sr, si, vr0[j] * sc[j], vi0[j] * sc[j]);
    }
    sr += __shfl_xor_sync(0xffffffffu, sr, 1 << (l - 1));
    si += __shfl_xor_sync(0xffffffffu, si, 1 << (l - 1));
  }
}

// Shared layout of a segment block: records (steps, stages, levels), the metadata
// cache and the arena, each part starting on a 16-byte boundary (the records are
// copied in 16-byte chunks, the arena in 8- or 16-byte values).
// After the level records come the item map (one byte per work item: its step) and,
// past the records, the lane table lt[mask][lane] = pext(2 lane, mask) for 6-bit masks.
struct SegLayout {
  int table, meta, arena;  // byte offsets
};
constexpr int SEG_TABLE_BYTES = 64 * 32;
__host__ __device__ __forceinline__ SegLayout seg_layout(int nsteps, int nstages, int nlevels,
                                                         int nitems, int nmeta) {
  const int rec = nsteps * (int)sizeof(KStep) + nstages * (int)sizeof(SegStage) +
                  nlevels * (int)sizeof(SegLevel) + nitems;
  SegLayout l;
  l.table = (rec + 15) & ~15;
  l.meta = l.table + SEG_TABLE_BYTES;
  l.arena = (l.meta + nmeta * (int)sizeof(Meta) + 15) & ~15;
  return l;
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::
                   "r"((unsigned int)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::
                   "r"((unsigned int)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Thread-block clusters: a segment launch may give each slice a cluster of C blocks
// (C = %cluster_nctarank; 1 without a cluster launch). Every block of the cluster
// keeps a full copy of the arena and of the metadata cache; a level's work items are
// spread over all C blocks, and each result is written into every block's copy
// through distributed shared memory, so all reads stay local. One cluster barrier
// (release / acquire) per dependency level makes a level's results visible.
__device__ __forceinline__ unsigned int cl_rank() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned int cl_size() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}
// the address of local shared variable p in block `rank` of the cluster
__device__ __forceinline__ unsigned int cl_map(const void* p, unsigned int rank) {
  const unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
  unsigned int r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st2(unsigned int a, float x, float y) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" :: "r"(a), "f"(x), "f"(y) : "memory");
}
// (a complex128 value is stored as two 8-byte words: only 8-byte alignment is needed)
__device__ __forceinline__ void cl_st2(unsigned int a, double x, double y) {
  asm volatile("st.shared::cluster.f64 [%0], %1;\n\tst.shared::cluster.f64 [%0+8], %2;"
               :: "r"(a), "d"(x), "d"(y) : "memory");
}
__device__ __forceinline__ void cl_st_s32(unsigned int a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" :: "r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_max(unsigned int a, unsigned int v) {
  asm volatile("red.shared::cluster.max.u32 [%0], %1;" :: "r"(a), "r"(v) : "memory");
}

template <typename R>
__device__ __forceinline__ void seg_store(const KStep& st, long long i, unsigned long long I,
                                          R sr, R si, R* data, R* arena, unsigned int ncl) {
  const long long oi = (long long)(I >> st.nsum);
  if (st.out_soff >= 0) {
    R* p = arena + 2 * (st.out_soff + oi);
    if (ncl == 1) {
      using C2 = typename CT<R>::c2;
      C2 v;
      v.x = sr;
      v.y = si;
      *reinterpret_cast<C2*>(p) = v;
    } else {
      for (unsigned int r = 0; r < ncl; ++r) cl_st2(cl_map(p, r), sr, si);
    }
  }
  if (st.out_global) store_out<R>(data, st.out_base + i * st.out_slice_stride + oi, sr, si);
}

template <typename R>
__global__ void __launch_bounds__(seg_threads<R>()) k_segment(const KStep* steps, int nsteps,
                                                        const SegStage* stages, int nstages,
                                                        const SegLevel* levels, int nlevels,
                                                        int nitems, R* data, Meta* meta,
                                                        long long slice_first, int n_shared,
                                                        int n_slice_t, long long batch) {
  extern __shared__ __align__(16) KStep seg_steps[];
  const unsigned int ncl = cl_size(), rank = ncl > 1 ? cl_rank() : 0u;
  const long long i = blockIdx.x / ncl;  // the slice of this block's cluster
  const unsigned long long sid = (unsigned long long)(slice_first + i);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  SegStage* sst = reinterpret_cast<SegStage*>(seg_steps + nsteps);
  SegLevel* slv = reinterpret_cast<SegLevel*>(sst + nstages);
  const int nmeta = n_shared + n_slice_t;
  const SegLayout lay = seg_layout(nsteps, nstages, nlevels, nitems, nmeta);
  char* sbase = reinterpret_cast<char*>(seg_steps);
  const unsigned char* imap = reinterpret_cast<const unsigned char*>(slv + nlevels);
  unsigned char* lt = reinterpret_cast<unsigned char*>(sbase + lay.table);
  Meta* mc = reinterpret_cast<Meta*>(sbase + lay.meta);
  R* arena = reinterpret_cast<R*>(sbase + lay.arena);
  // the records (16-byte chunks) and the metadata cache: asynchronous copies, all in
  // flight; meanwhile the lane table
  {
    const char* src = reinterpret_cast<const char*>(steps);
    for (int w = threadIdx.x; w < lay.table / 16; w += blockDim.x)
      cp_async16(sbase + 16 * w, src + 16 * w);
    for (int q = threadIdx.x; q < nmeta; q += blockDim.x) {
      const long long g = q < n_shared ? q : n_shared + (long long)(q - n_shared) * batch + i;
      cp_async8(mc + q, meta + g);
    }
    for (int q = threadIdx.x; q < SEG_TABLE_BYTES; q += blockDim.x) {
      const unsigned int mask = (unsigned int)q >> 5, x = ((unsigned int)q & 31u) << 1;
      unsigned int r = 0, k = 0;
      for (int bit = 0; bit < 6; ++bit)
        if ((mask >> bit) & 1u) r |= ((x >> bit) & 1u) << k++;
      lt[q] = (unsigned char)r;
    }
    cp_async_wait_all();
  }
  __syncthreads();
  // the launch's results start at max-abs 0 (every work item raises it)
  for (int q = threadIdx.x; q < nsteps; q += blockDim.x) mc[seg_steps[q].out_mslot].maxabs = 0u;
  // inputs from outside the run: one stage record per warp, asynchronous copies into the
  // arena (every block of a cluster its own copy)
  for (int q = warp; q < nstages; q += nwarps) {
    const SegStage sg = sst[q];
    long long src = sg.base + i * sg.slice_stride;
    if (sg.smask) src += (long long)(pext64(sid, sg.smask) << sg.sshift);
    for (int e = lane; e < sg.n; e += 32) {
      if constexpr (sizeof(R) == 4) cp_async8(arena + 2 * (sg.soff + e), data + 2 * (src + e));
      else cp_async16(arena + 2 * (sg.soff + e), data + 2 * (src + e));
    }
  }
  cp_async_wait_all();
  // every block of the cluster has started and reset its slots before any remote write
  if (ncl > 1) cl_sync();
  else __syncthreads();
  const int cl_warp = (int)rank * nwarps + warp, cl_warps = (int)ncl * nwarps;
  int ibase = 0;  // the level's first entry in the item map
  for (int L = 0; L < nlevels; ++L) {
    const SegLevel lv = slv[L];
    // work items of 32 value pairs over the cluster's warps; no barrier inside a level
    // (a level's steps read only earlier levels)
    for (int it = cl_warp; it < lv.items; it += cl_warps) {
      const KStep& st = seg_steps[imap[ibase + it]];
      const int chunk = it - st.item0;
      // lane j < m: operand j's scale and its arena offset for this chunk
      R scj = R(1);
      int e = 0, bj = 0;
      if (lane < st.m) {
        const KOp& o = st.op[lane];
        const Meta mt = mc[o.mslot];
        const int sj = scale_exp(mt.maxabs);
        scj = pow2_neg<R>(sj);
        e = mt.E + sj;
        const unsigned int um = o.umask;
        bj = o.soff + (int)(pext32r((unsigned int)chunk, um >> 6) << __popc(um & 63u));
      }
      e = __reduce_add_sync(0xffffffffu, e);
      R sc[MAXOP];
      int obase[MAXOP];
#pragma unroll
      for (int j = 0; j < MAXOP; ++j) {  // m is the same in every lane
        if (j >= st.m) break;
        sc[j] = __shfl_sync(0xffffffffu, scj, j);
        obase[j] = __shfl_sync(0xffffffffu, bj, j);
      }
      const long long npairs = 1ll << (st.u - 1);
      const long long g = (long long)chunk * 32 + lane;
      const bool active = g < npairs;
      const unsigned long long I = (unsigned long long)(active ? g : 0) << 1;
      R sr, si;
      seg_pair<R>(st, sc, obase, lt, active, lane, arena, sr, si);
      float mx = 0.f;
      if (active && (lane & ((1 << (st.nsum - 1)) - 1)) == 0) {
        seg_store<R>(st, i, I, sr, si, data, arena, ncl);
        mx = absmax(sr, si);
      }
      const unsigned int red = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
      // the result's metadata: max-abs raised by every item, the exponent set by item 0
      // (in a cluster, lane r updates block r's copy)
      if (ncl == 1) {
        if (lane == 0) {
          if (red != 0u) atomicMax(&mc[st.out_mslot].maxabs, red);
          if (chunk == 0) mc[st.out_mslot].E = e;
        }
      } else if ((unsigned int)lane < ncl) {
        if (red != 0u) cl_max(cl_map(&mc[st.out_mslot].maxabs, (unsigned int)lane), red);
        if (chunk == 0) cl_st_s32(cl_map(&mc[st.out_mslot].E, (unsigned int)lane), e);
      }
    }
    ibase += lv.items;
    if (ncl > 1) cl_sync();
    else __syncthreads();
  }
  // the launch's result metadata, from the (identical) cache of the cluster's first block
  if (rank == 0)
    for (int q = threadIdx.x; q < nsteps; q += blockDim.x) {
      const KStep& st = seg_steps[q];
      meta[st.out_meta + (st.out_meta_per_slice ? i : 0)] = mc[st.out_mslot];
    }
}

// Tiled kernel. Per slice, the U index space is cut into tiles of 2^TILE_UBITS
// elements; a block owns a contiguous range of tiles. Inside a tile a thread
// owns 4 consecutive U elements (U bits 0-1), the 256 threads cover U bits
// 2-9 and a loop of Q_ITERS iterations covers U bits 10-13.
//
// Operands come in two kinds. A "streaming" operand has indices among the loop
// or tile bits: its offset is tile part (computed per warp) + thread part
// (registers) + loop part (shared-memory table) and it is loaded every loop
// iteration, UNR iterations at a time; whether it holds U bit 0 / bit 1
// decides the load shape (32, 16 or 8 bytes). A "thread-constant" operand has
// indices among U bits 0-9 only: its values at a thread's four elements are the
// same for the whole tile, so the constant operands of each level are
// multiplied once per tile into per-level factors F.
//
// Levels (fused launches): level-0 operands multiply all four elements; the
// pair over U bit 0 is summed; level-1 operands multiply the two half sums,
// which are added (U bit 1); level l >= 2 operands multiply each lane's partial
// sum before the lanes that differ in U bit l are added (a shuffle).
//
// Scaling: operands whose exponents are moderate are multiplied unscaled (the
// result exponent is then sum E_j); a slice with an extreme operand exponent
// takes the scaled path (operand j times 2^-s_j, exponent sum (E_j + s_j)). The
// decision depends only on the slice's operand metadata, so all tiles agree.
constexpr int TILE_THREADS = 256;
constexpr int TILE_UBITS = 14;
constexpr int TILE_LOCAL_BITS = 10;  // U bits fixed by the thread inside a tile
constexpr int Q_BITS = TILE_UBITS - TILE_LOCAL_BITS;
constexpr int Q_ITERS = 1 << Q_BITS;
constexpr int TILED_MAXSTREAM = 6;
constexpr int MAX_LEVELS = 8;
constexpr int MAX_FUSED_SUM = kMaxFusedSum;  // levels 0 .. MAX_FUSED_SUM-1
constexpr int SCALE_FREE_EXP = 30;  // |s_j| above this takes the scaled path

template <typename R> struct V4 { R r[4], i[4]; };

// loads the 4 values (U elements 0..3 of the thread) of one operand
template <typename R>
__device__ __forceinline__ void load4(const R* __restrict__ p, bool b0, bool b1, V4<R>& v) {
  using C2 = typename CT<R>::c2;
  if constexpr (sizeof(R) == 4) {
    if (b0 && b1) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p));
      const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
      v.r[0] = a.x; v.i[0] = a.y; v.r[1] = a.z; v.i[1] = a.w;
      v.r[2] = b.x; v.i[2] = b.y; v.r[3] = b.z; v.i[3] = b.w;
    } else if (b0 || b1) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p));
      if (b0) {
        v.r[0] = v.r[2] = a.x; v.i[0] = v.i[2] = a.y; v.r[1] = v.r[3] = a.z; v.i[1] = v.i[3] = a.w;
      } else {
        v.r[0] = v.r[1] = a.x; v.i[0] = v.i[1] = a.y; v.r[2] = v.r[3] = a.z; v.i[2] = v.i[3] = a.w;
      }
    } else {
      const float2 a = __ldg(reinterpret_cast<const float2*>(p));
      v.r[0] = v.r[1] = v.r[2] = v.r[3] = a.x;
      v.i[0] = v.i[1] = v.i[2] = v.i[3] = a.y;
    }
  } else {
    const C2* q = reinterpret_cast<const C2*>(p);
    if (b0 && b1) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const C2 a = __ldg(q + e);
        v.r[e] = a.x; v.i[e] = a.y;
      }
    } else if (b0 || b1) {
      const C2 a = __ldg(q), b = __ldg(q + 1);
      if (b0) {
        v.r[0] = v.r[2] = a.x; v.i[0] = v.i[2] = a.y; v.r[1] = v.r[3] = b.x; v.i[1] = v.i[3] = b.y;
      } else {
        v.r[0] = v.r[1] = a.x; v.i[0] = v.i[1] = a.y; v.r[2] = v.r[3] = b.x; v.i[2] = v.i[3] = b.y;
      }
    } else {
      const C2 a = __ldg(q);
      v.r[0] = v.r[1] = v.r[2] = v.r[3] = a.x;
      v.i[0] = v.i[1] = v.i[2] = v.i[3] = a.y;
    }
  }
}

// per-thread products of the thread-constant operands, by level
template <typename R> struct ConstF {
  R f0r[4], f0i[4];   // level 0, at the four elements
  R f1r[2], f1i[2];   // level 1, at U bit 1 = 0 / 1
  R flr[MAX_LEVELS], fli[MAX_LEVELS];  // levels >= 2
  unsigned int levels;  // bit l: some constant operand at level l
};

// Variants of the tiled kernel (picked per launch by the autotuner): loop
// iterations whose loads are in flight together, and the minimum resident
// blocks per SM the register allocation must allow.
constexpr int N_VARIANTS = 3;
__host__ __device__ constexpr int variant_unr(int v, int m) {
  return v == 0 ? (m <= 2 ? 4 : (m <= 4 ? 2 : 1)) : (v == 1 ? (m <= 2 ? 2 : 1) : 1);
}
__host__ __device__ constexpr int variant_minb(int v) { return v == 0 ? 1 : (v == 1 ? 3 : 4); }

template <typename R, int MS, bool SCALE, int UNR>
__device__ __forceinline__ void tile_body(const KStep& st, const R* const (&base)[MS],
                                          const int (&thr)[MS], const bool (&b0)[MS],
                                          const bool (&b1)[MS], const int (&lev)[MS],
                                          const R (&sc)[MS], const ConstF<R>& F,
                                          const int (*qoff)[Q_ITERS], R* __restrict__ out,
                                          int tid, int lane, float& mx) {
  const int nsum = st.nsum;
#pragma unroll 1
  for (int q0 = 0; q0 < Q_ITERS; q0 += UNR) {
    V4<R> v[UNR][MS];
#pragma unroll
    for (int uu = 0; uu < UNR; ++uu)
#pragma unroll
      for (int j = 0; j < MS; ++j)
        load4<R>(base[j] + 2 * (thr[j] + qoff[j][q0 + uu]), b0[j], b1[j], v[uu][j]);
#pragma unroll
    for (int uu = 0; uu < UNR; ++uu) {
      R pr[4], pi[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        pr[e] = F.f0r[e];
        pi[e] = F.f0i[e];
      }
#pragma unroll
      for (int j = 0; j < MS; ++j) {
        if (lev[j] != 0) continue;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          R br = v[uu][j].r[e], bi = v[uu][j].i[e];
          if constexpr (SCALE) {
            br *= sc[j];
            bi *= sc[j];
          }
          cmul<R>(pr[e], pi[e], br, bi);
        }
      }
      R h0r = pr[0] + pr[1], h0i = pi[0] + pi[1];
      R h1r = pr[2] + pr[3], h1i = pi[2] + pi[3];
      const unsigned long long ubase = ((unsigned long long)(q0 + uu) << TILE_LOCAL_BITS) |
                                       ((unsigned)tid << 2);
      if (nsum == 1) {
        using C2 = typename CT<R>::c2;
        const long long o = (long long)(ubase >> 1);
        if constexpr (sizeof(R) == 4) {
          *reinterpret_cast<float4*>(out + 2 * o) = make_float4(h0r, h0i, h1r, h1i);
        } else {
          C2* w = reinterpret_cast<C2*>(out + 2 * o);
          w[0] = C2{h0r, h0i};
          w[1] = C2{h1r, h1i};
        }
        mx = fmaxf(mx, fmaxf(absmax(h0r, h0i), absmax(h1r, h1i)));
      } else {
        if (F.levels & 2u) {
          cmul<R>(h0r, h0i, F.f1r[0], F.f1i[0]);
          cmul<R>(h1r, h1i, F.f1r[1], F.f1i[1]);
        }
#pragma unroll
        for (int j = 0; j < MS; ++j) {
          if (lev[j] != 1) continue;
          R ar = v[uu][j].r[0], ai = v[uu][j].i[0], br = v[uu][j].r[2], bi = v[uu][j].i[2];
          if constexpr (SCALE) {
            ar *= sc[j]; ai *= sc[j]; br *= sc[j]; bi *= sc[j];
          }
          cmul<R>(h0r, h0i, ar, ai);
          cmul<R>(h1r, h1i, br, bi);
        }
        R sr = h0r + h1r, si = h0i + h1i;
#pragma unroll
        for (int l = 2; l < MAX_FUSED_SUM; ++l) {
          if (l >= nsum) break;
          if (F.levels & (1u << l)) cmul<R>(sr, si, F.flr[l], F.fli[l]);
#pragma unroll
          for (int j = 0; j < MS; ++j) {
            if (lev[j] != l) continue;
            R ar = v[uu][j].r[0], ai = v[uu][j].i[0];
            if constexpr (SCALE) {
              ar *= sc[j];
              ai *= sc[j];
            }
            cmul<R>(sr, si, ar, ai);
          }
          sr += __shfl_xor_sync(0xffffffffu, sr, 1 << (l - 2));
          si += __shfl_xor_sync(0xffffffffu, si, 1 << (l - 2));
        }
        if ((lane & ((1 << (nsum - 2)) - 1)) == 0) {
          store_out<R>(out, (long long)(ubase >> nsum), sr, si);
          mx = fmaxf(mx, absmax(sr, si));
        }
      }
    }
  }
}

// Operands 0..ms-1 of the launch are streaming (template MS == ms), operands
// ms..m-1 thread-constant.
template <typename R, int MS, int V>
__global__ void __launch_bounds__(TILE_THREADS, variant_minb(V))
    k_bucket_tiled(const KStep st, R* data, Meta* meta) {
  constexpr int UNR = variant_unr(V, MS);
  __shared__ int qoff[MS][Q_ITERS];
  __shared__ unsigned int blkmax;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  for (int e = tid; e < MS * Q_ITERS; e += TILE_THREADS) {
    const int j = e / Q_ITERS, q = e % Q_ITERS;
    qoff[j][q] = (int)pext64((unsigned long long)q << TILE_LOCAL_BITS, st.op[j].umask);
  }
  if (tid == 0) blkmax = 0u;
  __syncthreads();
  int thr[MS], lev[MS];
  bool b0[MS], b1[MS];
#pragma unroll
  for (int j = 0; j < MS; ++j) {
    thr[j] = (int)pext64((unsigned long long)tid << 2, st.op[j].umask);
    b0[j] = st.op[j].umask & 1u;
    b1[j] = (st.op[j].umask >> 1) & 1u;
    lev[j] = st.op[j].level;
  }
  const int m = st.m;
  const long long tiles_per_slice = 1ll << (st.u - TILE_UBITS);
  const long long ntiles = st.nslices * tiles_per_slice;
  const long long T0 = ntiles * blockIdx.x / gridDim.x;
  const long long T1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  long long cur_slice = T0 < T1 ? T0 / tiles_per_slice : -1;
  float mx = 0.f;
  for (long long T = T0; T < T1; ++T) {
    const long long i = T / tiles_per_slice;
    const long long Tl = T - i * tiles_per_slice;
    if (i != cur_slice) {  // block-uniform: flush the previous slice's max
      unsigned int v = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
      if (lane == 0 && v) atomicMax(&blkmax, v);
      __syncthreads();
      if (tid == 0) {
        if (blkmax)
          atomicMax(&meta[st.out_meta + (st.out_meta_per_slice ? cur_slice : 0)].maxabs, blkmax);
        blkmax = 0u;
      }
      __syncthreads();
      cur_slice = i;
      mx = 0.f;
    }
    // tile part of every operand's offset, computed by each warp (lane j: operand j)
    const unsigned long long sid = (unsigned long long)(st.slice_first + i);
    const unsigned long long Uhi = (unsigned long long)Tl << TILE_UBITS;
    long long myoff = 0;
    int mys = 0, myE = 0;
    if (lane < m) {
      const KOp& o = st.op[lane];
      myoff = o.base + i * o.slice_stride + (long long)pext64(Uhi, o.umask);
      if (o.smask) myoff += (long long)(pext64(sid, o.smask) << o.sshift);
      const Meta mt = meta[o.meta + (o.meta_per_slice ? i : 0)];
      mys = scale_exp(mt.maxabs);
      myE = mt.E;
    }
    const bool extreme =
        __any_sync(0xffffffffu, lane < m && (mys > SCALE_FREE_EXP || mys < -SCALE_FREE_EXP));
    const int ssum = __reduce_add_sync(0xffffffffu, mys);
    const int Esum = __reduce_add_sync(0xffffffffu, myE);
    const bool scaled =
        (st.flags & 1) || extreme || ssum > 2 * SCALE_FREE_EXP || ssum < -2 * SCALE_FREE_EXP;
    if (Tl == 0 && tid == 0)
      meta[st.out_meta + (st.out_meta_per_slice ? i : 0)].E = Esum + (scaled ? ssum : 0);
    const R* base[MS];
    R sc[MS];
#pragma unroll
    for (int j = 0; j < MS; ++j) {
      const long long off = __shfl_sync(0xffffffffu, myoff, j);
      base[j] = data + 2 * off;
      sc[j] = pow2_neg<R>(__shfl_sync(0xffffffffu, mys, j));
    }
    // thread-constant operands folded into per-level factors
    ConstF<R> F;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      F.f0r[e] = 1;
      F.f0i[e] = 0;
    }
    F.f1r[0] = F.f1r[1] = 1;
    F.f1i[0] = F.f1i[1] = 0;
#pragma unroll
    for (int l = 0; l < MAX_LEVELS; ++l) {
      F.flr[l] = 1;
      F.fli[l] = 0;
    }
    F.levels = 0u;
    for (int j = MS; j < m; ++j) {
      const long long off0 = __shfl_sync(0xffffffffu, myoff, j);
      const int sj = __shfl_sync(0xffffffffu, mys, j);
      const KOp& o = st.op[j];
      V4<R> c;
      load4<R>(data + 2 * (off0 + (long long)pext64((unsigned long long)tid << 2, o.umask)),
               o.umask & 1u, (o.umask >> 1) & 1u, c);
      const R scj = scaled ? pow2_neg<R>(sj) : R(1);
      const int l = o.level;
      F.levels |= 1u << l;
      if (l == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) cmul<R>(F.f0r[e], F.f0i[e], c.r[e] * scj, c.i[e] * scj);
      } else if (l == 1) {
        cmul<R>(F.f1r[0], F.f1i[0], c.r[0] * scj, c.i[0] * scj);
        cmul<R>(F.f1r[1], F.f1i[1], c.r[2] * scj, c.i[2] * scj);
      } else {
#pragma unroll
        for (int ll = 2; ll < MAX_LEVELS; ++ll)
          if (ll == l) cmul<R>(F.flr[ll], F.fli[ll], c.r[0] * scj, c.i[0] * scj);
      }
    }
    R* out = data + 2 * (st.out_base + i * st.out_slice_stride + (long long)(Uhi >> st.nsum));
    if (scaled)
      tile_body<R, MS, true, UNR>(st, base, thr, b0, b1, lev, sc, F, qoff, out, tid, lane, mx);
    else
      tile_body<R, MS, false, UNR>(st, base, thr, b0, b1, lev, sc, F, qoff, out, tid, lane, mx);
  }
  // final flush
  unsigned int v = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
  if (lane == 0 && v) atomicMax(&blkmax, v);
  __syncthreads();
  if (tid == 0 && cur_slice >= 0 && blkmax)
    atomicMax(&meta[st.out_meta + (st.out_meta_per_slice ? cur_slice : 0)].maxabs, blkmax);
}

// Per (slice, amplitude): product of the slice result's factors in FP64 with
// the exponent applied; partials[i][b], b over the 2^a open-index values.
template <typename R>
__global__ void k_finalize(const ScalarTerm* terms, int nterms, const R* data, const Meta* meta,
                           long long nslices, long long slice_first, int a, double2* partials) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (nslices << a)) return;
  const long long i = idx >> a;
  const unsigned int b = (unsigned int)(idx & ((1ll << a) - 1));
  const unsigned long long sid = (unsigned long long)(slice_first + i);
  double pr = 1.0, pi = 0.0;
  long long E = 0;
  for (int t = 0; t < nterms; ++t) {
    const ScalarTerm& s = terms[t];
    long long off = s.base + (s.per_slice ? i * s.slice_stride : 0);
    if (s.omask) off += (long long)pext64(b, s.omask);
    if (s.smask) off += (long long)pext64(sid, s.smask) << __popc(s.omask);
    const double vr = (double)data[2 * off], vi = (double)data[2 * off + 1];
    const double nr = pr * vr - pi * vi, ni = pr * vi + pi * vr;
    pr = nr;
    pi = ni;
    E += meta[s.meta + (s.per_slice ? i : 0)].E;
  }
  const int e = (int)max(-100000ll, min(100000ll, E));
  partials[idx] = make_double2(ldexp(pr, e), ldexp(pi, e));
}

// Fixed-order FP64 sum of a batch's slice results into the accumulators: block
// b handles amplitude b; thread t adds slices t, t+1024, ... in order, then a
// fixed tree.
__global__ void __launch_bounds__(1024) k_reduce(const double2* partials, long long n, int a,
                                                 double2* acc, int first_batch) {
  __shared__ double sr[1024], si[1024];
  const long long A = 1ll << a;
  const long long b = blockIdx.x;
  double r = 0.0, im = 0.0;
  for (long long j = threadIdx.x; j < n; j += 1024) {
    r += partials[j * A + b].x;
    im += partials[j * A + b].y;
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
      acc[b].x = sr[0];
      acc[b].y = si[0];
    } else {
      acc[b].x += sr[0];
      acc[b].y += si[0];
    }
  }
}

__global__ void k_write_out(const double2* acc, long long n_amps, double norm, double* out) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_amps) return;
  out[2 * b] = acc[b].x * norm;
  out[2 * b + 1] = acc[b].y * norm;
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

// resident blocks per SM of a kernel launched with TILE_THREADS threads (cached)
template <typename K>
static int resident_blocks(K kernel) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, TILE_THREADS, 0) != cudaSuccess ||
      n < 1)
    n = 2;
  return n;
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
    st.smask = t.kind == TK_SLICE ? 0ull : t.smask;
    for (int32_t l : t.labels) {  // open indices are the pos range [n_order, n_order + n_open)
      const int j = S.pos[l] - (int)(S.pos.size() - S.k - S.n_open);
      if (j >= 0 && j < S.n_open) st.omask |= 1u << j;
    }
    st.meta = t.meta;
    terms.push_back(st);
  }
  net->gate_stage.assign(gate_bytes + meta_bytes + terms.size() * sizeof(ScalarTerm), 0);
  unsigned char* g = net->gate_stage.data();
  Meta* gm = reinterpret_cast<Meta*>(g + gate_bytes);
  for (int64_t m = 0; m < S.n_shared_meta; ++m) gm[m] = Meta{0u, 0};
  for (const STensor& t : S.tensors) {
    if (t.kind != TK_GATE) continue;
    // the gate's values in the canonical order of its schedule labels, written straight
    // into the image (canonical bit b is the gate's axis axis_of[b]; no temporary copy)
    const Tensor& gt = net->tensors[t.gate];
    const int r = (int)gt.labels.size();
    int axis_of[32] = {};
    for (int b = 0; b < r; ++b)
      for (int ax = 0; ax < r; ++ax)
        if (gt.labels[ax] == t.labels[b]) axis_of[b] = ax;
    float mx = 0.f;
    for (size_t e = 0; e < ((size_t)1 << r); ++e) {
      size_t src = 0;
      for (int b = 0; b < r; ++b)
        if ((e >> b) & 1u) src |= (size_t)1 << axis_of[b];
      for (int c = 0; c < 2; ++c) {
        const double dv = gt.data[2 * src + c];
        const size_t at = (size_t)t.offset * 2 + 2 * e + c;
        if (S.precision == QT_FP64) {
          std::memcpy(g + at * sizeof(double), &dv, sizeof(double));
        } else {
          const float fv = (float)dv;
          std::memcpy(g + at * sizeof(float), &fv, sizeof(float));
        }
        mx = std::max(mx, (float)std::fabs(dv));
      }
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

static void segtab_dirty(qt_net* net);

qt_status upload(qt_net* net, void* ws, size_t bytes, void* stream, std::string& err) {
  const Schedule& S = net->sched;
  segtab_dirty(net);
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
  net->uploaded_gen = S.generation;
  net->uploaded_data = net->data_version;
  net->uploaded_ws = ws;
  return QT_OK;
}

static void fill_op(const Schedule& S, const SGroup& g, int j, KOp& o) {
  const STensor& t = S.tensors[g.ops[j]];
  const long long eb = S.elem_bytes;
  o = KOp{};
  unsigned int um = 0;
  for (int b = 0; b < g.u; ++b)
    if (std::find(t.labels.begin(), t.labels.end(), g.ulabels[b]) != t.labels.end())
      um |= 1u << b;
  o.umask = um;
  o.level = g.levels[j];
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
    if (g.region == 1 && t.nsliced) {
      o.smask = t.smask;
      o.sshift = t.rank - t.nsliced;
    }
  }
}

// A step ready to launch: its kernel arguments (slice_first patched per batch),
// the kernel chosen for it and the grid.
struct LaunchDesc {
  KStep k;
  GemmArgs ga;  // kind 3
  int group;    // schedule launch group
  int kind;     // 0 flat, 1 tiled, 3 GEMM form (pack A', pack B', GEMM), 4 GEMM form
                // (fold A', fold B', shared-memory tiled GEMM), 5 segment (a run of small
                // flat launches, one block per slice), 6 triangle form
  int variant;  // 0..2 tiled kernel variants, 3 GEMM form
  int gemm_mode;
  unsigned grid;
  int64_t bytes, flops;  // ledger counts per slice
  long long seg_off = 0;             // kind 5: byte offset of its records in the segment table
  int seg_count = 0, stage_count = 0, level_count = 0;
  long long seg_arena = 0;           // kind 5: shared-arena elements per block
  int seg_cl_max = 1;                // kind 5: largest cluster the device co-schedules (1..8)
  int seg_items = 0;                 // kind 5: work items over all levels (item-map bytes)
  bool alt_staging = false;          // kind 4: the tiled GEMM's other staging (VARIANT_GEMM_ALT)
  int g_last = -1;                   // last schedule group the launch covers (kind 5: a run)
};

constexpr int VARIANT_GEMM = 3;
constexpr int VARIANT_TRI = 4;
constexpr int VARIANT_FLAT = 5;  // the flat kernel for a launch the tiled kernel takes
constexpr int VARIANT_STREAM = 6;  // the GEMM form's streaming kernel
constexpr int VARIANT_UMMA = 7;    // the GEMM form on the tcgen05 tensor cores
// the FP32 tiled GEMM with its other staging: by default it stages rows of up to 32
// summed values with tensor copies and rows of 64 with cp.async (the tensor-copy ring of
// long rows is 2x slower on some launches and 1.5x faster on others); this variant swaps
constexpr int VARIANT_GEMM_ALT = 8;
constexpr int N_ALL_VARIANTS = 9;

static bool tc_precision(int p) { return p == QT_TF32 || p == QT_BF16 || p == QT_3XTF32; }

// GEMM-form launches use the warp-level mma.sync kernels (BF16 mode, or tcgen05 off)
static bool legacy_tc(const Schedule& S) {
  return S.precision == QT_BF16 || (tc_precision(S.precision) && S.tcgen05 == 2);
}

// products per input pair of the tcgen05 kernel in this mode (0: the mode does not use it)
static int umma_passes(const Schedule& S) {
  if (S.tcgen05 == 2) return 0;
  return S.precision == QT_TF32 ? 1 : (S.precision == QT_3XTF32 ? 3 : 0);
}

// GEMM flavour of a GEMM-form launch in a precision mode
static int gemm_mode_for(const Schedule& S, const SGroup& g) {
  const int mb = __builtin_popcount(g.mM), nb = __builtin_popcount(g.mN);
  const bool tc_shape = mb >= 4 && nb >= 3;  // at least one full 16 x 8 tile
  if (!legacy_tc(S)) return GEMM_SIMT;  // the FP32 GEMM (the tiled kernel where it applies)
  switch (S.precision) {
    case QT_TF32: return tc_shape ? GEMM_TC_TF32 : GEMM_SIMT;
    case QT_BF16: return tc_shape ? GEMM_TC_BF16 : GEMM_SIMT;
    case QT_3XTF32: return tc_shape ? GEMM_TC_3XTF32 : GEMM_SIMT;
    default: return GEMM_SIMT;
  }
}

static void fill_gemm(const Schedule& S, const SGroup& g, long long nslices, GemmArgs& a) {
  a = GemmArgs{};
  a.m = (int)g.ops.size();
  a.nsum = g.nsum;
  a.mK = g.mK;
  a.mSA = g.mSA;
  a.mSB = g.mSB;
  a.mM = g.mM;
  a.mN = g.mN;
  a.mBt = g.mBt;
  a.nslices = nslices;
  const STensor& out = S.tensors[g.out];
  const long long eb = S.elem_bytes;
  const bool per_slice = out.kind == TK_SLICE;
  const long long region = (long long)(per_slice ? S.off_slices : S.off_prefix) / eb;
  a.out_base = region + out.offset;
  a.out_slice_stride = per_slice ? S.slice_elems : 0;
  a.out_meta_per_slice = per_slice ? 1 : 0;
  a.out_meta = out.meta;
  a.scratch_a = region + g.scratch_a;
  a.scratch_b = region + g.scratch_b;
  a.scratch_stride = per_slice ? S.slice_elems : 0;
  for (int j = 0; j < a.m; ++j) {
    KOp o;
    fill_op(S, g, j, o);
    GOp& q = a.op[j];
    q.base = o.base;
    q.slice_stride = o.slice_stride;
    q.meta = o.meta;
    q.umask = o.umask;
    q.smask = o.smask;
    q.sshift = o.sshift;
    q.meta_per_slice = o.meta_per_slice;
    q.side = g.side[j];
  }
  a.gA = g.gA;
  a.gB = g.gB;
  // GEMM_TILE: each operand's indices in its side's big operand's bit numbering
  for (int j = 0; j < a.m; ++j) {
    const unsigned int X = a.op[a.op[j].side ? g.gB : g.gA].umask;
    unsigned int xm = 0;
    int k = 0;
    for (int b = 0; b < 32; ++b)
      if ((X >> b) & 1u) {
        if ((a.op[j].umask >> b) & 1u) xm |= 1u << k;
        ++k;
      }
    a.op[j].xmask = xm;
    if (j != g.gA && j != g.gB) (a.op[j].side ? a.fold_b : a.fold_a) = 1;
  }
  a.tb = gemm_tile_bits(a, g.u);
  a.tile_inner = gemm_tile_inner(a, g.u);
  a.stay = gemm_tile_stay(a);
  a.ws_elems = (long long)(S.total_bytes / 8);
  a.umma_shape = S.tcgen05 == 3 ? 0 : 1;  // wide products unless the long-run tiles are asked for
  a.umma_kc_max = S.tcgen05 == 4 ? 2 : 0;  // chunks of 4 summed values, to check the chunking
  gemm_tile_regs(a, S.tma_block);
}

// the tcgen05 kernel takes this GEMM-form launch in the schedule's mode
static bool umma_applies(const Schedule& S, const SGroup& g, long long nslices) {
  const int np = umma_passes(S);
  if (!g.gemm || !np) return false;
  GemmArgs a;
  fill_gemm(S, g, nslices, a);
  UmmaPlan p;
  return umma_plan(a, np, p);
}

// Triangle form of a launch (three large operands; see gemm.cu k_tri_tile).
static void fill_tri(const Schedule& S, const SGroup& g, long long nslices, GemmArgs& a) {
  a = GemmArgs{};
  a.m = (int)g.ops.size();
  a.nsum = g.nsum;
  a.nslices = nslices;
  const STensor& out = S.tensors[g.out];
  const long long eb = S.elem_bytes;
  const bool per_slice = out.kind == TK_SLICE;
  const long long region = (long long)(per_slice ? S.off_slices : S.off_prefix) / eb;
  a.out_base = region + out.offset;
  a.out_slice_stride = per_slice ? S.slice_elems : 0;
  a.out_meta_per_slice = per_slice ? 1 : 0;
  a.out_meta = out.meta;
  a.gA = a.gB = -1;
  a.reg_a = a.reg_b = a.reg_a2 = a.reg_b2 = -1;
  for (int j = 0; j < a.m; ++j) {
    KOp o;
    fill_op(S, g, j, o);
    GOp& q = a.op[j];
    q.base = o.base;
    q.slice_stride = o.slice_stride;
    q.meta = o.meta;
    q.umask = o.umask;
    q.smask = o.smask;
    q.sshift = o.sshift;
    q.meta_per_slice = o.meta_per_slice;
    q.tfold = g.tfold[j];
  }
  // operands inside C: folded into C' once per slice (scratch in C's own layout)
  const unsigned int C = a.op[g.tC].umask;
  for (int j = 0; j < a.m; ++j) {
    if (a.op[j].tfold != 1) continue;
    a.fold_a = 1;
    unsigned int xm = 0;
    int k = 0;
    for (int b = 0; b < 32; ++b)
      if ((C >> b) & 1u) {
        if ((a.op[j].umask >> b) & 1u) xm |= 1u << k;
        ++k;
      }
    a.op[j].xmask = xm;
  }
  const bool per_slice_out = S.tensors[g.out].kind == TK_SLICE;
  a.scratch_a = (long long)(per_slice_out ? S.off_slices : S.off_prefix) / S.elem_bytes + g.scratch_t;
  a.scratch_stride = per_slice_out ? S.slice_elems : 0;
  a.tA = g.tA;
  a.tB = g.tB;
  a.tC = g.tC;
  a.tK = g.tK;
  a.tX = g.tX;
  a.tY = g.tY;
  a.tb = tri_tile_bits(a, g.u);
  a.ws_elems = (long long)(S.total_bytes / 8);
  a.tile_inner = tri_tile_inner(a, g.u);
}

// Concurrency of the slice-phase launches inside a captured graph: per launch, the
// stream it goes to (0: the capturing stream) and the launches on other streams it
// waits for; a launch whose event someone waits for records it.
constexpr int kStreams = 4;
struct LaunchPlan {
  std::vector<int> stream;
  std::vector<std::vector<int>> wait;
  std::vector<char> record;
};

struct EngineCache {
  uint64_t generation = 0;
  std::vector<LaunchDesc> prefix, slice;
  LaunchPlan plan;
  cudaStream_t aux[kStreams] = {};       // aux[1..] join the capture by a fork event
  std::vector<cudaEvent_t> events;       // one per slice-phase launch
  cudaEvent_t fork = nullptr, join[kStreams] = {};
  std::vector<unsigned char> segtab;  // per segment launch: step records, stage records, levels
  const void* seg_ws = nullptr;    // workspace the table was last copied to
  uint64_t seg_gen = 0;
  // captured run
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;
  long long first = -1, count = -1;
  void* ws = nullptr;
  double* d_out = nullptr;
  ~EngineCache() {
    if (exec) cudaGraphExecDestroy(exec);
    if (capture) cudaStreamDestroy(capture);
    for (int k = 1; k < kStreams; ++k) {
      if (aux[k]) cudaStreamDestroy(aux[k]);
      if (join[k]) cudaEventDestroy(join[k]);
    }
    if (fork) cudaEventDestroy(fork);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
  }
};

static void segtab_dirty(qt_net* net) {
  if (net->engine) static_cast<EngineCache*>(net->engine)->seg_ws = nullptr;
}

// copies the segment table into the workspace when it is not there yet
static bool ensure_segtab(qt_net* net, EngineCache& c, char* base, cudaStream_t s,
                          std::string& err) {
  if (c.segtab.empty() || (c.seg_ws == base && c.seg_gen == c.generation)) return true;
  if (!cuda_ok(cudaMemcpyAsync(base + net->sched.off_segtab, c.segtab.data(), c.segtab.size(),
                               cudaMemcpyHostToDevice, s),
               "upload segment table", err))
    return false;
  c.seg_ws = base;
  c.seg_gen = c.generation;
  return true;
}

template <typename R>
using TiledFn = void (*)(const KStep, R*, Meta*);

template <typename R, int V>
static TiledFn<R> tiled_fn_v(int m) {
  switch (m) {
    case 1: return k_bucket_tiled<R, 1, V>;
    case 2: return k_bucket_tiled<R, 2, V>;
    case 3: return k_bucket_tiled<R, 3, V>;
    case 4: return k_bucket_tiled<R, 4, V>;
    case 5: return k_bucket_tiled<R, 5, V>;
    case 6: return k_bucket_tiled<R, 6, V>;
    default: return nullptr;
  }
}

template <typename R>
static TiledFn<R> tiled_fn(int v, int m) {
  return v == 0 ? tiled_fn_v<R, 0>(m) : (v == 1 ? tiled_fn_v<R, 1>(m) : tiled_fn_v<R, 2>(m));
}

template <typename R>
static int tiled_grid_cap(int v, int m) {
  static int cap[N_VARIANTS][TILED_MAXSTREAM + 1] = {};
  if (cap[v][m] == 0) cap[v][m] = num_sms() * resident_blocks(tiled_fn<R>(v, m));
  return cap[v][m];
}

template <typename R>
static bool make_desc(const Schedule& S, int gi, long long nslices, LaunchDesc& d,
                      std::string& err, int variant = -1) {
  const SGroup& st = S.groups[gi];
  if (variant < 0) {
    variant = st.gemm && (tc_precision(S.precision) || S.force_gemm)
                  ? (S.force_stream && !tc_precision(S.precision) ? VARIANT_STREAM : VARIANT_GEMM)
                  : (st.tri && S.force_tri ? VARIANT_TRI : 1);
    if (st.gemm && sizeof(R) == 4 && umma_passes(S) && umma_applies(S, st, nslices))
      variant = VARIANT_UMMA;
  }
  KStep& k = d.k;
  k = KStep{};
  k.m = (int)st.ops.size();
  k.u = st.u;
  k.nsum = st.nsum;
  k.nslices = nslices;
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
  k.flags = S.force_scaled ? 1 : 0;
  if (k.m > MAXOP) {
    err = "bucket with more operands than the kernels take";
    return false;
  }
  for (int j = 0; j < k.m; ++j) {
    fill_op(S, st, j, k.op[j]);
    k.op[j].tid = st.ops[j];
    k.op[j].soff = -1;
  }
  k.out_soff = -1;
  k.out_global = 1;
  // streaming operands (indices among the tiled kernel's loop or tile bits) first
  std::stable_partition(k.op, k.op + k.m, [](const KOp& o) { return (o.umask >> TILE_LOCAL_BITS) != 0u; });
  k.ms = 0;
  for (int j = 0; j < k.m; ++j) k.ms += (k.op[j].umask >> TILE_LOCAL_BITS) != 0u;
  d.group = gi;
  d.bytes = st.bytes * (S.elem_bytes / 8);
  d.flops = st.flops;
  const bool tiled = st.u >= TILE_UBITS && k.ms >= 1 && k.ms <= TILED_MAXSTREAM && st.nsum <= 7;
  d.kind = tiled ? 1 : 0;
  d.variant = variant;
  d.gemm_mode = -1;
  if (variant == VARIANT_UMMA && st.gemm && sizeof(R) == 4) {
    fill_gemm(S, st, nslices, d.ga);
    UmmaPlan up;
    const int np = umma_passes(S);
    if (np && umma_plan(d.ga, np, up)) {
      d.kind = 3;
      d.gemm_mode = np == 1 ? GEMM_UMMA_TF32 : GEMM_UMMA_3XTF32;
      d.grid = 0;
      return true;
    }
    variant = VARIANT_GEMM;  // the tensor-core kernel does not apply: the FP32 GEMM
  }
  if (variant == VARIANT_STREAM && st.gemm && sizeof(R) == 4 && !legacy_tc(S)) {
    fill_gemm(S, st, nslices, d.ga);
    if (gemm_stream_ok(d.ga)) {
      d.ga.use_stream = 1;
      d.kind = 4;
      d.gemm_mode = GEMM_TILE;
      d.grid = 0;
      return true;
    }
    variant = VARIANT_GEMM;  // the streaming kernel does not apply: the tiled GEMM
  }
  if ((variant == VARIANT_GEMM || variant == VARIANT_GEMM_ALT) && st.gemm && sizeof(R) == 4) {
    d.kind = 3;
    d.alt_staging = variant == VARIANT_GEMM_ALT;
    d.gemm_mode = gemm_mode_for(S, st);
    fill_gemm(S, st, nslices, d.ga);
    if (d.gemm_mode == GEMM_SIMT && d.ga.tb > 0) {
      d.gemm_mode = GEMM_TILE;
      d.kind = 4;
    }
    d.grid = 0;
    return true;
  }

  if (variant == VARIANT_TRI && st.tri && sizeof(R) == 4) {
    fill_tri(S, st, nslices, d.ga);
    if (d.ga.tb > 0) {
      d.kind = 6;
      d.grid = 0;
      return true;
    }
  }
  bool use_tiled = tiled;
  if (variant == VARIANT_FLAT) {
    use_tiled = false;
    d.kind = 0;
  } else if (variant >= VARIANT_GEMM) {
    d.variant = variant = 1;
  }
  if (use_tiled) {
    const long long ntiles = nslices << (st.u - TILE_UBITS);
    d.grid = (unsigned)std::min<long long>(ntiles, tiled_grid_cap<R>(variant, k.ms));
  } else {
    const long long total = nslices << (st.u - 1);
    const long long blocks = (total + 255) / 256;
    d.grid = (unsigned)std::max<long long>(1, std::min<long long>(blocks, (long long)num_sms() * 16));
  }
  return true;
}

// Which slice-phase launches may run at the same time. A launch reads its groups'
// per-slice operands and writes their results and their GEMM / triangle scratch
// (counted whatever kernel the autotuner picks); two launches conflict when one
// writes arena elements the other reads or writes (the arena reuses memory by
// liveness, so tensors are compared as element ranges). A launch goes to the stream
// whose last launch is its latest conflict, else to the least recently used stream,
// and waits for its latest conflict on every other stream.
struct Span {
  int64_t lo, hi;  // per-slice arena elements [lo, hi)
};

static void plan_streams(const Schedule& S, const std::vector<LaunchDesc>& list, LaunchPlan& P,
                         std::vector<std::vector<Span>>* reads = nullptr,
                         std::vector<std::vector<Span>>* writes = nullptr) {
  auto span = [](int64_t off, int64_t n) { return Span{off, off + (n + 63) / 64 * 64}; };
  const size_t n = list.size();
  std::vector<std::vector<Span>> rd(n), wr(n);
  for (size_t x = 0; x < n; ++x) {
    const LaunchDesc& d = list[x];
    const int last = d.g_last >= 0 ? d.g_last : d.group;
    for (int gi = d.group; gi <= last; ++gi) {
      const SGroup& g = S.groups[gi];
      for (int32_t tid : g.ops) {
        const STensor& t = S.tensors[tid];
        if (t.kind == TK_SLICE && !t.virt) rd[x].push_back(span(t.offset, (int64_t)1 << t.rank));
      }
      const STensor& o = S.tensors[g.out];
      if (o.kind == TK_SLICE) wr[x].push_back(span(o.offset, (int64_t)1 << o.rank));
      if (g.region == 1 && g.gemm) {
        const int kb = __builtin_popcount(g.mK), bt = __builtin_popcount(g.mBt);
        wr[x].push_back(span(g.scratch_a, (int64_t)1 << (bt + __builtin_popcount(g.mM) + kb)));
        wr[x].push_back(span(g.scratch_b, (int64_t)1 << (bt + __builtin_popcount(g.mN) + kb)));
      }
      if (g.region == 1 && g.tri) wr[x].push_back(span(g.scratch_t, (int64_t)1 << g.tCbits));
    }
  }
  auto meet = [](const std::vector<Span>& a, const std::vector<Span>& b) {
    for (const Span& p : a)
      for (const Span& q : b)
        if (p.lo < q.hi && q.lo < p.hi) return true;
    return false;
  };
  P.stream.assign(n, 0);
  P.wait.assign(n, {});
  P.record.assign(n, 0);
  int lastl[kStreams];
  for (int k = 0; k < kStreams; ++k) lastl[k] = -1;
  for (size_t m = 0; m < n; ++m) {
    int latest[kStreams];  // latest conflicting launch on each stream
    for (int k = 0; k < kStreams; ++k) latest[k] = -1;
    int top = -1;
    for (size_t l = 0; l < m; ++l)
      if (meet(wr[l], rd[m]) || meet(wr[l], wr[m]) || meet(rd[l], wr[m])) {
        latest[P.stream[l]] = std::max(latest[P.stream[l]], (int)l);
        top = std::max(top, (int)l);
      }
    int st = -1;
    if (top >= 0 && lastl[P.stream[top]] == top) st = P.stream[top];
    if (st < 0) {
      st = 0;
      for (int k = 1; k < kStreams; ++k)
        if (lastl[k] < lastl[st]) st = k;
    }
    P.stream[m] = st;
    for (int k = 0; k < kStreams; ++k)
      if (k != st && latest[k] >= 0) {
        P.wait[m].push_back(latest[k]);
        P.record[latest[k]] = 1;
      }
    lastl[st] = (int)m;
  }
  if (reads) *reads = rd;
  if (writes) *writes = wr;
}

// Segment launches: dynamic shared memory of a block and the largest cluster size (8,
// 4, 2, else 1) the device can co-schedule with it, asked once when the launch is
// planned (never during stream capture).
template <typename R>
static void seg_set_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_segment<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         SEG_SMEM_MAX);
    done = true;
  }
}

template <typename R>
static size_t seg_smem(const Schedule& S, const LaunchDesc& d) {
  const SegLayout l = seg_layout(d.seg_count, d.stage_count, d.level_count, d.seg_items,
                                 (int)(S.n_shared_meta + S.n_slice_meta_tensors));
  return (size_t)l.arena + (size_t)d.seg_arena * 2 * sizeof(R);
}

template <typename R>
static int seg_cluster_max(size_t smem) {
  seg_set_attr<R>();
  for (int c = 8; c > 1; c >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c);
    cfg.blockDim = dim3(seg_threads<R>());
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_segment<R>, &cfg) == cudaSuccess && n > 0) return c;
    cudaGetLastError();
  }
  return 1;
}

// Blocks per slice of a segment launch: the network's setting (QT_OPT_SEG_CLUSTER), or
// the largest of 8, 4, 2 whose clusters fill at most two blocks per SM, so that small
// slice batches spread each slice's work over several SMs; 1 for large batches. Never
// above what the device co-schedules.
static int seg_cluster_size(const qt_net* net, const LaunchDesc& d, long long nslices) {
  int c = net->seg_cluster;
  if (c == 0) {
    c = 8;
    while (c > 1 && nslices * c > 2ll * num_sms()) c >>= 1;
  }
  return std::min(c, d.seg_cl_max);
}

template <typename R>
static bool build_cache(qt_net* net, EngineCache& c, std::string& err) {
  const Schedule& S = net->sched;
  c.prefix.clear();
  c.slice.clear();
  for (int gi = 0; gi < (int)S.groups.size(); ++gi) {
    LaunchDesc d;
    const bool pre = S.groups[gi].region == 0;
    if (!make_desc<R>(S, gi, pre ? 1 : S.batch, d, err)) return false;
    (pre ? c.prefix : c.slice).push_back(d);
  }
  // runs of two or more consecutive small flat launches become one segment launch
  c.segtab.clear();
  const int nsh = (int)S.n_shared_meta;
  auto mslot_of = [&](long long g, bool per_slice) -> int {
    return per_slice ? nsh + (int)((g - nsh) / S.batch) : (int)g;
  };
  for (std::vector<LaunchDesc>* list : {&c.prefix, &c.slice}) {
    std::vector<LaunchDesc> merged;
    // Plans the run [i, j): its steps are ordered by dependency level, so every value a
    // step reads inside the run must come from the shared arena (a reordered step may
    // already have reused the global slot of a tensor that dies in the run); returns
    // false when some input or internal result does not fit.
    auto plan = [&](size_t i, size_t j, LaunchDesc& d, std::vector<KStep>& recs,
                    std::vector<SegStage>& stages, std::vector<SegLevel>& levels,
                    std::vector<unsigned char>& imap) -> bool {
      const int n = (int)(j - i);
      const int gi_last = (*list)[j - 1].group;
      std::map<int, int> producer;  // tid -> step index in the run
      std::vector<int> lev(n, 0);
      for (int q = 0; q < n; ++q) {
        const KStep& k = (*list)[i + q].k;
        for (int o = 0; o < k.m; ++o) {
          auto it = producer.find(k.op[o].tid);
          if (it != producer.end()) lev[q] = std::max(lev[q], lev[it->second] + 1);
        }
        producer[S.groups[(*list)[i + q].group].out] = q;
      }
      const int nlev = *std::max_element(lev.begin(), lev.end()) + 1;
      std::map<int, int> last_lev;  // last level reading each tensor inside the run
      for (int q = 0; q < n; ++q) {
        const KStep& k = (*list)[i + q].k;
        for (int o = 0; o < k.m; ++o) {
          auto it = last_lev.find(k.op[o].tid);
          if (it == last_lev.end() || it->second < lev[q]) last_lev[k.op[o].tid] = lev[q];
        }
      }
      const long long cap = (long long)(SEG_ARENA_BYTES / (2 * sizeof(R)));
      std::map<long long, long long> free_blocks{{0, cap}};
      long long peak = 0;
      auto take = [&](long long cnt) -> long long {
        cnt = (cnt + 1) & ~1ll;
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it)
          if (it->second >= cnt) {
            const long long off = it->first, rest = it->second - cnt;
            free_blocks.erase(it);
            if (rest > 0) free_blocks[off + cnt] = rest;
            peak = std::max(peak, off + cnt);
            return off;
          }
        return -1;
      };
      auto give = [&](long long off, long long cnt) {
        cnt = (cnt + 1) & ~1ll;
        auto it = free_blocks.emplace(off, cnt).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
          it->second += nx->second;
          free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
          auto pv = std::prev(it);
          if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            free_blocks.erase(it);
          }
        }
      };
      std::map<int, std::pair<long long, long long>> slot;  // tid -> (offset, elements)
      recs.clear();
      stages.clear();
      levels.clear();
      imap.clear();
      // inputs produced before the run: staged at the start, kept for the whole run
      int cum = 0;
      for (int q = 0; q < n; ++q) {
        const KStep& k = (*list)[i + q].k;
        const bool region1 = S.groups[(*list)[i + q].group].region == 1;
        for (int o = 0; o < k.m; ++o) {
          const int tid = k.op[o].tid;
          if (producer.count(tid) || slot.count(tid)) continue;
          const STensor& tt = S.tensors[tid];
          const long long cnt = 1ll << (tt.rank - (region1 ? tt.nsliced : 0));
          const long long off = take(cnt);
          if (off < 0) return false;
          slot[tid] = {off, cnt};
          stages.push_back(SegStage{k.op[o].base, k.op[o].slice_stride, k.op[o].smask,
                                    k.op[o].sshift, (int)cnt, (int)off, cum});
          cum += (int)cnt;
        }
      }
      d = (*list)[i];
      d.kind = 5;
      d.bytes = d.flops = 0;
      for (int L = 0; L < nlev; ++L) {
        // results no longer read at this level or later give their slot back
        for (auto it = slot.begin(); it != slot.end();) {
          auto ll = last_lev.find(it->first);
          if (producer.count(it->first) && (ll == last_lev.end() || ll->second < L)) {
            give(it->second.first, it->second.second);
            it = slot.erase(it);
          } else {
            ++it;
          }
        }
        SegLevel sl{(int)recs.size(), 0, 0, 0};
        int items = 0;
        for (int pass = 0; pass < 2; ++pass)  // warp steps, then block steps
          for (int q = 0; q < n; ++q) {
            if (lev[q] != L) continue;
            KStep k = (*list)[i + q].k;
            const bool warp_step = k.u <= 6;
            if (warp_step != (pass == 0)) continue;
            for (int o = 0; o < k.m; ++o) {
              auto it = slot.find(k.op[o].tid);
              if (it == slot.end()) return false;
              k.op[o].soff = (int)it->second.first;
              k.op[o].mslot = mslot_of(k.op[o].meta, k.op[o].meta_per_slice != 0);
            }
            const int out = S.groups[(*list)[i + q].group].out;
            const STensor& ot = S.tensors[out];
            k.out_soff = -1;
            k.out_mslot = mslot_of(k.out_meta, k.out_meta_per_slice != 0);
            if (last_lev.count(out)) {
              const long long cnt = 1ll << (ot.rank - (ot.kind == TK_SLICE ? ot.nsliced : 0));
              const long long off = take(cnt);
              if (off < 0) return false;
              k.out_soff = (int)off;
              slot[out] = {off, cnt};
            }
            k.out_global = (ot.last_use > gi_last || k.out_soff < 0) ? 1 : 0;
            k.item0 = items;
            const int nit = (int)std::max(1ll, (1ll << (k.u - 1)) / 32);
            items += nit;
            imap.insert(imap.end(), (size_t)nit, (unsigned char)recs.size());
            recs.push_back(k);
            (pass == 0 ? sl.nwarp : sl.nblock)++;
            d.bytes += (*list)[i + q].bytes;
            d.flops += (*list)[i + q].flops;
          }
        sl.items = items;
        levels.push_back(sl);
      }
      d.seg_count = n;
      d.seg_items = (int)imap.size();
      d.stage_count = (int)stages.size();
      d.level_count = nlev;
      d.seg_arena = peak;
      return seg_smem<R>(S, d) <= (size_t)SEG_SMEM_MAX;
    };
    for (size_t i = 0; i < list->size();) {
      size_t j = i;
      const int max_u = std::min(net->seg_max_u, SEG_MAX_U);
      auto small = [&](const LaunchDesc& d) { return d.kind == 0 && d.k.u <= max_u; };
      while (j < list->size() && small((*list)[j]) && j - i < (size_t)SEG_MAX_STEPS) ++j;
      LaunchDesc d;
      std::vector<KStep> recs;
      std::vector<SegStage> stages;
      std::vector<SegLevel> levels;
      std::vector<unsigned char> imap;
      bool ok = false;
      if (net->segments && S.n_shared_meta + S.n_slice_meta_tensors <= SEG_META_MAX)
        for (; j - i >= 2; --j)
          if (plan(i, j, d, recs, stages, levels, imap)) {
            ok = true;
            break;
          }
      if (!ok) {
        merged.push_back((*list)[i]);
        ++i;
        continue;
      }
      d.seg_cl_max = seg_cluster_max<R>(seg_smem<R>(S, d));
      // records start on 16 bytes and are read in 16-byte chunks
      c.segtab.resize((c.segtab.size() + 15) & ~(size_t)15, 0);
      d.seg_off = (long long)c.segtab.size();
      auto append = [&](const void* p, size_t bytes) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        c.segtab.insert(c.segtab.end(), b, b + bytes);
      };
      append(recs.data(), recs.size() * sizeof(KStep));
      append(stages.data(), stages.size() * sizeof(SegStage));
      append(levels.data(), levels.size() * sizeof(SegLevel));
      append(imap.data(), imap.size());
      c.segtab.resize((c.segtab.size() + 15) & ~(size_t)15, 0);
      d.g_last = (*list)[j - 1].group;
      merged.push_back(d);
      i = j;
    }
    *list = merged;
  }
  if (c.segtab.size() > S.groups.size() * kStepRecordBytes) {
    err = "segment tables exceed their workspace region";
    return false;
  }
  plan_streams(S, c.slice, c.plan);
  c.seg_ws = nullptr;
  if (c.exec) cudaGraphExecDestroy(c.exec);
  c.exec = nullptr;
  c.first = c.count = -1;
  c.generation = S.generation;
  return true;
}

template <typename R>
static void launch_desc(qt_net* net, const LaunchDesc& d0, long long nslices, long long slice_first,
                        char* base, cudaStream_t s) {
  const Schedule& S = net->sched;
  if (d0.kind == 5) {
    R* data = reinterpret_cast<R*>(base);
    Meta* meta = reinterpret_cast<Meta*>(base + S.off_meta);
    ProfRec pr{S.groups[d0.group].first, 5, nslices, d0.bytes * nslices, d0.flops * nslices,
               nullptr, nullptr};
    if (net->prof) prof_begin(net, s, pr);
    net->launches++;
    const KStep* tab = reinterpret_cast<const KStep*>(base + S.off_segtab + d0.seg_off);
    const SegStage* stab = reinterpret_cast<const SegStage*>(tab + d0.seg_count);
    const SegLevel* ltab = reinterpret_cast<const SegLevel*>(stab + d0.stage_count);
    seg_set_attr<R>();
    const int nsh = (int)S.n_shared_meta, nst = (int)S.n_slice_meta_tensors;
    const size_t smem = seg_smem<R>(S, d0);
    const int ncl = seg_cluster_size(net, d0, nslices);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nslices * ncl));
    cfg.blockDim = dim3(seg_threads<R>());
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)ncl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = ncl > 1 ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k_segment<R>, tab, d0.seg_count, stab, d0.stage_count, ltab,
                       d0.level_count, d0.seg_items, data, meta, slice_first, nsh, nst,
                       (long long)S.batch);
    if (net->prof) prof_end(net, s, pr);
    return;
  }
  KStep k = d0.k;
  k.nslices = nslices;
  k.slice_first = slice_first;
  unsigned grid = d0.grid;
  if (nslices != d0.k.nslices) {  // a short last batch
    LaunchDesc d;
    std::string e;
    make_desc<R>(S, d0.group, nslices, d, e, d0.variant);
    grid = d.grid;
  }
  R* data = reinterpret_cast<R*>(base);
  Meta* meta = reinterpret_cast<Meta*>(base + S.off_meta);
  // (profile class 7: the GEMM form's streaming kernel)
  // (profile class 7: the GEMM form's streaming kernel; 8: the tcgen05 GEMM)
  const bool umma = d0.kind == 3 &&
                    (d0.gemm_mode == GEMM_UMMA_TF32 || d0.gemm_mode == GEMM_UMMA_3XTF32);
  ProfRec pr{S.groups[d0.group].first,
             umma ? 8 : (d0.kind == 4 && d0.ga.use_stream ? 7 : d0.kind), nslices,
             d0.bytes * nslices, d0.flops * nslices, nullptr, nullptr};
  if (net->prof) prof_begin(net, s, pr);
  if (d0.kind == 6) {
    GemmArgs ga = d0.ga;
    ga.nslices = nslices;
    ga.slice_first = slice_first;
    ga.err = reinterpret_cast<int*>(base + S.off_err);
    ga.use_tma = net->tma ? 1 : 0;
    bool tma = false;
    net->launches += tri_launch(ga, reinterpret_cast<float*>(base), reinterpret_cast<GMeta*>(meta),
                                s, num_sms(), &tma);
    if (tma) net->tma_launches++;
    if (net->prof) prof_end(net, s, pr);
    return;
  }
  if (d0.kind >= 3) {
    GemmArgs ga = d0.ga;
    ga.nslices = nslices;
    ga.slice_first = slice_first;
    ga.err = reinterpret_cast<int*>(base + S.off_err);
    // default staging: tensor copies for rows of up to 32 summed values
    ga.use_tma = (net->tma && ((ga.nsum <= 5) != d0.alt_staging)) ? 1 : 0;
    bool tma = false;
    net->launches += gemm_launch(ga, d0.gemm_mode, reinterpret_cast<float*>(base),
                                 reinterpret_cast<GMeta*>(meta), s, num_sms(), &tma);
    if (tma && umma) net->umma_launches++;
    else if (tma) net->tma_launches++;
    if (ga.use_stream) net->stream_launches++;
    if (net->prof) prof_end(net, s, pr);
    return;
  }
  net->launches++;
  if (d0.kind == 1) {
    tiled_fn<R>(d0.variant, k.ms)<<<grid, TILE_THREADS, 0, s>>>(k, data, meta);
  } else {
    if (k.m <= 4) k_bucket_flat<R, 4><<<grid, 256, 0, s>>>(k, data, meta);
    else if (k.m <= 8) k_bucket_flat<R, 8><<<grid, 256, 0, s>>>(k, data, meta);
    else k_bucket_flat<R, MAXOP><<<grid, 256, 0, s>>>(k, data, meta);
  }
  if (net->prof) prof_end(net, s, pr);
}

template <typename R>
static qt_status enqueue_run(qt_net* net, EngineCache& c, long long first, long long count,
                             char* base, cudaStream_t s, double* d_out, std::string& err,
                             bool fork = false) {
  const Schedule& S = net->sched;
  const size_t ngm = n_gate_meta(S);
  Meta* meta = reinterpret_cast<Meta*>(base + S.off_meta);
  if (!cuda_ok(cudaMemsetAsync(base + S.off_err, 0, sizeof(int), s), "reset status", err))
    return QT_ECUDA;
  // prefix (contract_first): once, unsliced
  if (S.n_shared_meta > (int64_t)ngm &&
      !cuda_ok(cudaMemsetAsync(meta + ngm, 0, (S.n_shared_meta - ngm) * sizeof(Meta), s),
               "reset prefix meta", err))
    return QT_ECUDA;
  for (const LaunchDesc& d : c.prefix) launch_desc<R>(net, d, 1, 0, base, s);
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
    if (fork) {
      // fork: the other streams join the capture behind everything issued so far
      cudaEventRecord(c.fork, s);
      for (int k = 1; k < kStreams; ++k) cudaStreamWaitEvent(c.aux[k], c.fork, 0);
      for (size_t x = 0; x < c.slice.size(); ++x) {
        cudaStream_t st = c.plan.stream[x] ? c.aux[c.plan.stream[x]] : s;
        for (int w : c.plan.wait[x]) cudaStreamWaitEvent(st, c.events[w], 0);
        launch_desc<R>(net, c.slice[x], nb, b0, base, st);
        if (c.plan.record[x]) cudaEventRecord(c.events[x], st);
      }
      for (int k = 1; k < kStreams; ++k) {  // join
        cudaEventRecord(c.join[k], c.aux[k]);
        cudaStreamWaitEvent(s, c.join[k], 0);
      }
    } else {
      for (const LaunchDesc& d : c.slice) launch_desc<R>(net, d, nb, b0, base, s);
    }
    ProfRec pr{-1, 2, nb, 0, 0, nullptr, nullptr};
    if (net->prof) prof_begin(net, s, pr);
    net->launches += 2;
    const long long nthreads = nb * S.n_amps;
    k_finalize<R><<<(unsigned)((nthreads + 127) / 128), 128, 0, s>>>(
        terms, nterms, reinterpret_cast<const R*>(base), meta, nb, b0, S.n_open, partials);
    k_reduce<<<(unsigned)S.n_amps, 1024, 0, s>>>(partials, nb, S.n_open, acc,
                                                 first_batch ? 1 : 0);
    if (net->prof) prof_end(net, s, pr);
    first_batch = false;
  }
  net->launches++;
  k_write_out<<<(unsigned)((S.n_amps + 255) / 256), 256, 0, s>>>(acc, S.n_amps,
                                                                std::pow(2.0, -0.5 * net->n), d_out);
  if (!cuda_ok(cudaGetLastError(), "kernel launch", err)) return QT_ECUDA;
  return QT_OK;
}

// Autotuner: runs the schedule's first batch once, launching every tiled step
// with each kernel variant (forward then backward over the variants, so warm
// caches favour none), and keeps the fastest variant per step.
template <typename R>
static qt_status autotune_impl(qt_net* net, char* base, cudaStream_t s, std::string& report,
                               std::string& err) {
  if (!net->engine) net->engine = new EngineCache();
  EngineCache& c = *static_cast<EngineCache*>(net->engine);
  const Schedule& S = net->sched;
  if (c.generation != S.generation && !build_cache<R>(net, c, err)) return QT_ERANGE;
  if (!ensure_segtab(net, c, base, s, err)) return QT_ECUDA;
  const bool prof = net->prof;
  net->prof = false;
  struct Trial {
    std::vector<LaunchDesc>* list;
    size_t idx;
    int variant;
    cudaEvent_t a, b;
  };
  std::vector<Trial> trials;
  auto ev = [&]() {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  };
  auto run_list = [&](std::vector<LaunchDesc>& list, long long nb, long long b0) {
    for (size_t i = 0; i < list.size(); ++i) {
      LaunchDesc& d = list[i];
      const SGroup& grp = S.groups[d.group];
      // the FP32 GEMM, streaming and triangle kernels are candidates in every mode but
      // the legacy tensor-core one (they are at least as accurate as TF32 products)
      const bool can_gemm = grp.gemm && !legacy_tc(S) && sizeof(R) == 4;
      const bool can_tri = grp.tri && !legacy_tc(S) && sizeof(R) == 4;
      const bool can_umma = grp.gemm && sizeof(R) == 4 && umma_applies(S, grp, d.k.nslices);
      if (d.kind == 0 || d.kind == 5 ||
          ((d.kind == 3 || d.kind == 4) && (legacy_tc(S) || S.force_gemm)) ||
          (d.kind == 6 && S.force_tri) || (can_umma && (S.tcgen05 == 1 || S.tcgen05 == 3 || S.tcgen05 == 4))) {
        launch_desc<R>(net, d, nb, b0, base, s);
        continue;
      }
      std::vector<int> cands;
      for (int v = 0; v < N_VARIANTS; ++v) cands.push_back(v);
      if (can_umma) cands.push_back(VARIANT_UMMA);
      if (can_gemm) cands.push_back(VARIANT_GEMM);
      if (can_gemm && net->tma) cands.push_back(VARIANT_GEMM_ALT);
      if (can_gemm) {
        GemmArgs ga;
        fill_gemm(S, grp, d.k.nslices, ga);
        if (gemm_stream_ok(ga)) cands.push_back(VARIANT_STREAM);
      }
      if (can_tri) cands.push_back(VARIANT_TRI);
      if (grp.u <= 20) cands.push_back(VARIANT_FLAT);  // small launches: one pair per thread
      const int nv = (int)cands.size();
      for (int pass = 0; pass < 2; ++pass)
        for (int t = 0; t < nv; ++t) {
          const int v = cands[pass == 0 ? t : nv - 1 - t];
          LaunchDesc dv = d;
          std::string e2;
          make_desc<R>(S, d.group, d.k.nslices, dv, e2, v);
          Trial tr{&list, i, v, ev(), ev()};
          cudaEventRecord(tr.a, s);
          launch_desc<R>(net, dv, nb, b0, base, s);
          cudaEventRecord(tr.b, s);
          trials.push_back(tr);
        }
    }
  };
  const size_t ngm = n_gate_meta(S);
  Meta* meta = reinterpret_cast<Meta*>(base + S.off_meta);
  if (S.n_shared_meta > (int64_t)ngm)
    cudaMemsetAsync(meta + ngm, 0, (S.n_shared_meta - ngm) * sizeof(Meta), s);
  run_list(c.prefix, 1, 0);
  const long long nb = std::min<long long>(S.batch, S.nslices);
  if (S.n_slice_meta_tensors)
    cudaMemsetAsync(meta + S.n_shared_meta, 0,
                    (size_t)(S.n_slice_meta_tensors * S.batch) * sizeof(Meta), s);
  run_list(c.slice, nb, 0);
  qt_status st = QT_OK;
  if (!cuda_ok(cudaStreamSynchronize(s), "autotune run", err)) st = QT_ECUDA;
  std::vector<std::vector<float>> best;  // per (list, idx): ms per variant
  report = "[";
  if (st == QT_OK) {
    // accumulate times per step and variant
    struct Key { std::vector<LaunchDesc>* list; size_t idx; };
    std::vector<std::pair<Key, std::vector<float>>> acc;
    for (const Trial& tr : trials) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, tr.a, tr.b);
      if (acc.empty() || acc.back().first.list != tr.list || acc.back().first.idx != tr.idx)
        acc.push_back({Key{tr.list, tr.idx}, std::vector<float>(N_ALL_VARIANTS, 1e30f)});
      float& slot = acc.back().second[tr.variant];
      slot = slot >= 1e29f ? ms : slot + ms;
    }
    bool first = true;
    for (auto& kv : acc) {
      LaunchDesc& d = (*kv.first.list)[kv.first.idx];
      int bv = 0;
      for (int v = 1; v < N_ALL_VARIANTS; ++v)
        if (kv.second[v] < kv.second[bv]) bv = v;
      std::string e2;
      make_desc<R>(S, d.group, d.k.nslices, d, e2, bv);
      char buf[256];
      auto half = [](float x) { return x >= 1e29f ? -1.0 : x / 2.0; };
      std::snprintf(buf, sizeof buf,
                    "%s{\"step\":%d,\"variant\":%d,\"ms\":[%.4f,%.4f,%.4f,%.4f,%.4f,%.4f,%.4f,%.4f,%.4f]}",
                    first ? "" : ",", S.groups[d.group].first, bv, half(kv.second[0]),
                    half(kv.second[1]), half(kv.second[2]), half(kv.second[3]),
                    half(kv.second[4]), half(kv.second[5]), half(kv.second[6]),
                    half(kv.second[7]), half(kv.second[8]));
      report += buf;
      first = false;
    }
  }
  report += "]";
  for (const Trial& tr : trials) {
    cudaEventDestroy(tr.a);
    cudaEventDestroy(tr.b);
  }
  if (c.exec) {
    cudaGraphExecDestroy(c.exec);
    c.exec = nullptr;
  }
  c.first = c.count = -1;
  net->prof = prof;
  return st;
}

qt_status autotune(qt_net* net, void* ws, void* stream, std::string& report, std::string& err) {
  char* base = (char*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  if (net->sched.precision == QT_FP64) return autotune_impl<double>(net, base, s, report, err);
  return autotune_impl<float>(net, base, s, report, err);
}

constexpr long long kMaxGraphLaunches = 8192;

template <typename R>
static qt_status run_impl(qt_net* net, long long first, long long count, char* base,
                          cudaStream_t s, double* d_out, std::string& err) {
  if (!net->engine) net->engine = new EngineCache();
  EngineCache& c = *static_cast<EngineCache*>(net->engine);
  const Schedule& S = net->sched;
  if (c.generation != S.generation && !build_cache<R>(net, c, err)) return QT_ERANGE;
  if (!ensure_segtab(net, c, base, s, err)) return QT_ECUDA;
  const long long batches = (count + S.batch - 1) / S.batch;
  const long long nlaunch = (long long)c.prefix.size() + batches * ((long long)c.slice.size() + 2) + 1;
  if (!net->graphs || net->prof || nlaunch > kMaxGraphLaunches)
    return enqueue_run<R>(net, c, first, count, base, s, d_out, err);
  // captured once per (range, workspace, output, schedule), replayed afterwards
  if (!(c.exec && c.first == first && c.count == count && c.ws == (void*)base && c.d_out == d_out)) {
    if (c.exec) {
      cudaGraphExecDestroy(c.exec);
      c.exec = nullptr;
    }
    if (!c.capture &&
        !cuda_ok(cudaStreamCreateWithFlags(&c.capture, cudaStreamNonBlocking), "capture stream", err))
      return QT_ECUDA;
    // streams and events of the concurrent slice phase (fork / join inside the capture)
    const bool fork = net->concurrent && c.slice.size() > 1;
    if (fork) {
      for (int k = 1; k < kStreams; ++k) {
        if (!c.aux[k] && !cuda_ok(cudaStreamCreateWithFlags(&c.aux[k], cudaStreamNonBlocking),
                                  "aux stream", err))
          return QT_ECUDA;
        if (!c.join[k] &&
            !cuda_ok(cudaEventCreateWithFlags(&c.join[k], cudaEventDisableTiming), "event", err))
          return QT_ECUDA;
      }
      if (!c.fork && !cuda_ok(cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming), "event", err))
        return QT_ECUDA;
      while (c.events.size() < c.slice.size()) {
        cudaEvent_t e = nullptr;
        if (!cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event", err))
          return QT_ECUDA;
        c.events.push_back(e);
      }
    }
    if (!cuda_ok(cudaStreamBeginCapture(c.capture, cudaStreamCaptureModeThreadLocal),
                 "begin capture", err))
      return QT_ECUDA;
    const int64_t launches0 = net->launches;
    qt_status r = enqueue_run<R>(net, c, first, count, base, c.capture, d_out, err, fork);
    net->launches = launches0;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c.capture, &g);
    if (r != QT_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (!cuda_ok(e, "end capture", err)) return QT_ECUDA;
    e = cudaGraphInstantiate(&c.exec, g, 0);
    cudaGraphDestroy(g);
    if (!cuda_ok(e, "graph instantiate", err)) {
      c.exec = nullptr;
      return QT_ECUDA;
    }
    c.first = first;
    c.count = count;
    c.ws = base;
    c.d_out = d_out;
  }
  net->launches += nlaunch;
  if (!cuda_ok(cudaGraphLaunch(c.exec, s), "graph launch", err)) return QT_ECUDA;
  return QT_OK;
}

qt_status run(qt_net* net, long long first, long long count, void* ws, void* stream,
              double* d_out, std::string& err) {
  char* base = (char*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  if (net->sched.precision == QT_FP64) return run_impl<double>(net, first, count, base, s, d_out, err);
  return run_impl<float>(net, first, count, base, s, d_out, err);
}

// the device status word of a run: nonzero when a bounded wait gave up
// The slice phase's launches as the engine would capture them: per launch its first and
// last schedule group, kernel class, stream, the launches it waits for, and the per-slice
// arena ranges it reads and writes. Host work only.
template <typename R>
static bool launch_plan_impl(qt_net* net, std::string& out, std::string& err) {
  EngineCache tmp;
  if (!build_cache<R>(net, tmp, err)) return false;
  std::vector<std::vector<Span>> rd, wr;
  LaunchPlan P;
  plan_streams(net->sched, tmp.slice, P, &rd, &wr);
  std::ostringstream o;
  o << "{\"streams\":" << kStreams << ",\"launches\":[";
  auto spans = [&](const std::vector<Span>& v) {
    o << "[";
    for (size_t q = 0; q < v.size(); ++q) o << (q ? "," : "") << "[" << v[q].lo << "," << v[q].hi << "]";
    o << "]";
  };
  for (size_t x = 0; x < tmp.slice.size(); ++x) {
    const LaunchDesc& d = tmp.slice[x];
    o << (x ? "," : "") << "{\"group\":" << d.group << ",\"g_last\":"
      << (d.g_last >= 0 ? d.g_last : d.group) << ",\"kind\":" << d.kind
      << ",\"stream\":" << P.stream[x] << ",\"wait\":[";
    for (size_t q = 0; q < P.wait[x].size(); ++q) o << (q ? "," : "") << P.wait[x][q];
    o << "],\"reads\":";
    spans(rd[x]);
    o << ",\"writes\":";
    spans(wr[x]);
    if (d.kind != 5 && d.group >= 0 && net->sched.groups[d.group].gemm) {
      // a group with a GEMM form (whichever kernel runs it): summed indices, the U-bit
      // masks of each index class, the two large operands' index masks, the tiled
      // kernels' tile bits and staying side
      GemmArgs ga;
      fill_gemm(net->sched, net->sched.groups[d.group], d.k.nslices, ga);
      o << ",\"gemm\":{\"step\":" << net->sched.groups[d.group].first << ",\"nsum\":" << ga.nsum << ",\"mK\":" << ga.mK << ",\"mM\":" << ga.mM
        << ",\"mN\":" << ga.mN << ",\"mBt\":" << ga.mBt << ",\"mSA\":" << ga.mSA
        << ",\"mSB\":" << ga.mSB << ",\"umA\":" << (ga.gA >= 0 ? ga.op[ga.gA].umask : 0u)
        << ",\"umB\":" << (ga.gB >= 0 ? ga.op[ga.gB].umask : 0u) << ",\"tb\":" << ga.tb
        << ",\"stay\":" << ga.stay << ",\"fold_a\":" << ga.fold_a << ",\"fold_b\":"
        << ga.fold_b << ",\"scratch\":[" << ga.scratch_a << "," << ga.scratch_b << ","
        << ga.scratch_stride << "]";
      // the two large operands' element offsets, slice strides and slice-bit placement
      for (int side = 0; side < 2; ++side) {
        const int gi2 = side ? ga.gB : ga.gA;
        if (gi2 < 0) continue;
        const GOp& op = ga.op[gi2];
        o << (side ? ",\"B\":[" : ",\"A\":[") << op.base << "," << op.slice_stride << ","
          << op.smask << "," << op.sshift << "]";
      }
      o << "}";
    }
    if (d.kind == 5) {
      // the segment's dependency levels (warp steps, block steps) and per step its
      // operand count, union indices and summed indices
      const KStep* ks = reinterpret_cast<const KStep*>(tmp.segtab.data() + d.seg_off);
      const SegLevel* lv =
          reinterpret_cast<const SegLevel*>(reinterpret_cast<const SegStage*>(ks + d.seg_count) +
                                            d.stage_count);
      o << ",\"segment\":{\"arena\":" << d.seg_arena << ",\"stages\":" << d.stage_count
        << ",\"cluster_max\":" << d.seg_cl_max << ",\"levels\":[";
      for (int q = 0; q < d.level_count; ++q)
        o << (q ? "," : "") << "[" << lv[q].nwarp << "," << lv[q].nblock << "," << lv[q].items
          << "]";
      o << "],\"steps\":[";
      for (int q = 0; q < d.seg_count; ++q)
        o << (q ? "," : "") << "[" << ks[q].m << "," << ks[q].u << "," << ks[q].nsum << "]";
      o << "]}";
    }
    UmmaPlan up;
    if (d.kind == 3 && (d.gemm_mode == GEMM_UMMA_TF32 || d.gemm_mode == GEMM_UMMA_3XTF32) &&
        umma_plan(d.ga, d.gemm_mode == GEMM_UMMA_TF32 ? 1 : 3, up)) {
      // the tcgen05 tiling: masks over the launch's U bits, sizes, tile order
      o << ",\"umma\":{\"lside\":" << up.lside << ",\"nsum\":" << up.nsum << ",\"cb\":" << up.cb
        << ",\"gb\":" << up.gb << ",\"kc\":" << up.kc << ",\"passes\":" << up.passes << ",\"sraw\":" << up.sraw
        << ",\"splane\":" << up.splane << ",\"tmem_cols\":" << up.tmem_cols
        << ",\"smem\":" << umma_smem(up) << ",\"mlane\":" << up.mlane << ",\"mcol\":" << up.mcol
        << ",\"mgrp\":" << up.mgrp << ",\"mM\":" << d.ga.mM << ",\"mN\":" << d.ga.mN
        << ",\"mBt\":" << d.ga.mBt << ",\"mK\":" << d.ga.mK << ",\"cwb\":" << up.cwb
        << ",\"rb\":" << up.rb << ",\"chunk_out\":" << up.chunk_out << ",\"prefix\":" << up.prefix
        << ",\"lruns\":[";
      for (int q = 0; q < up.nlrun; ++q)
        o << (q ? "," : "") << "[" << up.lrun_start[q] << "," << up.lrun_len[q] << "]";
      o << "],\"cruns\":[";
      for (int q = 0; q < up.ncrun; ++q)
        o << (q ? "," : "") << "[" << up.crun_start[q] << "," << up.crun_len[q] << "]";
      o << "],\"rest\":[";
      for (int q = 0; q < up.nrest; ++q) o << (q ? "," : "") << up.rest[q];
      o << "]}";
    }
    o << "}";
  }
  o << "]}";
  out = o.str();
  return true;
}

qt_status launch_plan(qt_net* net, std::string& out, std::string& err) {
  const bool ok = net->sched.precision == QT_FP64 ? launch_plan_impl<double>(net, out, err)
                                                  : launch_plan_impl<float>(net, out, err);
  return ok ? QT_OK : QT_ERANGE;
}

qt_status read_status(const qt_net* net, const void* ws, void* stream, int* status,
                      std::string& err) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!cuda_ok(cudaMemcpyAsync(status, (const char*)ws + net->sched.off_err, sizeof(int),
                               cudaMemcpyDeviceToHost, s),
               "read status", err) ||
      !cuda_ok(cudaStreamSynchronize(s), "stream synchronize", err))
    return QT_ECUDA;
  return QT_OK;
}

// Angle sweep of the amplitude (the reuse of one plan for many angles): the gate and
// gate-meta images of n_sets angle sets (host, stride bytes apart) are copied to
// ws + staging_off.
// Each is copied in turn over the workspace's gate and meta regions and followed by a run
// of all slices (the captured graph replayed); the run's amplitudes (2 n_amps doubles) are
// copied to ws + results_off + s * 16 n_amps. Nothing waits on the host in between.
size_t stage_image_bytes(const qt_net* net) {
  const Schedule& S = net->sched;
  return (size_t)S.gate_elems * (size_t)S.elem_bytes + (size_t)S.n_shared_meta * sizeof(Meta);
}

qt_status sweep_run(qt_net* net, void* ws, void* stream, int n_sets, const void* images,
                    size_t staging_off, size_t stride, size_t results_off, std::string& err) {
  const Schedule& S = net->sched;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  const size_t gate_bytes = (size_t)S.gate_elems * (size_t)S.elem_bytes;
  const size_t meta_bytes = (size_t)S.n_shared_meta * sizeof(Meta);
  const size_t out_bytes = (size_t)16 * (size_t)S.n_amps;
  if (!cuda_ok(cudaMemcpyAsync(base + staging_off, images, stride * (size_t)n_sets,
                               cudaMemcpyHostToDevice, s),
               "upload of the angle sets", err))
    return QT_ECUDA;
  double* d_out = reinterpret_cast<double*>(base + S.off_acc + out_bytes);
  for (int k = 0; k < n_sets; ++k) {
    const char* img = base + staging_off + (size_t)k * stride;
    if (gate_bytes && !cuda_ok(cudaMemcpyAsync(base + S.off_gates, img, gate_bytes,
                                               cudaMemcpyDeviceToDevice, s),
                               "install gates", err))
      return QT_ECUDA;
    if (meta_bytes && !cuda_ok(cudaMemcpyAsync(base + S.off_meta, img + gate_bytes, meta_bytes,
                                               cudaMemcpyDeviceToDevice, s),
                               "install gate meta", err))
      return QT_ECUDA;
    qt_status r = run(net, 0, S.nslices, ws, stream, d_out, err);
    if (r != QT_OK) return r;
    if (!cuda_ok(cudaMemcpyAsync(base + results_off + (size_t)k * out_bytes, d_out, out_bytes,
                                 cudaMemcpyDeviceToDevice, s),
                 "collect amplitude", err))
      return QT_ECUDA;
  }
  return QT_OK;
}

qt_status download_result_status(const qt_net* net, const void* ws, const double* d_out,
                                 double* host, int64_t n_doubles, int* status, void* stream,
                                 std::string& err) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!cuda_ok(cudaMemcpyAsync(host, d_out, (size_t)n_doubles * sizeof(double),
                               cudaMemcpyDeviceToHost, s),
               "download result", err) ||
      !cuda_ok(cudaMemcpyAsync(status, (const char*)ws + net->sched.off_err, sizeof(int),
                               cudaMemcpyDeviceToHost, s),
               "read status", err) ||
      !cuda_ok(cudaStreamSynchronize(s), "stream synchronize", err))
    return QT_ECUDA;
  return QT_OK;
}

qt_status download_result(const double* d_out, double* host, int64_t n_doubles, void* stream,
                          std::string& err) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!cuda_ok(cudaMemcpyAsync(host, d_out, (size_t)n_doubles * sizeof(double),
                               cudaMemcpyDeviceToHost, s),
               "download result", err))
    return QT_ECUDA;
  if (!cuda_ok(cudaStreamSynchronize(s), "stream synchronize", err)) return QT_ECUDA;
  return QT_OK;
}

}  // namespace qt

namespace qt {
void* engine_detach(qt_net* net) {
  void* e = net->engine;
  net->engine = nullptr;
  return e;
}

void engine_restore(qt_net* net, void* saved) {
  delete static_cast<EngineCache*>(net->engine);
  net->engine = saved;
}
}  // namespace qt

qt_net::~qt_net() {
  delete static_cast<qt::EngineCache*>(engine);
  qt::prof_clear(this);
  for (void* e : prof_pool) cudaEventDestroy((cudaEvent_t)e);
}
