// GEMM form of a fused bucket launch (complex64 tensors).
//
// A launch whose two largest operands A, B hold every index of its union U
// (all other operands lying inside A or inside B) is a batched complex GEMM:
//   out[bt][m][n] = sum_k A'[bt][m][k] B'[bt][n][k],
// k: summed indices both A and B have; m (n): output indices only A (B) has;
// bt: output indices both have. A' is A times the operands folded into it (exact
// by distributivity: each operand of the nested sum only multiplies terms it
// is constant over), already summed over the summed indices only A has; B'
// likewise. The pack kernels write A', B' planar (re plane, im plane); the
// GEMM kernels multiply them on CUDA cores (FP32) or on the tensor cores
// (mma.sync TF32 m16n8k8, BF16 m16n8k16 with FP32 accumulation, or 3xTF32:
// a = a_hi + a_lo with a_hi = tf32(a), products a_hi b_hi + a_hi b_lo + a_lo b_hi),
// and the epilogue scatters each result to its place in the canonical layout
// of the output (index = the output's U bits, shifted down by the summed ones).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gemm.h"

namespace qt {

namespace {

__device__ __forceinline__ unsigned long long pext64g(unsigned long long x, unsigned long long m) {
  unsigned long long r = 0;
  int k = 0;
  while (m) {
    const int b = __ffsll((long long)m) - 1;
    r |= ((x >> b) & 1ull) << k;
    ++k;
    m &= m - 1;
  }
  return r;
}

__device__ __forceinline__ int scale_exp_g(unsigned int maxabs_bits) {
  if (maxabs_bits == 0u) return 0;
  const int s = (int)((maxabs_bits >> 23) & 0xffu) - 126;
  return max(-125, min(125, s));
}

__device__ __forceinline__ float pow2_neg_g(int s) { return __int_as_float((127 - s) << 23); }

__device__ __forceinline__ float absmax_g(float re, float im) { return fmaxf(fabsf(re), fabsf(im)); }

// Byte-sliced lookup tables in shared memory replace per-element bit loops:
// pdep(x, mask) for a dimension's index = sum over its bytes of T[byte][value],
// pext(U, umask) for an operand = sum over the four bytes of U of P[byte][value].
struct PdepLut {
  unsigned int t[3][256];
};

__device__ __forceinline__ void build_pdep(PdepLut& L, unsigned int mask) {
  for (int e = threadIdx.x; e < 3 * 256; e += blockDim.x) {
    const int c = e >> 8, v = e & 255;
    // the mask's set bits number c*8 .. c*8+7 take the bits of v
    unsigned int m = mask, r = 0;
    int k = 0;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      if (k >= 8 * c && k < 8 * c + 8 && ((v >> (k - 8 * c)) & 1)) r |= 1u << b;
      ++k;
    }
    L.t[c][v] = r;
  }
}

__device__ __forceinline__ unsigned int pdep_lut(const PdepLut& L, unsigned int x) {
  return L.t[0][x & 255] | L.t[1][(x >> 8) & 255] | L.t[2][(x >> 16) & 255];
}

__device__ __forceinline__ void build_pext(unsigned int (*P)[256], unsigned int umask) {
  for (int e = threadIdx.x; e < 4 * 256; e += blockDim.x) {
    const int c = e >> 8, v = e & 255;
    const unsigned int x = (unsigned int)v << (8 * c);
    unsigned int m = umask, r = 0;
    int k = 0;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      r |= ((x >> b) & 1u) << k;
      ++k;
    }
    P[c][v] = r;
  }
}

__device__ __forceinline__ unsigned int pext_lut(const unsigned int (*P)[256], unsigned int U) {
  return P[0][U & 255] + P[1][(U >> 8) & 255] + P[2][(U >> 16) & 255] + P[3][U >> 24];
}

constexpr int PACK_MAXOPS = 8;

// A' (side 0) or B' (side 1): one packed element (bt, x, k) per thread; the
// sum over the side's one-sided summed indices runs inside the thread.
__global__ void __launch_bounds__(256) k_gemm_pack(const GemmArgs a, int side, float* data,
                                                   const GMeta* meta) {
  __shared__ PdepLut Lk, Lx, Lb, Ls;
  __shared__ unsigned int P[PACK_MAXOPS][4][256];
  __shared__ int opj[PACK_MAXOPS];
  __shared__ int nops;
  const unsigned int mX = side ? a.mN : a.mM, mS = side ? a.mSB : a.mSA;
  build_pdep(Lk, a.mK);
  build_pdep(Lx, mX);
  build_pdep(Lb, a.mBt);
  build_pdep(Ls, mS);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int j = 0; j < a.m; ++j)
      if (a.op[j].side == side) opj[c++] = j;
    nops = c;
  }
  __syncthreads();
  for (int q = 0; q < nops; ++q) build_pext(P[q], a.op[opj[q]].umask);
  __syncthreads();
  const int kb = __popc(a.mK), xb = __popc(mX), bb = __popc(a.mBt), sb = __popc(mS);
  const long long per = 1ll << (bb + xb + kb);
  const long long total = a.nslices * per;
  float* plane = data + 2 * (side ? a.scratch_b : a.scratch_a);
  const long long sstride = 2 * a.scratch_stride;
  long long cur = -1;
  float sc[PACK_MAXOPS];
  long long obase[PACK_MAXOPS];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / per;
    const long long loc = e - i * per;
    if (i != cur) {  // per-slice operand bases and scales
      cur = i;
      const unsigned long long sid = (unsigned long long)(a.slice_first + i);
      for (int q = 0; q < nops; ++q) {
        const GOp& o = a.op[opj[q]];
        long long off = o.base + i * o.slice_stride;
        if (o.smask) off += (long long)(pext64g(sid, o.smask) << o.sshift);
        obase[q] = off;
        sc[q] = pow2_neg_g(scale_exp_g(meta[o.meta + (o.meta_per_slice ? i : 0)].maxabs));
      }
    }
    const unsigned int k = (unsigned int)(loc & ((1ll << kb) - 1));
    const unsigned int x = (unsigned int)((loc >> kb) & ((1ll << xb) - 1));
    const unsigned int bt = (unsigned int)(loc >> (kb + xb));
    const unsigned int U0 = pdep_lut(Lk, k) | pdep_lut(Lx, x) | pdep_lut(Lb, bt);
    float accr = 0.f, acci = 0.f;
    for (unsigned int t = 0; t < (1u << sb); ++t) {
      const unsigned int U = U0 | pdep_lut(Ls, t);
      float pr = 1.f, pi = 0.f;
      for (int q = 0; q < nops; ++q) {
        const float2 v = reinterpret_cast<const float2*>(data)[obase[q] + pext_lut(P[q], U)];
        const float vr = v.x * sc[q], vi = v.y * sc[q];
        const float nr = pr * vr - pi * vi, ni = pr * vi + pi * vr;
        pr = nr;
        pi = ni;
      }
      accr += pr;
      acci += pi;
    }
    float* pl = plane + i * sstride;
    pl[loc] = accr;
    pl[per + loc] = acci;
  }
}

__device__ __forceinline__ void write_meta_e(const GemmArgs& a, GMeta* meta, long long i) {
  int E = 0;
  for (int j = 0; j < a.m; ++j) {
    const GOp& o = a.op[j];
    const GMeta mt = meta[o.meta + (o.meta_per_slice ? i : 0)];
    E += mt.E + scale_exp_g(mt.maxabs);
  }
  meta[a.out_meta + (a.out_meta_per_slice ? i : 0)].E = E;
}

__device__ __forceinline__ void flush_max(const GemmArgs& a, GMeta* meta, long long i, float mx) {
  const unsigned int v = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
  if ((threadIdx.x & 31) == 0 && v)
    atomicMax(&meta[a.out_meta + (a.out_meta_per_slice ? i : 0)].maxabs, v);
}

__device__ __forceinline__ long long out_index_lut(const GemmArgs& a, const PdepLut& Lb,
                                                   const PdepLut& Lm, const PdepLut& Ln,
                                                   unsigned int bt, unsigned int m, unsigned int n) {
  return (long long)((pdep_lut(Lb, bt) | pdep_lut(Lm, m) | pdep_lut(Ln, n)) >> a.nsum);
}

// CUDA-core GEMM: one output element per thread, k summed in order
__global__ void __launch_bounds__(256) k_gemm_simt(const GemmArgs a, float* data, GMeta* meta) {
  __shared__ PdepLut Lb, Lm, Ln;
  build_pdep(Lb, a.mBt);
  build_pdep(Lm, a.mM);
  build_pdep(Ln, a.mN);
  __syncthreads();
  const int kb = __popc(a.mK), mb = __popc(a.mM), nb = __popc(a.mN), bb = __popc(a.mBt);
  const long long per = 1ll << (bb + mb + nb);
  const long long total = a.nslices * per;
  const int K = 1 << kb;
  const long long pa = 1ll << (bb + mb + kb), pb = 1ll << (bb + nb + kb);
  long long cur = -1;
  float mx = 0.f;
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += step) {
    const long long e = base + threadIdx.x;
    const bool active = e < total;
    const long long i = active ? e / per : cur;
    if (__any_sync(0xffffffffu, active && i != cur && cur >= 0)) {
      flush_max(a, meta, cur, mx);
      mx = 0.f;
    }
    cur = __shfl_sync(0xffffffffu, i, 0);
    if (active) {
      const long long loc = e - i * per;
      const unsigned int n = (unsigned int)(loc & ((1ll << nb) - 1));
      const unsigned int m = (unsigned int)((loc >> nb) & ((1ll << mb) - 1));
      const unsigned int bt = (unsigned int)(loc >> (nb + mb));
      const float* A = data + 2 * (a.scratch_a + i * a.scratch_stride);
      const float* B = data + 2 * (a.scratch_b + i * a.scratch_stride);
      const long long ra = ((long long)bt << (mb + kb)) | ((long long)m << kb);
      const long long rb = ((long long)bt << (nb + kb)) | ((long long)n << kb);
      float cr = 0.f, ci = 0.f;
      for (int k = 0; k < K; ++k) {
        const float ar = A[ra + k], ai = A[pa + ra + k], br = B[rb + k], bi = B[pb + rb + k];
        cr += ar * br - ai * bi;
        ci += ar * bi + ai * br;
      }
      const long long o = a.out_base + i * a.out_slice_stride + out_index_lut(a, Lb, Lm, Ln, bt, m, n);
      reinterpret_cast<float2*>(data)[o] = make_float2(cr, ci);
      mx = fmaxf(mx, fmaxf(fabsf(cr), fabsf(ci)));
      if (loc == 0) write_meta_e(a, meta, i);
    }
  }
  if (cur >= 0) flush_max(a, meta, cur, mx);
}

__device__ __forceinline__ unsigned int to_tf32(float x) {
  unsigned int r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned int (&a)[4],
                                         const unsigned int (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned int pack_bf16(float lo, float hi) {
  unsigned int r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned int (&a)[4],
                                         const unsigned int (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned int pext32g(unsigned int x, unsigned int m) {
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

__device__ __forceinline__ long long op_slice_base(const GOp& o, long long i,
                                                   unsigned long long sid) {
  long long off = o.base + i * o.slice_stride;
  if (o.smask) off += (long long)(pext64g(sid, o.smask) << o.sshift);
  return off;
}

// GEMM_TILE, fold: X' = X times the other operands of its side, all scaled by
// their 2^-s, in X's own canonical layout (no one-sided summed index, so nothing
// is summed here). An operand's index at X index x is pext(x, its xmask).
__global__ void __launch_bounds__(256) k_gemm_fold(const GemmArgs a, int side, float* data,
                                                   const GMeta* meta) {
  const GOp& X = a.op[side ? a.gB : a.gA];
  const int xb = __popc(X.umask);
  const unsigned int xall = (unsigned int)((1ull << xb) - 1ull);
  const long long total = a.nslices << xb;
  float2* out = reinterpret_cast<float2*>(data) + (side ? a.scratch_b : a.scratch_a);
  const float2* d2 = reinterpret_cast<const float2*>(data);
  long long cur = -1;
  long long base[GEMM_MAXOP];
  float sc[GEMM_MAXOP];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e >> xb;
    const unsigned int x = (unsigned int)(e & xall);
    if (i != cur) {
      cur = i;
      const unsigned long long sid = (unsigned long long)(a.slice_first + i);
#pragma unroll
      for (int j = 0; j < GEMM_MAXOP; ++j)
        if (j < a.m && a.op[j].side == side) {
          base[j] = op_slice_base(a.op[j], i, sid);
          sc[j] = pow2_neg_g(scale_exp_g(meta[a.op[j].meta + (a.op[j].meta_per_slice ? i : 0)].maxabs));
        }
    }
    float pr = 1.f, pi = 0.f;
#pragma unroll
    for (int j = 0; j < GEMM_MAXOP; ++j)
      if (j < a.m && a.op[j].side == side) {
        const unsigned int xm = a.op[j].xmask;
        const unsigned int idx = xm == xall ? x : pext32g(x, xm);
        const float2 v = d2[base[j] + idx];
        const float vr = v.x * sc[j], vi = v.y * sc[j];
        const float nr = pr * vr - pi * vi, ni = pr * vi + pi * vr;
        pr = nr;
        pi = ni;
      }
    out[i * a.scratch_stride + x] = make_float2(pr, pi);
  }
}

__device__ __forceinline__ unsigned int pdep32g(unsigned int x, unsigned int m) {
  unsigned int r = 0;
  int k = 0;
  while (m) {
    const int b = __ffs(m) - 1;
    r |= ((x >> k) & 1u) << b;
    ++k;
    m &= m - 1;
  }
  return r;
}

// Bit extract / deposit over a 32-bit mask computed by a whole warp, one lane per
// mask bit (every lane must call; all lanes get the result).
__device__ __forceinline__ unsigned int warp_pext(unsigned long long x, unsigned int m) {
  const int lane = threadIdx.x & 31;
  const unsigned int below = m & ((1u << lane) - 1u);
  const unsigned int bit = ((m >> lane) & 1u) ? (unsigned int)((x >> lane) & 1ull) : 0u;
  return __reduce_or_sync(0xffffffffu, bit << __popc(below));
}
__device__ __forceinline__ unsigned int warp_pdep(unsigned int x, unsigned int m) {
  const int lane = threadIdx.x & 31;
  const unsigned int below = m & ((1u << lane) - 1u);
  const unsigned int bit = ((m >> lane) & 1u) ? ((x >> __popc(below)) & 1u) : 0u;
  return __reduce_or_sync(0xffffffffu, bit << lane);
}

// Shared-memory mbarriers for asynchronous (TMA) copies, and a bounded wait on a
// barrier's phase: after kMbarSpins failed
// tries the wait gives up, raises *err and returns false (the caller's results are
// then invalid and the host reports a timeout) instead of spinning forever.
constexpr unsigned int kMbarSpins = 1u << 24;

__device__ __forceinline__ unsigned int smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned int parity) {
  unsigned int done = 0;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned int parity, int* err) {
  for (unsigned int it = 0; it < kMbarSpins; ++it) {
    unsigned int done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  if (err) atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// GEMM_TILE, the product: a tile is the 2^tb lowest output indices for fixed
// higher ones, i.e. the lowest nsum + tb bits of U. In the canonical layout those
// bits are the lowest bits of every operand, so the tile reads one contiguous
// block of A' (rows = A's output indices in the tile, columns = the K summed
// indices, all of which A and B share) and one of B', and writes its 2^tb outputs
// as one contiguous run. The operands' power-of-two scales multiply the finished
// sums.
//
// Tiles are numbered with the high output indices of one side (tile_inner, the
// indices only the smaller operand has) varying fastest, and each block takes one
// contiguous range of tile numbers. Consecutive tiles of a block then share the
// other side's block, which stays in shared memory: a side's block is copied
// only when its place changes. Each side has two buffers; the copies of the next
// tile (16-byte cp.async) overlap the products of this one, and one barrier per
// tile separates them. Warp 0 locates the tile after next meanwhile.
//
// Register blocking: with an A-only output bit rA and a B-only bit rB inside the
// tile, a thread computes the four outputs that differ in those two bits. They
// share two A rows and two B rows, so one k step is 4 shared-memory loads for
// 8 complex multiply-adds. The tile is the same for every tile number, so each
// thread's rows and outputs are computed once, before the loop.
constexpr int kTileQuads = 2;  // quads per thread: tiles of up to 2^11 outputs

__global__ void __launch_bounds__(256, 4) k_gemm_tile(const GemmArgs a, int u, float* data,
                                                   GMeta* meta) {
  extern __shared__ float4 gsm[];
  __shared__ long long s_loc[3][4];  // tile slots: slice, tau, A block, B block
  const int nsum = a.nsum, t = a.tb, c = u - nsum, h = c - t;
  const int K = 1 << nsum, RS = K + 2;  // row stride (complex): rows stay 16-byte aligned
  const int KC = K >> 1, lkc = nsum - 1;  // 16-byte chunks per row
  const GOp& OA = a.op[a.gA];
  const GOp& OB = a.op[a.gB];
  const unsigned int L = (nsum + t >= 32) ? 0xffffffffu : ((1u << (nsum + t)) - 1u);
  const int la = __popc(OA.umask & L), lb = __popc(OB.umask & L);
  const int rows_a = 1 << (la - nsum), rows_b = 1 << (lb - nsum);
  float2* sbase = reinterpret_cast<float2*>(gsm);  // A buffers 0, 1, then B buffers 0, 1
  const unsigned int ma = (OA.umask & L) >> nsum, mb = (OB.umask & L) >> nsum;
  const int T = 1 << t;
  const long long per = 1ll << h;
  const long long ntiles = a.nslices * per;
  const long long chunk = (ntiles + gridDim.x - 1) / gridDim.x;
  const long long w0 = (long long)blockIdx.x * chunk;
  const long long w1 = min(ntiles, w0 + chunk);
  const unsigned int inner = a.tile_inner, hmask = h >= 32 ? 0xffffffffu : ((1u << h) - 1u);
  const int pin = __popc(inner);
  const float2* d2 = reinterpret_cast<const float2*>(data);
  // tile w -> slot; called by all lanes of warp 0 (lane-parallel bit extracts)
  auto locate = [&](long long w, int slot) {
    const long long i = w >> h;
    const unsigned int tp = (unsigned int)(w & (per - 1));
    const unsigned int tau = inner ? (warp_pdep(tp & ((1u << pin) - 1u), inner) |
                                      warp_pdep(tp >> pin, ~inner & hmask))
                                   : tp;
    const unsigned long long sid = (unsigned long long)(a.slice_first + i);
    const unsigned int hiA = (OA.umask & ~L) >> (nsum + t), hiB = (OB.umask & ~L) >> (nsum + t);
    const long long pa = (long long)warp_pext(tau, hiA), pb = (long long)warp_pext(tau, hiB);
    if ((threadIdx.x & 31) == 0) {
      const long long ba = a.fold_a ? a.scratch_a + i * a.scratch_stride : op_slice_base(OA, i, sid);
      const long long bb = a.fold_b ? a.scratch_b + i * a.scratch_stride : op_slice_base(OB, i, sid);
      s_loc[slot][0] = i;
      s_loc[slot][1] = tau;
      s_loc[slot][2] = ba + (pa << la);
      s_loc[slot][3] = bb + (pb << lb);
    }
  };
  // one side's block (rows x K complex, contiguous) into buffer b of that side
  auto copy_rows = [&](long long src, float2* dst, int rows) {
    for (int e = threadIdx.x; e < rows * KC; e += blockDim.x)
      cp_async16(dst + (e >> lkc) * RS + 2 * (e & (KC - 1)), d2 + src + 2 * e);
  };
  float2* const bufA = sbase;
  float2* const bufB = sbase + 2 * rows_a * RS;
  // this thread's work in every tile: quads (blocked) or single outputs
  const bool blocked = a.reg_a >= 0;
  const unsigned int rmask = blocked ? ((1u << a.reg_a) | (1u << a.reg_b)) : 0u;
  const int items = blocked ? (T >> 2) : T;
  int nmine = 0;
  unsigned int o_of[kTileQuads];
  int ra0[kTileQuads], ra1[kTileQuads], rb0[kTileQuads], rb1[kTileQuads];
#pragma unroll
  for (int r = 0; r < kTileQuads; ++r) {
    const int q = threadIdx.x + r * blockDim.x;
    o_of[r] = 0u;
    ra0[r] = ra1[r] = rb0[r] = rb1[r] = 0;
    if (blocked && q < items) {
      const unsigned int o00 = pdep32g((unsigned)q, (unsigned)(T - 1) & ~rmask);
      o_of[r] = o00;
      ra0[r] = (int)pext32g(o00, ma) * RS;
      ra1[r] = (int)pext32g(o00 | (1u << a.reg_a), ma) * RS;
      rb0[r] = (int)pext32g(o00, mb) * RS;
      rb1[r] = (int)pext32g(o00 | (1u << a.reg_b), mb) * RS;
      nmine = r + 1;
    }
  }
  if (threadIdx.x < 32) {
    if (w0 < w1) locate(w0, 0);
    if (w0 + 1 < w1) locate(w0 + 1, 1);
  }
  __syncthreads();
  int ba = 0, bb = 0;  // buffers holding this tile's A and B blocks
  if (w0 < w1) {
    copy_rows(s_loc[0][2], bufA, rows_a);
    copy_rows(s_loc[0][3], bufB, rows_b);
    cp_async_commit();
  }
  long long cur = -1;
  float sc = 1.f, mx = 0.f;
  for (int j = 0, slot = 0; w0 + j < w1; ++j, slot = slot == 2 ? 0 : slot + 1) {
    const long long w = w0 + j;
    cp_async_wait<0>();
    __syncthreads();  // this tile's blocks are in; every thread is done with the last tile
    const int ns = slot == 2 ? 0 : slot + 1;  // the slots of tiles j + 1 and j + 2
    if (threadIdx.x < 32 && w + 2 < w1) locate(w + 2, ns == 2 ? 0 : ns + 1);
    int nba = ba, nbb = bb;
    if (w + 1 < w1) {
      if (s_loc[ns][2] != s_loc[slot][2]) {
        nba = ba ^ 1;
        copy_rows(s_loc[ns][2], bufA + nba * rows_a * RS, rows_a);
      }
      if (s_loc[ns][3] != s_loc[slot][3]) {
        nbb = bb ^ 1;
        copy_rows(s_loc[ns][3], bufB + nbb * rows_b * RS, rows_b);
      }
      cp_async_commit();
    }
    const long long i_c = s_loc[slot][0], tau_c = s_loc[slot][1];
    if (i_c != cur) {
      if (cur >= 0) flush_max(a, meta, cur, mx);
      mx = 0.f;
      cur = i_c;
      const float sa = a.fold_a ? 1.f
          : pow2_neg_g(scale_exp_g(meta[OA.meta + (OA.meta_per_slice ? i_c : 0)].maxabs));
      const float sb = a.fold_b ? 1.f
          : pow2_neg_g(scale_exp_g(meta[OB.meta + (OB.meta_per_slice ? i_c : 0)].maxabs));
      sc = sa * sb;
      if (tau_c == 0 && threadIdx.x == 0) write_meta_e(a, meta, i_c);
    }
    const float2* sA = bufA + ba * rows_a * RS;
    const float2* sB = bufB + bb * rows_b * RS;
    float2* out = reinterpret_cast<float2*>(data) + a.out_base + i_c * a.out_slice_stride +
                  (tau_c << t);
    if (blocked) {
#pragma unroll
      for (int r = 0; r < kTileQuads; ++r) {
        if (r >= nmine) break;
        const float4* pa0 = reinterpret_cast<const float4*>(sA + ra0[r]);
        const float4* pa1 = reinterpret_cast<const float4*>(sA + ra1[r]);
        const float4* pb0 = reinterpret_cast<const float4*>(sB + rb0[r]);
        const float4* pb1 = reinterpret_cast<const float4*>(sB + rb1[r]);
        float c00r = 0.f, c00i = 0.f, c01r = 0.f, c01i = 0.f, c10r = 0.f, c10i = 0.f,
              c11r = 0.f, c11i = 0.f;
#pragma unroll 2
        for (int k2 = 0; k2 < KC; ++k2) {
          const float4 x0 = pa0[k2], x1 = pa1[k2], y0 = pb0[k2], y1 = pb1[k2];
#define QT_CMAC2(CR, CI, P, Q)                                                          \
  CR = fmaf(P.x, Q.x, CR); CR = fmaf(-P.y, Q.y, CR); CI = fmaf(P.x, Q.y, CI);          \
  CI = fmaf(P.y, Q.x, CI); CR = fmaf(P.z, Q.z, CR); CR = fmaf(-P.w, Q.w, CR);          \
  CI = fmaf(P.z, Q.w, CI); CI = fmaf(P.w, Q.z, CI);
          QT_CMAC2(c00r, c00i, x0, y0)
          QT_CMAC2(c01r, c01i, x0, y1)
          QT_CMAC2(c10r, c10i, x1, y0)
          QT_CMAC2(c11r, c11i, x1, y1)
#undef QT_CMAC2
        }
        const unsigned int o00 = o_of[r];
        out[o00] = make_float2(c00r * sc, c00i * sc);
        out[o00 | (1u << a.reg_b)] = make_float2(c01r * sc, c01i * sc);
        out[o00 | (1u << a.reg_a)] = make_float2(c10r * sc, c10i * sc);
        out[o00 | rmask] = make_float2(c11r * sc, c11i * sc);
        mx = fmaxf(mx, fmaxf(fmaxf(absmax_g(c00r, c00i), absmax_g(c01r, c01i)),
                             fmaxf(absmax_g(c10r, c10i), absmax_g(c11r, c11i))) * sc);
      }
    } else {
      for (int o = threadIdx.x; o < T; o += blockDim.x) {
        const float4* pa = reinterpret_cast<const float4*>(sA + pext32g((unsigned)o, ma) * RS);
        const float4* pb = reinterpret_cast<const float4*>(sB + pext32g((unsigned)o, mb) * RS);
        float cr = 0.f, ci = 0.f;
#pragma unroll 4
        for (int k2 = 0; k2 < KC; ++k2) {
          const float4 x = pa[k2], y = pb[k2];
          cr = fmaf(x.x, y.x, cr);
          cr = fmaf(-x.y, y.y, cr);
          ci = fmaf(x.x, y.y, ci);
          ci = fmaf(x.y, y.x, ci);
          cr = fmaf(x.z, y.z, cr);
          cr = fmaf(-x.w, y.w, cr);
          ci = fmaf(x.z, y.w, ci);
          ci = fmaf(x.w, y.z, ci);
        }
        cr *= sc;
        ci *= sc;
        out[o] = make_float2(cr, ci);
        mx = fmaxf(mx, absmax_g(cr, ci));
      }
    }
    ba = nba;
    bb = nbb;
  }
  if (cur >= 0) flush_max(a, meta, cur, mx);
}

// GEMM form, streaming: for launches whose small side S (at most 12 indices) fits
// in shared memory whole and whose large side G has no operand folded into it.
// One thread per row of G (its K summed values, contiguous), loaded once with
// 16-byte streaming loads and multiplied with every row of S' that shares its
// batch indices (S' = S times its folded operands, staged per slice); the outputs
// of consecutive rows of G are consecutive when G holds the lowest output indices.
// The bit deposit of a row's output position and the extract of its S row use
// byte tables in shared memory.
// rows per thread and pass of the streaming kernel: up to 4 row loads in flight
__host__ __device__ constexpr int stream_rows(int nsum) { return nsum <= 1 ? 4 : (nsum == 2 ? 2 : 1); }

template <int NSUM>
__global__ void __launch_bounds__(256, NSUM <= 3 ? 4 : 2) k_gemm_stream(const GemmArgs a, float* data, GMeta* meta) {
  constexpr int K = 1 << NSUM, kStreamRows = stream_rows(NSUM);
  extern __shared__ float4 stm[];
  __shared__ PdepLut Lg;               // pdep over G's output indices
  __shared__ unsigned int Ps[4][256];  // pext over S's output indices
  const int gside = a.stay;            // 0: A is the large side G
  const GOp& OG = a.op[gside ? a.gB : a.gA];
  const GOp& OS = a.op[gside ? a.gA : a.gB];
  const int fold_s = gside ? a.fold_a : a.fold_b;
  const long long scr_s = gside ? a.scratch_a : a.scratch_b;
  const unsigned int Gm = OG.umask >> NSUM, Sm = OS.umask >> NSUM, Nm = Sm & ~Gm;
  const int rbits = __popc(Gm), nS = __popc(OS.umask), nN = __popc(Nm);
  float2* sS = reinterpret_cast<float2*>(stm);                             // 2^nS complex
  unsigned int* nTab = reinterpret_cast<unsigned int*>(sS + (1 << nS));  // S row part of nb
  unsigned int* oTab = nTab + (1 << nN);                                   // output part of nb
  build_pdep(Lg, Gm);
  build_pext(Ps, Sm);
  for (int e = threadIdx.x; e < (1 << nN); e += blockDim.x) {
    const unsigned int on = pdep32g((unsigned)e, Nm);
    oTab[e] = on;
    nTab[e] = pext32g(on, Sm);
  }
  const long long rows = 1ll << rbits;  // rows of G per slice (a multiple of the block)
  const long long total = a.nslices << rbits;
  const float2* d2 = reinterpret_cast<const float2*>(data);
  long long cur = -1;
  float sc = 1.f, mx = 0.f;
  // kStreamRows rows per thread per pass (consecutive runs of the block's rows), the
  // next pass's rows loaded before this pass's products (two register sets). Output
  // position and S row split into this thread's low 8 row bits (once) and the
  // block-uniform high bits (pdep and pext add over disjoint bit sets).
  const long long span = (long long)blockDim.x * kStreamRows;
  const long long step = (long long)gridDim.x * span;
  __syncthreads();  // the byte tables and nTab / oTab are complete
  const unsigned int oLo = pdep_lut(Lg, threadIdx.x & 255u);
  const unsigned int sLo = pext_lut(Ps, oLo);
  // a row's index is (pass base) + r * 256 + (thread): three disjoint bit ranges, so its
  // output position and S row are sums of three parts; the r parts are constants
  unsigned int oR[kStreamRows], sR[kStreamRows];
#pragma unroll
  for (int r = 0; r < kStreamRows; ++r) {
    oR[r] = pdep_lut(Lg, (unsigned int)(r * 256));
    sR[r] = pext_lut(Ps, oR[r]);
  }
  float4 gv[kStreamRows][K / 2], gn[kStreamRows][K / 2];
  auto load_pass = [&](long long b, float4 (&dst)[kStreamRows][K / 2]) {
    const long long ib = b >> rbits;
    const float2* gb = d2 + op_slice_base(OG, ib, (unsigned long long)(a.slice_first + ib));
#pragma unroll
    for (int r = 0; r < kStreamRows; ++r) {
      const unsigned int rG = (unsigned int)((b + threadIdx.x + r * blockDim.x) & (rows - 1));
      const float4* gp = reinterpret_cast<const float4*>(gb + (long long)rG * K);
#pragma unroll
      for (int q = 0; q < K / 2; ++q) dst[r][q] = __ldcs(gp + q);
    }
  };
  long long base = (long long)blockIdx.x * span;
  if (base < total) load_pass(base, gn);
  for (; base < total; base += step) {
#pragma unroll
    for (int r = 0; r < kStreamRows; ++r)
#pragma unroll
      for (int q = 0; q < K / 2; ++q) gv[r][q] = gn[r][q];
    if (base + step < total) load_pass(base + step, gn);
    const long long i = base >> rbits;  // the same for the whole block (rows is a multiple of span)
    if (i != cur) {
      if (cur >= 0) flush_max(a, meta, cur, mx);
      mx = 0.f;
      __syncthreads();  // the tables are built; the last slice's S' is no longer read
      const unsigned long long sid = (unsigned long long)(a.slice_first + i);
      if (fold_s && a.fold_in) {
        // S' = the product of the S side's operands, each times its scale, in operand
        // order (the arithmetic of k_gemm_fold, so the same values); a small S only
        // (its rebuild, once per slice, stalls the block)
        const int sside = gside ? 0 : 1;
        const unsigned int xall = (unsigned int)((1ull << nS) - 1ull);
        for (int e = threadIdx.x; e < (1 << nS); e += blockDim.x) {
          float pr = 1.f, pi = 0.f;
#pragma unroll 1
          for (int j = 0; j < a.m; ++j) {
            const GOp& o = a.op[j];
            if (o.side != sside) continue;
            const float fs =
                pow2_neg_g(scale_exp_g(meta[o.meta + (o.meta_per_slice ? i : 0)].maxabs));
            const unsigned int idx = o.xmask == xall ? (unsigned int)e : pext32g((unsigned int)e, o.xmask);
            const float2 v = d2[op_slice_base(o, i, sid) + idx];
            const float vr = v.x * fs, vi = v.y * fs;
            const float nr = pr * vr - pi * vi, ni = pr * vi + pi * vr;
            pr = nr;
            pi = ni;
          }
          sS[e] = make_float2(pr, pi);
        }
      } else {
        // S' from the fold kernel's scratch, or S itself times its scale
        const long long sb = fold_s ? scr_s + i * a.scratch_stride : op_slice_base(OS, i, sid);
        const float ss = fold_s ? 1.f
            : pow2_neg_g(scale_exp_g(meta[OS.meta + (OS.meta_per_slice ? i : 0)].maxabs));
        for (int e = threadIdx.x; e < (1 << nS); e += blockDim.x) {
          const float2 v = d2[sb + e];
          sS[e] = make_float2(v.x * ss, v.y * ss);
        }
      }
      sc = pow2_neg_g(scale_exp_g(meta[OG.meta + (OG.meta_per_slice ? i : 0)].maxabs));
      if ((base & (rows - 1)) == 0 && threadIdx.x == 0) write_meta_e(a, meta, i);
      cur = i;
      __syncthreads();
    }
    float2* out = reinterpret_cast<float2*>(data) + a.out_base + i * a.out_slice_stride;
    const unsigned int oB = pdep_lut(Lg, (unsigned int)(base & (rows - 1)));  // pass base
    const unsigned int sB = pext_lut(Ps, oB);
#pragma unroll
    for (int r = 0; r < kStreamRows; ++r) {
      const unsigned int oG = oLo | oR[r] | oB;
      const unsigned int sG = sLo + sR[r] + sB;
      for (int nb = 0; nb < (1 << nN); ++nb) {
        const float4* sp = reinterpret_cast<const float4*>(sS + (size_t)(sG + nTab[nb]) * K);
        float cr = 0.f, ci = 0.f;
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
          const float4 x = gv[r][q], y = sp[q];
          cr = fmaf(x.x, y.x, cr);
          cr = fmaf(-x.y, y.y, cr);
          ci = fmaf(x.x, y.y, ci);
          ci = fmaf(x.y, y.x, ci);
          cr = fmaf(x.z, y.z, cr);
          cr = fmaf(-x.w, y.w, cr);
          ci = fmaf(x.z, y.w, ci);
          ci = fmaf(x.w, y.z, ci);
        }
        cr *= sc;
        ci *= sc;
        __stcs(out + (oG | oTab[nb]), make_float2(cr, ci));
        mx = fmaxf(mx, absmax_g(cr, ci));
      }
    }
  }
  if (cur >= 0) flush_max(a, meta, cur, mx);
}

// GEMM_TILE with tensor-copy (TMA) staging and a producer warp: the same tiles,
// tile numbering, block ranges, register blocking and arithmetic (so the same
// results, bit for bit) as k_gemm_tile, with the summed-index count a
// compile-time constant. The workspace is seen by two 2-D tensor maps, rows of K
// complex (2K floats); a block of R rows is one or more box copies
// (cp.async.bulk.tensor.2d) completing on the buffer's "full" mbarrier. Each
// map's box is 2K + 4 floats wide: the 4 floats past the row lie outside the
// tensor and arrive as zeros, which pads every row in shared memory to K + 2
// complex (no bank conflicts) without any thread touching the data.
//
// Warp specialisation: warp 8 locates tiles (32 at a time, one per lane) and issues
// the copies, running ahead of the 8 consumer warps, which wait on a buffer's "full" barrier, compute, and
// arrive on its "empty" barrier; nothing else synchronises the block. The side
// whose block is shared by a group of tiles (the tiles differing only in the
// tile_inner indices) has two buffers and its next group's block is requested at
// the first tile of this group and issued as soon as its buffer is free; the other side has a ring of nmove buffers, one
// per tile. Every wait is bounded: on a timeout the block raises the status word
// and stops, waiting (bounded) for its copies still in flight; the host reports
// QT_ETIMEOUT.
__device__ __forceinline__ void tma_load_2d(void* smem, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(smem)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

constexpr int kTmaBoxRows = 256;  // rows per box copy (the hardware's limit)
constexpr int kTmaConsumers = 256;
constexpr int kTmaThreads = kTmaConsumers + 32;
constexpr int kMoveStagesMax = 4;

struct TmaSlot {
  long long i, out;  // slice, output offset (complex) of the tile
  float sc;          // the product of the operands' scales in that slice
  int first;         // the slice's first tile (tau = 0)
};

template <int NSUM, int WIDE>
__global__ void __launch_bounds__(kTmaThreads, 3) k_gemm_tma(
    const GemmArgs a, const __grid_constant__ CUtensorMap mapA,
    const __grid_constant__ CUtensorMap mapB, int u, int nmove, float* data, GMeta* meta) {
  constexpr int K = 1 << NSUM, RS = K + 2, KC = K / 2;
  extern __shared__ float4 gsm[];
  __shared__ TmaSlot s_slot[kMoveStagesMax];  // per ring buffer: its tile's slice, output, scale
  // barriers: 0, 1 the shared side's buffers, 2 + s the ring's
  __shared__ alignas(8) unsigned long long s_full[2 + kMoveStagesMax];
  __shared__ alignas(8) unsigned long long s_empty[2 + kMoveStagesMax];
  __shared__ volatile int s_fail;
  const int t = a.tb, c = u - NSUM, h = c - t;
  const GOp& OA = a.op[a.gA];
  const GOp& OB = a.op[a.gB];
  const unsigned int L = (NSUM + t >= 32) ? 0xffffffffu : ((1u << (NSUM + t)) - 1u);
  const int la = __popc(OA.umask & L), lb = __popc(OB.umask & L);
  const int rows_a = 1 << (la - NSUM), rows_b = 1 << (lb - NSUM);
  const int stay = a.stay, move = stay ^ 1;  // stay: 0 the groups share A's block, 1 B's
  const int rows_s = stay ? rows_b : rows_a, rows_m = stay ? rows_a : rows_b;
  // buffers of 1024-byte multiples from a 1024-byte aligned base
  const int szS = (rows_s * RS + 127) & ~127, szM = (rows_m * RS + 127) & ~127;  // float2
  // (offset from gsm itself, so the compiler keeps these shared-memory pointers)
  float2* const bufS = reinterpret_cast<float2*>(reinterpret_cast<char*>(gsm) +
                                                 ((1024u - (smem_u32(gsm) & 1023u)) & 1023u));
  float2* const bufM = bufS + 2 * szS;
  const long long ntiles = a.nslices << h;
  const long long chunk = (ntiles + gridDim.x - 1) / gridDim.x;
  const long long w0 = (long long)blockIdx.x * chunk;
  const long long w1 = min(ntiles, w0 + chunk);
  const int pin = __popc(a.tile_inner);
  const long long gmask = ((long long)1 << pin) - 1;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2 + nmove; ++b) {
      mbar_init(&s_full[b], 1);
      mbar_init(&s_empty[b], kTmaConsumers / 32);
    }
    mbar_fence_init();
    s_fail = 0;
  }
  __syncthreads();
  unsigned int issued = 0u;  // producer lane 0, barrier b: bit b some fill, bit 8 + b parity
  if (threadIdx.x >= kTmaConsumers) {
    // ---- producer warp ----
    // Windows of 32 tiles: lane l locates tile wb + l (scalar bit extracts, all lanes at
    // once), then lane 0 walks the window, reading each tile's numbers from its lane,
    // waiting for the buffers and issuing the copies.
    const int lane = threadIdx.x & 31;
    const unsigned int inner = a.tile_inner, hmask = h >= 32 ? 0xffffffffu : ((1u << h) - 1u);
    const unsigned int outer = ~inner & hmask, pmask = (1u << pin) - 1u;
    const unsigned int hiA = (OA.umask & ~L) >> (NSUM + t), hiB = (OB.umask & ~L) >> (NSUM + t);
    const CUtensorMap* mapS = stay ? &mapB : &mapA;
    const CUtensorMap* mapM = stay ? &mapA : &mapB;
    // tile w: slice, tau and the block offsets (complex) of the shared and other sides
    auto where = [&](long long w, long long& i, unsigned int& tau, long long& offS, long long& offM) {
      i = w >> h;
      const unsigned int tp = (unsigned int)(w & (((long long)1 << h) - 1));
      tau = inner ? (pdep32g(tp & pmask, inner) | pdep32g(tp >> pin, outer)) : tp;
      const unsigned long long sid = (unsigned long long)(a.slice_first + i);
      const long long oA = (a.fold_a ? a.scratch_a + i * a.scratch_stride : op_slice_base(OA, i, sid)) +
                           ((long long)pext32g(tau, hiA) << la);
      const long long oB = (a.fold_b ? a.scratch_b + i * a.scratch_stride : op_slice_base(OB, i, sid)) +
                           ((long long)pext32g(tau, hiB) << lb);
      offS = stay ? oB : oA;
      offM = stay ? oA : oB;
    };
    auto load = [&](const CUtensorMap* map, long long off, float2* dst, int rows, int b) {
      unsigned long long* bar = &s_full[b];
      const int box = min(rows, kTmaBoxRows);
      const int row0 = (int)(off >> NSUM);
      mbar_expect_tx(bar, (unsigned)(rows * RS * 8));
      for (int r = 0; r < rows; r += box) tma_load_2d(dst + r * RS, map, 0, row0 + r, bar);
      issued = (issued | (1u << b)) ^ (256u << b);
    };
    int ms = 0, f = 0;  // ring buffer of the tile and the fill count it reaches
    int pend_b = -1;    // lane 0: a shared-side buffer whose block waits for it to be free
    unsigned int pend_par = 0u;
    long long pend_off = 0;
    long long pi = -1;  // lane 0: the slice whose scale is in sc
    float sc = 1.f;
    bool ok = true;
    for (long long wb = w0; wb < w1 && ok; wb += 32) {
      const long long wl = wb + lane;
      long long li = 0, loffS = 0, loffM = 0, lnext = 0;
      unsigned int ltau = 0;
      if (wl < w1) {
        where(wl, li, ltau, loffS, loffM);
        // the next group's shared block, requested when tile wl starts a group
        const long long g1 = ((wl >> pin) + 1) << pin;
        if (g1 < w1 && (wl == w0 || (wl & gmask) == 0)) {
          long long i1, m1;
          unsigned int t1;
          where(g1, i1, t1, lnext, m1);
        }
      }
      const int nwin = (int)min(32ll, w1 - wb);
      for (int j = 0; j < nwin; ++j) {
        const long long w = wb + j;
        const long long i = __shfl_sync(0xffffffffu, li, j);
        const unsigned int tau = __shfl_sync(0xffffffffu, ltau, j);
        const long long offS = __shfl_sync(0xffffffffu, loffS, j);
        const long long offM = __shfl_sync(0xffffffffu, loffM, j);
        const long long onext = __shfl_sync(0xffffffffu, lnext, j);
        if (lane == 0) {
          if (s_fail) ok = false;
          if (ok && i != pi) {
            pi = i;
            sc = (a.fold_a ? 1.f
                           : pow2_neg_g(scale_exp_g(meta[OA.meta + (OA.meta_per_slice ? i : 0)].maxabs))) *
                 (a.fold_b ? 1.f
                           : pow2_neg_g(scale_exp_g(meta[OB.meta + (OB.meta_per_slice ? i : 0)].maxabs)));
          }
          // the ring buffer is free once the tile nmove earlier is done
          if (ok && f > 0) ok = mbar_wait(&s_empty[2 + ms], (unsigned)((f - 1) & 1), a.err);
          if (ok) {
            s_slot[ms].i = i;
            s_slot[ms].out = a.out_base + i * a.out_slice_stride + ((long long)tau << t);
            s_slot[ms].sc = sc;
            s_slot[ms].first = tau == 0u;
            load(mapM, offM, bufM + ms * szM, rows_m, 2 + ms);
            if (w == w0) load(mapS, offS, bufS, rows_s, 0);
          }
          // the next group's shared block: requested at this group's first tile, issued
          // as soon as its buffer is free (polled between ring tiles), at the latest
          // at the next group's first tile
          if (ok && (w == w0 || (w & gmask) == 0)) {
            if (pend_b >= 0) {
              ok = mbar_wait(&s_empty[pend_b], pend_par, a.err);
              if (ok) load(mapS, pend_off, bufS + pend_b * szS, rows_s, pend_b);
              pend_b = -1;
            }
            const long long g1 = ((w >> pin) + 1) << pin;
            if (ok && g1 < w1) {
              const int sgi = (int)((w >> pin) - (w0 >> pin));
              const int nb = (sgi + 1) & 1, fs = (sgi + 1) >> 1;
              if (fs == 0) {
                load(mapS, onext, bufS + nb * szS, rows_s, nb);
              } else {
                pend_b = nb;
                pend_par = (unsigned)((fs - 1) & 1);
                pend_off = onext;
              }
            }
          }
          if (ok && pend_b >= 0 && mbar_test(&s_empty[pend_b], pend_par)) {
            load(mapS, pend_off, bufS + pend_b * szS, rows_s, pend_b);
            pend_b = -1;
          }
          if (!ok) s_fail = 1;
        }
        if (++ms == nmove) {
          ms = 0;
          ++f;
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) break;
      }
    }
  } else {
    // ---- consumer warps ----
    // register block: NA rows of A x NB rows of B (the wide side's two bits reg_x, reg_x2)
    constexpr int NA = WIDE == 2 ? 4 : 2, NB = WIDE == 1 ? 4 : 2;
    constexpr int kItems = NA * NB == 4 ? kTileQuads : 1;  // tiles of up to 2^11 outputs
    const unsigned int ma = (OA.umask & L) >> NSUM, mb = (OB.umask & L) >> NSUM;
    const int T = 1 << t;
    const bool blocked = a.reg_a >= 0;
    const unsigned int amask = (blocked ? 1u << a.reg_a : 0u) | (WIDE == 2 ? 1u << a.reg_a2 : 0u);
    const unsigned int bmask = (blocked ? 1u << a.reg_b : 0u) | (WIDE == 1 ? 1u << a.reg_b2 : 0u);
    const unsigned int rmask = amask | bmask;
    const int items = blocked ? (T / (NA * NB)) : T;
    unsigned int aoff[NA], boff[NB];
#pragma unroll
    for (int x = 0; x < NA; ++x) aoff[x] = pdep32g((unsigned)x, amask);
#pragma unroll
    for (int y = 0; y < NB; ++y) boff[y] = pdep32g((unsigned)y, bmask);
    int nmine = 0;
    unsigned int o_of[kItems];
    int ra[kItems][NA], rb[kItems][NB];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int q = threadIdx.x + r * kTmaConsumers;
      o_of[r] = 0u;
#pragma unroll
      for (int x = 0; x < NA; ++x) ra[r][x] = 0;
#pragma unroll
      for (int y = 0; y < NB; ++y) rb[r][y] = 0;
      if (blocked && q < items) {
        const unsigned int o00 = pdep32g((unsigned)q, (unsigned)(T - 1) & ~rmask);
        o_of[r] = o00;
#pragma unroll
        for (int x = 0; x < NA; ++x) ra[r][x] = (int)pext32g(o00 | aoff[x], ma) * RS;
#pragma unroll
        for (int y = 0; y < NB; ++y) rb[r][y] = (int)pext32g(o00 | boff[y], mb) * RS;
        nmine = r + 1;
      }
    }
    long long cur = -1;
    float mx = 0.f;
    int ms = 0, sb = 0;            // ring buffer of the tile, shared-side buffer of its group
    unsigned int ph = 0u, phs = 0u;  // the fill parities they wait for
    long long gnext = ((w0 >> pin) + 1) << pin;  // first tile of the next group
    for (long long w = w0; w < w1; ++w) {
      if (w == gnext) {
        gnext += 1ll << pin;
        sb ^= 1;
        phs ^= (unsigned)(sb == 0);
      }
      const bool ok = mbar_wait(&s_full[2 + ms], ph, a.err) && mbar_wait(&s_full[sb], phs, a.err);
      if (!__all_sync(0xffffffffu, ok)) {  // the warp leaves together
        s_fail = 1;
        break;
      }
      const long long i_c = s_slot[ms].i;
      const float sc = s_slot[ms].sc;
      if (i_c != cur) {
        if (cur >= 0) flush_max(a, meta, cur, mx);
        mx = 0.f;
        cur = i_c;
        if (s_slot[ms].first && threadIdx.x == 0) write_meta_e(a, meta, i_c);
      }
      const float2* sA = stay ? bufM + ms * szM : bufS + sb * szS;
      const float2* sB = stay ? bufS + sb * szS : bufM + ms * szM;
      float2* out = reinterpret_cast<float2*>(data) + s_slot[ms].out;
      if (blocked) {
#pragma unroll
        for (int r = 0; r < kItems; ++r) {
          if (r >= nmine) break;
          float cr[NA][NB], ci[NA][NB];
#pragma unroll
          for (int x = 0; x < NA; ++x)
#pragma unroll
            for (int y = 0; y < NB; ++y) cr[x][y] = ci[x][y] = 0.f;
#pragma unroll
          for (int k2 = 0; k2 < KC; ++k2) {
            float4 xv[NA], yv[NB];
#pragma unroll
            for (int x = 0; x < NA; ++x) xv[x] = reinterpret_cast<const float4*>(sA + ra[r][x])[k2];
#pragma unroll
            for (int y = 0; y < NB; ++y) yv[y] = reinterpret_cast<const float4*>(sB + rb[r][y])[k2];
#pragma unroll
            for (int x = 0; x < NA; ++x)
#pragma unroll
              for (int y = 0; y < NB; ++y) {
                const float4 P = xv[x], Q = yv[y];
                cr[x][y] = fmaf(P.x, Q.x, cr[x][y]);
                cr[x][y] = fmaf(-P.y, Q.y, cr[x][y]);
                ci[x][y] = fmaf(P.x, Q.y, ci[x][y]);
                ci[x][y] = fmaf(P.y, Q.x, ci[x][y]);
                cr[x][y] = fmaf(P.z, Q.z, cr[x][y]);
                cr[x][y] = fmaf(-P.w, Q.w, cr[x][y]);
                ci[x][y] = fmaf(P.z, Q.w, ci[x][y]);
                ci[x][y] = fmaf(P.w, Q.z, ci[x][y]);
              }
          }
          const unsigned int o00 = o_of[r];
#pragma unroll
          for (int x = 0; x < NA; ++x)
#pragma unroll
            for (int y = 0; y < NB; ++y) {
              const float vr = cr[x][y] * sc, vi = ci[x][y] * sc;
              out[o00 | aoff[x] | boff[y]] = make_float2(vr, vi);
              mx = fmaxf(mx, absmax_g(vr, vi));
            }
        }
      } else {
        for (int o = threadIdx.x; o < T; o += kTmaConsumers) {
          const float4* pa = reinterpret_cast<const float4*>(sA + pext32g((unsigned)o, ma) * RS);
          const float4* pb = reinterpret_cast<const float4*>(sB + pext32g((unsigned)o, mb) * RS);
          float cr = 0.f, ci = 0.f;
#pragma unroll
          for (int k2 = 0; k2 < KC; ++k2) {
            const float4 x = pa[k2], y = pb[k2];
            cr = fmaf(x.x, y.x, cr);
            cr = fmaf(-x.y, y.y, cr);
            ci = fmaf(x.x, y.y, ci);
            ci = fmaf(x.y, y.x, ci);
            cr = fmaf(x.z, y.z, cr);
            cr = fmaf(-x.w, y.w, cr);
            ci = fmaf(x.z, y.w, ci);
            ci = fmaf(x.w, y.z, ci);
          }
          cr *= sc;
          ci *= sc;
          out[o] = make_float2(cr, ci);
          mx = fmaxf(mx, absmax_g(cr, ci));
        }
      }
      // release the tile's buffers: one arrival per warp once all its lanes are done
      __syncwarp();
      if ((threadIdx.x & 31) == 0) {
        mbar_arrive(&s_empty[2 + ms]);
        if (w + 1 == w1 || w + 1 == gnext) mbar_arrive(&s_empty[sb]);
      }
      if (++ms == nmove) {
        ms = 0;
        ph ^= 1u;
      }
    }
    if (cur >= 0) flush_max(a, meta, cur, mx);
  }
  __syncthreads();
  if (s_fail && threadIdx.x == kTmaConsumers) {
    // bounded waits for the copies still in flight into this block's shared memory
    for (int b = 0; b < 2 + nmove; ++b)
      if ((issued >> b) & 1u) mbar_wait(&s_full[b], ((issued >> (8 + b)) & 1u) ^ 1u, nullptr);
  }
}

// Tensor-core GEMM: one warp per (slice, bt, 16-row m tile, 8-column n tile).
// Fragment layouts of mma.m16n8k8 (tf32) / m16n8k16 (bf16), with g = lane / 4,
// t = lane % 4: A row g (+8), columns t (+4) [tf32] or 2t, 2t+1 (+8) [bf16];
// B column g, rows t (+4) [tf32] or 2t, 2t+1 (+8) [bf16]; C rows g (+8),
// columns 2t, 2t+1. The launch requires M >= 16 and N >= 8 (powers of two, so
// every tile is full); k beyond K (K < 8, or K < 16 in BF16) reads as 0.
template <int MODE>
__global__ void __launch_bounds__(128) k_gemm_tc(const GemmArgs a, float* data, GMeta* meta) {
  __shared__ PdepLut Lb, Lm, Ln;
  build_pdep(Lb, a.mBt);
  build_pdep(Lm, a.mM);
  build_pdep(Ln, a.mN);
  __syncthreads();
  const int kb = __popc(a.mK), mb = __popc(a.mM), nb = __popc(a.mN), bb = __popc(a.mBt);
  const int K = 1 << kb;
  const int mt = (1 << mb) / 16, nt = (1 << nb) / 8;
  const long long per = (long long)mt * nt << bb;
  const long long items = a.nslices * per;
  const long long pa = 1ll << (bb + mb + kb), pb = 1ll << (bb + nb + kb);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long warps = (long long)gridDim.x * (blockDim.x / 32);
  constexpr int KSTEP = MODE == GEMM_TC_BF16 ? 16 : 8;
  const bool kfull = K >= KSTEP;
  long long cur = -1;
  float mx = 0.f;
  for (long long w = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < items;
       w += warps) {
    const long long i = w / per;
    const long long r = w - i * per;
    const int ntile = (int)(r % nt);
    const int mtile = (int)((r / nt) % mt);
    const unsigned int bt = (unsigned int)(r / ((long long)nt * mt));
    if (i != cur) {
      if (cur >= 0) flush_max(a, meta, cur, mx);
      cur = i;
      mx = 0.f;
    }
    const int m0 = mtile * 16, n0 = ntile * 8;
    // row pointers of this lane's fragment rows
    const float* A0 = data + 2 * (a.scratch_a + i * a.scratch_stride) +
                      ((((long long)bt << mb) + m0 + g) << kb);
    const float* A8 = A0 + (8ll << kb);
    const float* Bn = data + 2 * (a.scratch_b + i * a.scratch_stride) +
                      ((((long long)bt << nb) + n0 + g) << kb);
    auto kv = [&](const float* P, int k) -> float { return (kfull || k < K) ? P[k] : 0.f; };
    float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
    if constexpr (MODE == GEMM_TC_BF16) {
      for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + 2 * t;
        unsigned int ar_[4], ai_[4], nai_[4], br_[2], bi_[2];
        ar_[0] = pack_bf16(kv(A0, ka), kv(A0, ka + 1));
        ar_[1] = pack_bf16(kv(A8, ka), kv(A8, ka + 1));
        ar_[2] = pack_bf16(kv(A0, ka + 8), kv(A0, ka + 9));
        ar_[3] = pack_bf16(kv(A8, ka + 8), kv(A8, ka + 9));
        ai_[0] = pack_bf16(kv(A0 + pa, ka), kv(A0 + pa, ka + 1));
        ai_[1] = pack_bf16(kv(A8 + pa, ka), kv(A8 + pa, ka + 1));
        ai_[2] = pack_bf16(kv(A0 + pa, ka + 8), kv(A0 + pa, ka + 9));
        ai_[3] = pack_bf16(kv(A8 + pa, ka + 8), kv(A8 + pa, ka + 9));
#pragma unroll
        for (int q = 0; q < 4; ++q) nai_[q] = ai_[q] ^ 0x80008000u;
        br_[0] = pack_bf16(kv(Bn, ka), kv(Bn, ka + 1));
        br_[1] = pack_bf16(kv(Bn, ka + 8), kv(Bn, ka + 9));
        bi_[0] = pack_bf16(kv(Bn + pb, ka), kv(Bn + pb, ka + 1));
        bi_[1] = pack_bf16(kv(Bn + pb, ka + 8), kv(Bn + pb, ka + 9));
        mma_bf16(cr, ar_, br_);
        mma_bf16(cr, nai_, bi_);
        mma_bf16(ci, ar_, bi_);
        mma_bf16(ci, ai_, br_);
      }
    } else {
      for (int k0 = 0; k0 < K; k0 += 8) {
        const float far[4] = {kv(A0, k0 + t), kv(A8, k0 + t), kv(A0, k0 + t + 4), kv(A8, k0 + t + 4)};
        const float fai[4] = {kv(A0 + pa, k0 + t), kv(A8 + pa, k0 + t), kv(A0 + pa, k0 + t + 4),
                              kv(A8 + pa, k0 + t + 4)};
        const float fbr[2] = {kv(Bn, k0 + t), kv(Bn, k0 + t + 4)};
        const float fbi[2] = {kv(Bn + pb, k0 + t), kv(Bn + pb, k0 + t + 4)};
        unsigned int arh[4], aih[4], naih[4], brh[2], bih[2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          arh[q] = to_tf32(far[q]);
          aih[q] = to_tf32(fai[q]);
          naih[q] = aih[q] ^ 0x80000000u;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          brh[q] = to_tf32(fbr[q]);
          bih[q] = to_tf32(fbi[q]);
        }
        mma_tf32(cr, arh, brh);
        mma_tf32(cr, naih, bih);
        mma_tf32(ci, arh, bih);
        mma_tf32(ci, aih, brh);
        if constexpr (MODE == GEMM_TC_3XTF32) {
          unsigned int arl[4], ail[4], nail[4], brl[2], bil[2];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            arl[q] = to_tf32(far[q] - __uint_as_float(arh[q]));
            ail[q] = to_tf32(fai[q] - __uint_as_float(aih[q]));
            nail[q] = ail[q] ^ 0x80000000u;
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            brl[q] = to_tf32(fbr[q] - __uint_as_float(brh[q]));
            bil[q] = to_tf32(fbi[q] - __uint_as_float(bih[q]));
          }
          mma_tf32(cr, arh, brl);
          mma_tf32(cr, naih, bil);
          mma_tf32(ci, arh, bil);
          mma_tf32(ci, aih, brl);
          mma_tf32(cr, arl, brh);
          mma_tf32(cr, nail, bih);
          mma_tf32(ci, arl, bih);
          mma_tf32(ci, ail, brh);
        }
      }
    }
    const long long obase = a.out_base + i * a.out_slice_stride;
    const unsigned int ub = pdep_lut(Lb, bt);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + g + (q >= 2 ? 8 : 0);
      const int n = n0 + 2 * t + (q & 1);
      const unsigned int U = ub | pdep_lut(Lm, (unsigned)m) | pdep_lut(Ln, (unsigned)n);
      reinterpret_cast<float2*>(data)[obase + (U >> a.nsum)] = make_float2(cr[q], ci[q]);
      mx = fmaxf(mx, fmaxf(fabsf(cr[q]), fabsf(ci[q])));
    }
    if (r == 0 && lane == 0) write_meta_e(a, meta, i);
  }
  if (cur >= 0) flush_max(a, meta, cur, mx);
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Triangle form of a fused launch: three large operands A, B, C, every summed
// index in exactly two of them (K: A and B, X: A and C, Y: B and C), so
//   out[o] = sum_k w(k) sum_x A[o; k, x] sum_y B[o; k, y] C'[o; x, y],
// C' = C times the operands inside C, w = the product of the summed-only
// operands inside K. Against the elementwise nested sum (3 loads per U element)
// this reads |X||Y| + |K|(|X| + |Y|) values per output instead of 3|K||X||Y|.
// A tile is the 2^tb lowest output indices for fixed higher ones (the lowest
// nsum + tb bits of U), so each operand's block is contiguous; the blocks are
// copied into shared memory transposed ([summed column][row], 8-byte async
// copies, two buffers), making the lanes' rows (consecutive outputs) consecutive
// words. Thread 0 locates the tile after next while the block works.
struct TriLayout {
  // per operand: la local bits, s summed bits, r rows, n elements, p column stride
  // (rows + 1, odd: consecutive columns of one row fall in different banks)
  int laA, laB, laC, sA, sB, sC, rA, rB, rC, nA, nB, nC, pA, pB, pC, zA, zB, zC, nK, nX, nY, buf;
  size_t off_cf, off_rt, off_col, off_w, bytes;
};

__host__ __device__ inline int popc_h(unsigned int x) {
#ifdef __CUDA_ARCH__
  return __popc(x);
#else
  return __builtin_popcount(x);
#endif
}

__host__ __device__ inline TriLayout tri_layout(const GemmArgs& a, int t) {
  TriLayout l{};
  const unsigned int L = (a.nsum + t >= 32) ? 0xffffffffu : ((1u << (a.nsum + t)) - 1u);
  const unsigned int Sm = (1u << a.nsum) - 1u;
  const unsigned int mA = a.op[a.tA].umask, mB = a.op[a.tB].umask, mC = a.op[a.tC].umask;
  l.laA = popc_h(mA & L); l.laB = popc_h(mB & L); l.laC = popc_h(mC & L);
  l.sA = popc_h(mA & Sm); l.sB = popc_h(mB & Sm); l.sC = popc_h(mC & Sm);
  l.rA = 1 << (l.laA - l.sA); l.rB = 1 << (l.laB - l.sB); l.rC = 1 << (l.laC - l.sC);
  l.nA = 1 << l.laA; l.nB = 1 << l.laB; l.nC = 1 << l.laC;
  l.pA = l.rA + 1; l.pB = l.rB + 1; l.pC = l.rC + 1;
  l.zA = l.pA << l.sA; l.zB = l.pB << l.sB; l.zC = l.pC << l.sC;  // padded sizes
  l.nK = 1 << popc_h(a.tK); l.nX = 1 << popc_h(a.tX); l.nY = 1 << popc_h(a.tY);
  l.buf = l.zA + l.zB + l.zC;
  size_t off = (size_t)2 * l.buf * 8;            // two buffers of complex64
  l.off_cf = 0;
  l.off_rt = off;  off += (size_t)3 * 2 * (1u << t);  // row tables (uint16)
  off = (off + 15) / 16 * 16;
  l.off_col = off; off += (size_t)4 * (2 * l.nK + l.nX + l.nY + l.nX * l.nY);
  off = (off + 15) / 16 * 16;
  l.off_w = off;   off += (size_t)8 * l.nK;
  l.bytes = off;
  return l;
}

// C' = C times the operands inside C, once per slice, in C's own layout (the
// triangle form's fold; an operand's index at C index x is pext(x, its xmask)).
__global__ void __launch_bounds__(256) k_tri_fold(const GemmArgs a, float* data, const GMeta* meta) {
  const GOp& X = a.op[a.tC];
  const int xb = __popc(X.umask);
  const unsigned int xall = (unsigned int)((1ull << xb) - 1ull);
  const long long total = a.nslices << xb;
  float2* out = reinterpret_cast<float2*>(data) + a.scratch_a;
  const float2* d2 = reinterpret_cast<const float2*>(data);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e >> xb;
    const unsigned int x = (unsigned int)(e & xall);
    const unsigned long long sid = (unsigned long long)(a.slice_first + i);
    float pr = 1.f, pi = 0.f;
    for (int j = 0; j < a.m; ++j) {
      const GOp& o = a.op[j];
      if (j != a.tC && o.tfold != 1) continue;
      const float sc = pow2_neg_g(scale_exp_g(meta[o.meta + (o.meta_per_slice ? i : 0)].maxabs));
      const unsigned int idx = j == a.tC ? x : pext32g(x, o.xmask);
      const float2 v = d2[op_slice_base(o, i, sid) + idx];
      const float vr = v.x * sc, vi = v.y * sc;
      const float nr = pr * vr - pi * vi, ni = pr * vi + pi * vr;
      pr = nr;
      pi = ni;
    }
    out[i * a.scratch_stride + x] = make_float2(pr, pi);
  }
}

template <int NX, int NY>
__global__ void __launch_bounds__(256) k_tri_tile(const GemmArgs a, int u, float* data,
                                                  GMeta* meta) {
  extern __shared__ float4 trsm[];
  __shared__ long long s_loc[3][5];   // tile slots: slice, tau, A, B, C block starts
  __shared__ float s_sc;
  const int nsum = a.nsum, t = a.tb, c = u - nsum, h = c - t;
  const TriLayout ly = tri_layout(a, t);
  const unsigned int L = (nsum + t >= 32) ? 0xffffffffu : ((1u << (nsum + t)) - 1u);
  const unsigned int Sm = (1u << nsum) - 1u;
  const GOp& OA = a.op[a.tA];
  const GOp& OB = a.op[a.tB];
  const GOp& OC = a.op[a.tC];
  char* sm = reinterpret_cast<char*>(trsm);
  float2* bufs = reinterpret_cast<float2*>(sm);
  unsigned short* RA = reinterpret_cast<unsigned short*>(sm + ly.off_rt);
  const int T = 1 << t;
  unsigned short* RB = RA + T;
  unsigned short* RC = RB + T;
  // column offsets: pext over disjoint bit sets adds, so A's column of (k, x) is
  // ka[k] + xa[x] and B's of (k, y) is kb[k] + yb[y] (times the column stride)
  int* ka = reinterpret_cast<int*>(sm + ly.off_col);
  int* kb = ka + ly.nK;
  int* xa = kb + ly.nK;
  int* yb = xa + NX;
  int* colC = yb + NY;
  float2* W = reinterpret_cast<float2*>(sm + ly.off_w);
  const int nK = ly.nK;
  {
    const unsigned int ma = (OA.umask & L) >> nsum, mb = (OB.umask & L) >> nsum,
                       mc = (OC.umask & L) >> nsum;
    for (int o = threadIdx.x; o < T; o += blockDim.x) {
      RA[o] = (unsigned short)pext32g((unsigned)o, ma);
      RB[o] = (unsigned short)pext32g((unsigned)o, mb);
      RC[o] = (unsigned short)pext32g((unsigned)o, mc);
    }
    for (int k = threadIdx.x; k < nK; k += blockDim.x) {
      const unsigned int U = pdep32g((unsigned)k, a.tK);
      ka[k] = (int)pext32g(U, OA.umask & Sm) * ly.pA;
      kb[k] = (int)pext32g(U, OB.umask & Sm) * ly.pB;
    }
    for (int x = threadIdx.x; x < NX; x += blockDim.x)
      xa[x] = (int)pext32g(pdep32g((unsigned)x, a.tX), OA.umask & Sm) * ly.pA;
    for (int y = threadIdx.x; y < NY; y += blockDim.x)
      yb[y] = (int)pext32g(pdep32g((unsigned)y, a.tY), OB.umask & Sm) * ly.pB;
    for (int e = threadIdx.x; e < NX * NY; e += blockDim.x) {
      const unsigned int U = pdep32g((unsigned)(e / NY), a.tX) | pdep32g((unsigned)(e % NY), a.tY);
      colC[e] = (int)pext32g(U, OC.umask & Sm) * ly.pC;
    }
  }
  const long long per = 1ll << h;
  const long long ntiles = a.nslices * per;
  const unsigned int inner = a.tile_inner, hmask = h >= 32 ? 0xffffffffu : ((1u << h) - 1u);
  const int pin = __popc(inner);
  const float2* d2 = reinterpret_cast<const float2*>(data);
  // tile w -> slot; called by all lanes of warp 0 (lane-parallel bit extracts)
  auto locate = [&](long long w, int slot) {
    const long long i = w / per;
    const unsigned int tp = (unsigned int)(w - i * per);
    const unsigned int tau = inner ? (warp_pdep(tp & ((1u << pin) - 1u), inner) |
                                      warp_pdep(tp >> pin, ~inner & hmask))
                                   : tp;
    const unsigned long long sid = (unsigned long long)(a.slice_first + i);
    const int sh = nsum + t;
    const long long pa = (long long)warp_pext(tau, (OA.umask & ~L) >> sh);
    const long long pb = (long long)warp_pext(tau, (OB.umask & ~L) >> sh);
    const long long pc = (long long)warp_pext(tau, (OC.umask & ~L) >> sh);
    if ((threadIdx.x & 31) == 0) {
      s_loc[slot][0] = i;
      s_loc[slot][1] = tau;
      s_loc[slot][2] = op_slice_base(OA, i, sid) + (pa << ly.laA);
      s_loc[slot][3] = op_slice_base(OB, i, sid) + (pb << ly.laB);
      const long long cb = a.fold_a ? a.scratch_a + i * a.scratch_stride : op_slice_base(OC, i, sid);
      s_loc[slot][4] = cb + (pc << ly.laC);
    }
  };
  auto issue = [&](int slot, float2* dst) {
    const float2* srcA = d2 + s_loc[slot][2];
    const float2* srcB = d2 + s_loc[slot][3];
    const float2* srcC = d2 + s_loc[slot][4];
    float2* dA = dst;
    float2* dB = dA + ly.zA;
    float2* dC = dB + ly.zB;
    for (int e = threadIdx.x; e < ly.nA; e += blockDim.x)
      cp_async8(dA + (e & ((1 << ly.sA) - 1)) * ly.pA + (e >> ly.sA), srcA + e);
    for (int e = threadIdx.x; e < ly.nB; e += blockDim.x)
      cp_async8(dB + (e & ((1 << ly.sB) - 1)) * ly.pB + (e >> ly.sB), srcB + e);
    for (int e = threadIdx.x; e < ly.nC; e += blockDim.x)
      cp_async8(dC + (e & ((1 << ly.sC) - 1)) * ly.pC + (e >> ly.sC), srcC + e);
    cp_async_commit();
  };
  const long long G = gridDim.x;
  long long w = blockIdx.x;
  if (threadIdx.x < 32) {
    if (w < ntiles) locate(w, 0);
    if (w + G < ntiles) locate(w + G, 1);
  }
  __syncthreads();
  if (w < ntiles) issue(0, bufs);
  long long cur = -1;
  float mx = 0.f;
  bool has_w = false;
  for (int j = 0; j < a.m; ++j) has_w |= a.op[j].tfold == 2;
  for (int jt = 0; w < ntiles; ++jt, w += G) {
    const int slot = jt % 3;
    if (w + G < ntiles) {
      issue((jt + 1) % 3, bufs + ((jt + 1) & 1) * ly.buf);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    if (threadIdx.x < 32 && w + 2 * G < ntiles) locate(w + 2 * G, (jt + 2) % 3);
    const long long i_c = s_loc[slot][0], tau_c = s_loc[slot][1];
    if (i_c != cur) {
      // per slice: the weight over K and the scales of A, B (and C unless folded)
      if (has_w) {
        const unsigned long long sid = (unsigned long long)(a.slice_first + i_c);
        for (int k = threadIdx.x; k < nK; k += blockDim.x) {
          float wr = 1.f, wi = 0.f;
          const unsigned int U = pdep32g((unsigned)k, a.tK);
          for (int q = 0; q < a.m; ++q) {
            const GOp& o = a.op[q];
            if (o.tfold != 2) continue;
            const float sc = pow2_neg_g(scale_exp_g(meta[o.meta + (o.meta_per_slice ? i_c : 0)].maxabs));
            const float2 v = d2[op_slice_base(o, i_c, sid) + pext32g(U, o.umask)];
            const float vr = v.x * sc, vi = v.y * sc;
            const float nr = wr * vr - wi * vi, ni = wr * vi + wi * vr;
            wr = nr;
            wi = ni;
          }
          W[k] = make_float2(wr, wi);
        }
      }
      if (threadIdx.x == 0) {
        float sc = pow2_neg_g(scale_exp_g(meta[OA.meta + (OA.meta_per_slice ? i_c : 0)].maxabs)) *
                   pow2_neg_g(scale_exp_g(meta[OB.meta + (OB.meta_per_slice ? i_c : 0)].maxabs));
        if (!a.fold_a)
          sc *= pow2_neg_g(scale_exp_g(meta[OC.meta + (OC.meta_per_slice ? i_c : 0)].maxabs));
        s_sc = sc;
      }
    }
    __syncthreads();
    if (i_c != cur) {
      if (cur >= 0) flush_max(a, meta, cur, mx);
      mx = 0.f;
      cur = i_c;
      if (tau_c == 0 && threadIdx.x == 0) write_meta_e(a, meta, i_c);
    }
    const float2* sA = bufs + (jt & 1) * ly.buf;
    const float2* sB = sA + ly.zA;
    const float2* sC = sB + ly.zB;
    float2* out = reinterpret_cast<float2*>(data) + a.out_base + i_c * a.out_slice_stride +
                  (tau_c << t);
    const float sc = s_sc;
    int xo[NX], yo[NY];
#pragma unroll
    for (int x = 0; x < NX; ++x) xo[x] = xa[x];
#pragma unroll
    for (int y = 0; y < NY; ++y) yo[y] = yb[y];
    for (int o = threadIdx.x; o < T; o += blockDim.x) {
      const float2* pa = sA + RA[o];
      const float2* pb = sB + RB[o];
      const int rc = RC[o];
      float cvr[NX * NY], cvi[NX * NY];
#pragma unroll
      for (int xy = 0; xy < NX * NY; ++xy) {
        const float2 v = sC[colC[xy] + rc];
        cvr[xy] = v.x;
        cvi[xy] = v.y;
      }
      float accr = 0.f, acci = 0.f;
      for (int k = 0; k < nK; ++k) {
        const float2* pak = pa + ka[k];
        const float2* pbk = pb + kb[k];
        float bvr[NY], bvi[NY];
#pragma unroll
        for (int y = 0; y < NY; ++y) {
          const float2 v = pbk[yo[y]];
          bvr[y] = v.x;
          bvi[y] = v.y;
        }
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int x = 0; x < NX; ++x) {
          float yr = 0.f, yi = 0.f;
#pragma unroll
          for (int y = 0; y < NY; ++y) {
            yr = fmaf(bvr[y], cvr[x * NY + y], yr);
            yr = fmaf(-bvi[y], cvi[x * NY + y], yr);
            yi = fmaf(bvr[y], cvi[x * NY + y], yi);
            yi = fmaf(bvi[y], cvr[x * NY + y], yi);
          }
          const float2 av = pak[xo[x]];
          sr = fmaf(av.x, yr, sr);
          sr = fmaf(-av.y, yi, sr);
          si = fmaf(av.x, yi, si);
          si = fmaf(av.y, yr, si);
        }
        if (has_w) {
          const float2 wk = W[k];
          accr = fmaf(wk.x, sr, accr);
          accr = fmaf(-wk.y, si, accr);
          acci = fmaf(wk.x, si, acci);
          acci = fmaf(wk.y, sr, acci);
        } else {
          accr += sr;
          acci += si;
        }
      }
      accr *= sc;
      acci *= sc;
      out[o] = make_float2(accr, acci);
      mx = fmaxf(mx, absmax_g(accr, acci));
    }
    __syncthreads();
  }
  if (cur >= 0) flush_max(a, meta, cur, mx);
}

using TriFn = void (*)(const GemmArgs, int, float*, GMeta*);

template <int NX, int NY>
TriFn tri_fn_xy() {
  return k_tri_tile<NX, NY>;
}

TriFn tri_fn(int nx, int ny) {
  switch (nx * 8 + ny) {
    case 1 * 8 + 1: return tri_fn_xy<1, 1>();
    case 2 * 8 + 1: return tri_fn_xy<2, 1>();
    case 4 * 8 + 1: return tri_fn_xy<4, 1>();
    case 8 * 8 + 1: return tri_fn_xy<8, 1>();
    case 16 * 8 + 1: return tri_fn_xy<16, 1>();
    case 2 * 8 + 2: return tri_fn_xy<2, 2>();
    case 4 * 8 + 2: return tri_fn_xy<4, 2>();
    case 8 * 8 + 2: return tri_fn_xy<8, 2>();
    case 4 * 8 + 4: return tri_fn_xy<4, 4>();
    default: return nullptr;
  }
}

// Triangle form with tensor-copy (TMA) staging and a producer warp: the same tiles
// and the same sum as k_tri_tile, with the operand blocks in their natural layout
// (row = the operand's output indices in the tile, column = its summed indices),
// each row padded by 2 complex (box copies 4 floats wider than the row, the excess
// lying outside the tensor and arriving as zeros). A row stride of 4 words modulo
// 32 makes 16-byte loads by lanes on consecutive rows conflict-free, so the
// consumers read the summed values in pairs: the two values of the operand's
// lowest summed index (a K index, or for A an X index, for B a Y index). Per k the
// x sum is taken first: u_y = sum_x A[k,x] C'[x,y], then sum_y u_y B[k,y]
// (NX NY + NY complex multiply-adds per k).
//
// Warp 8 locates 32 tiles at a time (one per lane), waits for a ring stage to be
// free, writes the tile's slice, output offset, scale and K weights into the
// stage's slot and issues the copies of A's, B's and C's blocks, completing on
// the stage's "full" barrier; the 8 consumer warps compute one output per thread
// and arrive on the stage's "empty" barrier. Waits are bounded as in k_gemm_tma.
constexpr int kTriStages = 2;
constexpr int kTriMaxK = 64;

struct TriSlot {
  long long i, out;
  float sc;
  int first;
  float2 w[kTriMaxK];  // the weights over K of the tile's slice
};

// One output of the triangle form from its A, B and C' rows in shared memory
// (natural layout): A's and B's summed values are read two at a time, over k when
// PAIRA_K (PAIRB_K), else over x (y).
template <int NX, int NY, bool PAIRA_K, bool PAIRB_K>
__device__ __forceinline__ float2 tri_one(const float2* pa, const float2* pb, const float2* pc,
                                          const int* ka, const int* kb, const int (&xa)[NX],
                                          const int (&yb)[NY], const int (&cc)[NX * NY], int nK,
                                          bool has_w, const float2* wk) {
  float cvr[NX * NY], cvi[NX * NY];
#pragma unroll
  for (int xy = 0; xy < NX * NY; ++xy) {
    const float2 v = pc[cc[xy]];
    cvr[xy] = v.x;
    cvi[xy] = v.y;
  }
  float accr = 0.f, acci = 0.f;
#pragma unroll 2
  for (int k0 = 0; k0 < nK; k0 += 2) {
    float ar[2][NX], ai[2][NX], br[2][NY], bi[2][NY];
    if (PAIRA_K) {
      const float2* q = pa + ka[k0];
#pragma unroll
      for (int x = 0; x < NX; ++x) {
        const float4 v = *reinterpret_cast<const float4*>(q + xa[x]);
        ar[0][x] = v.x; ai[0][x] = v.y; ar[1][x] = v.z; ai[1][x] = v.w;
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const float2* q = pa + ka[k0 + kk];
#pragma unroll
        for (int x = 0; x < NX; x += 2) {
          const float4 v = *reinterpret_cast<const float4*>(q + xa[x]);
          ar[kk][x] = v.x; ai[kk][x] = v.y; ar[kk][x + 1] = v.z; ai[kk][x + 1] = v.w;
        }
      }
    }
    if (PAIRB_K) {
      const float2* q = pb + kb[k0];
#pragma unroll
      for (int y = 0; y < NY; ++y) {
        const float4 v = *reinterpret_cast<const float4*>(q + yb[y]);
        br[0][y] = v.x; bi[0][y] = v.y; br[1][y] = v.z; bi[1][y] = v.w;
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const float2* q = pb + kb[k0 + kk];
#pragma unroll
        for (int y = 0; y < NY; y += 2) {
          const float4 v = *reinterpret_cast<const float4*>(q + yb[y]);
          br[kk][y] = v.x; bi[kk][y] = v.y; br[kk][y + 1] = v.z; bi[kk][y + 1] = v.w;
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int y = 0; y < NY; ++y) {
        float ur = 0.f, ui = 0.f;
#pragma unroll
        for (int x = 0; x < NX; ++x) {
          ur = fmaf(ar[kk][x], cvr[x * NY + y], ur);
          ur = fmaf(-ai[kk][x], cvi[x * NY + y], ur);
          ui = fmaf(ar[kk][x], cvi[x * NY + y], ui);
          ui = fmaf(ai[kk][x], cvr[x * NY + y], ui);
        }
        sr = fmaf(ur, br[kk][y], sr);
        sr = fmaf(-ui, bi[kk][y], sr);
        si = fmaf(ur, bi[kk][y], si);
        si = fmaf(ui, br[kk][y], si);
      }
      if (has_w) {
        const float2 w = wk[k0 + kk];
        accr = fmaf(w.x, sr, accr);
        accr = fmaf(-w.y, si, accr);
        acci = fmaf(w.x, si, acci);
        acci = fmaf(w.y, sr, acci);
      } else {
        accr += sr;
        acci += si;
      }
    }
  }
  return make_float2(accr, acci);
}

constexpr int kTriOutsPerThread = 2;  // tiles of up to 512 outputs

template <int NX, int NY>
__global__ void __launch_bounds__(kTmaThreads, 2) k_tri_tma(
    const GemmArgs a, const __grid_constant__ CUtensorMap mapA,
    const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapC, int u,
    float* data, GMeta* meta) {
  extern __shared__ float4 trsm[];
  __shared__ TriSlot s_slot[kTriStages];
  __shared__ alignas(8) unsigned long long s_full[kTriStages];
  __shared__ alignas(8) unsigned long long s_empty[kTriStages];
  __shared__ int s_col[2 * kTriMaxK + NX + NY + NX * NY];  // ka, kb, xa, yb, colC
  __shared__ volatile int s_fail;
  const int nsum = a.nsum, t = a.tb, h = u - nsum - t;
  const unsigned int L = (nsum + t >= 32) ? 0xffffffffu : ((1u << (nsum + t)) - 1u);
  const unsigned int Sm = (1u << nsum) - 1u;
  const GOp& OA = a.op[a.tA];
  const GOp& OB = a.op[a.tB];
  const GOp& OC = a.op[a.tC];
  const int sA = __popc(OA.umask & Sm), sB = __popc(OB.umask & Sm), sC = __popc(OC.umask & Sm);
  const int laA = __popc(OA.umask & L), laB = __popc(OB.umask & L), laC = __popc(OC.umask & L);
  const int rA = 1 << (laA - sA), rB = 1 << (laB - sB), rC = 1 << (laC - sC);
  const int PA = (1 << sA) + 2, PB = (1 << sB) + 2, PC = (1 << sC) + 2;  // row strides (complex)
  const int zA = (rA * PA + 127) & ~127, zB = (rB * PB + 127) & ~127, zC = (rC * PC + 127) & ~127;
  const int zS = zA + zB + zC;  // one stage (float2)
  float2* const stage0 = reinterpret_cast<float2*>(reinterpret_cast<char*>(trsm) +
                                                   ((1024u - (smem_u32(trsm) & 1023u)) & 1023u));
  const int nK = 1 << __popc(a.tK);
  bool has_w = false;
  for (int j = 0; j < a.m; ++j) has_w |= a.op[j].tfold == 2;
  const long long ntiles = a.nslices << h;
  const long long chunk = (ntiles + gridDim.x - 1) / gridDim.x;
  const long long w0 = (long long)blockIdx.x * chunk;
  const long long w1 = min(ntiles, w0 + chunk);
  int* ka = s_col;
  int* kb = ka + nK;
  int* xa = kb + nK;
  int* yb = xa + NX;
  int* colC = yb + NY;
  if (threadIdx.x == 0) {
    for (int b = 0; b < kTriStages; ++b) {
      mbar_init(&s_full[b], 1);
      mbar_init(&s_empty[b], kTmaConsumers / 32);
    }
    mbar_fence_init();
    s_fail = 0;
  }
  // column of (k, x) in A's row = ka[k] + xa[x] (pext over disjoint bit sets adds)
  for (int k = threadIdx.x; k < nK; k += blockDim.x) {
    const unsigned int U = pdep32g((unsigned)k, a.tK);
    ka[k] = (int)pext32g(U, OA.umask & Sm);
    kb[k] = (int)pext32g(U, OB.umask & Sm);
  }
  for (int x = threadIdx.x; x < NX; x += blockDim.x)
    xa[x] = (int)pext32g(pdep32g((unsigned)x, a.tX), OA.umask & Sm);
  for (int y = threadIdx.x; y < NY; y += blockDim.x)
    yb[y] = (int)pext32g(pdep32g((unsigned)y, a.tY), OB.umask & Sm);
  for (int e = threadIdx.x; e < NX * NY; e += blockDim.x) {
    const unsigned int U = pdep32g((unsigned)(e / NY), a.tX) | pdep32g((unsigned)(e % NY), a.tY);
    colC[e] = (int)pext32g(U, OC.umask & Sm);
  }
  __syncthreads();
  unsigned int issued = 0u;  // producer lane 0, barrier b: bit b some fill, bit 8 + b parity
  if (threadIdx.x >= kTmaConsumers) {
    // ---- producer warp ----
    const int lane = threadIdx.x & 31;
    const unsigned int inner = a.tile_inner, hmask = h >= 32 ? 0xffffffffu : ((1u << h) - 1u);
    const int pin = __popc(inner);
    const unsigned int outer = ~inner & hmask, pmask = (1u << pin) - 1u;
    const int sh = nsum + t;
    const unsigned int hiA = (OA.umask & ~L) >> sh, hiB = (OB.umask & ~L) >> sh,
                       hiC = (OC.umask & ~L) >> sh;
    const unsigned int bytes = (unsigned)((rA * PA + rB * PB + rC * PC) * 8);
    auto load = [&](const CUtensorMap* map, long long off, float2* dst, int rows, int P, int s, int b) {
      const int box = min(rows, kTmaBoxRows);
      const int row0 = (int)(off >> s);
      for (int r = 0; r < rows; r += box) tma_load_2d(dst + r * P, map, 0, row0 + r, &s_full[b]);
    };
    int ms = 0, f = 0;
    long long pi = -1;
    float sc = 1.f;
    float2 wl0 = make_float2(1.f, 0.f), wl1 = make_float2(1.f, 0.f);  // W[lane], W[lane + 32]
    bool ok = true;
    for (long long wb = w0; wb < w1 && ok; wb += 32) {
      const long long wl = wb + lane;
      long long li = 0, oa = 0, ob = 0, oc = 0;
      unsigned int ltau = 0;
      if (wl < w1) {
        li = wl >> h;
        const unsigned int tp = (unsigned int)(wl & (((long long)1 << h) - 1));
        ltau = inner ? (pdep32g(tp & pmask, inner) | pdep32g(tp >> pin, outer)) : tp;
        const unsigned long long sid = (unsigned long long)(a.slice_first + li);
        oa = op_slice_base(OA, li, sid) + ((long long)pext32g(ltau, hiA) << laA);
        ob = op_slice_base(OB, li, sid) + ((long long)pext32g(ltau, hiB) << laB);
        const long long cb = a.fold_a ? a.scratch_a + li * a.scratch_stride : op_slice_base(OC, li, sid);
        oc = cb + ((long long)pext32g(ltau, hiC) << laC);
      }
      const int nwin = (int)min(32ll, w1 - wb);
      for (int j = 0; j < nwin; ++j) {
        const long long i = __shfl_sync(0xffffffffu, li, j);
        const unsigned int tau = __shfl_sync(0xffffffffu, ltau, j);
        const long long offA = __shfl_sync(0xffffffffu, oa, j);
        const long long offB = __shfl_sync(0xffffffffu, ob, j);
        const long long offC = __shfl_sync(0xffffffffu, oc, j);
        if (i != pi) {  // a new slice: its scale (lane 0) and weights over K (all lanes)
          pi = i;
          if (lane == 0) {
            sc = pow2_neg_g(scale_exp_g(meta[OA.meta + (OA.meta_per_slice ? i : 0)].maxabs)) *
                 pow2_neg_g(scale_exp_g(meta[OB.meta + (OB.meta_per_slice ? i : 0)].maxabs));
            if (!a.fold_a)
              sc *= pow2_neg_g(scale_exp_g(meta[OC.meta + (OC.meta_per_slice ? i : 0)].maxabs));
          }
          if (has_w) {
            const unsigned long long sid = (unsigned long long)(a.slice_first + i);
            for (int half = 0; half < 2; ++half) {
              const int k = lane + 32 * half;
              float wr = 1.f, wi = 0.f;
              if (k < nK) {
                const unsigned int U = pdep32g((unsigned)k, a.tK);
                for (int q = 0; q < a.m; ++q) {
                  const GOp& o = a.op[q];
                  if (o.tfold != 2) continue;
                  const float s = pow2_neg_g(scale_exp_g(meta[o.meta + (o.meta_per_slice ? i : 0)].maxabs));
                  const float2 v = reinterpret_cast<const float2*>(data)[op_slice_base(o, i, sid) +
                                                                        pext32g(U, o.umask)];
                  const float vr = v.x * s, vi = v.y * s;
                  const float nr = wr * vr - wi * vi, ni = wr * vi + wi * vr;
                  wr = nr;
                  wi = ni;
                }
              }
              if (half) wl1 = make_float2(wr, wi);
              else wl0 = make_float2(wr, wi);
            }
          }
        }
        // the stage is free once the tile kTriStages earlier is done
        if (lane == 0) {
          if (s_fail) ok = false;
          if (ok && f > 0) ok = mbar_wait(&s_empty[ms], (unsigned)((f - 1) & 1), a.err);
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) {
          if (lane == 0) s_fail = 1;
          break;
        }
        if (has_w) {
          if (lane < nK) s_slot[ms].w[lane] = wl0;
          if (lane + 32 < nK) s_slot[ms].w[lane + 32] = wl1;
        }
        if (lane == 0) {
          s_slot[ms].i = i;
          s_slot[ms].out = a.out_base + i * a.out_slice_stride + ((long long)tau << t);
          s_slot[ms].sc = sc;
          s_slot[ms].first = tau == 0u;
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) {
          float2* st = stage0 + ms * zS;
          mbar_expect_tx(&s_full[ms], bytes);
          load(&mapA, offA, st, rA, PA, sA, ms);
          load(&mapB, offB, st + zA, rB, PB, sB, ms);
          load(&mapC, offC, st + zA + zB, rC, PC, sC, ms);
          issued = (issued | (1u << ms)) ^ (256u << ms);
        }
        if (++ms == kTriStages) {
          ms = 0;
          ++f;
        }
      }
    }
  } else {
    // ---- consumer warps ----
    const int T = 1 << t;
    const unsigned int ma = (OA.umask & L) >> nsum, mb = (OB.umask & L) >> nsum,
                       mc = (OC.umask & L) >> nsum;
    // pairs: A's lowest summed index is K's lowest (pairs over k) or X's (pairs over x)
    const bool pairA_k = ((OA.umask & Sm) & (0u - (OA.umask & Sm))) & a.tK;
    const bool pairB_k = ((OB.umask & Sm) & (0u - (OB.umask & Sm))) & a.tK;
    // this thread's outputs (the same in every tile) and their rows, once
    int nmine = 0, ro[kTriOutsPerThread], rA_[kTriOutsPerThread], rB_[kTriOutsPerThread],
        rC_[kTriOutsPerThread];
#pragma unroll
    for (int r = 0; r < kTriOutsPerThread; ++r) {
      const int o = threadIdx.x + r * kTmaConsumers;
      ro[r] = o;
      rA_[r] = (int)pext32g((unsigned)o, ma) * PA;
      rB_[r] = (int)pext32g((unsigned)o, mb) * PB;
      rC_[r] = (int)pext32g((unsigned)o, mc) * PC;
      if (o < T) nmine = r + 1;
    }
    int xr[NX], yr[NY], cr[NX * NY];
#pragma unroll
    for (int x = 0; x < NX; ++x) xr[x] = xa[x];
#pragma unroll
    for (int y = 0; y < NY; ++y) yr[y] = yb[y];
#pragma unroll
    for (int e = 0; e < NX * NY; ++e) cr[e] = colC[e];
    long long cur = -1;
    float mx = 0.f;
    int ms = 0;
    unsigned int ph = 0u;
    for (long long w = w0; w < w1; ++w) {
      const bool ok = mbar_wait(&s_full[ms], ph, a.err);
      if (!__all_sync(0xffffffffu, ok)) {
        s_fail = 1;
        break;
      }
      const TriSlot& sl = s_slot[ms];
      const long long i_c = sl.i;
      const float sc = sl.sc;
      if (i_c != cur) {
        if (cur >= 0) flush_max(a, meta, cur, mx);
        mx = 0.f;
        cur = i_c;
        if (sl.first && threadIdx.x == 0) write_meta_e(a, meta, i_c);
      }
      const float2* stA = stage0 + ms * zS;
      const float2* stB = stA + zA;
      const float2* stC = stB + zB;
      float2* out = reinterpret_cast<float2*>(data) + sl.out;
#pragma unroll
      for (int r = 0; r < kTriOutsPerThread; ++r) {
        if (r >= nmine) break;
        float2 v;
        if (pairA_k && pairB_k)
          v = tri_one<NX, NY, true, true>(stA + rA_[r], stB + rB_[r], stC + rC_[r], ka, kb, xr, yr,
                                          cr, nK, has_w, sl.w);
        else if (pairA_k)
          v = tri_one<NX, NY, true, false>(stA + rA_[r], stB + rB_[r], stC + rC_[r], ka, kb, xr,
                                           yr, cr, nK, has_w, sl.w);
        else if (pairB_k)
          v = tri_one<NX, NY, false, true>(stA + rA_[r], stB + rB_[r], stC + rC_[r], ka, kb, xr,
                                           yr, cr, nK, has_w, sl.w);
        else
          v = tri_one<NX, NY, false, false>(stA + rA_[r], stB + rB_[r], stC + rC_[r], ka, kb, xr,
                                            yr, cr, nK, has_w, sl.w);
        v.x *= sc;
        v.y *= sc;
        out[ro[r]] = v;
        mx = fmaxf(mx, absmax_g(v.x, v.y));
      }
      __syncwarp();
      if ((threadIdx.x & 31) == 0) mbar_arrive(&s_empty[ms]);
      if (++ms == kTriStages) {
        ms = 0;
        ph ^= 1u;
      }
    }
    if (cur >= 0) flush_max(a, meta, cur, mx);
  }
  __syncthreads();
  if (s_fail && threadIdx.x == kTmaConsumers) {
    for (int b = 0; b < kTriStages; ++b)
      if ((issued >> b) & 1u) mbar_wait(&s_full[b], ((issued >> (8 + b)) & 1u) ^ 1u, nullptr);
  }
}


using TriTmaFn = void (*)(const GemmArgs, const CUtensorMap, const CUtensorMap, const CUtensorMap,
                          int, float*, GMeta*);

TriTmaFn tri_tma_fn(int nx, int ny) {
  switch (nx * 8 + ny) {
    case 2 * 8 + 1: return k_tri_tma<2, 1>;
    case 4 * 8 + 1: return k_tri_tma<4, 1>;
    case 8 * 8 + 1: return k_tri_tma<8, 1>;
    case 2 * 8 + 2: return k_tri_tma<2, 2>;
    case 4 * 8 + 2: return k_tri_tma<4, 2>;
    default: return nullptr;
  }
}

constexpr size_t kTriSmemMax = 100 * 1024;

}  // namespace

constexpr size_t kTileSmemMax = 100 * 1024;
// Largest tile: 2^11 outputs, i.e. at most kTileQuads quads per thread of 256.
constexpr int kTileMaxBits = 11;

static size_t tile_smem(const GemmArgs& a, int t) {
  // two buffers of each side's block, rows padded to K + 2 complex
  const unsigned int L = (a.nsum + t >= 32) ? 0xffffffffu : ((1u << (a.nsum + t)) - 1u);
  const long long ra = 1ll << (__builtin_popcount(a.op[a.gA].umask & L) - a.nsum);
  const long long rb = 1ll << (__builtin_popcount(a.op[a.gB].umask & L) - a.nsum);
  return (size_t)(2 * (ra + rb) * ((1ll << a.nsum) + 2) * 8);
}

int gemm_tile_bits(const GemmArgs& a, int u) {
  if (a.mSA || a.mSB || a.gA < 0 || a.gB < 0) return 0;
  if (__builtin_popcount(a.op[a.gA].umask) > 30 || __builtin_popcount(a.op[a.gB].umask) > 30)
    return 0;
  const int c = u - a.nsum;
  for (int t = std::min(c, kTileMaxBits); t >= 5; --t)
    if (tile_smem(a, t) + 3072 <= kTileSmemMax) return t;
  return 0;
}

void gemm_tile_regs(GemmArgs& a, int block_mode) {
  // the highest (reg_x) and second highest (reg_x2) A-only and B-only output bits
  // inside the tile (-1: none)
  a.reg_a = a.reg_b = a.reg_a2 = a.reg_b2 = -1;
  a.wide = 0;
  for (int b = 0; b < a.tb; ++b) {
    if ((a.mM >> (a.nsum + b)) & 1u) {
      a.reg_a2 = a.reg_a;
      a.reg_a = b;
    }
    if ((a.mN >> (a.nsum + b)) & 1u) {
      a.reg_b2 = a.reg_b;
      a.reg_b = b;
    }
  }
  if (a.reg_a < 0 || a.reg_b < 0 || a.tb < 3) {
    a.reg_a = a.reg_b = a.reg_a2 = a.reg_b2 = -1;
    return;
  }
  // a 2 x 4 (or 4 x 2) block when the wide side's rows are shared by more lanes of a
  // warp: a warp's lanes take the five lowest tile bits outside the block's bits, and
  // a shared-memory wavefront serves 8 distinct 16-byte rows
  auto wavefronts = [&](unsigned int rmask, unsigned int side) {
    int n = 0, seen = 0;
    for (int b = 0; b < a.tb && seen < 5; ++b) {
      if ((rmask >> b) & 1u) continue;
      ++seen;
      n += (side >> (a.nsum + b)) & 1u;
    }
    return std::max(1, (1 << n) / 8);
  };
  if (block_mode == 1) return;
  if (block_mode == 2 || block_mode == 3) {  // a wide block whenever a second bit exists
    const bool b_ok = a.reg_b2 >= 0 && a.tb >= 4, a_ok = a.reg_a2 >= 0 && a.tb >= 4;
    if (block_mode == 2) a.wide = b_ok ? 1 : (a_ok ? 2 : 0);
    else a.wide = a_ok ? 2 : (b_ok ? 1 : 0);
    return;
  }
  const unsigned int uA = a.op[a.gA].umask, uB = a.op[a.gB].umask;
  const unsigned int r2 = (1u << a.reg_a) | (1u << a.reg_b);
  // (a wider block costs registers: taken only for a quarter fewer wavefronts or more)
  const int cost22 = 2 * wavefronts(r2, uA) + 2 * wavefronts(r2, uB);  // per 4 outputs
  int best = 3 * cost22 / 2;  // per 8 outputs, x 3/4
  if (a.reg_b2 >= 0 && a.tb >= 4) {
    const unsigned int rm = r2 | (1u << a.reg_b2);
    const int c = 2 * wavefronts(rm, uA) + 4 * wavefronts(rm, uB);
    if (c < best) {
      best = c;
      a.wide = 1;
    }
  }
  if (a.reg_a2 >= 0 && a.tb >= 4) {
    const unsigned int rm = r2 | (1u << a.reg_a2);
    const int c = 4 * wavefronts(rm, uA) + 2 * wavefronts(rm, uB);
    if (c < best) {
      best = c;
      a.wide = 2;
    }
  }
}

unsigned int gemm_tile_inner(const GemmArgs& a, int u) {
  // the high output bits of the side whose block is smaller go innermost, so
  // consecutive tiles share the larger side's block
  const int t = a.tb, hb = u - a.nsum - t;
  if (t <= 0 || hb <= 0) return 0u;
  const bool a_larger = gemm_tile_stay(a) == 0;
  const unsigned int only = a_larger ? a.mN : a.mM;  // indices of the smaller side only
  unsigned int inner = 0;
  for (int b = 0; b < hb; ++b)
    if ((only >> (a.nsum + t + b)) & 1u) inner |= 1u << b;
  return inner;
}

int gemm_tile_stay(const GemmArgs& a) {
  return __builtin_popcount(a.op[a.gA].umask) >= __builtin_popcount(a.op[a.gB].umask) ? 0 : 1;
}

int tri_tile_bits(const GemmArgs& a, int u) {
  if (a.tA < 0) return 0;
  const int nx = 1 << __builtin_popcount(a.tX), ny = 1 << __builtin_popcount(a.tY);
  if (!tri_fn(nx, ny)) return 0;
  const int c = u - a.nsum;
  for (int t = std::min(c, 10); t >= 7; --t) {
    const TriLayout l = tri_layout(a, t);
    if (l.bytes <= kTriSmemMax && l.zA < (1 << 30) && l.rA <= 65535 && l.rB <= 65535 &&
        l.rC <= 65535)
      return t;
  }
  return 0;
}

static bool row_map(CUtensorMap& m, float* data, long long ws_elems, int nsum, int box_rows);

// The workspace as rows of 2^s complex, boxes 2^(s+1) + 4 floats wide (padding as above).
static bool cols_map(CUtensorMap& m, float* data, long long ws_elems, int s, int box_rows) {
  return row_map(m, data, ws_elems, s, box_rows);
}

constexpr size_t kTriTmaSmemMax = 110 * 1024;  // two blocks per SM

// The tensor-copy triangle kernel's shared memory (0: not applicable).
static size_t tri_tma_smem(const GemmArgs& a) {
  const unsigned int L = (a.nsum + a.tb >= 32) ? 0xffffffffu : ((1u << (a.nsum + a.tb)) - 1u);
  const unsigned int Sm = (1u << a.nsum) - 1u;
  size_t z = 0;
  const int ops[3] = {a.tA, a.tB, a.tC};
  for (int q = 0; q < 3; ++q) {
    const unsigned int m = a.op[ops[q]].umask;
    const int s = __builtin_popcount(m & Sm), la = __builtin_popcount(m & L);
    if (s < 1 || s > 6) return 0;
    const long long rows = 1ll << (la - s), P = (1ll << s) + 2;
    z += (size_t)((rows * P + 127) & ~127ll);
  }
  return 2 * z * 8 + 1024;
}

// Every block a triangle tile reads starts on a whole row of its operand.
static bool tri_rows_aligned(const GemmArgs& a) {
  const unsigned int Sm = (1u << a.nsum) - 1u;
  const int ops[3] = {a.tA, a.tB, a.tC};
  for (int q = 0; q < 3; ++q) {
    const GOp& o = a.op[ops[q]];
    const long long C = 1ll << __builtin_popcount(o.umask & Sm);
    if (q == 2 && a.fold_a) {
      if (a.scratch_a % C || a.scratch_stride % C) return false;
    } else {
      if (o.base % C || o.slice_stride % C) return false;
      if (o.smask && (1ll << o.sshift) % C) return false;
    }
  }
  return true;
}

unsigned int tri_tile_inner(const GemmArgs& a, int u) {
  // consecutive tiles share A's or B's block: the high output bits missing from A or B
  // are visited innermost
  const int hb = u - a.nsum - a.tb;
  const unsigned int AB = a.op[a.tA].umask & a.op[a.tB].umask;
  unsigned int inner = 0;
  for (int b = 0; b < hb && a.tb > 0; ++b)
    if (!((AB >> (a.nsum + a.tb + b)) & 1u)) inner |= 1u << b;
  return inner;
}

int tri_launch(const GemmArgs& a, float* data, GMeta* meta, cudaStream_t s, int sms,
               bool* used_tma) {
  if (used_tma) *used_tma = false;
  int u = 0;
  for (unsigned int m = a.op[a.tA].umask | a.op[a.tB].umask | a.op[a.tC].umask; m; m >>= 1) ++u;
  const int nx = 1 << __builtin_popcount(a.tX), ny = 1 << __builtin_popcount(a.tY);
  TriFn fn = tri_fn(nx, ny);
  static bool attr[5][5] = {};
  const int ix = __builtin_ctz(nx), iy = __builtin_ctz(ny);
  if (!attr[ix][iy]) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriSmemMax);
    attr[ix][iy] = true;
  }
  int n = 0;
  if (a.fold_a) {
    const long long work = a.nslices << __builtin_popcount(a.op[a.tC].umask);
    const long long g = std::min<long long>((work + 255) / 256, (long long)sms * 16);
    k_tri_fold<<<(unsigned)std::max<long long>(1, g), 256, 0, s>>>(a, data, meta);
    ++n;
  }
  // tensor-copy staging when the kernel exists for the shape and the rows line up, with
  // its own tile: the largest of 2^9 .. 2^7 outputs whose two-stage ring fits
  TriTmaFn tfn = tri_tma_fn(nx, ny);
  if (a.use_tma && a.err && tfn && a.tK && tri_rows_aligned(a)) {
    GemmArgs b = a;
    size_t tsm = 0;
    for (int t = std::min(9, u - a.nsum); t >= 7 && !tsm; --t) {
      b.tb = t;
      const size_t z = tri_tma_smem(b);
      if (z && z <= kTriTmaSmemMax) tsm = z;
    }
    if (tsm) {
      b.tile_inner = tri_tile_inner(b, u);
      const unsigned int L = (b.nsum + b.tb >= 32) ? 0xffffffffu : ((1u << (b.nsum + b.tb)) - 1u);
      const unsigned int Sm = (1u << b.nsum) - 1u;
      CUtensorMap mp[3];
      const int ops[3] = {b.tA, b.tB, b.tC};
      bool ok = true;
      for (int q = 0; q < 3 && ok; ++q) {
        const unsigned int m = b.op[ops[q]].umask;
        const int sq = __builtin_popcount(m & Sm), la = __builtin_popcount(m & L);
        ok = cols_map(mp[q], data, b.ws_elems, sq, std::min(1 << (la - sq), 256));
      }
      if (ok) {
        cudaFuncSetAttribute(tfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriTmaSmemMax);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tfn, kTmaThreads, tsm) !=
            cudaSuccess)
          per_sm = 1;
        const long long nt = b.nslices << (u - b.nsum - b.tb);
        const unsigned grid = (unsigned)std::max<long long>(
            1, std::min<long long>(nt, (long long)sms * std::max(1, per_sm)));
        tfn<<<grid, kTmaThreads, tsm, s>>>(b, mp[0], mp[1], mp[2], u, data, meta);
        if (used_tma) *used_tma = true;
        return n + 1;
      }
    }
  }
  const long long ntiles = a.nslices << (u - a.nsum - a.tb);
  const TriLayout l = tri_layout(a, a.tb);
  const int threads = std::min(256, 1 << a.tb);
  const int per_sm = std::max<int>(1, std::min<int>(8, (int)((220 * 1024) / (l.bytes + 2048))));
  const unsigned grid =
      (unsigned)std::max<long long>(1, std::min<long long>(ntiles, (long long)sms * per_sm));
  fn<<<grid, threads, l.bytes, s>>>(a, u, data, meta);
  return n + 1;
}

// cuTensorMapEncodeTiled, from the driver through the runtime (no link-time libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// The workspace as rows of K complex (2K floats); boxes of box_rows rows, 2K + 4
// floats wide (the last 4 lie outside every row and arrive as zeros: padding).
static bool row_map(CUtensorMap& m, float* data, long long ws_elems, int nsum, int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  const long long K = 1ll << nsum;
  const long long rows = ws_elems / K;
  if (!fn || rows < 1 || rows > 0x7fffffffll || 2 * K + 4 > 256) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * K), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(K * 8)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * K + 4), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, data, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Every block a tile can read starts on a whole row of K complex.
static bool rows_aligned(const GemmArgs& a) {
  const long long K = 1ll << a.nsum;
  for (int side = 0; side < 2; ++side) {
    const GOp& o = a.op[side ? a.gB : a.gA];
    if (side ? a.fold_b : a.fold_a) {
      if ((side ? a.scratch_b : a.scratch_a) % K || a.scratch_stride % K) return false;
    } else {
      if (o.base % K || o.slice_stride % K) return false;
      if (o.smask && o.sshift < a.nsum) return false;
    }
  }
  return true;
}

// shared side: two buffers; the other side: a ring of nmove buffers
static size_t tma_smem(const GemmArgs& a, int nmove) {
  const unsigned int L = (a.nsum + a.tb >= 32) ? 0xffffffffu : ((1u << (a.nsum + a.tb)) - 1u);
  const long long RS = (1ll << a.nsum) + 2;
  const long long ra = 1ll << (__builtin_popcount(a.op[a.gA].umask & L) - a.nsum);
  const long long rb = 1ll << (__builtin_popcount(a.op[a.gB].umask & L) - a.nsum);
  const long long szA = (ra * RS + 127) & ~127ll, szB = (rb * RS + 127) & ~127ll;
  const long long szS = a.stay ? szB : szA, szM = a.stay ? szA : szB;
  return (size_t)((2 * szS + nmove * szM) * 8 + 1024);
}

typedef void (*TmaFn)(const GemmArgs, const CUtensorMap, const CUtensorMap, int, int, float*,
                      GMeta*);

template <int WIDE>
static TmaFn tma_fn_w(int nsum) {
  switch (nsum) {
    case 1: return k_gemm_tma<1, WIDE>;
    case 2: return k_gemm_tma<2, WIDE>;
    case 3: return k_gemm_tma<3, WIDE>;
    case 4: return k_gemm_tma<4, WIDE>;
    case 5: return k_gemm_tma<5, WIDE>;
    case 6: return k_gemm_tma<6, WIDE>;
    default: return nullptr;
  }
}

static TmaFn tma_fn(int nsum, int wide) {
  return wide == 1 ? tma_fn_w<1>(nsum) : (wide == 2 ? tma_fn_w<2>(nsum) : tma_fn_w<0>(nsum));
}

bool gemm_stream_ok(const GemmArgs& a) {
  if (a.mSA || a.mSB || a.gA < 0 || a.gB < 0 || a.nsum < 1 || a.nsum > 5) return false;
  const int gs = gemm_tile_stay(a);
  const GOp& G = a.op[gs ? a.gB : a.gA];
  const GOp& S = a.op[gs ? a.gA : a.gB];
  if (gs ? a.fold_b : a.fold_a) return false;  // nothing folded into the large side
  const unsigned int Gm = G.umask >> a.nsum, Sm = S.umask >> a.nsum;
  // (the row's output position comes from 3 byte tables: at most 24 row indices)
  return __builtin_popcount(S.umask) <= 12 && __builtin_popcount(Gm) >= 10 &&
         __builtin_popcount(Gm) <= 24 && __builtin_popcount(Sm & ~Gm) <= 10;
}

typedef void (*StreamFn)(const GemmArgs, float*, GMeta*);

static StreamFn stream_fn(int nsum) {
  switch (nsum) {
    case 1: return k_gemm_stream<1>;
    case 2: return k_gemm_stream<2>;
    case 3: return k_gemm_stream<3>;
    case 4: return k_gemm_stream<4>;
    case 5: return k_gemm_stream<5>;
    default: return nullptr;
  }
}

int gemm_launch(const GemmArgs& a, int mode_in, float* data, GMeta* meta, cudaStream_t s, int sms,
                bool* used_tma) {
  if (used_tma) *used_tma = false;
  int mode = mode_in;
  if (mode == GEMM_UMMA_TF32 || mode == GEMM_UMMA_3XTF32) {
    // tcgen05 tensor cores: the folds of A' and B', then one launch; a launch the
    // kernel cannot take (alignment, tensor maps) runs as the FP32 tiled GEMM
    UmmaPlan p;
    if (umma_plan(a, mode == GEMM_UMMA_TF32 ? 1 : 3, p)) {
      int n = 0;
      for (int side = 0; side < 2; ++side) {
        if (!(side ? a.fold_b : a.fold_a)) continue;
        const long long work = a.nslices << __builtin_popcount(a.op[side ? a.gB : a.gA].umask);
        const long long g = std::min<long long>((work + 255) / 256, (long long)sms * 16);
        k_gemm_fold<<<(unsigned)std::max<long long>(1, g), 256, 0, s>>>(a, side, data, meta);
        ++n;
      }
      if (umma_launch(a, p, data, meta, s, sms)) {
        if (used_tma) *used_tma = true;
        return n + 1;
      }
      // the folds already ran; the tiled kernel below folds again (same values)
    }
    mode = a.tb > 0 ? GEMM_TILE : GEMM_SIMT;
  }
  if (mode == GEMM_TILE && a.use_stream) {
    int n = 0;
    const int gs = gemm_tile_stay(a);
    // a small side of at most 256 elements is folded inside the kernel (one element per
    // thread); a larger one by the fold kernel into its scratch first
    GemmArgs as = a;
    const int s_bits = __builtin_popcount(a.op[gs ? a.gA : a.gB].umask);
    as.fold_in = (gs ? a.fold_a : a.fold_b) && s_bits <= 8;
    if ((gs ? a.fold_a : a.fold_b) && !as.fold_in) {
      const int side = gs ? 0 : 1;
      const long long work = a.nslices << __builtin_popcount(a.op[side ? a.gB : a.gA].umask);
      const long long g = std::min<long long>((work + 255) / 256, (long long)sms * 16);
      k_gemm_fold<<<(unsigned)std::max<long long>(1, g), 256, 0, s>>>(a, side, data, meta);
      ++n;
    }
    const GOp& G = a.op[gs ? a.gB : a.gA];
    const GOp& S = a.op[gs ? a.gA : a.gB];
    const unsigned int Gm = G.umask >> a.nsum, Sm = S.umask >> a.nsum;
    const size_t smem = ((size_t)8 << __builtin_popcount(S.umask)) +
                        ((size_t)8 << __builtin_popcount(Sm & ~Gm));
    const long long total = a.nslices << __builtin_popcount(Gm);
    StreamFn fn = stream_fn(a.nsum);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    // one block per resident slot: a single wave, so the next-pass prefetch never restarts
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, 256, smem) !=
        cudaSuccess)
      per_sm = 4;
    const unsigned grid = (unsigned)std::max<long long>(
        1, std::min<long long>(total / (256 * stream_rows(a.nsum)),
                               (long long)sms * std::max(1, per_sm)));
    fn<<<grid, 256, smem, s>>>(as, data, meta);
    return n + 1;
  }
  if (mode == GEMM_TILE) {
    int n = 0;
    for (int side = 0; side < 2; ++side) {
      if (!(side ? a.fold_b : a.fold_a)) continue;
      const long long work = a.nslices << __builtin_popcount(a.op[side ? a.gB : a.gA].umask);
      const long long g = std::min<long long>((work + 255) / 256, (long long)sms * 16);
      k_gemm_fold<<<(unsigned)std::max<long long>(1, g), 256, 0, s>>>(a, side, data, meta);
      ++n;
    }
    int u = 0;
    for (unsigned int m = a.mK | a.mSA | a.mSB | a.mM | a.mN | a.mBt; m; m >>= 1) ++u;
    const long long ntiles = a.nslices << (u - a.nsum - a.tb);
    // one block per resident slot (each block takes one range of tiles)
    // one block per resident slot (each block takes one range of tiles)
    auto grid_for = [&](const void* f, int threads, size_t smem) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem) != cudaSuccess)
        per_sm = 1;
      per_sm = std::max(1, per_sm);
      return (unsigned)std::max<long long>(1, std::min<long long>(ntiles, (long long)sms * per_sm));
    };
    // tensor-copy staging when the rows line up and the maps encode; the ring as
    // deep as it can be without fewer resident blocks than a ring of 2
    TmaFn fn = tma_fn(a.nsum, a.wide);
    if (a.use_tma && a.err && fn && tma_smem(a, 2) <= kTileSmemMax && rows_aligned(a)) {
      const unsigned int L = (a.nsum + a.tb >= 32) ? 0xffffffffu : ((1u << (a.nsum + a.tb)) - 1u);
      const int ra = 1 << (__builtin_popcount(a.op[a.gA].umask & L) - a.nsum);
      const int rb = 1 << (__builtin_popcount(a.op[a.gB].umask & L) - a.nsum);
      CUtensorMap mA, mB;
      if (row_map(mA, data, a.ws_elems, a.nsum, std::min(ra, 256)) &&
          row_map(mB, data, a.ws_elems, a.nsum, std::min(rb, 256))) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemMax);
        const size_t per2 = (220 * 1024) / (tma_smem(a, 2) + 1024);
        int nmove = 2;
        for (int m = kMoveStagesMax; m > 2; --m)
          if (tma_smem(a, m) <= kTileSmemMax && (220 * 1024) / (tma_smem(a, m) + 1024) >= per2) {
            nmove = m;
            break;
          }
        const size_t tsm = tma_smem(a, nmove);
        fn<<<grid_for((const void*)fn, kTmaThreads, tsm), kTmaThreads, tsm, s>>>(a, mA, mB, u, nmove,
                                                                                  data, meta);
        if (used_tma) *used_tma = true;
        return n + 1;
      }
    }
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_gemm_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTileSmemMax);
      attr = true;
    }
    const size_t smem = tile_smem(a, a.tb);
    k_gemm_tile<<<grid_for((const void*)k_gemm_tile, 256, smem), 256, smem, s>>>(a, u, data, meta);
    return n + 1;
  }
  const int kb = __builtin_popcount(a.mK), bb = __builtin_popcount(a.mBt);
  const long long pa = a.nslices << (bb + __builtin_popcount(a.mM) + kb);
  const long long pb = a.nslices << (bb + __builtin_popcount(a.mN) + kb);
  auto grid_for = [&](long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    return (unsigned)std::max<long long>(1, std::min<long long>(g, (long long)sms * 16));
  };
  k_gemm_pack<<<grid_for(pa, 256), 256, 0, s>>>(a, 0, data, meta);
  k_gemm_pack<<<grid_for(pb, 256), 256, 0, s>>>(a, 1, data, meta);
  const int mb = __builtin_popcount(a.mM), nb = __builtin_popcount(a.mN);
  if (mode == GEMM_SIMT) {
    const long long outs = a.nslices << (bb + mb + nb);
    k_gemm_simt<<<grid_for(outs, 256), 256, 0, s>>>(a, data, meta);
  } else {
    const long long items = a.nslices * (long long)((1 << mb) / 16) * ((1 << nb) / 8) << bb;
    const unsigned grid = grid_for(items * 32, 128);
    if (mode == GEMM_TC_TF32) k_gemm_tc<GEMM_TC_TF32><<<grid, 128, 0, s>>>(a, data, meta);
    else if (mode == GEMM_TC_BF16) k_gemm_tc<GEMM_TC_BF16><<<grid, 128, 0, s>>>(a, data, meta);
    else k_gemm_tc<GEMM_TC_3XTF32><<<grid, 128, 0, s>>>(a, data, meta);
  }
  return 3;
}

}  // namespace qt
