// GEMM form of a fused bucket launch on the fifth-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), complex64 tensors.
//
// The launch computes out[bt][m][n] = sum_k A'[bt][m][k] B'[bt][n][k] (gemm.cu
// describes the form). In the canonical layout the K summed indices are the
// lowest bits of both operands, so a row of an operand (its other indices fixed)
// is K contiguous complex numbers, (re, im) interleaved. A complex product is
// one real product of doubled size:
//   L^[l][2k] = Lr[l][k], L^[l][2k+1] = Li[l][k]        (the natural row)
//   C^[2c][.] = (Cr0, -Ci0, Cr1, -Ci1, ...),  C^[2c+1][.] = (Ci0, Cr0, Ci1, Cr1, ...)
// so that (L^ C^T)[l][2c] = Re sum_k L C and [l][2c+1] = Im sum_k L C: the
// accumulator row of lane l holds (re, im) pairs, i.e. complex64 columns.
// One operand side L (the lane side) gives the MMA's 128 rows, the other side C
// gives its columns. For TF32 the inputs are split, x = hi + lo with hi = tf32(x)
// (round to nearest) and lo = tf32(x - hi); three products hi.hi + hi.lo + lo.hi
// ("3xTF32") keep the sum within FP32 accuracy, one product hi.hi is plain TF32.
//
// A tile: one slice, G values of batch indices (each its own accumulator), 128
// lane-side rows and Nt column-side rows. The host picks them by walking the output
// indices from the lowest, so the tile covers the longest prefix of output indices
// that tensor memory allows (two accumulator buffers of G x 2 Nt columns): a warp's
// outputs are then long contiguous runs. A work unit is one group value of a tile:
// its 128 lane-side rows are one TMA box (a multi-dimensional tensor map over the
// row bits they span) and its Nt column-side rows another.
//
// Warp roles (448 threads): warps 0-3 epilogue (tensor-memory lanes 0-127),
// warps 4-11 converters, warp 12 producer, warp 13 MMA issuer.
//   producer:   unit u's two boxes (cp.async.bulk.tensor) into raw slot u % SR -> raw_full
//   converters: raw rows -> split planes in the canonical no-swizzle K-major layout
//               (8-row x 16-byte core matrices), plane slot u % SP  -> op_full, raw_empty
//   issuer:     tcgen05.mma into accumulator (tile % 2, group), tcgen05.commit
//                                                                   -> op_empty, acc_full
//   epilogue:   per chunk of a warp's outputs: tcgen05.ld, power-of-two scale, a padded
//               shared-memory staging in output order, coalesced 16-byte stores of the
//               contiguous runs, max-abs                            -> acc_empty
// Every mbarrier wait is bounded in time: on a timeout the block raises the workspace
// status word, all roles leave their loops, the block waits (bounded) for its copies
// and products still in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "gemm.h"

namespace qt {

namespace {

// ------------------------------ device helpers ------------------------------

__device__ __forceinline__ unsigned long long u_pext64(unsigned long long x, unsigned long long m) {
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

__device__ __forceinline__ unsigned int u_pext32(unsigned int x, unsigned int m) {
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

__device__ __forceinline__ int u_scale_exp(unsigned int maxabs_bits) {
  if (maxabs_bits == 0u) return 0;
  const int s = (int)((maxabs_bits >> 23) & 0xffu) - 126;
  return max(-125, min(125, s));
}

__device__ __forceinline__ float u_pow2_neg(int s) { return __int_as_float((127 - s) << 23); }

__device__ __forceinline__ long long u_slice_base(const GOp& o, long long i,
                                                  unsigned long long sid) {
  long long off = o.base + i * o.slice_stride;
  if (o.smask) off += (long long)(u_pext64(sid, o.smask) << o.sshift);
  return off;
}

__device__ __forceinline__ unsigned int u_smem(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}

// every wait gives up after this many nanoseconds of the global timer
constexpr unsigned long long kUmmaWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long u_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

__device__ __forceinline__ void u_mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(u_smem(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void u_mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(u_smem(bar)) : "memory");
}
__device__ __forceinline__ void u_mbar_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(u_smem(bar)),
               "r"(bytes)
               : "memory");
}
// Wait for the phase of the given parity, bounded in time: non-blocking tests with a
// short sleep between them, giving up after kUmmaWaitNs of the global timer (then
// false, and *err raised).
__device__ __forceinline__ bool u_mbar_wait(unsigned long long* bar, unsigned int parity,
                                            int* err) {
  unsigned long long t0 = 0;
  for (unsigned int it = 0;; ++it) {
    unsigned int done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(u_smem(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) {
      t0 = u_now();
    } else if ((it & 63u) == 0u) {
      if (u_now() - t0 > kUmmaWaitNs) break;
    }
    if (it > 256u) __nanosleep(64);
  }
  if (err) atomicExch(err, 1);
  return false;
}

// one box of a 3- to 5-dimensional tensor map (coordinate 0 in every dimension but the
// last, the row offset) into shared memory, completing on the mbarrier
// one unit's box: x (floats, a multiple of 4) selects the chunk of the summed values
__device__ __forceinline__ void u_box(void* smem, const CUtensorMap* map, int rank, int x, int row,
                                      unsigned long long* bar) {
  const unsigned long long m = reinterpret_cast<unsigned long long>(map);
  if (rank == 3)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(u_smem(smem)),
        "l"(m), "r"(x), "r"(0), "r"(row), "r"(u_smem(bar))
        : "memory");
  else if (rank == 4)
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %3, %4}], [%5];\n" ::"r"(u_smem(smem)),
        "l"(m), "r"(x), "r"(0), "r"(row), "r"(u_smem(bar))
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %3, %3, %4}], [%5];\n" ::"r"(u_smem(smem)),
        "l"(m), "r"(x), "r"(0), "r"(row), "r"(u_smem(bar))
        : "memory");
}

__device__ __forceinline__ void u_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void u_tc_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void u_tc_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Shared-memory matrix descriptor of tcgen05.mma: start address, leading (K
// direction) and stride (8-row direction) byte offsets, all >> 4; version 1 at
// bit 46; layout type 0 (no swizzle) at bits 61-63.
__device__ __forceinline__ unsigned long long u_desc(unsigned int saddr, unsigned int lbo,
                                                     unsigned int sbo) {
  return (unsigned long long)((saddr >> 4) & 0x3fffu) |
         ((unsigned long long)((lbo >> 4) & 0x3fffu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma.kind::tf32: D F32 (bits 4-5 = 1), A and B
// TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr unsigned int u_idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned int)(n >> 3) << 17) |
         ((unsigned int)(m >> 4) << 24);
}

__device__ __forceinline__ void u_mma_tf32(unsigned int d_tmem, unsigned long long a_desc,
                                           unsigned long long b_desc, unsigned int idesc,
                                           int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// the mbarrier receives one arrival once every tcgen05.mma this thread issued before is done
__device__ __forceinline__ void u_mma_commit(unsigned long long* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          u_smem(bar))
      : "memory");
}

// N consecutive 32-bit columns of this thread's lane (N = 4, 8, 16, 32), into v[0..N)
template <int N>
__device__ __forceinline__ void u_tmem_ld(unsigned int taddr, float* v) {
  unsigned int* r = reinterpret_cast<unsigned int*>(v);
  if constexpr (N == 4) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
  } else if constexpr (N == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr)
        : "memory");
  } else if constexpr (N == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
  } else {
    static_assert(N == 32, "tcgen05.ld width");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
  }
}
__device__ __forceinline__ void u_tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ unsigned int u_tf32(float x) {
  unsigned int r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo (each a TF32 value in a 32-bit word)
__device__ __forceinline__ void u_split(float x, float& hi, float& lo) {
  const unsigned int h = u_tf32(x);
  hi = __uint_as_float(h);
  lo = __uint_as_float(u_tf32(x - hi));
}

__device__ __forceinline__ float u_absmax(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }


constexpr int kUmmaThreads = 448;
constexpr int kMaxRaw = 8, kMaxPlane = 4;

// byte offset of (row r, 16-byte chunk q) in a plane of R rows (canonical no-swizzle
// K-major: core matrices of 8 rows x 16 bytes, the R/8 of one chunk contiguous)
__device__ __forceinline__ unsigned int u_core_off(int r, int q, int R) {
  return (unsigned int)(q * (R * 16) + (r >> 3) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ unsigned int u_dep(unsigned int x, unsigned int m) {
  unsigned int v = 0u;
  for (int k = 0; m; ++k, m &= m - 1)
    if ((x >> k) & 1u) v |= m & (~m + 1u);
  return v;
}

// staging position of chunk-local output index e (complex): 2 complex of padding after
// every 16, so the rows of 16 lanes writing 16 complex apart fall in different banks
__device__ __forceinline__ unsigned int u_phys(unsigned int e) { return e + 2u * (e >> 4); }

template <int G, int CW>
__global__ void __launch_bounds__(kUmmaThreads, 1) k_gemm_umma(
    const GemmArgs a, const UmmaPlan p, const __grid_constant__ CUtensorMap mapL,
    const __grid_constant__ CUtensorMap mapC, float* data, GMeta* meta) {
  constexpr int CHUNK = 32 * CW * G;  // complex per epilogue chunk of a warp
  extern __shared__ float4 usm[];
  __shared__ alignas(8) unsigned long long s_raw_full[kMaxRaw], s_raw_empty[kMaxRaw];
  __shared__ alignas(8) unsigned long long s_op_full[kMaxPlane], s_op_empty[kMaxPlane];
  __shared__ alignas(8) unsigned long long s_acc_full[2], s_acc_empty[2];
  __shared__ unsigned int s_tmem;
  __shared__ volatile int s_fail;
  // abort path: the phase parity each raw slot's last copy completes and that of the
  // issuer's last commit on each plane slot (-1: none)
  __shared__ int s_fill_par[kMaxRaw], s_commit_par[kMaxPlane];

  const int nsum = p.nsum, kc = p.kc, lq = kc - 1;
  const int NC = 1 << (nsum - kc);    // chunks of the summed values per group
  const int Q = 1 << lq;              // 16-byte pieces per row chunk (2 complex each)
  const int Nt = 1 << p.cb, R2 = 2 * Nt;
  const int rowB = 8 << kc;           // bytes per row chunk
  const int SR = p.sraw, SP = p.splane;
  const GOp& OL = a.op[p.lside ? a.gB : a.gA];
  const GOp& OC = a.op[p.lside ? a.gA : a.gB];
  const int foldL = p.lside ? a.fold_b : a.fold_a, foldC = p.lside ? a.fold_a : a.fold_b;
  const long long scrL = p.lside ? a.scratch_b : a.scratch_a;
  const long long scrC = p.lside ? a.scratch_a : a.scratch_b;

  // shared memory (1024-byte aligned): raw units, plane slots, staging, run starts
  char* const base = reinterpret_cast<char*>(usm) + ((1024u - (u_smem(usm) & 1023u)) & 1023u);
  const unsigned int unitL = 128u * rowB, unit_b = (unitL + Nt * rowB + 1023u) & ~1023u;
  const unsigned int plL = 128u * rowB, plC = (unsigned int)R2 * rowB;
  const unsigned int plane_b =
      ((plL + plC) * (p.passes == 3 ? 2u : 1u) + 1023u) & ~1023u;  // Lhi, Chi, [Llo, Clo]
  char* const raw = base;
  char* const planes = raw + SR * unit_b;
  float2* const stage = reinterpret_cast<float2*>(planes + SP * plane_b);
  constexpr unsigned int kStageC = CHUNK + CHUNK / 8;  // complex per warp, padding included
  unsigned int* const runstart = reinterpret_cast<unsigned int*>(stage + 4 * kStageC);
  const int nruns = CHUNK >> p.rb;

  const long long per = 1ll << p.nrest;
  const long long ntiles = a.nslices * per;
  const long long chunk = (ntiles + gridDim.x - 1) / gridDim.x;
  const long long w0 = (long long)blockIdx.x * chunk;
  const long long w1 = min(ntiles, w0 + chunk);
  const long long nunits = w1 > w0 ? (w1 - w0) * G * NC : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kMaxRaw; ++s) {
      u_mbar_init(&s_raw_full[s], 1);
      u_mbar_init(&s_raw_empty[s], 256);
      s_fill_par[s] = -1;
    }
    for (int s = 0; s < kMaxPlane; ++s) {
      u_mbar_init(&s_op_full[s], 256);
      u_mbar_init(&s_op_empty[s], 1);
      s_commit_par[s] = -1;
    }
    for (int s = 0; s < 2; ++s) {
      u_mbar_init(&s_acc_full[s], 1);
      u_mbar_init(&s_acc_empty[s], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_fail = 0;
  }
  // the output offset of each run of a chunk (the chunk's bits above rb, deposited)
  {
    const unsigned int hi = p.chunk_out & ~((1u << p.rb) - 1u);
    for (int r = threadIdx.x; r < nruns; r += blockDim.x) runstart[r] = u_dep((unsigned)r, hi);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     u_smem(&s_tmem)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    u_tc_before_sync();
  }
  __syncthreads();
  u_tc_after_sync();
  const unsigned int tmem = s_tmem;
  // per rest bit k (lane k): its contribution to the tile's lane-side row, column-side
  // row and output offset (sums over the set bits of a tile number give the tile's)
  const unsigned int uL = OL.umask >> nsum, uC = OC.umask >> nsum;
  unsigned int kRow = 0u, kCol = 0u, kOut = 0u;
  if (lane < p.nrest) {
    const unsigned int bit = (1u << p.rest[lane]) >> nsum;
    kRow = u_pext32(bit, uL);
    kCol = u_pext32(bit, uC);
    kOut = bit;
  }

  if (warp == 12) {
    // ---------------- producer ----------------
    const unsigned int gl = lane < G ? u_pext32(u_dep((unsigned)lane, p.mgrp) >> nsum, uL) : 0u;
    const unsigned int gc = lane < G ? u_pext32(u_dep((unsigned)lane, p.mgrp) >> nsum, uC) : 0u;
    const int rankL = p.nlrun + 2, rankC = p.ncrun + 2;
    long long rowL0 = 0, rowC0 = 0;
    for (long long u = 0; u < nunits; ++u) {
      const int slot = (int)(u % SR);
      const long long gu = u / NC;  // unit u: group gu % G of tile gu / G, chunk u % NC
      const int c = (int)(u % NC);
      const int g = (int)(gu & (G - 1));
      if (g == 0 && c == 0) {
        const long long w = w0 + (gu / G);
        const long long i = w >> p.nrest;
        const unsigned int tp = (unsigned int)(w & (per - 1));
        const unsigned int on = (tp >> lane) & 1u;
        const unsigned int dl = __reduce_add_sync(0xffffffffu, on ? kRow : 0u);
        const unsigned int dc = __reduce_add_sync(0xffffffffu, on ? kCol : 0u);
        const unsigned long long sid = (unsigned long long)(a.slice_first + i);
        const long long bL = foldL ? scrL + i * a.scratch_stride : u_slice_base(OL, i, sid);
        const long long bC = foldC ? scrC + i * a.scratch_stride : u_slice_base(OC, i, sid);
        rowL0 = (bL >> nsum) + dl;
        rowC0 = (bC >> nsum) + dc;
      }
      const int rl = (int)(rowL0 + __shfl_sync(0xffffffffu, gl, g));
      const int rc = (int)(rowC0 + __shfl_sync(0xffffffffu, gc, g));
      bool ok = !s_fail;
      if (ok && u >= SR) ok = u_mbar_wait(&s_raw_empty[slot], (unsigned)(((u / SR) - 1) & 1), a.err);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        s_fail = 1;
        break;
      }
      if (lane == 0) {
        char* dst = raw + slot * unit_b;
        u_mbar_expect_tx(&s_raw_full[slot], unitL + (unsigned int)Nt * rowB);
        s_fill_par[slot] = (int)((u / SR) & 1);
        u_box(dst, &mapL, rankL, c << (kc + 1), rl, &s_raw_full[slot]);
        u_box(dst + unitL, &mapC, rankC, c << (kc + 1), rc, &s_raw_full[slot]);
      }
      __syncwarp();
    }
  } else if (warp >= 4 && warp < 12) {
    // ---------------- converters: raw rows -> split planes ----------------
    const int t = threadIdx.x - 128;
    for (long long u = 0; u < nunits; ++u) {
      const int slot = (int)(u % SR), ps = (int)(u % SP);
      bool ok = !s_fail && u_mbar_wait(&s_raw_full[slot], (unsigned)((u / SR) & 1), a.err);
      if (ok && u >= SP) ok = u_mbar_wait(&s_op_empty[ps], (unsigned)(((u / SP) - 1) & 1), a.err);
      if (!__all_sync(0xffffffffu, ok)) {
        s_fail = 1;
        break;
      }
      const char* src = raw + slot * unit_b;
      char* const pLhi = planes + ps * plane_b;
      char* const pChi = pLhi + plL;
      char* const pLlo = pChi + plC;
      char* const pClo = pLlo + plL;
      // lane side: the natural row, split
      const int nl = 128 << lq;
#pragma unroll 2
      for (int e = t; e < nl; e += 256) {
        const int r = e >> lq, q = e & (Q - 1);
        const float4 x = *reinterpret_cast<const float4*>(src + (size_t)e * 16);
        const unsigned int off = u_core_off(r, q, 128);
        float4 hi, lo;
        u_split(x.x, hi.x, lo.x);
        u_split(x.y, hi.y, lo.y);
        u_split(x.z, hi.z, lo.z);
        u_split(x.w, hi.w, lo.w);
        *reinterpret_cast<float4*>(pLhi + off) = hi;
        if (p.passes == 3) *reinterpret_cast<float4*>(pLlo + off) = lo;
      }
      // column side: each row becomes its (re) and (im) rows 2c, 2c+1
      const int nc = Nt << lq;
      for (int e = t; e < nc; e += 256) {
        const int c = e >> lq, q = e & (Q - 1);
        const float4 x = *reinterpret_cast<const float4*>(src + unitL + (size_t)e * 16);
        const float4 xr = make_float4(x.x, -x.y, x.z, -x.w);
        const float4 xi = make_float4(x.y, x.x, x.w, x.z);
        const unsigned int offr = u_core_off(2 * c, q, R2), offi = u_core_off(2 * c + 1, q, R2);
        float4 hr, lr, hm, lm;
        u_split(xr.x, hr.x, lr.x);
        u_split(xr.y, hr.y, lr.y);
        u_split(xr.z, hr.z, lr.z);
        u_split(xr.w, hr.w, lr.w);
        u_split(xi.x, hm.x, lm.x);
        u_split(xi.y, hm.y, lm.y);
        u_split(xi.z, hm.z, lm.z);
        u_split(xi.w, hm.w, lm.w);
        *reinterpret_cast<float4*>(pChi + offr) = hr;
        *reinterpret_cast<float4*>(pChi + offi) = hm;
        if (p.passes == 3) {
          *reinterpret_cast<float4*>(pClo + offr) = lr;
          *reinterpret_cast<float4*>(pClo + offi) = lm;
        }
      }
      u_fence_proxy_async();  // the planes, written by threads, are read by the tensor cores
      u_mbar_arrive(&s_op_full[ps]);
      u_mbar_arrive(&s_raw_empty[slot]);
    }
  } else if (warp == 13) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const unsigned int idesc = u_idesc_tf32(128, R2);
      const unsigned int lboL = 128 * 16, lboC = (unsigned int)R2 * 16;
      const int ksteps = (2 << kc) / 8;  // the doubled chunk over 8 per tf32 MMA
      for (long long u = 0; u < nunits; ++u) {
        const int ps = (int)(u % SP);
        const long long gu = u / NC;
        const long long j = gu / G;
        const int c = (int)(u % NC);
        const int g = (int)(gu & (G - 1)), b = (int)(j & 1);
        bool ok = !s_fail && u_mbar_wait(&s_op_full[ps], (unsigned)((u / SP) & 1), a.err);
        if (ok && g == 0 && c == 0 && j >= 2)
          ok = u_mbar_wait(&s_acc_empty[b], (unsigned)(((j >> 1) - 1) & 1), a.err);
        if (!ok) {
          s_fail = 1;
          break;
        }
        u_tc_after_sync();
        const unsigned int pL = u_smem(planes + ps * plane_b);
        const unsigned int aLhi = pL, aChi = pL + plL, aLlo = aChi + plC, aClo = aLlo + plL;
        const unsigned int d = tmem + (unsigned int)((b * G + g) * R2);
        int acc = c > 0 ? 1 : 0;  // a group's later chunks add to its accumulator
        // (lo, hi), (hi, lo) first: the small terms accumulate before the large one
        for (int pass = (p.passes == 3 ? 0 : 2); pass < 3; ++pass) {
          const unsigned int la = pass == 0 ? aLlo : aLhi;
          const unsigned int cb = pass == 1 ? aClo : aChi;
          for (int k = 0; k < ksteps; ++k) {
            u_mma_tf32(d, u_desc(la + (unsigned int)k * 2 * lboL, lboL, 128),
                       u_desc(cb + (unsigned int)k * 2 * lboC, lboC, 128), idesc, acc);
            acc = 1;
          }
        }
        u_mma_commit(&s_op_empty[ps]);
        s_commit_par[ps] = (int)((u / SP) & 1);
        if (g == G - 1 && c == NC - 1) u_mma_commit(&s_acc_full[b]);
      }
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---------------- epilogue: warps 0-3, tensor-memory lanes 0-127 ----------------
    // chunk-local output positions (additive over disjoint bit sets) of this lane, of
    // each group and of each column inside a chunk
    const unsigned int lowcols = u_dep((1u << p.cwb) - 1u, p.mcol);
    const unsigned int sL = u_pext32(u_dep((unsigned)lane, p.mlane) >> nsum, p.chunk_out);
    const unsigned int outW = u_dep((unsigned)(warp * 32), p.mlane) >> nsum;  // lanes 5, 6
    unsigned int sG[G], sC[CW];
#pragma unroll
    for (int g = 0; g < G; ++g) sG[g] = u_pext32(u_dep((unsigned)g, p.mgrp) >> nsum, p.chunk_out);
#pragma unroll
    for (int c = 0; c < CW; ++c) sC[c] = u_pext32(u_dep((unsigned)c, lowcols) >> nsum, p.chunk_out);
    const unsigned int trow = tmem + ((unsigned int)(warp * 32) << 16);
    float2* const d2 = reinterpret_cast<float2*>(data);
    float2* const stg = stage + warp * kStageC;
    const int nchunks = Nt / CW;
    long long cur = -1;
    float mx = 0.f, sc = 1.f;
    for (long long j = 0; w0 + j < w1; ++j) {
      const int b = (int)(j & 1);
      const bool ok = !s_fail && u_mbar_wait(&s_acc_full[b], (unsigned)((j >> 1) & 1), a.err);
      if (!__all_sync(0xffffffffu, ok)) {
        s_fail = 1;
        break;
      }
      u_tc_after_sync();
      const long long w = w0 + j;
      const long long ti = w >> p.nrest;
      const unsigned int tp = (unsigned int)(w & (per - 1));
      const unsigned int tout = __reduce_add_sync(0xffffffffu, ((tp >> lane) & 1u) ? kOut : 0u);
      if (ti != cur) {
        if (cur >= 0) {
          const unsigned int v = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
          if (lane == 0 && v)
            atomicMax(&meta[a.out_meta + (a.out_meta_per_slice ? cur : 0)].maxabs, v);
        }
        mx = 0.f;
        cur = ti;
        sc = (a.fold_a ? 1.f
                       : u_pow2_neg(u_scale_exp(meta[a.op[a.gA].meta +
                                                     (a.op[a.gA].meta_per_slice ? cur : 0)].maxabs))) *
             (a.fold_b ? 1.f
                       : u_pow2_neg(u_scale_exp(meta[a.op[a.gB].meta +
                                                     (a.op[a.gB].meta_per_slice ? cur : 0)].maxabs)));
        if (tp == 0u && threadIdx.x == 0) {
          int E = 0;
          for (int q = 0; q < a.m; ++q) {
            const GOp& o = a.op[q];
            const GMeta mt = meta[o.meta + (o.meta_per_slice ? cur : 0)];
            E += mt.E + u_scale_exp(mt.maxabs);
          }
          meta[a.out_meta + (a.out_meta_per_slice ? cur : 0)].E = E;
        }
      }
      const long long obase = a.out_base + ti * a.out_slice_stride + (long long)(tout + outW);
      for (int k = 0; k < nchunks; ++k) {
        float v[G][2 * CW];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const unsigned int col = (unsigned int)((b * G + g) * R2 + 2 * k * CW);
          if constexpr (2 * CW <= 32) {
            u_tmem_ld<2 * CW>(trow + col, v[g]);
          } else {
            u_tmem_ld<32>(trow + col, v[g]);
            u_tmem_ld<32>(trow + col + 32, v[g] + 32);
          }
        }
        u_tmem_wait_ld();
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
          for (int c = 0; c < CW; ++c) {
            const float2 z = make_float2(v[g][2 * c] * sc, v[g][2 * c + 1] * sc);
            mx = fmaxf(mx, u_absmax(z));
            stg[u_phys(sL + sG[g] + sC[c])] = z;
          }
        __syncwarp();
        const long long cbase = obase + (long long)(u_dep((unsigned)(k << p.cwb), p.mcol) >> nsum);
        const unsigned int rmask = (1u << p.rb) - 1u;
#pragma unroll 4
        for (int it = 0; it < CHUNK / 64; ++it) {
          const unsigned int e = 2u * (unsigned)(lane + 32 * it);
          const float4 val = *reinterpret_cast<const float4*>(stg + u_phys(e));
          *reinterpret_cast<float4*>(d2 + cbase + runstart[e >> p.rb] + (e & rmask)) = val;
        }
        __syncwarp();
      }
      u_tc_before_sync();
      u_mbar_arrive(&s_acc_empty[b]);
    }
    if (cur >= 0) {
      const unsigned int v = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
      if (lane == 0 && v) atomicMax(&meta[a.out_meta + (a.out_meta_per_slice ? cur : 0)].maxabs, v);
    }
  }
  __syncthreads();
  if (s_fail) {
    // bounded waits for what may still be in flight: each raw slot's last copy and the
    // issuer's last products (a phase already passed returns at once)
    if (threadIdx.x == 12 * 32)
      for (int s = 0; s < kMaxRaw; ++s)
        if (s_fill_par[s] >= 0) u_mbar_wait(&s_raw_full[s], (unsigned)s_fill_par[s], nullptr);
    if (threadIdx.x == 13 * 32)
      for (int s = 0; s < kMaxPlane; ++s)
        if (s_commit_par[s] >= 0) u_mbar_wait(&s_op_empty[s], (unsigned)s_commit_par[s], nullptr);
    __syncthreads();
  }
  if (warp == 0) {
    u_tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

}  // namespace

// ------------------------------------ host ------------------------------------

namespace {

typedef CUresult (*UEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

UEncodeFn u_encode() {
  static UEncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault,
                                         &r) == cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<UEncodeFn>(q);
  }
  return fn;
}

// The workspace seen as: rows of 2^nsum complex (dimension 0, 2^(nsum+1) floats), one
// dimension per run of row bits (extent 2^len, stride 2^start rows) and a last
// dimension of single rows (the box's origin row). The box: whole rows, every run,
// one origin -- the rows of one unit, in the order of their row bits.
bool u_unit_map(CUtensorMap& m, float* data, long long ws_elems, int nsum, int kc, int nrun,
                const int* start, const int* len) {
  UEncodeFn fn = u_encode();
  const long long K = 1ll << nsum;
  const long long rows = ws_elems / K;
  if (!fn || rows < 1 || rows > 0x7fffffffll || kc < 2 || kc > nsum || (2 << kc) > 256 ||
      nrun < 1 || nrun > 3)
    return false;
  const int rank = nrun + 2;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5];
  dims[0] = (cuuint64_t)(2 * K);
  box[0] = (cuuint32_t)(2 << kc);  // one chunk of the row
  for (int r = 0; r < nrun; ++r) {
    dims[1 + r] = (cuuint64_t)1 << len[r];
    strides[r] = (cuuint64_t)(K * 8) << start[r];
    box[1 + r] = (cuuint32_t)1 << len[r];
  }
  dims[rank - 1] = (cuuint64_t)rows;
  strides[rank - 2] = (cuuint64_t)(K * 8);
  box[rank - 1] = 1;
  for (int d = 0; d < rank; ++d) estr[d] = 1;
  return fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, data, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr size_t kUmmaSmemMax = 225 * 1024;

unsigned int lowest_bits(unsigned int m, int n) {
  unsigned int r = 0;
  for (int k = 0; k < n && m; ++k, m &= m - 1) r |= m & (~m + 1u);
  return r;
}

// runs of consecutive positions among the row bits of `bits` in an operand with index
// mask umask (row bit = the operand's index bit minus nsum); false if more than 3
bool row_runs(unsigned int bits, unsigned int umask, int nsum, int& n, int* start, int* len) {
  n = 0;
  int prev = -2;
  for (unsigned int m = bits; m; m &= m - 1) {
    const int ub = __builtin_ctz(m);
    const int rbit = __builtin_popcount(umask & ((1u << ub) - 1u)) - nsum;
    if (rbit == prev + 1) {
      ++len[n - 1];
    } else {
      if (n == 3) return false;
      start[n] = rbit;
      len[n] = 1;
      ++n;
    }
    prev = rbit;
  }
  return n >= 1;
}

}  // namespace

size_t umma_smem(const UmmaPlan& p) {
  const int G = 1 << p.gb, Nt = 1 << p.cb;
  const size_t rowB = (size_t)8 << p.kc;
  const size_t unit = (((size_t)(128 + Nt) * rowB) + 1023) & ~(size_t)1023;
  const size_t plane = (((size_t)(128 + 2 * Nt) * rowB * (p.passes == 3 ? 2 : 1)) + 1023) & ~(size_t)1023;
  const int cw = 1 << p.cwb;
  const size_t chunk = (size_t)32 * cw * G;
  const size_t stage = 4 * (chunk + chunk / 8) * 8;
  const size_t runs = (chunk >> p.rb) * 4;
  return 1024 + (size_t)p.sraw * unit + (size_t)p.splane * plane + stage + runs;
}

bool umma_plan(const GemmArgs& a, int passes, UmmaPlan& best) {
  best = UmmaPlan{};
  if (a.mSA || a.mSB || a.gA < 0 || a.gB < 0 || a.nsum < 2 || a.nsum > 6) return false;
  if (passes != 1 && passes != 3) return false;
  const int ns = a.nsum;
  if (a.mK != (1u << ns) - 1u) return false;
  int u = 0;
  for (unsigned int m = a.mK | a.mM | a.mN | a.mBt; m; m >>= 1) ++u;
  bool found = false;
  for (int lside = 0; lside < 2; ++lside) {
    UmmaPlan p{};
    const unsigned int lonly = lside ? a.mN : a.mM, conly = lside ? a.mM : a.mN;
    if (__builtin_popcount(lonly) < 7 || __builtin_popcount(conly) < 3) continue;
    p.lside = lside;
    p.nsum = ns;
    p.passes = passes;
    p.mlane = lowest_bits(lonly, 7);
    // walk the output indices from the lowest while the tile can take them: two
    // accumulator buffers of G x 2 Nt columns (Nt at least 8) in 512, G at most 16
    int G = 1, Nt = 1, b = ns;
    for (; b < u; ++b) {
      const unsigned int bit = 1u << b;
      if (bit & p.mlane) continue;
      if (bit & lonly) break;
      if (bit & a.mBt) {
        // (wide products: only the batch indices among the two lowest output indices)
        if (2 * G > 16 || 2 * G * std::max(Nt, 8) > 128 || (a.umma_shape == 1 && b > ns + 1))
          break;
        p.mgrp |= bit;
        G *= 2;
        continue;
      }
      if (2 * Nt > 128 || G * std::max(2 * Nt, 8) > 128) break;
      p.mcol |= bit;
      Nt *= 2;
    }
    p.prefix = b - ns;
    // the MMA's N is at least 16; wide products: as many columns as tensor memory holds
    const int want = a.umma_shape == 1 ? std::min(128, 128 / G) : 8;
    while (Nt < want) {
      const unsigned int m = conly & ~p.mcol;
      if (!m) break;
      p.mcol |= m & (~m + 1u);
      Nt *= 2;
    }
    if (Nt < 8) continue;
    p.cb = __builtin_ctz((unsigned)Nt);
    p.gb = __builtin_ctz((unsigned)G);
    const unsigned int uL = a.op[lside ? a.gB : a.gA].umask, uC = a.op[lside ? a.gA : a.gB].umask;
    if (!row_runs(p.mlane, uL, ns, p.nlrun, p.lrun_start, p.lrun_len)) continue;
    if (!row_runs(p.mcol, uC, ns, p.ncrun, p.crun_start, p.crun_len)) continue;
    // epilogue chunks: 32 lanes x CW columns x G groups, at most 1024 complex
    const int cw = std::min(Nt, 32 / G);
    p.cwb = __builtin_ctz((unsigned)cw);
    const unsigned int lanes5 = lowest_bits(p.mlane, 5);
    p.chunk_out = (p.mgrp | lanes5 | lowest_bits(p.mcol, p.cwb)) >> ns;
    p.rb = 0;
    while ((p.chunk_out >> p.rb) & 1u) ++p.rb;
    if (p.rb < 1) continue;
    // the tiles: the column side's further indices vary fastest (consecutive tiles
    // share the lane-side rows), then everything else from the lowest up
    const unsigned int outall = (a.mM | a.mN | a.mBt) & ~((1u << ns) - 1u);
    const unsigned int restm = outall & ~(p.mlane | p.mcol | p.mgrp);
    p.nrest = 0;
    for (unsigned int m = restm & conly; m; m &= m - 1) p.rest[p.nrest++] = __builtin_ctz(m);
    for (unsigned int m = restm & ~conly; m; m &= m - 1) p.rest[p.nrest++] = __builtin_ctz(m);
    if (p.nrest > 31) continue;
    int cols = 32;
    while (cols < 4 * G * Nt) cols <<= 1;
    if (cols > 512) continue;
    p.tmem_cols = cols;
    // as many units of raw rows in flight as shared memory holds (TMA latency), then
    // plane slots (converters ahead of the tensor cores)
    p.sraw = 2;
    p.splane = 1;
    // the summed values in chunks (at least 4 complex: one tf32 MMA of K = 8) when the
    // whole rows of two raw units and a plane slot do not fit
    p.kc = a.umma_kc_max > 0 ? std::min(ns, std::max(2, a.umma_kc_max)) : ns;
    while (p.kc > 2 && umma_smem(p) > kUmmaSmemMax) --p.kc;
    if (p.kc < ns) {
      // chunked anyway: smaller chunks for 4 raw units and 2 plane slots in flight
      p.sraw = 4;
      p.splane = 2;
      while (p.kc > 2 && umma_smem(p) > kUmmaSmemMax) --p.kc;
      if (umma_smem(p) > kUmmaSmemMax) {
        p.sraw = 2;
        p.splane = 1;
      }
    }
    if (umma_smem(p) > kUmmaSmemMax) continue;
    for (bool grew = true; grew;) {
      grew = false;
      if (p.sraw < kMaxRaw) {
        ++p.sraw;
        if (umma_smem(p) <= kUmmaSmemMax) grew = true;
        else --p.sraw;
      }
      if (p.splane < kMaxPlane && p.sraw >= 4) {
        ++p.splane;
        if (umma_smem(p) <= kUmmaSmemMax) grew = true;
        else --p.splane;
      }
    }
    if (!found || p.prefix > best.prefix) {
      best = p;
      found = true;
    }
  }
  return found;
}

typedef void (*UmmaFn)(const GemmArgs, const UmmaPlan, const CUtensorMap, const CUtensorMap,
                       float*, GMeta*);

static UmmaFn umma_fn(int gb, int cwb) {
  const int G = 1 << gb, CW = 1 << cwb;
  if (G == 16 && CW == 2) return k_gemm_umma<16, 2>;
  if (G == 8 && CW == 4) return k_gemm_umma<8, 4>;
  if (G == 4 && CW == 8) return k_gemm_umma<4, 8>;
  if (G == 2 && CW == 16) return k_gemm_umma<2, 16>;
  if (G == 2 && CW == 8) return k_gemm_umma<2, 8>;
  if (G == 1 && CW == 32) return k_gemm_umma<1, 32>;
  if (G == 1 && CW == 16) return k_gemm_umma<1, 16>;
  if (G == 1 && CW == 8) return k_gemm_umma<1, 8>;
  return nullptr;
}

bool umma_rows_aligned(const GemmArgs& a) {
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

bool umma_launch(const GemmArgs& a, const UmmaPlan& p, float* data, GMeta* meta, cudaStream_t s,
                 int sms) {
  UmmaFn fn = umma_fn(p.gb, p.cwb);
  if (!fn || !a.err || !umma_rows_aligned(a)) return false;
  // the epilogue's 16-byte stores start on 2-complex boundaries of the output
  if (a.out_base % 2 || a.out_slice_stride % 2) return false;
  CUtensorMap mL, mC;
  if (!u_unit_map(mL, data, a.ws_elems, p.nsum, p.kc, p.nlrun, p.lrun_start, p.lrun_len) ||
      !u_unit_map(mC, data, a.ws_elems, p.nsum, p.kc, p.ncrun, p.crun_start, p.crun_len))
    return false;
  const size_t smem = umma_smem(p);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return false;
  const long long ntiles = a.nslices << p.nrest;
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(ntiles, sms));
  fn<<<grid, kUmmaThreads, smem, s>>>(a, p, mL, mC, data, meta);
  return true;
}

}  // namespace qt
