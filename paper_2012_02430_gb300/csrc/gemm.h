// Launch arguments of the GEMM form of a fused bucket launch (gemm.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

namespace qt {

enum { GEMM_SIMT = 0, GEMM_TC_TF32 = 1, GEMM_TC_BF16 = 2, GEMM_TC_3XTF32 = 3 };

constexpr int GEMM_MAXOP = 12;

struct GMeta {
  unsigned int maxabs;
  int E;
};

struct GOp {
  long long base, slice_stride, meta;
  unsigned int umask, smask;
  int sshift, meta_per_slice, side, pad;
};

struct GemmArgs {
  int m, nsum;
  unsigned int mK, mSA, mSB, mM, mN, mBt;
  long long nslices, slice_first;
  long long out_base, out_slice_stride, out_meta;
  int out_meta_per_slice, pad;
  long long scratch_a, scratch_b, scratch_stride;  // elements (complex64 units)
  GOp op[GEMM_MAXOP];
};

// pack A', pack B', GEMM; returns the number of kernels launched
int gemm_launch(const GemmArgs& a, int mode, float* data, GMeta* meta, cudaStream_t s, int sms);

}  // namespace qt
