// The proposal network's training kernels: a 2-hidden-layer ReLU MLP
// x (F) -> H -> H -> 1, trained on the GPU with mean-squared error and Adam.
// Parameter layout (one float array): W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
// Every reduction is a fixed-order loop of one thread, so results are
// reproducible run to run (the gradient check compares them with FP64 NumPy).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qt_internal.h"

namespace qt {
void set_last_error(const std::string& msg);
int mlp_param_count(int nf, int hidden);
}  // namespace qt

struct qt_mlp {
  int nf = 0, hidden = 0, max_batch = 0, params = 0;
  int64_t t = 0;  // Adam step
  size_t off_p = 0, off_g = 0, off_m = 0, off_v = 0, off_h1 = 0, off_h2 = 0, off_y = 0, off_dy = 0,
         off_d2 = 0, off_d1 = 0, off_loss = 0, total = 0;
};

namespace {

struct Net {
  const float *W1, *b1, *W2, *b2, *w3, *b3;
};

__device__ __forceinline__ Net net_of(const float* p, int F, int H) {
  Net n;
  n.W1 = p;
  n.b1 = n.W1 + H * F;
  n.W2 = n.b1 + H;
  n.b2 = n.W2 + H * H;
  n.w3 = n.b2 + H;
  n.b3 = n.w3 + H;
  return n;
}

__global__ void k_fwd1(const float* p, int F, int H, const float* x, int B, float* h1) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * H) return;
  const int b = idx / H, j = idx % H;
  const Net n = net_of(p, F, H);
  float a = n.b1[j];
  for (int i = 0; i < F; ++i) a += n.W1[j * F + i] * x[b * F + i];
  h1[idx] = a > 0.f ? a : 0.f;
}

__global__ void k_fwd2(const float* p, int F, int H, const float* h1, int B, float* h2) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * H) return;
  const int b = idx / H, j = idx % H;
  const Net n = net_of(p, F, H);
  float a = n.b2[j];
  for (int i = 0; i < H; ++i) a += n.W2[j * H + i] * h1[b * H + i];
  h2[idx] = a > 0.f ? a : 0.f;
}

__global__ void k_fwd3(const float* p, int F, int H, const float* h2, int B, float* y) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const Net n = net_of(p, F, H);
  float a = n.b3[0];
  for (int i = 0; i < H; ++i) a += n.w3[i] * h2[b * H + i];
  y[b] = a;
}

// loss = mean (y - t)^2 and dL/dy (one block, fixed order)
__global__ void __launch_bounds__(256) k_loss(const float* y, const float* t, int B, float* dy,
                                              float* loss) {
  __shared__ float sh[256];
  float acc = 0.f;
  for (int b = threadIdx.x; b < B; b += 256) {
    const float d = y[b] - t[b];
    dy[b] = 2.f * d / (float)B;
    acc += d * d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / (float)B;
}

__global__ void k_bwd2(const float* p, int F, int H, const float* dy, const float* h2, int B,
                       float* d2) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * H) return;
  const int b = idx / H, j = idx % H;
  const Net n = net_of(p, F, H);
  d2[idx] = h2[idx] > 0.f ? dy[b] * n.w3[j] : 0.f;
}

__global__ void k_bwd1(const float* p, int F, int H, const float* d2, const float* h1, int B,
                       float* d1) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * H) return;
  const int b = idx / H, i = idx % H;
  const Net n = net_of(p, F, H);
  float a = 0.f;
  for (int j = 0; j < H; ++j) a += d2[b * H + j] * n.W2[j * H + i];
  d1[idx] = h1[idx] > 0.f ? a : 0.f;
}

// gradient of every parameter: one thread each, summing over the batch in order
__global__ void k_grad(int F, int H, const float* x, const float* h1, const float* h2,
                       const float* dy, const float* d2, const float* d1, int B, float* g) {
  const int P = H * F + H + H * H + H + H + 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  float a = 0.f;
  int r = k;
  if (r < H * F) {
    const int j = r / F, i = r % F;
    for (int b = 0; b < B; ++b) a += d1[b * H + j] * x[b * F + i];
  } else if ((r -= H * F) < H) {
    for (int b = 0; b < B; ++b) a += d1[b * H + r];
  } else if ((r -= H) < H * H) {
    const int j = r / H, i = r % H;
    for (int b = 0; b < B; ++b) a += d2[b * H + j] * h1[b * H + i];
  } else if ((r -= H * H) < H) {
    for (int b = 0; b < B; ++b) a += d2[b * H + r];
  } else if ((r -= H) < H) {
    for (int b = 0; b < B; ++b) a += dy[b] * h2[b * H + r];
  } else {
    for (int b = 0; b < B; ++b) a += dy[b];
  }
  g[k] = a;
}

// Adam (Kingma and Ba 2015): bias corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t
__global__ void k_adam(float* p, const float* g, float* m, float* v, int P, float lr, float beta1,
                       float beta2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const float gk = g[k];
  const float mk = beta1 * m[k] + (1.f - beta1) * gk;
  const float vk = beta2 * v[k] + (1.f - beta2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float mh = mk / c1, vh = vk / c2;
  p[k] -= lr * mh / (sqrtf(vh) + eps);
}

qt_status fail(qt_status s, const std::string& msg) {
  qt::set_last_error(msg);
  return s;
}

bool ok_cuda(cudaError_t e, const char* what, std::string& err) {
  if (e == cudaSuccess) return true;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

qt_status check(const qt_mlp* M, void* ws, size_t bytes, const char* who) {
  if (!M || !ws) return fail(QT_EINVAL, std::string(who) + ": null argument");
  if ((uintptr_t)ws % 256) return fail(QT_EINVAL, std::string(who) + ": workspace not 256-byte aligned");
  if (bytes < M->total) return fail(QT_ENOMEM, std::string(who) + ": workspace too small");
  return QT_OK;
}

// forward pass into the workspace activations
void forward(const qt_mlp* M, char* ws, const float* x, int B, cudaStream_t s) {
  const float* p = reinterpret_cast<const float*>(ws + M->off_p);
  float* h1 = reinterpret_cast<float*>(ws + M->off_h1);
  float* h2 = reinterpret_cast<float*>(ws + M->off_h2);
  float* y = reinterpret_cast<float*>(ws + M->off_y);
  const int n = B * M->hidden;
  k_fwd1<<<(n + 255) / 256, 256, 0, s>>>(p, M->nf, M->hidden, x, B, h1);
  k_fwd2<<<(n + 255) / 256, 256, 0, s>>>(p, M->nf, M->hidden, h1, B, h2);
  k_fwd3<<<(B + 255) / 256, 256, 0, s>>>(p, M->nf, M->hidden, h2, B, y);
}

void backward(const qt_mlp* M, char* ws, const float* x, const float* t, int B, float* loss,
              cudaStream_t s) {
  const float* p = reinterpret_cast<const float*>(ws + M->off_p);
  float* g = reinterpret_cast<float*>(ws + M->off_g);
  const float* h1 = reinterpret_cast<const float*>(ws + M->off_h1);
  const float* h2 = reinterpret_cast<const float*>(ws + M->off_h2);
  const float* y = reinterpret_cast<const float*>(ws + M->off_y);
  float* dy = reinterpret_cast<float*>(ws + M->off_dy);
  float* d2 = reinterpret_cast<float*>(ws + M->off_d2);
  float* d1 = reinterpret_cast<float*>(ws + M->off_d1);
  const int n = B * M->hidden;
  k_loss<<<1, 256, 0, s>>>(y, t, B, dy, loss);
  k_bwd2<<<(n + 255) / 256, 256, 0, s>>>(p, M->nf, M->hidden, dy, h2, B, d2);
  k_bwd1<<<(n + 255) / 256, 256, 0, s>>>(p, M->nf, M->hidden, d2, h1, B, d1);
  k_grad<<<(M->params + 127) / 128, 128, 0, s>>>(M->nf, M->hidden, x, h1, h2, dy, d2, d1, B, g);
}

}  // namespace

extern "C" {

qt_status qt_mlp_create(int32_t n_features, int32_t hidden, int32_t max_batch, qt_mlp** out) {
  if (!out) return fail(QT_EINVAL, "qt_mlp_create: out is NULL");
  *out = nullptr;
  if (n_features < 1 || hidden < 1 || max_batch < 1 || n_features > 1024 || hidden > 1024 ||
      max_batch > (1 << 24))
    return fail(QT_EINVAL, "qt_mlp_create: sizes out of range");
  qt_mlp* M = new (std::nothrow) qt_mlp();
  if (!M) return fail(QT_ENOMEM, "qt_mlp_create: out of host memory");
  M->nf = n_features;
  M->hidden = hidden;
  M->max_batch = max_batch;
  M->params = qt::mlp_param_count(n_features, hidden);
  const size_t P = (size_t)M->params * 4, BH = (size_t)max_batch * hidden * 4,
               B = (size_t)max_batch * 4;
  size_t off = 0;
  M->off_p = off; off = a256(off + P);
  M->off_g = off; off = a256(off + P);
  M->off_m = off; off = a256(off + P);
  M->off_v = off; off = a256(off + P);
  M->off_h1 = off; off = a256(off + BH);
  M->off_h2 = off; off = a256(off + BH);
  M->off_y = off; off = a256(off + B);
  M->off_dy = off; off = a256(off + B);
  M->off_d2 = off; off = a256(off + BH);
  M->off_d1 = off; off = a256(off + BH);
  M->off_loss = off; off = a256(off + 16);
  M->total = off;
  *out = M;
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_mlp_workspace_size(const qt_mlp* M, size_t* bytes, int32_t* n_params) {
  if (!M) return fail(QT_EINVAL, "qt_mlp_workspace_size: null handle");
  if (bytes) *bytes = M->total;
  if (n_params) *n_params = M->params;
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_mlp_set_params(qt_mlp* M, void* ws, size_t bytes, const float* params, void* stream) {
  qt_status s = check(M, ws, bytes, "qt_mlp_set_params");
  if (s != QT_OK) return s;
  if (!params) return fail(QT_EINVAL, "qt_mlp_set_params: null params");
  std::string err;
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  const size_t P = (size_t)M->params * 4;
  if (!ok_cuda(cudaMemcpyAsync(base + M->off_p, params, P, cudaMemcpyHostToDevice, st), "params", err) ||
      !ok_cuda(cudaMemsetAsync(base + M->off_m, 0, P, st), "adam m", err) ||
      !ok_cuda(cudaMemsetAsync(base + M->off_v, 0, P, st), "adam v", err) ||
      !ok_cuda(cudaStreamSynchronize(st), "sync", err))
    return fail(QT_ECUDA, "qt_mlp_set_params: " + err);
  M->t = 0;
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_mlp_get_params(const qt_mlp* M, void* ws, size_t bytes, float* params, void* stream) {
  qt_status s = check(M, ws, bytes, "qt_mlp_get_params");
  if (s != QT_OK) return s;
  if (!params) return fail(QT_EINVAL, "qt_mlp_get_params: null params");
  std::string err;
  cudaStream_t st = (cudaStream_t)stream;
  if (!ok_cuda(cudaMemcpyAsync(params, (char*)ws + M->off_p, (size_t)M->params * 4,
                               cudaMemcpyDeviceToHost, st), "params", err) ||
      !ok_cuda(cudaStreamSynchronize(st), "sync", err))
    return fail(QT_ECUDA, "qt_mlp_get_params: " + err);
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_mlp_forward(qt_mlp* M, void* ws, size_t bytes, const float* d_x, int32_t batch,
                         float* d_y, void* stream) {
  qt_status s = check(M, ws, bytes, "qt_mlp_forward");
  if (s != QT_OK) return s;
  if (!d_x || !d_y || batch < 1 || batch > M->max_batch)
    return fail(QT_EINVAL, "qt_mlp_forward: bad input, output or batch");
  cudaStream_t st = (cudaStream_t)stream;
  forward(M, (char*)ws, d_x, batch, st);
  std::string err;
  if (!ok_cuda(cudaMemcpyAsync(d_y, (char*)ws + M->off_y, (size_t)batch * 4,
                               cudaMemcpyDeviceToDevice, st), "copy y", err) ||
      !ok_cuda(cudaGetLastError(), "launch", err))
    return fail(QT_ECUDA, "qt_mlp_forward: " + err);
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_mlp_gradients(qt_mlp* M, void* ws, size_t bytes, const float* d_x, const float* d_t,
                           int32_t batch, float* d_grad, float* d_loss, void* stream) {
  qt_status s = check(M, ws, bytes, "qt_mlp_gradients");
  if (s != QT_OK) return s;
  if (!d_x || !d_t || !d_grad || !d_loss || batch < 1 || batch > M->max_batch)
    return fail(QT_EINVAL, "qt_mlp_gradients: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  forward(M, base, d_x, batch, st);
  backward(M, base, d_x, d_t, batch, d_loss, st);
  std::string err;
  if (!ok_cuda(cudaMemcpyAsync(d_grad, base + M->off_g, (size_t)M->params * 4,
                               cudaMemcpyDeviceToDevice, st), "copy grad", err) ||
      !ok_cuda(cudaGetLastError(), "launch", err))
    return fail(QT_ECUDA, "qt_mlp_gradients: " + err);
  qt::set_last_error("");
  return QT_OK;
}

qt_status qt_mlp_train_step(qt_mlp* M, void* ws, size_t bytes, const float* d_x, const float* d_t,
                            int32_t batch, float lr, float* d_loss, void* stream) {
  qt_status s = check(M, ws, bytes, "qt_mlp_train_step");
  if (s != QT_OK) return s;
  if (!d_x || !d_t || !d_loss || batch < 1 || batch > M->max_batch || !(lr > 0.f))
    return fail(QT_EINVAL, "qt_mlp_train_step: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  forward(M, base, d_x, batch, st);
  backward(M, base, d_x, d_t, batch, d_loss, st);
  M->t += 1;
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 - std::pow((double)beta1, (double)M->t));
  const float c2 = (float)(1.0 - std::pow((double)beta2, (double)M->t));
  k_adam<<<(M->params + 255) / 256, 256, 0, st>>>(
      reinterpret_cast<float*>(base + M->off_p), reinterpret_cast<const float*>(base + M->off_g),
      reinterpret_cast<float*>(base + M->off_m), reinterpret_cast<float*>(base + M->off_v),
      M->params, lr, beta1, beta2, eps, c1, c2);
  std::string err;
  if (!ok_cuda(cudaGetLastError(), "launch", err)) return fail(QT_ECUDA, "qt_mlp_train_step: " + err);
  qt::set_last_error("");
  return QT_OK;
}

void qt_mlp_free(qt_mlp* M) { delete M; }

}  // extern "C"
