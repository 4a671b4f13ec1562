// qt_contract_static: the end-to-end contraction with its device scratch in a
// fixed array inside this library instead of a caller workspace.
//
// Who needs it: callers that cannot allocate device memory themselves, e.g. a
// plugin running inside a host application that owns the CUDA allocator and
// forbids cudaMalloc from third-party code, or code on a path that must not
// allocate (real-time loops, memory-capped sandboxes). They pass their inputs
// (the network built on the host) and outputs (two host doubles) as usual; the
// intermediate tensors, gate copies and bookkeeping live in g_static_ws.
//
// The array is a file-scope __device__ object of kStaticWorkspaceBytes: every
// GPU on which this library's module is loaded holds it until the process
// exits. In host code its name is only a host-side stand-in, so the device
// address is obtained once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels as the workspace pointer.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "qt_internal.h"

namespace qt {
qt_status upload(qt_net* net, void* ws, size_t bytes, void* stream, std::string& err);
qt_status run(qt_net* net, long long first, long long count, void* ws, void* stream,
              double* d_out, std::string& err);
qt_status download_result(const double* d_out, double* host, int64_t n_doubles, void* stream,
                          std::string& err);
void set_last_error(const std::string& msg);  // api.cpp: the message qt_last_error() returns
}  // namespace qt

namespace {

constexpr size_t kStaticWorkspaceBytes = size_t(64) << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_ws[kStaticWorkspaceBytes];

std::mutex g_setup_mu;
void* g_static_ptr[kMaxDevices] = {};

qt_status fail(qt_status s, const std::string& m) {
  qt::set_last_error(m);
  return s;
}

// Device address of g_static_ws on the current device (set up on first use).
qt_status static_workspace(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(QT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(QT_EINVAL, "device ordinal beyond the table");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || !p)
      return fail(QT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return QT_OK;
}

}  // namespace

extern "C" {

qt_status qt_prepare(qt_net* net, int32_t precision, int32_t batch, size_t* workspace_bytes);
const char* qt_last_error(void);

qt_status qt_contract_static(qt_net* net, int32_t precision, void* stream, double* amp_re,
                             double* amp_im) {
  if (!net || !amp_re || !amp_im) return fail(QT_EINVAL, "qt_contract_static: null argument");
  if (!net->ordered) return fail(QT_ESTATE, "qt_contract_static: call qt_order first");
  if (!net->open.empty())
    return fail(QT_ESTATE, "qt_contract_static: the network has open qubits");
  void* ws = nullptr;
  qt_status s = static_workspace(&ws);
  if (s != QT_OK) return s;
  // the caller's prepared schedule (if any) is put back before returning
  const bool had_schedule = net->sched.valid;
  const int32_t old_precision = net->sched.precision;
  const int32_t old_batch = (int32_t)net->sched.batch;
  auto restore = [&]() {
    size_t unused = 0;
    if (had_schedule) qt_prepare(net, old_precision, old_batch, &unused);
  };
  // the largest slice batch whose schedule fits the static array
  size_t need = 0;
  s = qt_prepare(net, precision, 1, &need);
  if (s != QT_OK) {
    std::string m = std::string("qt_contract_static: ") + qt_last_error();
    restore();
    return fail(s, m);
  }
  if (need > kStaticWorkspaceBytes) {
    restore();
    return fail(QT_ENOMEM, "qt_contract_static: the network needs " + std::to_string(need) +
                               " bytes of device scratch; the static workspace holds " +
                               std::to_string(kStaticWorkspaceBytes));
  }
  int64_t lo = 1, hi = net->sched.nslices;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) / 2;
    s = qt_prepare(net, precision, (int32_t)std::min<int64_t>(mid, 1 << 30), &need);
    if (s != QT_OK) {
      std::string m = std::string("qt_contract_static: ") + qt_last_error();
      restore();
      return fail(s, m);
    }
    if (need <= kStaticWorkspaceBytes) lo = mid;
    else hi = mid - 1;
  }
  s = qt_prepare(net, precision, (int32_t)lo, &need);
  if (s != QT_OK) {
    std::string m = std::string("qt_contract_static: ") + qt_last_error();
    restore();
    return fail(s, m);
  }
  // no tracing events and no graph capture on this path: it creates no CUDA objects
  const bool prof = net->prof, graphs = net->graphs;
  net->prof = false;
  net->graphs = false;
  std::string err;
  s = qt::upload(net, ws, kStaticWorkspaceBytes, stream, err);
  double* d_out = reinterpret_cast<double*>((char*)ws + net->sched.off_acc + 16);
  if (s == QT_OK) s = qt::run(net, 0, net->sched.nslices, ws, stream, d_out, err);
  double h[2] = {0.0, 0.0};
  if (s == QT_OK) s = qt::download_result(d_out, h, 2, stream, err);
  net->prof = prof;
  net->graphs = graphs;
  restore();
  if (s != QT_OK) return fail(s, "qt_contract_static: " + err);
  *amp_re = h[0];
  *amp_im = h[1];
  qt::set_last_error("");
  return QT_OK;
}

}  // extern "C"
