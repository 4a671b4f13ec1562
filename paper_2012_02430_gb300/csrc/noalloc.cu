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
// exits. In host code its name is only a host-side stand-in, so every call
// asks for its device address on the current device (cudaGetSymbolAddress,
// which allocates nothing) and passes that address to the kernels as the
// workspace pointer. The first call on a device also loads the module there.
#include <cuda_runtime.h>

#include <new>
#include <string>
#include <utility>

#include "qt_internal.h"

namespace qt {
qt_status upload(qt_net* net, void* ws, size_t bytes, void* stream, std::string& err);
qt_status run(qt_net* net, long long first, long long count, void* ws, void* stream,
              double* d_out, std::string& err);
qt_status download_result(const double* d_out, double* host, int64_t n_doubles, void* stream,
                          std::string& err);
qt_status read_status(const qt_net* net, const void* ws, void* stream, int* status,
                      std::string& err);
void set_last_error(const std::string& msg);  // api.cpp: the message qt_last_error() returns
}  // namespace qt

namespace {

constexpr size_t kStaticWorkspaceBytes = size_t(64) << 20;  // 64 MiB per device

__device__ __align__(256) unsigned char g_static_ws[kStaticWorkspaceBytes];

qt_status fail(qt_status s, const std::string& m) {
  qt::set_last_error(m);
  return s;
}

// Device address of g_static_ws on the current device. Asked for on every call rather
// than cached, so that a context torn down and created again (cudaDeviceReset) never
// leaves a stale address behind.
qt_status static_workspace(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
  if (e != cudaSuccess || !p)
    return fail(QT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = p;
  return QT_OK;
}

// The caller's planning state, put back exactly on every return: the prepared schedule,
// what was last uploaded where, and the engine cache (launch descriptors, autotuned
// kernel choices, captured graph). The static call plans and runs on its own copies.
struct SavedState {
  qt_net* net;
  qt::Schedule sched;
  uint64_t uploaded_gen, uploaded_data;
  const void* uploaded_ws;
  bool prof, graphs;
  void* engine;
  explicit SavedState(qt_net* n)
      : net(n), sched(n->sched), uploaded_gen(n->uploaded_gen), uploaded_data(n->uploaded_data),
        uploaded_ws(n->uploaded_ws), prof(n->prof), graphs(n->graphs),
        engine(qt::engine_detach(n)) {}
  ~SavedState() {
    net->sched = std::move(sched);
    net->uploaded_gen = uploaded_gen;
    net->uploaded_data = uploaded_data;
    net->uploaded_ws = uploaded_ws;
    net->stage_dirty = true;  // the host gate staging was rebuilt for the static call
    net->prof = prof;
    net->graphs = graphs;
    qt::engine_restore(net, engine);
  }
};

}  // namespace

extern "C" {

qt_status qt_contract_static(qt_net* net, int32_t precision, void* stream, double* amp_re,
                             double* amp_im) {
  if (!net || !amp_re || !amp_im) return fail(QT_EINVAL, "qt_contract_static: null argument");
  if (!net->ordered) return fail(QT_ESTATE, "qt_contract_static: call qt_order first");
  if (!net->open.empty())
    return fail(QT_ESTATE, "qt_contract_static: the network has open qubits");
  void* ws = nullptr;
  qt_status s = static_workspace(&ws);
  if (s != QT_OK) return s;
  std::string err;
  double h[2] = {0.0, 0.0};
  try {
    SavedState saved(net);
    // the largest slice batch whose schedule fits the static array
    s = qt::prepare_fitting(net, precision, kStaticWorkspaceBytes, nullptr, nullptr, err);
    if (s == QT_ENOMEM)
      err += " (the static workspace holds " + std::to_string(kStaticWorkspaceBytes) + " bytes)";
    // no tracing events and no graph capture on this path: it creates no CUDA objects
    net->prof = false;
    net->graphs = false;
    if (s == QT_OK) s = qt::upload(net, ws, kStaticWorkspaceBytes, stream, err);
    double* d_out = reinterpret_cast<double*>((char*)ws + net->sched.off_acc + 16);
    if (s == QT_OK) s = qt::run(net, 0, net->sched.nslices, ws, stream, d_out, err);
    if (s == QT_OK) s = qt::download_result(d_out, h, 2, stream, err);
    // the status word sits at this schedule's offset: read before the caller's comes back
    int status = 0;
    if (s == QT_OK) s = qt::read_status(net, ws, stream, &status, err);
    if (s == QT_OK && status) {
      s = QT_ETIMEOUT;
      err = "a bounded device wait gave up";
    }
  } catch (const std::bad_alloc&) {
    s = QT_ENOMEM;
    err = "out of host memory";
  }
  if (s != QT_OK) return fail(s, "qt_contract_static: " + err);
  *amp_re = h[0];
  *amp_im = h[1];
  qt::set_last_error("");
  return QT_OK;
}

}  // extern "C"
