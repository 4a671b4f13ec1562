"""Python binding of the C ABI in include/qtensor.h (argument marshalling only).

The functions below carry the C names and forward to libqtensor.so through
ctypes; every step of the contraction runs in the library's CUDA kernels.
PyTorch is used only for device memory (the caller-owned workspace) and for the
current CUDA stream. Importing this module loads the in-tree library and
raises ImportError when it is missing: there is no fallback path.
"""

from __future__ import annotations

import ctypes as C
import json
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libqtensor.so")

QT_OK, QT_EINVAL, QT_ENOMEM, QT_ECUDA, QT_ETIMEOUT, QT_ESTATE, QT_ERANGE = range(7)
QT_GREEDY_MINFILL, QT_GREEDY_MINDEG = 0, 1
QT_FP32_SIMT, QT_TF32, QT_BF16, QT_3XTF32, QT_FP64 = 0, 1, 2, 3, 4
QT_OPT_FUSION, QT_OPT_GRAPHS, QT_OPT_GEMM, QT_OPT_SEGMENTS, QT_OPT_TRIANGLE, QT_OPT_TMA = 1, 2, 3, 4, 5, 6
QT_OPT_CONCURRENT = 7
QT_OPT_TCGEN05 = 8
QT_OPT_SCALED = 9
QT_OPT_SEG_CLUSTER = 10
QT_PROPOSAL_FEATURES = 16
QT_MAX_OPEN = 16

STATUS_NAMES = {0: "QT_OK", 1: "QT_EINVAL", 2: "QT_ENOMEM", 3: "QT_ECUDA",
                4: "QT_ETIMEOUT", 5: "QT_ESTATE", 6: "QT_ERANGE"}


class QtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libqtensor.so not built ({LIB_PATH}); run __graft_entry__.build()")
lib = C.CDLL(LIB_PATH)

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)
_u8p = C.POINTER(C.c_uint8)
_vp = C.c_void_p

_SIGS = {
    "qt_build_network": [_i32p, C.c_int32, C.c_int32, C.c_int32, _f64p, _f64p, _u8p,
                         C.POINTER(_vp)],
    "qt_set_angles": [_vp, _f64p, _f64p],
    "qt_set_bitstring": [_vp, _u8p],
    "qt_set_open": [_vp, _i32p, C.c_int32],
    "qt_contract_batch": [_vp, C.c_int32, _vp, C.c_size_t, _vp, _f64p],
    "qt_contract_sweep": [_vp, C.c_int32, C.c_int32, _f64p, _f64p, _vp, C.c_size_t, _vp, _f64p],
    "qt_order": [_vp, C.c_int32, C.c_uint64, _i32p],
    "qt_order_rgreedy": [_vp, C.c_double, C.c_int32, C.c_uint64, _i32p],
    "qt_slice": [_vp, C.c_int32, C.c_int32, C.c_int32, _i32p, _i32p],
    "qt_get_order": [_vp, _i32p, C.c_int32, _i32p],
    "qt_get_widths": [_vp, _i32p, C.c_int32, _i32p],
    "qt_get_slices": [_vp, _i32p, C.c_int32, _i32p, _i32p],
    "qt_get_tensor": [_vp, C.c_int32, _i32p, _i32p, _f64p],
    "qt_num_tensors": [_vp, _i32p, _i32p],
    "qt_prepare": [_vp, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)],
    "qt_stats": [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)],
    "qt_launch_plan": [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)],
    "qt_upload": [_vp, _vp, C.c_size_t, _vp],
    "qt_run": [_vp, C.c_int64, C.c_int64, _vp, C.c_size_t, _vp, _vp],
    "qt_contract": [_vp, C.c_int32, _vp, C.c_size_t, _vp, _f64p, _f64p],
    "qt_profile": [_vp, C.c_int32],
    "qt_contract_static": [_vp, C.c_int32, _vp, _f64p, _f64p],
    "qt_set_option": [_vp, C.c_int32, C.c_int64],
    "qt_plan_info": [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_double)],
    "qt_slice_dataset": [_vp, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float), _i32p,
                         C.c_int32, _i32p],
    "qt_slice_learned": [_vp, C.POINTER(C.c_float), C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                         C.c_int32, C.c_int32, C.c_int32, _i32p, _i32p],
    "qt_order_dataset": [_vp, C.c_int32, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float),
                         C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)],
    "qt_order_learned": [_vp, C.POINTER(C.c_float), C.c_int32, C.c_int32, C.c_int32,
                         C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "qt_mlp_forward_host": [C.POINTER(C.c_float), C.c_int32, C.c_int32, C.POINTER(C.c_float),
                            C.c_int32, C.POINTER(C.c_float)],
    "qt_mlp_create": [C.c_int32, C.c_int32, C.c_int32, C.POINTER(_vp)],
    "qt_mlp_workspace_size": [_vp, C.POINTER(C.c_size_t), _i32p],
    "qt_mlp_set_params": [_vp, _vp, C.c_size_t, C.POINTER(C.c_float), _vp],
    "qt_mlp_get_params": [_vp, _vp, C.c_size_t, C.POINTER(C.c_float), _vp],
    "qt_mlp_forward": [_vp, _vp, C.c_size_t, _vp, C.c_int32, _vp, _vp],
    "qt_mlp_gradients": [_vp, _vp, C.c_size_t, _vp, _vp, C.c_int32, _vp, _vp, _vp],
    "qt_mlp_train_step": [_vp, _vp, C.c_size_t, _vp, _vp, C.c_int32, C.c_float, _vp, _vp],
    "qt_energy_build": [_i32p, C.c_int32, C.c_int32, C.c_int32, _f64p, _f64p, C.c_int32,
                        C.POINTER(_vp)],
    "qt_energy_set_angles": [_vp, _f64p, _f64p],
    "qt_energy_prepare": [_vp, C.c_int32, C.POINTER(C.c_size_t)],
    "qt_energy_upload": [_vp, _vp, C.c_size_t, _vp],
    "qt_energy_run": [_vp, _vp, C.c_size_t, _vp, _vp, _vp],
    "qt_energy_autotune": [_vp, _vp, C.c_size_t, _vp, _i32p],
    "qt_energy_compute": [_vp, C.c_int32, _vp, C.c_size_t, _vp, _f64p, _f64p],
    "qt_energy_get_order": [_vp, C.c_int32, _i32p, C.c_int32, _i32p, _i32p, _i32p],
    "qt_energy_stats": [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)],
    "qt_energy_sweep_prepare": [_vp, C.c_int32, C.POINTER(C.c_size_t)],
    "qt_energy_sweep": [_vp, C.c_int32, _f64p, _f64p, _vp, C.c_size_t, _vp, _vp, _vp],
    "qt_energy_sweep_upload": [_vp, C.c_int32, _f64p, _f64p, _vp, C.c_size_t, _vp],
    "qt_energy_sweep_run": [_vp, C.c_int32, _vp, C.c_size_t, _vp, _vp, _vp],
    "qt_autotune": [_vp, _vp, C.c_size_t, _vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)],
    "qt_profile_read": [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)],
}
for _name, _args in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = C.c_int
lib.qt_mlp_free.argtypes = [_vp]
lib.qt_mlp_free.restype = None
lib.qt_energy_free.argtypes = [_vp]
lib.qt_energy_free.restype = None
lib.qt_free.argtypes = [_vp]
lib.qt_free.restype = None
lib.qt_last_error.argtypes = []
lib.qt_last_error.restype = C.c_char_p
lib.qt_version.argtypes = []
lib.qt_version.restype = C.c_char_p


def _check(status: int):
    if status != QT_OK:
        raise QtError(status, lib.qt_last_error().decode())


def _arr(ctype, values):
    values = list(values)
    return (ctype * max(1, len(values)))(*values)


# ----------------------------- C-named functions -----------------------------

def qt_build_network(edges, n_vertices, p, gammas, betas, bitstring):
    flat = [int(x) for e in edges for x in e]
    out = _vp()
    _check(lib.qt_build_network(_arr(C.c_int32, flat), int(n_vertices), len(edges), int(p),
                                _arr(C.c_double, gammas), _arr(C.c_double, betas),
                                _arr(C.c_uint8, bitstring), C.byref(out)))
    return out


def qt_set_angles(net, gammas, betas):
    _check(lib.qt_set_angles(net, _arr(C.c_double, gammas), _arr(C.c_double, betas)))


def qt_set_bitstring(net, bitstring):
    _check(lib.qt_set_bitstring(net, _arr(C.c_uint8, bitstring)))


def qt_set_open(net, qubits):
    qubits = [int(q) for q in qubits]
    _check(lib.qt_set_open(net, _arr(C.c_int32, qubits) if qubits else None, len(qubits)))


def qt_order(net, algo=QT_GREEDY_MINFILL, seed=0):
    w = C.c_int32()
    _check(lib.qt_order(net, int(algo), int(seed), C.byref(w)))
    return w.value


def qt_order_rgreedy(net, tau, q, seed):
    w = C.c_int32()
    _check(lib.qt_order_rgreedy(net, float(tau), int(q), int(seed), C.byref(w)))
    return w.value


def qt_slice(net, width_limit, max_vars, r=1):
    k, w = C.c_int32(), C.c_int32()
    _check(lib.qt_slice(net, int(width_limit), int(max_vars), int(r), C.byref(k), C.byref(w)))
    return k.value, w.value


def _get_list(fn, net, *extra):
    n = C.c_int32()
    _check(fn(net, None, 0, C.byref(n), *extra))
    buf = (C.c_int32 * max(1, n.value))()
    _check(fn(net, buf, n.value, C.byref(n), *extra))
    return list(buf[: n.value])


def qt_get_order(net):
    return _get_list(lib.qt_get_order, net)


def qt_get_widths(net):
    return _get_list(lib.qt_get_widths, net)


def qt_get_slices(net):
    step = C.c_int32()
    vars_ = _get_list(lib.qt_get_slices, net, C.byref(step))
    return vars_, step.value


def qt_num_tensors(net):
    c, nv = C.c_int32(), C.c_int32()
    _check(lib.qt_num_tensors(net, C.byref(c), C.byref(nv)))
    return c.value, nv.value


def qt_get_tensor(net, t):
    rank = C.c_int32()
    _check(lib.qt_get_tensor(net, int(t), None, C.byref(rank), None))
    labels = (C.c_int32 * max(1, rank.value))()
    data = (C.c_double * (2 << rank.value))()
    _check(lib.qt_get_tensor(net, int(t), labels, C.byref(rank), data))
    return list(labels[: rank.value]), list(data)


def qt_prepare(net, precision=QT_FP32_SIMT, batch=1):
    n = C.c_size_t()
    _check(lib.qt_prepare(net, int(precision), int(batch), C.byref(n)))
    return n.value


def qt_stats(net):
    n = C.c_size_t()
    _check(lib.qt_stats(net, None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(lib.qt_stats(net, buf, n.value, C.byref(n)))
    return json.loads(buf.value.decode())


def qt_launch_plan(net):
    """The slice-phase launches' streams, waits and workspace ranges (a dict)."""
    n = C.c_size_t()
    _check(lib.qt_launch_plan(net, None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(lib.qt_launch_plan(net, buf, n.value, C.byref(n)))
    return json.loads(buf.value.decode())


def qt_upload(net, workspace_ptr, workspace_bytes, stream_ptr):
    _check(lib.qt_upload(net, _vp(workspace_ptr), int(workspace_bytes), _vp(stream_ptr)))


def qt_run(net, first, count, workspace_ptr, workspace_bytes, stream_ptr, d_out_ptr):
    _check(lib.qt_run(net, int(first), int(count), _vp(workspace_ptr), int(workspace_bytes),
                      _vp(stream_ptr), _vp(d_out_ptr)))


def qt_contract(net, precision, workspace_ptr, workspace_bytes, stream_ptr):
    re, im = C.c_double(), C.c_double()
    _check(lib.qt_contract(net, int(precision), _vp(workspace_ptr), int(workspace_bytes),
                           _vp(stream_ptr), C.byref(re), C.byref(im)))
    return complex(re.value, im.value)


def qt_contract_batch(net, precision, workspace_ptr, workspace_bytes, stream_ptr, a):
    """The 2^a amplitudes of a network with a open qubits; entry b has bit j = open qubit j."""
    buf = (C.c_double * (2 << a))()
    _check(lib.qt_contract_batch(net, int(precision), _vp(workspace_ptr), int(workspace_bytes),
                                 _vp(stream_ptr), buf))
    return [complex(buf[2 * b], buf[2 * b + 1]) for b in range(1 << a)]


def qt_contract_sweep(net, precision, gammas, betas, workspace_ptr, workspace_bytes, stream_ptr):
    """Amplitudes for n angle sets (gammas, betas: n lists of p angles) with one plan."""
    n = len(gammas)
    if n != len(betas):
        raise ValueError("gammas and betas need the same number of sets")
    flat_g = [float(x) for row in gammas for x in row]
    flat_b = [float(x) for row in betas for x in row]
    buf = (C.c_double * (2 * max(n, 1)))()
    _check(lib.qt_contract_sweep(net, int(precision), int(n), _arr(C.c_double, flat_g),
                                 _arr(C.c_double, flat_b), _vp(workspace_ptr), int(workspace_bytes),
                                 _vp(stream_ptr), buf))
    return [complex(buf[2 * s], buf[2 * s + 1]) for s in range(n)]


def qt_contract_static(net, precision, stream_ptr):
    re, im = C.c_double(), C.c_double()
    _check(lib.qt_contract_static(net, int(precision), _vp(stream_ptr), C.byref(re), C.byref(im)))
    return complex(re.value, im.value)


def qt_set_option(net, option, value):
    _check(lib.qt_set_option(net, int(option), int(value)))


def qt_autotune(net, workspace_ptr, workspace_bytes, stream_ptr):
    n = C.c_size_t()
    buf = C.create_string_buffer(1 << 16)
    _check(lib.qt_autotune(net, _vp(workspace_ptr), int(workspace_bytes), _vp(stream_ptr), buf,
                           len(buf), C.byref(n)))
    return json.loads(buf.value.decode())


def qt_profile(net, enable):
    _check(lib.qt_profile(net, 1 if enable else 0))


def qt_profile_read(net):
    n = C.c_size_t()
    _check(lib.qt_profile_read(net, None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(lib.qt_profile_read(net, buf, n.value, C.byref(n)))
    return json.loads(buf.value.decode())


def qt_free(net):
    lib.qt_free(net)


def qt_version():
    return lib.qt_version().decode()


def qt_energy_build(edges, n_vertices, p, gammas, betas, algo=QT_GREEDY_MINFILL):
    flat = [int(x) for e in edges for x in e]
    out = _vp()
    _check(lib.qt_energy_build(_arr(C.c_int32, flat), int(n_vertices), len(edges), int(p),
                               _arr(C.c_double, gammas), _arr(C.c_double, betas), int(algo),
                               C.byref(out)))
    return out


def qt_energy_set_angles(h, gammas, betas):
    _check(lib.qt_energy_set_angles(h, _arr(C.c_double, gammas), _arr(C.c_double, betas)))


def qt_energy_prepare(h, precision=QT_FP32_SIMT):
    n = C.c_size_t()
    _check(lib.qt_energy_prepare(h, int(precision), C.byref(n)))
    return n.value


def qt_energy_upload(h, workspace_ptr, workspace_bytes, stream_ptr):
    _check(lib.qt_energy_upload(h, _vp(workspace_ptr), int(workspace_bytes), _vp(stream_ptr)))


def qt_energy_run(h, workspace_ptr, workspace_bytes, stream_ptr, d_zz_ptr, d_energy_ptr):
    _check(lib.qt_energy_run(h, _vp(workspace_ptr), int(workspace_bytes), _vp(stream_ptr),
                             _vp(d_zz_ptr), _vp(d_energy_ptr)))


def qt_energy_autotune(h, workspace_ptr, workspace_bytes, stream_ptr):
    t = C.c_int32()
    _check(lib.qt_energy_autotune(h, _vp(workspace_ptr), int(workspace_bytes), _vp(stream_ptr),
                                  C.byref(t)))
    return t.value


def qt_energy_compute(h, precision, workspace_ptr, workspace_bytes, stream_ptr, n_edges):
    zz = (C.c_double * max(1, n_edges))()
    en = C.c_double()
    _check(lib.qt_energy_compute(h, int(precision), _vp(workspace_ptr), int(workspace_bytes),
                                 _vp(stream_ptr), zz, C.byref(en)))
    return en.value, list(zz[:n_edges])


def qt_energy_get_order(h, edge):
    n, nv, w = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib.qt_energy_get_order(h, int(edge), None, 0, C.byref(n), C.byref(nv), C.byref(w)))
    buf = (C.c_int32 * max(1, n.value))()
    _check(lib.qt_energy_get_order(h, int(edge), buf, n.value, C.byref(n), C.byref(nv), C.byref(w)))
    return list(buf[: n.value]), nv.value, w.value


def qt_energy_stats(h):
    n = C.c_size_t()
    _check(lib.qt_energy_stats(h, None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(lib.qt_energy_stats(h, buf, n.value, C.byref(n)))
    return json.loads(buf.value.decode())


def qt_energy_free(h):
    lib.qt_energy_free(h)


class Energy:
    """Owns a qt_energy handle and a torch-allocated workspace."""

    def __init__(self, edges, n_vertices, p, gammas, betas, algo=QT_GREEDY_MINFILL):
        self.n_edges = len(edges)
        self.handle = qt_energy_build(edges, n_vertices, p, gammas, betas, algo)
        self.workspace = None

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            qt_energy_free(h)
            self.handle = None

    def _stream(self):
        import torch
        return torch.cuda.current_stream().cuda_stream

    def prepare(self, precision=QT_FP32_SIMT, device="cuda"):
        import torch
        need = qt_energy_prepare(self.handle, precision)
        if self.workspace is None or self.workspace.numel() < need:
            self.workspace = None
            self.workspace = torch.empty(need, dtype=torch.uint8, device=device)
        return need

    def upload(self):
        qt_energy_upload(self.handle, self.workspace.data_ptr(), self.workspace.numel(),
                         self._stream())

    def autotune(self):
        return qt_energy_autotune(self.handle, self.workspace.data_ptr(), self.workspace.numel(),
                                  self._stream())

    def run(self, zz, energy):
        qt_energy_run(self.handle, self.workspace.data_ptr(), self.workspace.numel(),
                      self._stream(), zz.data_ptr(), energy.data_ptr())

    def compute(self, precision=QT_FP32_SIMT):
        return qt_energy_compute(self.handle, precision, self.workspace.data_ptr(),
                                 self.workspace.numel(), self._stream(), self.n_edges)

    def stats(self):
        return qt_energy_stats(self.handle)

    def sweep_prepare(self, n_sets, device="cuda"):
        """Workspace for angle sweeps of up to n_sets sets (after prepare)."""
        import torch
        need = C.c_size_t()
        _check(lib.qt_energy_sweep_prepare(self.handle, int(n_sets), C.byref(need)))
        self.sweep_ws = torch.empty(need.value, dtype=torch.uint8, device=device)
        return need.value

    def sweep_upload(self, gammas, betas):
        flat_g = [float(x) for row in gammas for x in row]
        flat_b = [float(x) for row in betas for x in row]
        _check(lib.qt_energy_sweep_upload(self.handle, len(gammas), _arr(C.c_double, flat_g),
                                          _arr(C.c_double, flat_b), _vp(self.sweep_ws.data_ptr()),
                                          int(self.sweep_ws.numel()), _vp(self._stream())))

    def sweep_run(self, n_sets, energies, zz=None):
        _check(lib.qt_energy_sweep_run(self.handle, int(n_sets), _vp(self.sweep_ws.data_ptr()),
                                       int(self.sweep_ws.numel()), _vp(self._stream()),
                                       _vp(energies.data_ptr()),
                                       _vp(zz.data_ptr()) if zz is not None else None))

    def sweep(self, gammas, betas, energies, zz=None):
        """Energies of len(gammas) angle sets (each a list of p angles) into the float64
        CUDA tensor `energies`; per-edge <Z_u Z_v> into `zz` [n_sets][n_edges] if given."""
        flat_g = [float(x) for row in gammas for x in row]
        flat_b = [float(x) for row in betas for x in row]
        _check(lib.qt_energy_sweep(self.handle, len(gammas), _arr(C.c_double, flat_g),
                                   _arr(C.c_double, flat_b), _vp(self.sweep_ws.data_ptr()),
                                   int(self.sweep_ws.numel()), _vp(self._stream()),
                                   _vp(energies.data_ptr()),
                                   _vp(zz.data_ptr()) if zz is not None else None))


# ------------------------ convenience wrapper (torch) ------------------------

class Network:
    """Owns a qt_net handle and, once prepared, a torch-allocated device workspace."""

    def __init__(self, edges, n_vertices, p, gammas, betas, bitstring):
        self.n, self.p = int(n_vertices), int(p)
        self.handle = qt_build_network(edges, n_vertices, p, gammas, betas, bitstring)
        self.workspace = None
        self.ws_bytes = 0
        self.open = []

    def set_open(self, qubits):
        """Leave these qubits' output indices open: contract_batch then gives 2^a amplitudes."""
        qt_set_open(self.handle, qubits)
        self.open = [int(q) for q in qubits]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            qt_free(h)
            self.handle = None

    def order(self, algo=QT_GREEDY_MINFILL):
        return qt_order(self.handle, algo)

    def slice(self, width_limit, max_vars, r=1):
        return qt_slice(self.handle, width_limit, max_vars, r)

    def prepare(self, precision=QT_FP32_SIMT, batch=1, device="cuda"):
        import torch
        self.ws_bytes = qt_prepare(self.handle, precision, batch)
        if self.workspace is None or self.workspace.numel() < self.ws_bytes:
            self.workspace = None
            self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        return self.ws_bytes

    def stats(self):
        return qt_stats(self.handle)

    def _stream(self):
        import torch
        return torch.cuda.current_stream().cuda_stream

    def autotune(self):
        return qt_autotune(self.handle, self.workspace.data_ptr(), self.workspace.numel(),
                           self._stream())

    def upload(self):
        qt_upload(self.handle, self.workspace.data_ptr(), self.workspace.numel(), self._stream())

    def run(self, first, count, out):
        """Device-resident run; out is a float64 CUDA tensor with >= 2 * 2^a elements."""
        qt_run(self.handle, first, count, self.workspace.data_ptr(), self.workspace.numel(),
               self._stream(), out.data_ptr())

    def contract(self, precision=QT_FP32_SIMT):
        return qt_contract(self.handle, precision, self.workspace.data_ptr(),
                           self.workspace.numel(), self._stream())

    def contract_sweep(self, gammas, betas, precision=QT_FP32_SIMT):
        """Amplitudes for several angle sets with this network's order and slicing. The
        workspace grows to hold every set's gate image beside the prepared schedule."""
        import torch
        st = self.stats()
        need = st["workspace_bytes"] + len(gammas) * (st["upload_bytes"] + 512) + 1024
        if self.workspace.numel() < need:
            dev = self.workspace.device
            self.workspace = None
            self.workspace = torch.empty(need, dtype=torch.uint8, device=dev)
        return qt_contract_sweep(self.handle, precision, gammas, betas, self.workspace.data_ptr(),
                                 self.workspace.numel(), self._stream())

    def contract_batch(self, precision=QT_FP32_SIMT):
        return qt_contract_batch(self.handle, precision, self.workspace.data_ptr(),
                                 self.workspace.numel(), self._stream(), len(self.open))
