"""Learned proposals for the slicing search: data generation, GPU training, evaluation.

The simulator generates its own training data: for seeded random 3-regular QAOA
networks (N = 50..150, p = 1, 2), every candidate (step s, slice vertex v) of the
first slicing round is ordered greedily once (qt_slice_dataset) and labelled with
the plan width it gives, placed between the round's best (0) and worst (1) width. The MLP is trained on the GPU by the library's own
kernels (qt_mlp_train_step: forward, backward, Adam). The planner then verifies
only the top-m scored candidates per round (qt_slice_learned).

    python -m paper_2012_02430_gb300.learn train        # data/proposal_mlp.json (GPU)
    python -m paper_2012_02430_gb300.learn train-order  # data/order_mlp.json (GPU):
        elimination-step proposals, trained on rollouts of the simulator's own orderings
"""

from __future__ import annotations

import ctypes as C
import json
import math
import os
import sys
import time

import numpy as np

from . import qtensor as Q
from .inputs import SplitMix64, qaoa_instance

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "data", "proposal_mlp.json")
NF = Q.QT_PROPOSAL_FEATURES if hasattr(Q, "QT_PROPOSAL_FEATURES") else 16
TRAIN_SET = [(n, p, 7000 + 37 * n + 11 * p + r) for n in range(50, 151, 10) for p in (1, 2)
             for r in range(2)]
HELD_OUT = [(n, p, 90000 + 13 * n + p) for n in (60, 80, 100, 120, 140) for p in (1, 2)]


def dataset_of(edges, n, p, gammas, betas, z, topv=3, algo=Q.QT_GREEDY_MINFILL):
    h = Q.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        Q.qt_order(h, algo)
        cnt = C.c_int32()
        Q._check(Q.lib.qt_slice_dataset(h, topv, None, None, None, 0, C.byref(cnt)))
        k = cnt.value
        f = (C.c_float * max(1, k * NF))()
        lab = (C.c_float * max(1, k))()
        meta = (C.c_int32 * max(1, 3 * k))()
        Q._check(Q.lib.qt_slice_dataset(h, topv, f, lab, meta, k, C.byref(cnt)))
        X = np.frombuffer(f, dtype=np.float32, count=k * NF).reshape(k, NF).copy()
        Y = np.frombuffer(lab, dtype=np.float32, count=k).copy()
        M = np.frombuffer(meta, dtype=np.int32, count=3 * k).reshape(k, 3).copy()
        return X, Y, M
    finally:
        Q.qt_free(h)


def round_targets(M):
    """Training target of each candidate of one round: its plan width placed between the
    round's best (0) and worst (1) width, so the model learns to rank within a round."""
    w = M[:, 2].astype(np.float64)
    lo, hi = w.min(), w.max()
    return ((w - lo) / max(1.0, hi - lo)).astype(np.float32)


def make_dataset(instances, topv=3):
    Xs, Ys = [], []
    for n, p, seed in instances:
        edges, g, b, z = qaoa_instance(n, p, seed)
        X, _, M = dataset_of(edges, n, p, g, b, z, topv)
        Xs.append(X)
        Ys.append(round_targets(M))
    return np.concatenate(Xs), np.concatenate(Ys)


def init_params(nf, hidden, seed):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, from SplitMix64."""
    rng = SplitMix64(seed)
    out = []

    def block(rows, cols):
        bound = math.sqrt(6.0 / cols)
        return [(2.0 * rng.uniform() - 1.0) * bound for _ in range(rows * cols)]

    out += block(hidden, nf) + [0.0] * hidden
    out += block(hidden, hidden) + [0.0] * hidden
    out += block(1, hidden) + [0.0]
    return np.array(out, dtype=np.float32)


class GPUMLP:
    """The library's MLP kernels on a torch-allocated workspace."""

    def __init__(self, nf, hidden, max_batch):
        import torch
        self.torch = torch
        self.nf, self.hidden, self.max_batch = nf, hidden, max_batch
        h = C.c_void_p()
        Q._check(Q.lib.qt_mlp_create(nf, hidden, max_batch, C.byref(h)))
        self.h = h
        n = C.c_size_t()
        npar = C.c_int32()
        Q._check(Q.lib.qt_mlp_workspace_size(h, C.byref(n), C.byref(npar)))
        self.n_params = npar.value
        self.ws = torch.empty(n.value, dtype=torch.uint8, device="cuda")

    def __del__(self):
        if getattr(self, "h", None):
            Q.lib.qt_mlp_free(self.h)
            self.h = None

    def _s(self):
        return C.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _ws(self):
        return C.c_void_p(self.ws.data_ptr()), C.c_size_t(self.ws.numel())

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        Q._check(Q.lib.qt_mlp_set_params(self.h, *self._ws(), p.ctypes.data_as(C.POINTER(C.c_float)),
                                         self._s()))

    def get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        Q._check(Q.lib.qt_mlp_get_params(self.h, *self._ws(), p.ctypes.data_as(C.POINTER(C.c_float)),
                                         self._s()))
        return p

    def forward(self, x_dev):
        y = self.torch.empty(x_dev.shape[0], dtype=self.torch.float32, device="cuda")
        Q._check(Q.lib.qt_mlp_forward(self.h, *self._ws(), C.c_void_p(x_dev.data_ptr()),
                                      x_dev.shape[0], C.c_void_p(y.data_ptr()), self._s()))
        return y

    def gradients(self, x_dev, t_dev):
        g = self.torch.empty(self.n_params, dtype=self.torch.float32, device="cuda")
        loss = self.torch.empty(1, dtype=self.torch.float32, device="cuda")
        Q._check(Q.lib.qt_mlp_gradients(self.h, *self._ws(), C.c_void_p(x_dev.data_ptr()),
                                        C.c_void_p(t_dev.data_ptr()), x_dev.shape[0],
                                        C.c_void_p(g.data_ptr()), C.c_void_p(loss.data_ptr()),
                                        self._s()))
        return g, loss

    def train_step(self, x_dev, t_dev, lr, loss_dev):
        Q._check(Q.lib.qt_mlp_train_step(self.h, *self._ws(), C.c_void_p(x_dev.data_ptr()),
                                         C.c_void_p(t_dev.data_ptr()), x_dev.shape[0],
                                         C.c_float(lr), C.c_void_p(loss_dev.data_ptr()),
                                         self._s()))


def train(X, Y, hidden=64, steps=3000, batch=1024, lr=2e-3, seed=12345):
    """Minibatch Adam on the GPU; minibatches drawn with SplitMix64. Returns (params, log)."""
    import torch
    mlp = GPUMLP(X.shape[1], hidden, batch)
    mlp.set_params(init_params(X.shape[1], hidden, seed))
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    rng = SplitMix64(seed + 1)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    log = []
    n = X.shape[0]
    idx_buf = np.zeros(batch, dtype=np.int64)
    t0 = time.time()
    for step in range(steps):
        for i in range(batch):
            idx_buf[i] = rng.below(n)
        idx = torch.from_numpy(idx_buf).cuda()
        xb = Xd.index_select(0, idx).contiguous()
        tb = Yd.index_select(0, idx).contiguous()
        mlp.train_step(xb, tb, lr, loss)
        if step % 250 == 0 or step == steps - 1:
            log.append((step, float(loss.item())))
    torch.cuda.synchronize()
    full_mse = float(((mlp_forward_full(mlp, Xd) - Yd) ** 2).mean().item())
    return mlp.get_params(), {"log": log, "train_mse": full_mse, "seconds": time.time() - t0}


def mlp_forward_full(mlp, Xd):
    import torch
    out = []
    for i in range(0, Xd.shape[0], mlp.max_batch):
        out.append(mlp.forward(Xd[i:i + mlp.max_batch].contiguous()))
    return torch.cat(out)


# ---------------------------------------------------------------------------
# Learned elimination steps: at a step of a greedy ordering the candidates are the
# STEP_TOPC vertices best by the greedy key; features and rollout labels come from
# qt_order_dataset, the model ranks candidates within a step, qt_order_learned
# orders with it (greedy as judge).
# ---------------------------------------------------------------------------
ORDER_WEIGHTS = os.path.join(HERE, "data", "order_mlp.json")
STEP_TOPC = 4
STEP_STRIDE = 4


def order_dataset_of(edges, n, p, gammas, betas, z, topc=STEP_TOPC, stride=STEP_STRIDE,
                     algo=Q.QT_GREEDY_MINFILL):
    h = Q.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        Q.qt_order(h, algo)
        cnt = C.c_int32()
        Q._check(Q.lib.qt_order_dataset(h, topc, stride, None, None, None, 0, C.byref(cnt)))
        k = cnt.value
        f = (C.c_float * max(1, k * NF))()
        lab = (C.c_float * max(1, k))()
        meta = (C.c_int32 * max(1, 3 * k))()
        Q._check(Q.lib.qt_order_dataset(h, topc, stride, f, lab, meta, k, C.byref(cnt)))
        X = np.frombuffer(f, dtype=np.float32, count=k * NF).reshape(k, NF).copy()
        L = np.frombuffer(lab, dtype=np.float32, count=k).copy()
        M = np.frombuffer(meta, dtype=np.int32, count=3 * k).reshape(k, 3).copy()
        return X, L, M
    finally:
        Q.qt_free(h)


def step_targets(L, M):
    """Each candidate's rollout log2 cost placed between its step's best (0) and worst (1)
    candidate, so the model learns to rank the candidates of a step."""
    Y = np.zeros_like(L)
    for t in np.unique(M[:, 0]):
        sel = M[:, 0] == t
        lo, hi = L[sel].min(), L[sel].max()
        Y[sel] = (L[sel] - lo) / max(1e-6, hi - lo)
    return Y


def make_order_dataset(instances, topc=STEP_TOPC, stride=STEP_STRIDE):
    Xs, Ys = [], []
    for n, p, seed in instances:
        edges, g, b, z = qaoa_instance(n, p, seed)
        X, L, M = order_dataset_of(edges, n, p, g, b, z, topc, stride)
        Xs.append(X)
        Ys.append(step_targets(L, M))
    return np.concatenate(Xs), np.concatenate(Ys)


def order_with(instance, params=None, hidden=64, topc=STEP_TOPC, judge=0):
    """Orders one instance greedily (params None) or with the learned steps; returns
    (width, log2 sum of 2^w, learned order kept)."""
    n, p, seed = instance
    edges, g, b, z = qaoa_instance(n, p, seed)
    h = Q.qt_build_network(edges, n, p, g, b, z)
    try:
        if params is None:
            w = Q.qt_order(h, Q.QT_GREEDY_MINFILL)
            kept = 0
        else:
            Q.qt_order(h, Q.QT_GREEDY_MINFILL)
            pa = np.ascontiguousarray(params, dtype=np.float32)
            wc, kc = C.c_int32(), C.c_int32()
            Q._check(Q.lib.qt_order_learned(h, pa.ctypes.data_as(C.POINTER(C.c_float)), hidden,
                                            topc, judge, C.byref(wc), C.byref(kc)))
            w, kept = wc.value, kc.value
        widths = Q.qt_get_widths(h)
        return w, math.log2(sum(math.ldexp(1.0, x) for x in widths)), kept
    finally:
        Q.qt_free(h)


def save(params, hidden, info, path=WEIGHTS):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"n_features": NF, "hidden": hidden, "params": [float(x) for x in params],
                   "train_instances": TRAIN_SET, **info}, f)


def load(path=WEIGHTS):
    with open(path) as f:
        d = json.load(f)
    return np.array(d["params"], dtype=np.float32), int(d["hidden"]), d


def plan_with(instance, mode, params=None, hidden=64, topv=3, topm=4, spread=4, width_drop=1,
              max_vars=1):
    """Slices one instance and returns the plan summary. Modes: 'paper' (qt_slice, every
    step with the max-degree vertex), 'full' (every (s, v) candidate), 'budget' (spread
    evenly spaced candidates, no model), 'learned' (the model's topm plus spread)."""
    n, p, seed = instance
    edges, g, b, z = qaoa_instance(n, p, seed)
    h = Q.qt_build_network(edges, n, p, g, b, z)
    try:
        w0 = Q.qt_order(h, Q.QT_GREEDY_MINFILL)
        lim = max(1, w0 - width_drop)
        t0 = time.perf_counter()
        k, w = C.c_int32(), C.c_int32()
        if mode == "paper":
            Q._check(Q.lib.qt_slice(h, lim, max_vars, 1, C.byref(k), C.byref(w)))
        else:
            pp, tm, sp = None, 0, spread
            if mode == "learned":
                pa = np.ascontiguousarray(params, dtype=np.float32)
                pp = pa.ctypes.data_as(C.POINTER(C.c_float))
                tm = topm
            elif mode == "full":
                sp = 1 << 30
            Q._check(Q.lib.qt_slice_learned(h, pp, hidden, lim, max_vars, 1, topv, tm, sp,
                                            C.byref(k), C.byref(w)))
        dt = time.perf_counter() - t0
        runs, cost = C.c_int64(), C.c_double()
        Q._check(Q.lib.qt_plan_info(h, C.byref(runs), C.byref(cost)))
        return {"width0": w0, "width": w.value, "k": k.value, "greedy_runs": runs.value,
                "log2_cost": math.log2(cost.value), "seconds": dt}
    finally:
        Q.qt_free(h)


def evaluate_order(params, hidden, instances=None, topc=STEP_TOPC):
    """Greedy vs learned steps (alone, and with greedy as judge) on held-out networks:
    per instance (width, log2 cost) of each."""
    rows = []
    for inst in instances or HELD_OUT:
        g = order_with(inst)
        lone = order_with(inst, params, hidden, topc, judge=0)
        judged = order_with(inst, params, hidden, topc, judge=1)
        rows.append({"instance": list(inst), "greedy": g[:2], "learned": lone[:2],
                     "judged": judged[:2], "kept": judged[2]})
    return rows


def main(argv):
    if len(argv) > 1 and argv[1] == "train-order":
        out = argv[2] if len(argv) > 2 else ORDER_WEIGHTS
        t0 = time.time()
        X, Y = make_order_dataset(TRAIN_SET, STEP_TOPC, 2)
        t_data = time.time() - t0
        print(f"dataset: {X.shape[0]} step candidates from {len(TRAIN_SET)} networks "
              f"({t_data:.1f} s)", flush=True)
        params, info = train(X, Y)
        info["dataset_size"] = int(X.shape[0])
        info["dataset_seconds"] = t_data
        info["topc"] = STEP_TOPC
        info["stride"] = 2
        rows = evaluate_order(params, 64)
        info["held_out"] = rows
        save(params, 64, info, out)
        print(json.dumps({k: v for k, v in info.items() if k not in ("log", "held_out")}), flush=True)
        for r in rows:
            print(r)
        g = np.array([r["greedy"] for r in rows])
        lo = np.array([r["learned"] for r in rows])
        ju = np.array([r["judged"] for r in rows])
        print("mean width greedy %.2f learned %.2f judged %.2f; mean log2 cost greedy %.3f "
              "learned %.3f judged %.3f" % (g[:, 0].mean(), lo[:, 0].mean(), ju[:, 0].mean(),
                                            g[:, 1].mean(), lo[:, 1].mean(), ju[:, 1].mean()))
    elif len(argv) > 1 and argv[1] == "train":
        X, Y = make_dataset(TRAIN_SET)
        print(f"dataset: {X.shape[0]} candidates from {len(TRAIN_SET)} networks", flush=True)
        params, info = train(X, Y)
        info["dataset_size"] = int(X.shape[0])
        save(params, 64, info)
        print(json.dumps({k: v for k, v in info.items() if k != "log"}), flush=True)
        print(info["log"][-3:])
    else:
        print(__doc__)


if __name__ == "__main__":
    main(sys.argv)
