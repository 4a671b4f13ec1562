"""Benchmark: slices/s of the sliced bucket-elimination amplitude on one GB300.

Workload (one "step" = one pass of the whole hot path): the amplitude of p=2
QAOA MaxCut on a seeded random 3-regular graph with N=80 vertices (seed 1002),
greedy min-fill order, step-dependent slicing to contraction width <= 26, all
2^k slices contracted on the GPU (complex64 steps, FP64 slice sum) and summed
into one amplitude. Synthetic data: the paper's workload is itself synthetic
(random 3-regular graphs), drawn here from a fixed seed.

Printed: one JSON line (rank 0). `value` is device-resident throughput (gate
tensors already in HBM); `e2e` goes through qt_contract with host inputs
(new angles every step: host network rebuild, upload, contraction, download).
`roofline` is the dominant kernel's algorithmic bytes over its live
CUDA-event launch times. `cpu_baseline` is the FP64 oracle on a bounded sample.
`--impl reference` times the oracle alone as the reference arm.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "slices/s & complex TFLOP/s vs plain FP32 greedy GPU path at rel.err<=1e-5"
WORKLOAD = dict(n=80, p=2, seed=1002, width_limit=26, max_vars=20, r=1, algo="greedy-minfill")
L2_FLUSH_BYTES = 512 << 20
PRECISIONS = {"fp32": 0, "tf32": 1, "bf16": 2, "3xtf32": 3, "fp64": 4}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock

# DRAM bytes (read + write) of the large launches of one amplitude pass of this workload,
# per step (a step's fold kernel included), from one ncu capture of the profiled pass
# (GB300, 1 GPU; `python bench.py --profile-pass` exited 0 first):
#   ncu --nvtx --nvtx-include "qt_pass/" --clock-control none --csv --log-file dram.csv
#       --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       python bench.py --profile-pass
# Each entry holds the kernel class the capture ran for that step: the roofline line's
# `traffic` averages the dominant class's steps that this run also gave to that class,
# and lists them with their algorithmic bytes. Used only while the kernel sources hash to
# STEP_DRAM_SOURCES (the sources the capture ran); after any change it is null.
STEP_DRAM_BYTES = {
    120: (7, 481.5e6),  # k_gemm_stream<1> (small side folded in the kernel): read 268.5 / write 213.0 MB
    131: (7, 212.3e6),  # k_gemm_stream<1>: 134.3 / 78.0
    132: (6, 440.4e6),  # k_tri_fold + k_tri_tma<4,2>: 413.4 / 27.0
}
# (under ncu the autotuner gave steps 117, 121 and 127 to the tiled GEMM's cp.async staging,
# which the timed run does not use there, so they have no entry)
STEP_DRAM_SOURCES = "f6d7dbfefd5ae8c3"
KERNEL_SOURCES = ("engine.cu", "gemm.cu", "umma.cu", "gemm.h", "qt_internal.h")


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2012_02430_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=list(PRECISIONS))
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: every rank its own amplitude; strong: one amplitude's slices "
                         "sharded over the ranks (partial sums exchanged)")
    ap.add_argument("--no-modes", action="store_true", help="skip the precision-mode table")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-slices", type=int, default=1)
    ap.add_argument("--no-all-cores", action="store_true",
                    help="skip the oracle timed over all host cores")
    ap.add_argument("--profile-pass", action="store_true",
                    help="for ncu: plan, autotune and warm the amplitude path, then run one pass "
                         "inside the NVTX range 'qt_pass' (direct launches) and print its launch list")
    ap.add_argument("--profile-sampled", action="store_true",
                    help="for ncu: a batch of 16 slices of the N=120 p=3 schedule (rank 28) in "
                         "--precision, planned and uploaded, then one run inside the NVTX range "
                         "'qt_sampled'")
    ap.add_argument("--tcgen05", type=int, default=0, choices=[0, 1, 3, 4],
                    help="with --profile-pass: QT_OPT_TCGEN05 (1: the tcgen05 GEMM kernel on every "
                         "GEMM-form launch it applies to, in the tf32 / 3xtf32 precisions)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def instance(rank):
    from paper_2012_02430_gb300.inputs import qaoa_instance, random_bitstring
    edges, gammas, betas, z = qaoa_instance(WORKLOAD["n"], WORKLOAD["p"], WORKLOAD["seed"])
    if rank:  # weak scaling: every rank its own bitstring of the same circuit
        z = random_bitstring(WORKLOAD["n"], WORKLOAD["seed"] + 7919 * rank)
    return edges, gammas, betas, z


# ------------------------------- CPU oracle ---------------------------------

def oracle_sample(n_slices, rank=0):
    """Times the FP64 oracle on `n_slices` slices of the workload (plan built first)."""
    from oracle import contract, network, ordering, slicing
    edges, gammas, betas, z = instance(rank)
    tensors, nv, norm = network.build_network(WORKLOAD["n"], edges, WORKLOAD["p"], gammas, betas, z)
    adj = ordering.adjacency_matrix(network.line_graph(tensors, nv), nv)
    plan = slicing.step_dependent_slicing(adj, ordering.MIN_FILL, WORKLOAD["width_limit"],
                                          WORKLOAD["max_vars"], WORKLOAD["r"])
    k = len(plan["sliced"])
    ids = list(range(min(n_slices, 1 << k)))
    t0 = time.perf_counter()
    contract.contract_amplitude(tensors, plan["order"], plan["sliced"], plan["slice_step"], ids)
    dt = time.perf_counter() - t0
    return len(ids), dt, k


def cpu_threads_used():
    # numpy.einsum (the oracle's contraction primitive) runs on one thread
    return 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


_WORKER_PLAN = None


def _oracle_worker_init(plan):
    global _WORKER_PLAN
    _WORKER_PLAN = plan


def _oracle_slice_worker(sid):
    """One slice of the workload on the oracle, in a spawned process (plan from the parent;
    sid < 0: start-up only)."""
    import time as _t
    from oracle import contract
    tensors, order, sliced, step = _WORKER_PLAN
    if sid < 0:
        return 0j, 0.0
    t0 = _t.perf_counter()
    total, _ = contract.contract_amplitude(tensors, order, sliced, step, [sid])
    return complex(total), _t.perf_counter() - t0


def oracle_all_cores():
    """Every slice of the workload at once, one spawned process per slice up to the host's
    cores (the paper's slice-level parallelism), the partial sums added in slice order.
    Timed from the first slice's start to the last one's end inside the workers."""
    import multiprocessing as mp
    ncpu = os.cpu_count() or 1
    from oracle import network, ordering, slicing
    edges, gammas, betas, z = instance(0)
    tensors, nv, norm = network.build_network(WORKLOAD["n"], edges, WORKLOAD["p"], gammas, betas, z)
    adj = ordering.adjacency_matrix(network.line_graph(tensors, nv), nv)
    plan = slicing.step_dependent_slicing(adj, ordering.MIN_FILL, WORKLOAD["width_limit"],
                                          WORKLOAD["max_vars"], WORKLOAD["r"])
    nsl = 1 << len(plan["sliced"])
    procs = min(ncpu, nsl)
    ctx = mp.get_context("spawn")
    wplan = (tensors, plan["order"], plan["sliced"], plan["slice_step"])
    with ctx.Pool(procs, initializer=_oracle_worker_init, initargs=(wplan,)) as pool:
        pool.map(_oracle_slice_worker, [-1] * procs)  # start-up and imports, untimed
        t0 = time.perf_counter()
        res = pool.map(_oracle_slice_worker, list(range(nsl)))
        wall = time.perf_counter() - t0
    amp = sum((r[0] for r in res), 0j) * norm
    return {"value": nsl / wall, "unit": "slices/s", "cores": procs, "host_cores": ncpu,
            "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"all {nsl} slices, one process per slice ({procs} processes of "
                      f"{ncpu} cores), FP64 numpy.einsum, partial sums added in slice order",
            "seconds": wall, "amplitude": [amp.real, amp.imag]}


def reference_arm(args):
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    per_step = max(1, args.cpu_sample_slices)
    for _ in range(args.warmup):
        oracle_sample(per_step)
    total_slices, total_t, k = 0, 0.0, 0
    for _ in range(args.steps):
        ns, dt, k = oracle_sample(per_step)
        total_slices += ns
        total_t += dt
    v = total_slices / total_t
    sample = (f"{per_step} of the 2^{k} slices per step (prefix + per-slice bucket elimination, "
              f"complex128 numpy.einsum), plan built outside the timed region")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "slices/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": "qaoa-maxcut-amplitude N=80 p=2 3-regular seed=1002 "
                               "min-fill sliced to width<=26", **WORKLOAD},
        "cpu_baseline": {"value": v, "unit": "slices/s", "cores": cpu_threads_used(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------- clocks --------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------- GPU arm -------------------------------------

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def ours(args):
    import torch

    from paper_2012_02430_gb300 import qtensor as Q

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    prec = PRECISIONS[args.precision]
    edges, gammas, betas, z = instance(rank)
    net = Q.Network(edges, WORKLOAD["n"], WORKLOAD["p"], gammas, betas, z)
    t_plan = time.perf_counter()
    width = net.order(Q.QT_GREEDY_MINFILL)
    k, sliced_width = net.slice(WORKLOAD["width_limit"], WORKLOAD["max_vars"], WORKLOAD["r"])
    t_plan = time.perf_counter() - t_plan
    nslices = 1 << k
    net.prepare(prec, batch=nslices)
    st = net.stats()
    net.upload()
    tuned = net.autotune()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    from paper_2012_02430_gb300 import dist as qdist
    if args.scaling == "strong":
        lo, hi = qdist.slice_range(nslices, rank, world)
        if hi <= lo:
            raise SystemExit("strong scaling needs at least one slice per rank")

        def step():
            net.run(lo, hi - lo, out)
    else:
        def step():
            net.run(0, nslices, out)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed between steps (outside the event pairs)
    launches0 = net.stats()["launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = net.stats()["launches"] - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    units = nslices if args.scaling == "strong" else world * nslices
    value = units * args.steps / (total_ms / 1e3)
    if args.scaling == "strong":
        amp = qdist.sharded_sum(qdist.gpu_partial(net, out), nslices, rank, world, device="cuda")
    else:
        amp = complex(out[0].item(), out[1].item())
    flops_per_step = st["prefix_flops"] + st["slice_flops"] * nslices
    bytes_per_step = (st["prefix_bytes"] + st["slice_bytes"] * nslices) * (st["elem_bytes"] // 8)
    tflops = (1 if args.scaling == "strong" else world) * flops_per_step * args.steps / (
        total_ms / 1e3) / 1e12

    # per-launch times of the same workload (events around every launch)
    Q.qt_profile(net.handle, 1)
    for i in range(max(1, min(args.steps, 5))):
        flush.fill_(i & 0xFF)
        step()
    recs = Q.qt_profile_read(net.handle)
    Q.qt_profile(net.handle, 0)
    by_kind = {}
    step_bytes = {}  # (kind, step) -> algorithmic bytes of one launch
    for r in recs:
        d = by_kind.setdefault(r["kernel"], {"ms": 0.0, "bytes": 0, "flops": 0, "n": 0})
        d["ms"] += r["ms"]
        d["bytes"] += r["bytes"]
        d["flops"] += r["flops"]
        d["n"] += 1
        step_bytes[(r["kernel"], r["step"])] = r["bytes"]
    kind_names = {0: "k_bucket_flat", 1: "k_bucket_tiled", 2: "k_finalize+k_reduce",
                  3: "gemm_form (k_gemm_pack x2 + k_gemm_tc/simt)",
                  4: "gemm_tile (k_gemm_fold + k_gemm_tma)", 5: "k_segment",
                  6: "k_tri_tma", 7: "gemm_stream (k_gemm_fold + k_gemm_stream)",
                  8: "gemm_tcgen05 (k_gemm_fold + k_gemm_umma)"}
    tot_ms = sum(d["ms"] for d in by_kind.values()) or 1.0
    dom = max(by_kind, key=lambda kk: by_kind[kk]["ms"])
    d = by_kind[dom]
    hbm_peak, peak_src = measured_peaks()
    secs = d["ms"] / 1e3 if d["ms"] > 0 else 1e-30
    intensity = d["flops"] / max(1, d["bytes"])
    ridge = FP32_PEAK_TFLOPS * 1e12 / (hbm_peak * 1e9)
    if prec != Q.QT_FP64 and intensity > ridge:
        achieved = d["flops"] / secs / 1e12
        roofline = {"bound": "alu", "kernel": kind_names[dom], "achieved": achieved,
                    "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS,
                    "peak_source": "FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flops x 2.07 GHz",
                    "hbm_achieved_gbs": d["bytes"] / secs / 1e9,
                    "hbm_frac_of_measured": d["bytes"] / secs / 1e9 / hbm_peak}
    else:
        achieved = d["bytes"] / secs / 1e9
        roofline = {"bound": "hbm", "kernel": kind_names[dom], "achieved": achieved,
                    "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                    "peak_source": f"{peak_src} hbm_gbs"}
    per_launch_bytes = d["bytes"] / max(1, d["n"])
    src_hash = kernel_sources_hash()
    # measured DRAM bytes of the dominant class's steps that the capture also ran in it
    covered = sorted(stp for (kk, stp) in step_bytes
                     if kk == dom and STEP_DRAM_BYTES.get(stp, (None,))[0] == dom)
    traffic = traffic_alg = None
    if src_hash == STEP_DRAM_SOURCES and covered:
        traffic = sum(STEP_DRAM_BYTES[stp][1] for stp in covered) / len(covered)
        traffic_alg = sum(step_bytes[(dom, stp)] for stp in covered) / len(covered)
    roofline.update({"traffic": traffic,
                     "traffic_unit": "bytes per launch (ncu dram read + write)",
                     "traffic_steps": covered if traffic is not None else [],
                     "algorithmic_bytes_per_launch_of_traffic_steps": traffic_alg,
                     "traffic_sources": {"measured_on": STEP_DRAM_SOURCES, "now": src_hash},
                     "algorithmic_bytes_per_launch": per_launch_bytes,
                     "launches": d["n"], "flop_per_byte": intensity,
                     "ridge_flop_per_byte": ridge,
                     "share": {kind_names[kk]: by_kind[kk]["ms"] / tot_ms for kk in by_kind}})

    # the plain FP32 greedy GPU path: one launch per bucket (no fused groups), default
    # kernel variants, same slices; device-resident like `value`
    plain = Q.Network(edges, WORKLOAD["n"], WORKLOAD["p"], gammas, betas, z)
    Q.qt_set_option(plain.handle, Q.QT_OPT_FUSION, 0)
    plain.order(Q.QT_GREEDY_MINFILL)
    plain.slice(WORKLOAD["width_limit"], WORKLOAD["max_vars"], WORKLOAD["r"])
    plain.prepare(prec, batch=nslices)
    plain.upload()
    pout = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(3):
        plain.run(0, nslices, pout)
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        pev[i][0].record(stream)
        plain.run(0, nslices, pout)
        pev[i][1].record(stream)
    torch.cuda.synchronize()
    plain_ms = sum(a.elapsed_time(b) for a, b in pev)
    plain_amp = complex(pout[0].item(), pout[1].item())
    plain_line = {"value": nslices * args.steps / (plain_ms / 1e3), "unit": "slices/s",
                  "ms_per_step": plain_ms / args.steps,
                  "complex_tflops": flops_per_step * args.steps / (plain_ms / 1e3) / 1e12,
                  "launch_bytes_per_step": plain.stats()["slice_launch_bytes"] * nslices,
                  "rel_diff_vs_value": abs(plain_amp - amp) / abs(plain_amp)}
    del plain

    energy_line = batched_energy(args, Q, torch, flush, stream)
    sweep_line = angle_sweep(args, Q, torch, flush, stream)
    batch_line = batched_amplitudes(args, Q, torch, edges, gammas, betas, z, prec, flush, stream,
                                    total_ms / args.steps)
    order_line = orderings(Q, edges, gammas, betas, z)
    modes_line = None if args.no_modes else precision_modes(Q, torch, edges, gammas, betas, z,
                                                            flush, stream)
    c3_line = None if args.no_modes else mixed_precision_c3(args, Q, torch, flush, stream)
    paper_line = None if args.no_modes else paper_shape_amplitude(args, Q, torch, flush, stream)
    c5_line = None if args.no_modes else planner_comparison(Q)

    # end to end: host inputs -> amplitude on the host, through qt_contract
    from paper_2012_02430_gb300.inputs import random_angles
    e2e_steps = max(3, min(args.steps, 10))
    gstage = st.get("workspace_bytes", 0)
    for i in range(max(3, args.warmup)):  # untimed: the first call re-captures the graph
        g2, b2 = random_angles(WORKLOAD["p"], 4000 + i)
        Q.qt_set_angles(net.handle, g2, b2)
        net.contract(prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        g2, b2 = random_angles(WORKLOAD["p"], 5000 + i)
        Q.qt_set_angles(net.handle, g2, b2)
        net.contract(prec)
    t_e2e = time.perf_counter() - t0
    h2d = gate_upload_bytes(st)
    e2e = {"value": world * nslices * e2e_steps / t_e2e, "unit": "slices/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16,
           "ms_per_step": 1e3 * t_e2e / e2e_steps,
           "includes": "qt_set_angles (host tensors) + qt_contract (H2D gates, all slices, D2H amplitude, stream sync)"}
    del gstage

    # angle sweep of the amplitude: 16 sets through one qt_contract_sweep call
    n_sw = 16
    sw_sets = [random_angles(WORKLOAD["p"], 6000 + i) for i in range(n_sw)]
    sw_g = [list(g2) for g2, _ in sw_sets]
    sw_b = [list(b2) for _, b2 in sw_sets]
    net.contract_sweep(sw_g, sw_b, prec)  # warm: workspace, graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.contract_sweep(sw_g, sw_b, prec)
    t_sw = time.perf_counter() - t0
    amp_sweep_line = {"workload": f"{n_sw} angle sets of the same amplitude, one qt_contract_sweep",
                      "ms_per_sweep": 1e3 * t_sw, "amplitudes_per_s": n_sw / t_sw,
                      "slices_per_s": n_sw * nslices / t_sw,
                      "includes": "host gate images of every set, one H2D, per set: gate copy "
                                  "+ graph replay, one D2H of the amplitudes"}

    line = {
        "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None,
        "dtype": "c128" if prec == Q.QT_FP64 else "c64", "data": "synthetic",
        "config": {"workload": "qaoa-maxcut-amplitude N=80 p=2 3-regular seed=1002 "
                               "min-fill sliced to width<=26",
                   **WORKLOAD, "k": k, "slices": nslices, "width": width,
                   "sliced_width": sliced_width, "precision": args.precision,
                   "l2": "flushed between steps (512 MiB write outside the timed events)",
                   "autotuned_variants": {str(t["step"]): t["variant"] for t in tuned},
                   "plan_seconds": t_plan},
        "complex_tflops": tflops, "ledger_flops_per_step": flops_per_step,
        "ledger_bytes_per_step": bytes_per_step,
        "launch_bytes_per_step": (st["prefix_launch_bytes"] + st["slice_launch_bytes"] * nslices)
        * (st["elem_bytes"] // 8),
        "plain_fp32_greedy_path": plain_line,
        "batched_energy": energy_line,
        "batched_amplitudes": batch_line,
        "angle_sweep": sweep_line,
        "amplitude_sweep": amp_sweep_line,
        "orderings": order_line,
        "precision_modes": modes_line,
        "mixed_precision_n120_p3": c3_line,
        "paper_shape_n210_p1": paper_line,
        "learned_vs_greedy_n210_p3": c5_line,
        "amplitude": [amp.real, amp.imag],
        "gpu_launches": launches,
        "roofline": roofline, "clocks": clk, "e2e": e2e,
    }
    # the whole pass against HBM: the fused launches' algorithmic bytes over the step time
    pass_bytes = line["launch_bytes_per_step"]
    hbm_peak, peak_src = measured_peaks()
    line["pass_roofline"] = {"bound": "hbm", "algorithmic_bytes": pass_bytes,
                             "achieved": pass_bytes / (total_ms / args.steps / 1e3) / 1e9,
                             "peak": hbm_peak, "unit": "GB/s",
                             "frac": pass_bytes / (total_ms / args.steps / 1e3) / 1e9 / hbm_peak,
                             "peak_source": f"{peak_src} hbm_gbs"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns, dt, _ = oracle_sample(args.cpu_sample_slices)
        line["cpu_baseline"] = {"value": ns / dt, "unit": "slices/s", "cores": cpu_threads_used(),
                                "host_cores": os.cpu_count(), "cpu_model": cpu_model(),
                                "kind": "oracle",
                                "sample": f"{ns} slice(s) of the same workload, FP64 oracle "
                                          f"(numpy.einsum bucket elimination), {dt:.1f} s"}
        if not args.no_all_cores:
            line["cpu_baseline_all_cores"] = oracle_all_cores()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


ENERGY_WORKLOAD = dict(n=1000, p=2, seed=1004)
# mixed precision: p=3 on a random 3-regular graph with N=120, sliced with 43 variables so
# that every slice's widest step has 28 indices (each slice fixes all sliced indices after
# the first round's step); accuracy on the N=50 p=3 stand-in over 64 seeded bitstrings
C3_WORKLOAD = dict(n=120, p=3, seed=1003, width_limit=28, max_vars=43, r=1)
C3_STAND_IN = dict(n=50, p=3, seed=1003, width_drop=6, max_vars=10, bitstrings=64)
C3_SAMPLED = 1024


PAPER_SHAPE = dict(n=210, p=1, seed=1005, width_limit=30, max_vars=12, r=1)
C5_WORKLOAD = dict(n=210, p=3, seed=1005, width_limit=30, max_vars=12, r=1)


def paper_shape_amplitude(args, Q, torch, flush, stream):
    """The paper's own experiment shape (one amplitude of p=1 QAOA on a 210-vertex random
    3-regular graph; Sec. VIII ran it on 1,024 Theta nodes): sliced to rank 30 and every
    slice contracted on one GPU (FP32, autotuned, CUDA events, L2 flushed)."""
    from paper_2012_02430_gb300.inputs import qaoa_instance
    w = PAPER_SHAPE
    edges, g, b, z = qaoa_instance(w["n"], w["p"], w["seed"])
    net = Q.Network(edges, w["n"], w["p"], g, b, z)
    width = net.order(Q.QT_GREEDY_MINFILL)
    t0 = time.perf_counter()
    k, planned = net.slice(w["width_limit"], w["max_vars"], w["r"])
    t_plan = time.perf_counter() - t0
    net.prepare(Q.QT_FP32_SIMT, batch=1)
    need1 = net.stats()["workspace_bytes"]
    batch = max(1, min(1 << k, int((96 << 30) // max(1, need1))))
    net.prepare(Q.QT_FP32_SIMT, batch=batch)
    st = net.stats()
    net.upload()
    net.autotune()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    net.run(0, 1 << k, out)
    times = []
    for i in range(3):
        flush.fill_(i & 0xFF)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        net.run(0, 1 << k, out)
        e.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(e))
    ms = statistics.median(times)
    flops = st["prefix_flops"] + st["slice_flops"] * (1 << k)
    return {"workload": "amplitude of p=1 QAOA MaxCut, random 3-regular N=210 seed 1005, "
                        "min-fill, sliced to rank 30, all slices",
            "greedy_width": width, "k": k, "slices": 1 << k, "planned_width": planned,
            "executed_slice_width": st["slice_width"], "batch": batch,
            "workspace_gb": st["workspace_bytes"] / 1e9, "ms_per_amplitude": ms,
            "slices_per_s": (1 << k) / (ms / 1e3), "complex_tflops": flops / (ms / 1e3) / 1e12,
            "plan_seconds": t_plan, "amplitude": [out[0].item(), out[1].item()],
            "context": "the paper: one amplitude of this shape (its decomposition: width 44) on "
                       "1,024 nodes of Theta; widths differ with the gate decomposition"}


def planner_comparison(Q):
    """Slicing plans of N=210 p=3 QAOA (rank target 30, 12 sliced variables) by the
    paper's search (every step up to the peak, max-degree vertex), the learned proposals
    (the committed GPU-trained model's top 8 per round) and the same budget without a
    model (8 candidates evenly spaced): plan width, log2 plan cost (sum of 2^w), greedy
    ordering runs and seconds. Greedy (no slicing) for reference."""
    import ctypes as C
    import math
    import numpy as np
    from paper_2012_02430_gb300 import learn
    from paper_2012_02430_gb300.inputs import qaoa_instance
    params, hidden, _ = learn.load()
    w = C5_WORKLOAD
    edges, g, b, z = qaoa_instance(w["n"], w["p"], w["seed"])
    res = {"workload": f"N={w['n']} p={w['p']} seed {w['seed']}, width target "
                       f"{w['width_limit']}, {w['max_vars']} sliced variables"}
    for mode in ("greedy", "paper_search", "learned_top8", "budget8_no_model"):
        h = Q.qt_build_network(edges, w["n"], w["p"], g, b, z)
        try:
            w0 = Q.qt_order(h, Q.QT_GREEDY_MINFILL)
            k, wd = C.c_int32(0), C.c_int32(w0)
            t0 = time.perf_counter()
            if mode == "paper_search":
                Q._check(Q.lib.qt_slice(h, w["width_limit"], w["max_vars"], w["r"], C.byref(k),
                                        C.byref(wd)))
            elif mode != "greedy":
                pa = np.ascontiguousarray(params, dtype=np.float32)
                pp = pa.ctypes.data_as(C.POINTER(C.c_float)) if mode == "learned_top8" else None
                Q._check(Q.lib.qt_slice_learned(h, pp, hidden, w["width_limit"], w["max_vars"],
                                                w["r"], 3, 8 if pp is not None else 0,
                                                0 if pp is not None else 8, C.byref(k),
                                                C.byref(wd)))
            dt = time.perf_counter() - t0
            runs, cost = C.c_int64(), C.c_double()
            Q._check(Q.lib.qt_plan_info(h, C.byref(runs), C.byref(cost)))
            res[mode] = {"plan_width": wd.value, "k": k.value,
                         "log2_plan_cost": math.log2(cost.value),
                         "greedy_runs": runs.value, "seconds": dt}
        finally:
            Q.qt_free(h)
    res["elimination_orders"] = order_comparison(Q)
    return res


def order_comparison(Q):
    """Unsliced elimination orders of the N=210 p=3 and N=120 p=3 networks: min-fill,
    min-degree, one Boltzmann-randomised greedy run (rgreedy, tau 0.1) and the learned
    elimination-step proposals (the committed model picks among the 4 best min-fill
    candidates at every step; min-fill judges, 2 ordering runs): width, log2 of the sum
    of 2^w over the steps, and seconds."""
    import json
    import math
    import numpy as np
    from paper_2012_02430_gb300 import learn
    from paper_2012_02430_gb300.inputs import qaoa_instance
    with open(learn.ORDER_WEIGHTS) as f:
        d = json.load(f)
    params, hidden = np.array(d["params"], dtype=np.float32), int(d["hidden"])
    out = {}
    for n, p, seed in ((C5_WORKLOAD["n"], C5_WORKLOAD["p"], C5_WORKLOAD["seed"]),
                       (C3_WORKLOAD["n"], C3_WORKLOAD["p"], C3_WORKLOAD["seed"])):
        edges, g, b, z = qaoa_instance(n, p, seed)
        row = {}
        h = Q.qt_build_network(edges, n, p, g, b, z)
        try:
            for name, run in (("min_fill", lambda: Q.qt_order(h, Q.QT_GREEDY_MINFILL)),
                              ("min_degree", lambda: Q.qt_order(h, Q.QT_GREEDY_MINDEG)),
                              ("rgreedy_q1", lambda: Q.qt_order_rgreedy(h, 0.1, 1, 1))):
                t0 = time.perf_counter()
                run()
                dt = time.perf_counter() - t0
                ws = Q.qt_get_widths(h)
                row[name] = {"width": max(ws),
                             "log2_cost": math.log2(sum(math.ldexp(1.0, x) for x in ws)),
                             "seconds": dt}
        finally:
            Q.qt_free(h)
        t0 = time.perf_counter()
        wd, lc, kept = learn.order_with((n, p, seed), params, hidden, learn.STEP_TOPC, 1)
        row["learned_judged"] = {"width": wd, "log2_cost": lc, "learned_kept": bool(kept),
                                 "seconds": time.perf_counter() - t0}
        out[f"N={n} p={p} seed {seed}"] = row
    return out


def mixed_precision_c3(args, Q, torch, flush, stream):
    """Sampled-slice throughput of the N=120 p=3 schedule (1,024 consecutive slice ids
    from a seeded offset; slices are independent units of the amplitude, Eq. 2) in FP32
    and split TF32, with the projected time to the full amplitude; and each precision
    mode's relative error on 64 seeded bitstrings of the N=50 p=3 stand-in against the
    FP64 path (which the GPU tests hold within 1e-10 of the oracle)."""
    import statistics as stats
    from paper_2012_02430_gb300.inputs import qaoa_instance, random_bitstring, random_slice_ids
    w = C3_WORKLOAD
    edges, g, b, z = qaoa_instance(w["n"], w["p"], w["seed"])
    sampled = {}
    for name in ("fp32", "3xtf32"):
        net = Q.Network(edges, w["n"], w["p"], g, b, z)
        width = net.order(Q.QT_GREEDY_MINFILL)
        t0 = time.perf_counter()
        k, planned = net.slice(w["width_limit"], w["max_vars"], w["r"])
        t_plan = time.perf_counter() - t0
        net.prepare(PRECISIONS[name], batch=1)
        st1 = net.stats()
        batch = max(1, min(C3_SAMPLED, int((64 << 30) // max(1, st1["workspace_bytes"]))))
        net.prepare(PRECISIONS[name], batch=batch)
        st = net.stats()
        net.upload()
        net.autotune()
        first = random_slice_ids(k, 1, 4242)[0] & ~(C3_SAMPLED - 1)
        first = min(first, (1 << k) - C3_SAMPLED)
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        net.run(first, C3_SAMPLED, out)
        torch.cuda.synchronize()
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        net.run(first, C3_SAMPLED, out)
        e.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(e)
        sps = C3_SAMPLED / (ms / 1e3)
        sampled[name] = {"slices_per_s": sps,
                         "complex_tflops": st["slice_flops"] * C3_SAMPLED / (ms / 1e3) / 1e12,
                         "ms_per_1024_slices": ms, "batch": batch,
                         "projected_seconds_to_amplitude": (2.0 ** k) / sps,
                         "projected_years_to_amplitude": (2.0 ** k) / sps / 3.156e7}
        sampled["schedule"] = {"n": w["n"], "p": w["p"], "seed": w["seed"], "greedy_width": width,
                               "k": k, "executed_slice_width": st["slice_width"],
                               "prefix_width": st["prefix_width"], "planned_width": planned,
                               "slice_flops": st["slice_flops"], "first_slice_id": first,
                               "plan_seconds": t_plan}
        del net
    # accuracy over 64 bitstrings of the stand-in
    si = C3_STAND_IN
    e2, g2, b2, z2 = qaoa_instance(si["n"], si["p"], si["seed"])
    bits = [random_bitstring(si["n"], 9000 + q) for q in range(si["bitstrings"])]
    amps = {}
    for name in ("fp64", "fp32", "3xtf32", "tf32", "bf16"):
        net = Q.Network(e2, si["n"], si["p"], g2, b2, z2)
        wd = net.order(Q.QT_GREEDY_MINFILL)
        k2, _ = net.slice(wd - si["width_drop"], si["max_vars"], 1)
        net.prepare(PRECISIONS[name], batch=1 << k2)
        res = []
        for zq in bits:
            Q.qt_set_bitstring(net.handle, zq)
            res.append(net.contract(PRECISIONS[name]))
        amps[name] = res
        del net
    acc = {"stand_in": f"N={si['n']} p={si['p']} seed {si['seed']}, greedy width - "
                       f"{si['width_drop']}, {si['bitstrings']} seeded bitstrings",
           "reference": "the FP64 path (held within 1e-10 of the oracle by the GPU tests)"}
    for name in ("fp32", "3xtf32", "tf32", "bf16"):
        errs = [abs(x - r) / abs(r) for x, r in zip(amps[name], amps["fp64"])]
        acc[name] = {"max_rel_err": max(errs), "median_rel_err": stats.median(errs)}
    return {"sampled_slices": sampled, "accuracy_64_bitstrings": acc}


def precision_modes(Q, torch, edges, gammas, betas, z, flush, stream, reps=5):
    """Every precision mode on the same workload (autotuned, device-resident, CUDA events,
    L2 flushed between runs): ms per amplitude and rel.err against the FP64 path (which the
    GPU tests hold within 1e-10 of the oracle)."""
    res, ref = {}, None
    for name in ("fp64", "fp32", "3xtf32", "tf32", "bf16"):
        net = Q.Network(edges, WORKLOAD["n"], WORKLOAD["p"], gammas, betas, z)
        net.order(Q.QT_GREEDY_MINFILL)
        k, _ = net.slice(WORKLOAD["width_limit"], WORKLOAD["max_vars"], WORKLOAD["r"])
        net.prepare(PRECISIONS[name], batch=1 << k)
        net.upload()
        net.autotune()
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        for _ in range(3):
            net.run(0, 1 << k, out)
        tot = 0.0
        for i in range(reps):
            flush.fill_(i & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            net.run(0, 1 << k, out)
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        amp = complex(out[0].item(), out[1].item())
        ref = amp if ref is None else ref
        st = net.stats()
        res[name] = {"ms_per_amplitude": tot / reps, "slices_per_s": (1 << k) / (tot / reps / 1e3),
                     "rel_err_vs_fp64": abs(amp - ref) / abs(ref),
                     "tensor_core_shape_flop_fraction": st["tensor_core_shape_flops"] / st["job_flops"]}
        del net
    return res


def batched_energy(args, Q, torch, flush, stream):
    """Secondary measurement: the p=2 MaxCut energy of a random 3-regular graph with
    N=1000 (1500 lightcone networks) as one persistent launch (CUDA-graph replay),
    device-resident, autotuned block size; CUDA events, L2 flushed between evaluations."""
    from paper_2012_02430_gb300.inputs import qaoa_instance
    n, p, seed = ENERGY_WORKLOAD["n"], ENERGY_WORKLOAD["p"], ENERGY_WORKLOAD["seed"]
    edges, g, b, _ = qaoa_instance(n, p, seed)
    en = Q.Energy(edges, n, p, g, b)
    en.prepare(Q.QT_FP32_SIMT)
    en.upload()
    threads = en.autotune()
    zz = torch.zeros(len(edges), dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(3):
        en.run(zz, E)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        en.run(zz, E)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b2) for a, b2 in ev) / args.steps
    st = en.stats()
    t0 = time.perf_counter()
    for _ in range(3):
        E_host, _ = en.compute(Q.QT_FP32_SIMT)
    e2e_ms = 1e3 * (time.perf_counter() - t0) / 3
    return {"workload": f"p={p} MaxCut energy, random 3-regular N={n} seed={seed}, "
                        f"{len(edges)} lightcone networks, one persistent launch",
            "edges_per_s": len(edges) / (ms / 1e3), "ms_per_energy": ms,
            "energy": float(E.item()), "e2e_ms_per_energy": e2e_ms,
            "e2e_includes": "upload of gates and step tables, launch, D2H of zz and energy",
            "block_threads": threads, "blocks": st["blocks"], "lightcone_width_hist": st["width_hist"],
            "ledger_flops": st["flops"], "launch_bytes": st["bytes"],
            "upload_bytes": st["upload_bytes"]}


SWEEP_SETS = 64  # angle sets of the sweep measurement


def angle_sweep(args, Q, torch, flush, stream):
    """Energies of SWEEP_SETS angle sets of the batched-energy graph in one persistent
    launch over (set, edge) work items (orders and schedules reused): device time of the
    launch (gate images already resident), and end to end with the host gate images,
    the copies and the D2H of the energies."""
    from paper_2012_02430_gb300.inputs import qaoa_instance, random_angles
    n, p, seed = ENERGY_WORKLOAD["n"], ENERGY_WORKLOAD["p"], ENERGY_WORKLOAD["seed"]
    edges, g, b, _ = qaoa_instance(n, p, seed)
    en = Q.Energy(edges, n, p, g, b)
    en.prepare(Q.QT_FP32_SIMT)
    en.upload()
    en.autotune()
    sets = [random_angles(p, 7000 + q) for q in range(SWEEP_SETS)]
    gs, bs = [x[0] for x in sets], [x[1] for x in sets]
    en.sweep_prepare(SWEEP_SETS)
    energies = torch.zeros(SWEEP_SETS, dtype=torch.float64, device="cuda")
    en.sweep_upload(gs, bs)
    for _ in range(3):
        en.sweep_run(SWEEP_SETS, energies)
    reps = max(3, min(args.steps, 10))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for i in range(reps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        en.sweep_run(SWEEP_SETS, energies)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b2) for a, b2 in ev) / reps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        en.sweep(gs, bs, energies)
        host = energies.cpu()
    e2e_ms = 1e3 * (time.perf_counter() - t0) / 3
    return {"workload": f"{SWEEP_SETS} angle sets of the p={p} N={n} energy, one launch",
            "ms_per_sweep": ms, "energies_per_s": SWEEP_SETS / (ms / 1e3),
            "lightcones_per_s": SWEEP_SETS * len(edges) / (ms / 1e3),
            "e2e_ms_per_sweep": e2e_ms,
            "e2e_includes": "host gate images for every set, H2D, launch, D2H of the energies",
            "energy_first_set": float(host[0].item())}


BATCH_OPEN = 8  # open qubits of the batched-amplitude measurement: 2^8 amplitudes


def batched_amplitudes(args, Q, torch, edges, gammas, betas, z, prec, flush, stream, ms_single):
    """Sec. VII: the same circuit with BATCH_OPEN output indices left open (the lowest-id
    qubits), planned with the same rule and width limit; 2^a amplitudes per contraction.
    Device-resident, autotuned, CUDA events, L2 flushed between runs."""
    n, p = WORKLOAD["n"], WORKLOAD["p"]
    net = Q.Network(edges, n, p, gammas, betas, z)
    net.set_open(list(range(BATCH_OPEN)))
    w = net.order(Q.QT_GREEDY_MINFILL)
    k, sw = net.slice(WORKLOAD["width_limit"], WORKLOAD["max_vars"], WORKLOAD["r"])
    net.prepare(prec, batch=1 << k)
    net.upload()
    net.autotune()
    out = torch.zeros(2 << BATCH_OPEN, dtype=torch.float64, device="cuda")
    for _ in range(3):
        net.run(0, 1 << k, out)
    reps = max(3, min(args.steps, 10))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for i in range(reps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        net.run(0, 1 << k, out)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b2) for a, b2 in ev) / reps
    return {"open_qubits": BATCH_OPEN, "amplitudes": 1 << BATCH_OPEN, "width": w, "k": k,
            "sliced_width": sw, "ms_per_batch": ms, "amplitudes_per_s": (1 << BATCH_OPEN) / (ms / 1e3),
            "ms_single_amplitude": ms_single,
            "cost_ratio_vs_single": ms / ms_single}


def orderings(Q, edges, gammas, betas, z, taus=(0.1, 0.3, 1.0), q=128, seed=1):
    """Sec. V.A: contraction width of the bench circuit under the greedy rules and rgreedy
    (best of q Boltzmann-weighted runs), with the host planner's wall time."""
    n, p = WORKLOAD["n"], WORKLOAD["p"]
    h = Q.qt_build_network(edges, n, p, gammas, betas, z)
    res = {}
    try:
        for name, algo in (("greedy_minfill", Q.QT_GREEDY_MINFILL), ("greedy_mindeg", Q.QT_GREEDY_MINDEG)):
            t0 = time.perf_counter()
            res[name] = {"width": Q.qt_order(h, algo), "seconds": time.perf_counter() - t0}
        for tau in taus:
            t0 = time.perf_counter()
            w = Q.qt_order_rgreedy(h, tau, q, seed)
            res[f"rgreedy_tau{tau}_q{q}"] = {"width": w, "seconds": time.perf_counter() - t0}
    finally:
        Q.qt_free(h)
    return res


def gate_upload_bytes(st):
    """Bytes of the host-to-device copies of one qt_contract (gates, gate meta, scalar table)."""
    return int(st.get("upload_bytes", 0))


def profile_pass(args):
    """One amplitude pass of the bench workload for ncu (--nvtx --nvtx-include qt_pass/):
    same plan, precision, batch and autotuned variants as the timed steps; no L2 flush."""
    import torch

    from paper_2012_02430_gb300 import qtensor as Q
    prec = PRECISIONS[args.precision]
    edges, gammas, betas, z = instance(0)
    net = Q.Network(edges, WORKLOAD["n"], WORKLOAD["p"], gammas, betas, z)
    net.order(Q.QT_GREEDY_MINFILL)
    k, _ = net.slice(WORKLOAD["width_limit"], WORKLOAD["max_vars"], WORKLOAD["r"])
    Q.qt_set_option(net.handle, Q.QT_OPT_GRAPHS, 0)
    Q.qt_set_option(net.handle, Q.QT_OPT_TCGEN05, args.tcgen05)
    net.prepare(prec, batch=1 << k)
    net.upload()
    net.autotune()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(max(3, args.warmup)):
        net.run(0, 1 << k, out)
    Q.qt_profile(net.handle, 1)
    net.run(0, 1 << k, out)
    torch.cuda.synchronize()
    recs = Q.qt_profile_read(net.handle)
    Q.qt_profile(net.handle, 0)
    torch.cuda.nvtx.range_push("qt_pass")
    net.run(0, 1 << k, out)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"profile_pass": [[r["step"], r["kernel"], round(r["ms"], 4)] for r in recs],
                      "amplitude": [out[0].item(), out[1].item()]}))


def profile_sampled(args):
    """A 16-slice batch of the N=120 p=3 schedule (the many-slice workload's plan; 4 GB of
    workspace) for ncu (--nvtx --nvtx-include qt_sampled/): no autotuning, so the kernel
    choices are the defaults of --precision and --tcgen05."""
    import torch

    from paper_2012_02430_gb300 import qtensor as Q
    from paper_2012_02430_gb300.inputs import qaoa_instance, random_slice_ids
    w = C3_WORKLOAD
    edges, g, b, z = qaoa_instance(w["n"], w["p"], w["seed"])
    net = Q.Network(edges, w["n"], w["p"], g, b, z)
    Q.qt_set_option(net.handle, Q.QT_OPT_GRAPHS, 0)
    Q.qt_set_option(net.handle, Q.QT_OPT_TCGEN05, args.tcgen05)
    net.order(Q.QT_GREEDY_MINFILL)
    k, _ = net.slice(w["width_limit"], w["max_vars"], w["r"])
    net.prepare(PRECISIONS[args.precision], batch=16)
    net.upload()
    first = random_slice_ids(k, 1, 4242)[0] & ~1023
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    net.run(first, 16, out)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("qt_sampled")
    net.run(first, 16, out)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"profile_sampled": {"k": k, "first_slice": first, "slices": 16,
                                          "workspace_gb": net.stats()["workspace_bytes"] / 1e9,
                                          "tcgen05_gemm_launches": net.stats()["tcgen05_gemm_launches"],
                                          "sum": [out[0].item(), out[1].item()]}}))


def main():
    args = parse()
    if args.profile_sampled:
        profile_sampled(args)
        return
    if args.profile_pass:
        profile_pass(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
