#!/usr/bin/env python
"""Throughput of one hash-encoded neural-volume training step (config 2) on GB300.

A step is one pass of the training hot path over a 2^18-point batch: Philox
sampling of the points and trilinear ground truth from a 128^3 blob volume,
hash encoding (L16 F2 T2^19), MLP forward, L2 loss, hand-written backward with
the table scatter-add, and the dense Adam update of all 16.8 M parameters.
The metric is training samples per second (decoded samples through the
forward + backward); the JSON line also carries the dominant kernel's
roofline, the end-to-end number through the C ABI with host buffers, and the
FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp16|bf16] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decoded samples/s (hash enc+MLP fwd/bwd), 1080p frame ms; PSNR vs FP64 oracle"
UNIT = "samples/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto", choices=["auto", "fp32", "fp16", "bf16"])
    ap.add_argument("--cpu-points", type=int, default=1 << 18, help="oracle sample size (points)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default="", choices=["", "train_cfg2", "render1080p"],
                    help="run one profiling case instead of the benchmark")
    ap.add_argument("--extras", default="cfg2_quality,cfg3_render,cfg4_inloop,cfg5_ooc",
                    help="comma list of extra measurements (empty for none)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region (median SM clock, throttle reasons)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    from paper_2207_11620_gb300 import replicas
    return replicas.setup()


def barrier(ws):
    from paper_2207_11620_gb300 import replicas
    replicas.barrier(ws)


def max_over_ranks(ws, v):
    from paper_2207_11620_gb300 import replicas
    return replicas.max_over_ranks(ws, v)


# ------------------------------------------------------------------- oracle ---

def oracle_step_rate(cpu_points: int):
    """FP64 oracle on a bounded sample of the config-2 step: one training step on
    `cpu_points` points plus the dense Adam over all parameters, extrapolated to a
    2^18-point step.  Returns (samples/s, threads, seconds, description)."""
    import oracle as O
    from paper_2207_11620_gb300 import configs as CF
    from paper_2207_11620_gb300 import inputs as I
    c = CF.CFG2["net"]
    net = O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)
    params = I.init_params(net.n_table, net.n_weights, seed=5, dims=c.dims)
    vol = I.blob_volume(CF.CFG2["volume"], seed=CF.CFG2["volume_seed"])
    x = O.sample_points(1234, 0, 0, cpu_points)
    t = O.trilinear(vol, x).astype(np.float32)
    tr = O.Trainer(net, params)
    t0 = time.perf_counter()
    tr.step(x, t)
    t_step = time.perf_counter() - t0
    p, g, m, v = tr.params.copy(), tr.grads.copy(), tr.m.copy(), tr.v.copy()
    t0 = time.perf_counter()
    O.adam(p, g, m, v, 2)
    t_adam = time.perf_counter() - t0
    per_point = max(t_step - t_adam, 1e-12) / cpu_points
    batch = CF.CFG2["batch"]
    rate = batch / (t_adam + batch * per_point)
    desc = (f"one oracle training step on {cpu_points} of the 2^18 config-2 points (forward, backward and "
            f"the dense Adam over {net.n_params} params on {O.num_threads()} threads); per-point cost "
            f"extrapolated to a 2^18-point step")
    return rate, O.num_threads(), t_step + t_adam, desc


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    rates = []
    secs = 0.0
    desc = ""
    threads = 1
    for i in range(args.warmup + args.steps):
        r, threads, s, desc = oracle_step_rate(args.cpu_points)  # the sample of ours' cpu_baseline
        if i >= args.warmup:
            rates.append(r)
            secs += s
    value = float(statistics.median(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "cfg2 training step: 128^3 blob volume, L16 F2 T2^19 Nmin16 b1.38, "
                               "MLP 32-64-64-1, 2^18 points, L2, Adam", "global_batch": 1 << 18},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ roofline ---

# the sources the config-2 step's kernels (k_encode_tiles, k_mlp_tc, k_fold_replicas, k_adam) compile from
STEP_SOURCES = ("k_grid.cu", "k_tc.cu", "k_adam.cu", "tc_grid.cuh", "tc_ptx.cuh", "nv_internal.cuh")


def csrc_digest():
    """SHA-256 over the CUDA sources of the config-2 step's kernels (names and contents)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2207_11620_gb300", "csrc")
    h = hashlib.sha256()
    for name in STEP_SOURCES:
        h.update(name.encode())
        with open(os.path.join(d, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def ncu_traffic(kernel):
    """(DRAM bytes per launch of a kernel from the committed ncu summary, note).

    The summary records the digest of the CUDA sources it was captured from; once
    the sources differ the figure no longer describes the kernel and is withheld."""
    p = os.path.join(ROOT, "profiles", "dram_traffic_cfg2.txt")
    if not os.path.exists(p):
        return None, "no committed capture"
    digest, val = None, None
    for line in open(p):
        if line.startswith("# csrc_sha256"):
            digest = line.split()[-1]
        f = line.split("#", 1)[0].split()
        if len(f) >= 2 and f[0] == kernel:
            val = int(f[1])
    if val is None:
        return None, "kernel not in the committed capture"
    if digest != csrc_digest():
        return None, "the step kernels' sources changed since the committed capture (profiles/dram_traffic_cfg2.txt)"
    return val, "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, committed capture " \
                "(profiles/dram_traffic_cfg2.txt) of these sources"


def l2_peaks(nv, torch):
    """Measured rates (accesses/s) of scattered 16-byte FP32 vector reductions into a 64 MiB buffer and of
    scattered 16-byte loads from a 32 MiB buffer -- the L2-resident sizes of config 2's FP32 table gradient
    and 16-bit tables -- by the library's measurement kernels; median of 5 launches of 2^26 accesses."""
    ops = 1 << 26
    red_buf = torch.zeros((1 << 22, 4), dtype=torch.float32, device="cuda")
    ld_buf = torch.ones((1 << 21, 4), dtype=torch.float32, device="cuda")
    sink = torch.zeros(1024, dtype=torch.int32, device="cuda")

    def rate(fn):
        fn(0)
        torch.cuda.synchronize()
        ts = []
        for s in range(1, 6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(s)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ops / (statistics.median(ts) / 1e3)
    red = rate(lambda s: nv.peak_scatter(red_buf, ops, seed=s))
    ld = rate(lambda s: nv.peak_gather(ld_buf, ops, sink, seed=s))
    l1 = rate(lambda s: nv.peak_gather(ld_buf[: 1 << 11], ops, sink, seed=s))
    del red_buf, ld_buf
    return {"scatter_reductions_per_s": red, "gather_loads_per_s": ld, "l1_gather_loads_per_s": l1,
            "how": "2^26 scattered 16-byte FP32 vector reductions into 64 MiB / 16-byte loads from 32 MiB / "
                   "16-byte loads from an L1-resident 32 KiB, median of 5 launches (nv_peak_scatter / "
                   "nv_peak_gather)"}


def roofline_of(kind, avg, prec, pk, pk_kind, batch, n_visit, n_table, d, L, F, l2pk=None):
    """Roofline of one kernel of the config-2 step from its live average launch time.

    Algorithmic bytes / FLOPs per launch (per unit x units):
      adam     34 B per parameter it visits (read p, g, m, v; write p, m, v, g = 0, 16-bit shadow);
               32 in FP32.  n_visit: the parameters in blocks that hold a weight or a hash slot a
               point of [0,1]^3 can reach (nv_adam_span); the other blocks stay unchanged.  Bound: HBM
      encode   per point: 8 corners x L levels x F 16-bit features gathered (8 L F 2 B) + the 8
               voxels of the trilinear target (32 B).  Bound: scattered loads that resolve in L1 / L2
               (the 16-bit tables are L2-resident), against the measured rate of scattered 16-byte
               loads x 16 B.  Also reported against HBM: those bytes + the feature row (2 D0 B) and
               target (4 B) written
      mlp      tensor-core path, per point: the table-gradient scatter, 8 corners x L x F FP32
               reductions (8 L F 4 B).  Bound: scattered vector reductions that resolve in L2 (the
               FP32 table gradient is L2-resident), against the measured rate of scattered 16-byte
               FP32 reductions x 16 B.  Also reported: against HBM, those bytes + the feature row
               read (2 D0 B) + the target (4 B); tensor FLOPs 2 (D0 64 + 64 64) forward + 2 (2 64 64
               + 2 64 D0) backward.  FP32 path: those FLOPs on CUDA cores"""
    ms = avg[kind]
    D0 = d[0]
    flops = 2 * batch * (D0 * 64 + 64 * 64) + 2 * batch * (2 * 64 * 64 + 2 * 64 * D0)
    if kind == "mlp" and prec == "fp32":
        ach = flops / (ms / 1e3) / 1e12
        peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        return {"kernel": "k_mlp_f32x", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "traffic_note": "not captured",
                "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x max SM clock",
                "algorithmic_flops_per_launch": flops, "avg_ms": ms}
    name = {"adam": "k_adam", "encode": "k_encode_tiles", "mlp": "k_mlp_tc"}[kind]
    traffic, note = ncu_traffic(name)
    if kind == "adam":
        bytes_ = n_visit * (32 + (2 if prec != "fp32" else 0))
        ach = bytes_ / (ms / 1e3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": traffic, "traffic_note": note,
                "peak_kind": pk_kind + " (copy)", "algorithmic_bytes_per_launch": bytes_, "avg_ms": ms,
                "params_visited_per_launch": n_visit}
    if kind == "encode":
        l2_bytes = batch * (8 * L * F * 2 + 8 * 4)
        hbm_bytes = l2_bytes + batch * (2 * D0 + 4)
        loads = batch * (L * (5 if F == 2 else 6) + 8)  # 16-byte loads issued: 5 per level at F = 2, 6 at F = 4
        peak_rate = l2pk["gather_loads_per_s"]
        kind_note = "measured: scattered 16-byte loads from 32 MiB (nv_peak_gather) x 16 B"
        issued = {"loads_per_launch": loads, "achieved_per_s": loads / (ms / 1e3), "peak_per_s": peak_rate,
                  "frac": loads / (ms / 1e3) / peak_rate}
        limiter = ("L1 / L2 request rate of the scattered 16-byte gathers; the coarse levels hit in L1 and "
                   "the 16-bit tables in L2, so DRAM carries a fraction of these bytes")
    else:
        l2_bytes = batch * (8 * L * F * 4)
        hbm_bytes = l2_bytes + batch * (2 * D0 + 4)
        reds = batch * L * (6 if F == 2 else 8)  # 16-byte reductions issued: 6 per level at F = 2 (x-paired)
        peak_rate = l2pk["scatter_reductions_per_s"]
        kind_note = "measured: scattered 16-byte FP32 vector reductions into 64 MiB (nv_peak_scatter) x 16 B"
        issued = {"reductions_per_launch": reds, "achieved_per_s": reds / (ms / 1e3), "peak_per_s": peak_rate,
                  "frac": reds / (ms / 1e3) / peak_rate}
        limiter = ("L2 vector reductions of the fused table-gradient scatter (the FP32 table gradient stays "
                   "L2-resident); the tensor pipe is not the limit")
    ach = l2_bytes / (ms / 1e3) / 1e9
    peak = peak_rate * 16 / 1e9
    r = {"kernel": name, "bound": "l2", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
         "traffic": traffic, "traffic_note": note, "peak_kind": kind_note,
         "algorithmic_bytes_per_launch": l2_bytes, "avg_ms": ms, "limiter": limiter,
         "issued_16B_accesses": issued,
         "hbm": {"achieved": hbm_bytes / (ms / 1e3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": hbm_bytes / (ms / 1e3) / 1e9 / pk["hbm_gbs"], "peak_kind": pk_kind + " (copy)",
                 "algorithmic_bytes_per_launch": hbm_bytes}}
    if kind == "mlp":
        peak_t = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        ach_t = flops / (ms / 1e3) / 1e12
        r["tensor"] = {"achieved": ach_t, "peak": peak_t, "unit": "TFLOP/s", "frac": ach_t / peak_t,
                       "algorithmic_flops_per_launch": flops, "peak_kind": pk_kind + " (bf16 sustained; "
                       "the FP16 dense rate is the same)"}
    return r


# ---------------------------------------------------------------------- ours ---

def run_ours(args):
    import torch
    from paper_2207_11620_gb300 import build as B
    from paper_2207_11620_gb300 import configs as CF
    from paper_2207_11620_gb300 import inputs as I
    from paper_2207_11620_gb300 import nv

    ws, rank, local = dist_setup(args.gpus)
    if rank == 0:
        B.build()
    barrier(ws)
    cfg = CF.CFG2
    c = cfg["net"]
    prec = args.prec
    if prec == "auto":
        prec = "fp16"
    try:
        net = nv.NeuralVolume(prec=prec, **c.kwargs())
    except nv.NvError as e:
        if args.prec == "auto" and e.status == 6:
            prec = "fp32"
            net = nv.NeuralVolume(prec=prec, **c.kwargs())
        else:
            raise
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=5 + rank, dims=c.dims)
    net.set_params(params)
    vol = torch.from_numpy(I.blob_volume(cfg["volume"], seed=cfg["volume_seed"])).cuda()
    batch = cfg["batch"]
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    # one GPU: nv_train_step samples the batch inside its gather kernel.  N GPUs: data
    # parallel (one network replicated, each rank sampling and training on its own
    # 2^18-point shard of an N x 2^18 global batch, one all-reduce of the gradient per step)
    if ws > 1:
        from paper_2207_11620_gb300 import dp
        dps = dp.DataParallelStep(net)

        def step(i):
            x, t = nv.sample(vol, batch, seed=1000 + rank, step=i)
            return dps.step_shard(x, t, ws * batch)

        def step_host(hx, ht, loss_host=None):
            return dps.step_shard(hx.cuda(non_blocking=True), ht.cuda(non_blocking=True), ws * batch)
    else:
        def step(i):
            net.train_step(n=batch, vol=vol, seed=1000 + rank, loss_out=loss)
            return loss

        def step_host(hx, ht, loss_host=None):
            # the step's last kernel writes the loss into the pinned host buffer
            net.train_step(hx, ht, loss_out=loss if loss_host is None else loss_host)
            return loss if loss_host is None else None

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = ev0.elapsed_time(ev1)
    # the same steps again with CUDA events around every kernel (the per-kernel
    # durations of the rooflines; the events themselves add a few us per step,
    # so the step time above is taken without them)
    net.profile(True)
    for k in ("mlp", "adam", "finish", "encode", "scatter"):
        net.profile_read(k)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for i in range(args.steps):
        step(args.warmup + args.steps + i)
    pe1.record(stream)
    torch.cuda.synchronize()
    ms_profiled = pe0.elapsed_time(pe1)
    net.profile(False)
    k_mlp = net.profile_read("mlp")
    k_adam = net.profile_read("adam")
    k_fin = net.profile_read("finish")
    ms_max = max_over_ranks(ws, ms)
    from paper_2207_11620_gb300 import replicas
    value = replicas.job_throughput(ws, batch * args.steps, ms_max / 1e3)

    # end to end through the C ABI: batches from pinned host memory, every step's loss
    # written into pinned host memory by the step's last kernel (one GPU) or copied
    # there from the device (data parallel)
    n_e2e = 4
    host_x, host_t = [], []
    for j in range(n_e2e):
        x, t = nv.sample(vol, batch, seed=77 + rank, step=j)
        host_x.append(x.cpu().pin_memory())
        host_t.append(t.cpu().pin_memory())
    loss_host = torch.zeros(1, dtype=torch.float64).pin_memory()
    for j in range(2):
        step_host(host_x[j], host_t[j])
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall = time.perf_counter()
    e0.record(stream)
    for i in range(args.steps):
        lo = step_host(host_x[i % n_e2e], host_t[i % n_e2e], loss_host)
        if lo is not None:  # data parallel: the global loss is a device tensor
            loss_host.copy_(lo, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    barrier(ws)
    e2e_ms = max(e0.elapsed_time(e1), 1e3 * t_wall)
    e2e_ms = max_over_ranks(ws, e2e_ms)
    e2e_value = replicas.job_throughput(ws, batch * args.steps, e2e_ms / 1e3)
    clk = clocks.stop()
    # fresh-run sanity: the loss stays finite
    assert np.isfinite(loss_host.item())

    if rank != 0:
        return 0
    pk, pk_kind = peaks()
    l2pk = l2_peaks(nv, torch)
    kt = {k: net.profile_read(k) for k in ("encode", "scatter")}
    kt["mlp"], kt["adam"], kt["finish"] = k_mlp, k_adam, k_fin
    avg = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in kt.items()}
    n_params, n_table = net.n_params, net.n_table
    n_visit = net.adam_span()
    d = c.dims
    D0 = d[0]
    dom = max(("encode", "mlp", "adam"), key=lambda k: kt[k][0])
    roof = roofline_of(dom, avg, prec, pk, pk_kind, batch, n_visit, n_table, d, c.L, c.F, l2pk)
    roof_others = {k: roofline_of(k, avg, prec, pk, pk_kind, batch, n_visit, n_table, d, c.L, c.F, l2pk)
                   for k in ("encode", "mlp", "adam") if avg.get(k) and k != dom}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f16", "bf16": "bf16"}[prec], "data": "synthetic",
        "config": {"workload": "cfg2 training step: 128^3 blob volume, L16 F2 T2^19 Nmin16 b1.38, MLP 32-64-64-1, "
                               "2^18 points sampled on the GPU, L2 loss, Adam",
                   "global_batch": ws * batch, "mlp_precision": prec, "n_params": n_params,
                   "adam_params_visited": n_visit,
                   "l2": "working set > L2: each step's Adam streams params, grads, m, v of the visited "
                         "blocks (%.0f MB)" % (n_visit * 16 / 1e6),
                   "parallelism": f"dp{ws}: one network, an all-reduce of its gradient per step" if ws > 1
                                  else "single"},
        "roofline": roof,
        "rooflines_other_kernels": roof_others,
        "l2_access_peaks": l2pk,
        "kernels_ms_per_step": {k: v for k, v in avg.items() if v > 0},
        "ms_per_step_with_kernel_events": ms_profiled / args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": batch * 16, "d2h_bytes_per_step": 8},
        "gpu_launches": args.steps * (sum(1 for k in ("encode", "mlp", "scatter", "adam", "finish") if kt[k][1])
                                      + (1 if ws > 1 else 0)),
        "clocks": clk,
    }
    if ws == 1:
        line["render_1080p"] = bench_render_1080p(nv, I, CF, torch, min(max(args.steps, 3), 20), pk, pk_kind, l2pk,
                                                  cpu=not args.no_cpu_baseline)
    if ws == 1 and args.extras:
        line["extra"] = run_extras(args, pk, pk_kind, l2pk)
    if ws == 1 and not args.no_cpu_baseline:
        rate, threads, secs, desc = oracle_step_rate(args.cpu_points)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
                                "seconds": secs}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- extras ---

def _psnr(mse):
    import math
    return 10.0 * math.log10(1.0 / mse) if mse > 0 else float("inf")


def extra_cfg2_quality(nv, I, CF, torch, steps=1000, pk=None):
    """Config 2 as specified: 1000 steps of 2^18 points, FP32 vs FP16 MLP; volume PSNR.
    The FP32 path's step (one fused encode + MLP + scatter kernel on CUDA cores,
    k_mlp_f32x, then Adam) is set against the CUDA cores' FP32 FMA rate: 152 SMs x 128
    lanes x 2 FLOP x the maximum SM clock."""
    cfg = CF.CFG2
    c = cfg["net"]
    vol = torch.from_numpy(I.blob_volume(cfg["volume"], seed=cfg["volume_seed"])).cuda()
    out = {}
    for prec in ("fp32", "fp16", "bf16"):
        net = nv.NeuralVolume(prec=prec, **c.kwargs())
        net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims))
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(steps):
            net.train_step(n=cfg["batch"], vol=vol, seed=31, loss_out=loss)
        e1.record()
        torch.cuda.synchronize()
        mse = net.volume_mse(vol).item()
        out[prec] = {"steps": steps, "ms_per_step": e0.elapsed_time(e1) / steps, "final_loss": loss.item(),
                     "volume_psnr_db": _psnr(mse)}
        if prec == "fp32" and pk:
            # the MLP kernel alone, timed with events over a few more steps
            net.profile(True)
            net.profile_read("mlp")
            for i in range(20):
                net.train_step(n=cfg["batch"], vol=vol, seed=31, loss_out=loss)
            t, nl = net.profile_read("mlp")
            net.profile(False)
            ms = t / max(nl, 1)
            D0 = c.dims[0]
            flops = 2 * cfg["batch"] * (D0 * 64 + 64 * 64 + 64) + 2 * cfg["batch"] * (2 * 64 * 64 + 2 * 64 * D0 + 64)
            peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            ach = flops / (ms / 1e3) / 1e12
            out[prec]["roofline"] = {"kernel": "k_mlp_f32x", "bound": "alu", "achieved": ach, "peak": peak,
                                     "unit": "TFLOP/s", "frac": ach / peak, "avg_ms": ms,
                                     "algorithmic_flops_per_launch": flops,
                                     "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x max SM clock"}
        net.close()
    return out


def _render_setup(nv, I, torch, cfg, vt):
    lut = torch.from_numpy(I.ramp_lut(alpha_floor=cfg["alpha_floor"])).cuda()
    _, mu = nv.macrocells_build(vt, cfg["cell"], lut)
    D = vt.shape[0]
    opts = dict(step=cfg["step_voxels"] / D, alpha_exp=cfg["step_voxels"], et=cfg["et"], K=cfg["K"])
    return lut, mu, opts


def _median_frame_ms(torch, frames, fn):
    """Median device time of `frames` calls of fn (CUDA events around each), after one warm-up call."""
    img = fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
    for a, b in ev:
        a.record()
        img = fn()
        b.record()
    torch.cuda.synchronize()
    return img, statistics.median(a.elapsed_time(b) for a, b in ev)


def _time_render(r, torch, frames, **kw):
    return _median_frame_ms(torch, frames, lambda: r.render(**kw))


def extra_cfg3_render(nv, I, CF, torch, train_steps=None, frames=9):
    """Config 3: 512^3 volume, T2^21 network trained with config 2's recipe, 1080p
    perspective march (0.5 voxel, 16^3 macrocells, ET 0.99) with FP16 and BF16
    inference; PSNR of each neural image against the raw-volume image."""
    cfg = CF.CFG3
    c = cfg["net"]
    D = cfg["volume"]
    vt = I.blob_volume_torch(D, cfg["volume_seed"], "cuda")
    lut, mu, opts = _render_setup(nv, I, torch, cfg, vt)
    W, H = cfg["image"]
    cam = I.perspective_camera(W, H, cfg["vfov"], cfg["eye"], cfg["target"])
    mc = (mu, cfg["cell"], vt.shape)
    r = nv.Renderer(W * H, K=cfg["K"])
    raw, raw_ms = _time_render(r, torch, frames, cam=cam, lut=lut, opts=opts, raw=vt, mc=mc)
    raw = raw.clone()
    it, ns = r.stats()
    out = {"image": [W, H], "raw_ms": raw_ms, "raw_samples_per_frame": ns, "raw_iterations": it}
    _, raw_pt_ms = _median_frame_ms(torch, frames, lambda: r.render_pt(
        cam, lut, dict(density=float(D), light=(0.0, 0.8, -0.6), max_bounces=8, seed=3), mc, raw=vt))
    out["raw_path_tracing_1spp_ms"] = raw_pt_ms
    steps = train_steps or cfg["train_steps"]
    for prec in ("fp16", "bf16"):
        net = nv.NeuralVolume(prec=prec, **c.kwargs())
        net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims))
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(steps):
            net.train_step(n=cfg["batch"], vol=vt, seed=11, loss_out=loss)
        e1.record()
        torch.cuda.synchronize()
        img, ms = _time_render(r, torch, frames, cam=cam, lut=lut, opts=opts, net=net, mc=mc)
        it, ns = r.stats()
        mse = nv.image_mse(img, raw).item()
        # the same frame by in-shader inference (Sec. 5.1): one megakernel
        sam = torch.zeros(1, dtype=torch.int64, device="cuda")
        is_img = torch.empty_like(img)
        is_img, is_ms = _median_frame_ms(
            torch, frames, lambda: nv.render_inshader(net, cam, lut, opts, mc=mc, out=is_img, samples=sam))
        # adaptive step (Sec. 5.3, Eq. 3): s1 = the fixed step, s2 = one macrocell
        ad_opts = dict(opts, step_max=opts["step"] * 2 * cfg["cell"])
        ad_img, ad_ms = _time_render(r, torch, frames, cam=cam, lut=lut, opts=ad_opts, net=net, mc=mc)
        ad_it, ad_ns = r.stats()
        ad_psnr = _psnr(nv.image_mse(ad_img, raw).item())
        # single-shot heuristic shadows and path tracing (Sec. 5.2.2) of the same network
        light = (0.0, 0.8, -0.6)
        sh_img, sh_ms = _time_render(r, torch, frames, cam=cam, lut=lut,
                                     opts=dict(opts, shade=1, light=light, ambient=0.25), net=net, mc=mc)
        sh_it, sh_ns = r.stats()
        # the same shadows by the in-shader megakernel
        is_sh = torch.empty_like(sh_img)
        is_sh, is_sh_ms = _median_frame_ms(
            torch, frames, lambda: nv.render_inshader(net, cam, lut, dict(opts, shade=1, light=light, ambient=0.25),
                                                      mc=mc, out=is_sh))
        pt_opts = dict(density=float(D), light=light, max_bounces=8, seed=3)
        _, pt_ms = _median_frame_ms(torch, frames, lambda: r.render_pt(cam, lut, pt_opts, mc, net=net))
        pt_it, pt_ns = r.stats()
        out_pt = {"frame_ms": pt_ms, "tentative_collisions_per_frame": pt_ns, "iterations": pt_it,
                  "network_samples_per_s": pt_ns / (pt_ms / 1e3), "density": float(D), "max_bounces": 8}
        out[prec] = {"train_steps": steps, "train_ms_per_step": e0.elapsed_time(e1) / steps,
                     "frame_ms": ms, "samples_per_frame": ns, "iterations": it,
                     "decoded_samples_per_s": ns / (ms / 1e3), "image_psnr_db": _psnr(mse),
                     "volume_psnr_db": _psnr(net.volume_mse(vt).item()),
                     "inshader": {"frame_ms": is_ms, "samples_per_frame": int(sam.item()),
                                  "max_abs_diff_vs_streaming": float((is_img - img).abs().max().item()),
                                  "streaming_speedup": is_ms / ms},
                     "adaptive_step": {"step_max_voxels": cfg["step_voxels"] * 2 * cfg["cell"], "frame_ms": ad_ms,
                                       "samples_per_frame": ad_ns, "iterations": ad_it, "image_psnr_db": ad_psnr},
                     "single_shot_shadows": {"frame_ms": sh_ms, "samples_per_frame": sh_ns, "iterations": sh_it,
                                             "inshader_frame_ms": is_sh_ms,
                                             "inshader_max_abs_diff": float((is_sh - sh_img).abs().max().item())},
                     "path_tracing_1spp": out_pt}
        if prec == "fp16":
            # samples per ray and iteration (Fig. 13's K): the image does not depend on K
            sweep = {}
            for k in (1, 2, 4, 8, 16):
                rk = nv.Renderer(W * H, K=k)
                img_k, ms_k = _time_render(rk, torch, frames, cam=cam, lut=lut, opts=dict(opts, K=k), net=net, mc=mc)
                it_k, ns_k = rk.stats()
                sweep[str(k)] = {"frame_ms": ms_k, "iterations": it_k, "samples_per_frame": ns_k,
                                 "max_abs_diff_vs_k%d" % cfg["K"]: float((img_k - img).abs().max().item())}
                rk.close()
            out["k_sweep_fp16"] = sweep
        net.close()
    # frame time and quality against the table size (Fig. 12's log2 T), FP16, same recipe
    t_sweep = {}
    for log2T in (17, 19, 21):
        kw = dict(c.kwargs(), log2T=log2T)
        net = nv.NeuralVolume(prec="fp16", **kw)
        net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims))
        for i in range(steps):
            net.train_step(n=cfg["batch"], vol=vt, seed=11)
        img, ms = _time_render(r, torch, frames, cam=cam, lut=lut, opts=opts, net=net, mc=mc)
        it, ns = r.stats()
        t_sweep[str(log2T)] = {"n_params": net.n_params, "compression_ratio": D ** 3 / net.n_params,
                               "frame_ms": ms, "samples_per_frame": ns,
                               "image_psnr_db": _psnr(nv.image_mse(img, raw).item()),
                               "volume_psnr_db": _psnr(net.volume_mse(vt).item())}
        net.close()
    out["log2T_sweep_fp16"] = t_sweep
    r.close()
    del vt
    torch.cuda.empty_cache()
    return out


# warp instructions per sample and level of the render gather (ncu, trained 1080p frame)
RENDER_GATHER_INSTR_PER_SAMPLE_LEVEL = 112


def gather_roofline(ns, g_ms, L, F, D0, pk, pk_kind, l2pk):
    """Roofline of the render gather (k_encode_tiles in inference) over one frame of ns
    decoded samples: 8 corners x L levels x F 16-bit features per sample (512 B at L16
    F2), each corner one load of its 2F-byte entry (8 loads per level).  The K samples
    of a ray sit in adjacent lanes and neighbouring rays share most corners, so these
    loads resolve in L1: the bytes are set against the measured rate of scattered
    16-byte loads from an L1-resident buffer (x 16 B) and from an L2-resident one.
    Lanes that share an address share a sector, so the issued loads can exceed the
    scattered-load rate; what bounds the kernel is instruction issue (ncu: 2.8 of 4
    instructions per SM cycle, no pipe above 40%).  Its own HBM traffic is the
    coordinates read (12 B) and the feature row written (2 D0 B) per sample."""
    g_bytes = ns * 8 * L * F * 2
    g_ach = g_bytes / (g_ms / 1e3) / 1e9
    loads = ns * L * 8
    l1 = l2pk["l1_gather_loads_per_s"]
    hbm = ns * (12 + 2 * D0) / (g_ms / 1e3) / 1e9
    out = {"kernel": "k_encode_tiles", "bound": "l1", "achieved": g_ach, "peak": l1 * 16 / 1e9, "unit": "GB/s",
            "frac": g_ach / (l1 * 16 / 1e9),
            "peak_kind": "measured: scattered 16-byte loads from an L1-resident 32 KiB (nv_peak_gather) x 16 B",
            "algorithmic_bytes_per_frame": g_bytes, "ms_per_frame": g_ms,
            "limiter": "instruction issue (ncu: 2.8 of 4 per SM cycle, ALU / FMA / LSU pipes 36 / 39 / 19%); "
                       "profiles/k_encode_tiles_render1080p.md",
            "issued_corner_loads": {"per_frame": loads, "bytes_each": 2 * F, "achieved_per_s": loads / (g_ms / 1e3),
                                    "scattered_16B_load_peak_per_s": l1, "frac": loads / (g_ms / 1e3) / l1},
            "l2": {"achieved": g_ach, "peak": l2pk["gather_loads_per_s"] * 16 / 1e9, "unit": "GB/s",
                   "frac": g_ach / (l2pk["gather_loads_per_s"] * 16 / 1e9),
                   "peak_kind": "measured: scattered 16-byte loads from 32 MiB (nv_peak_gather) x 16 B"},
            "hbm": {"achieved": hbm, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": hbm / pk["hbm_gbs"],
                    "peak_kind": pk_kind + " (copy)", "bytes_per_sample": 12 + 2 * D0}}
    if F == 2 and D0 == 32:
        # the bound itself: warp instructions issued against the SMs' issue rate (one per SM
        # sub-partition and cycle at the maximum clock), with the instructions per sample and
        # level of the committed ncu capture of this kernel on this workload
        import torch
        try:
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        except Exception:  # no device to ask: GB300's count
            sms = 152
        ipl = RENDER_GATHER_INSTR_PER_SAMPLE_LEVEL
        achieved = ipl * ns * L / 32 / (g_ms / 1e3)
        peak = 4 * sms * pk.get("sm_max_mhz", 2070.0) * 1e6
        out["issue"] = {"warp_instructions_per_sample_and_level": ipl, "achieved_per_s": achieved,
                        "peak_per_s": peak, "frac": achieved / peak,
                        "source": "ncu sm__inst_executed of k_encode_tiles on this frame, "
                                  "profiles/k_encode_tiles_render1080p.md"}
    return out


def oracle_render_rate(net, params, cam, lut, opts, mu, shape, stride=10):
    """The FP64 oracle renders every stride-th pixel of every stride-th row of the frame
    (1920x1080 -> 192x108) with the network's parameters; returns (ms per full frame
    extrapolated from the per-ray cost, threads, seconds, rays)."""
    import oracle as O
    W, H = cam["width"], cam["height"]
    pix = np.array([py * W + px for py in range(stride // 2, H, stride) for px in range(stride // 2, W, stride)],
                   np.int64)
    onet = O.Net(L=net.L, F=net.F, log2T=net.log2T, Nmin=net.Nmin, b=net.b, dims=net.dims)
    nz, ny, nx = shape
    o = dict(opts, mc_cell=int(opts.get("mc_cell", 0)), dims=(nz, ny, nx))
    t0 = time.perf_counter()
    O.render_pixels(cam, lut, o, pix, net=onet, params=params, mumax=mu)
    secs = time.perf_counter() - t0
    return 1e3 * secs * (W * H) / len(pix), O.num_threads(), secs, len(pix)


def bench_render_1080p(nv, I, CF, torch, frames, pk, pk_kind, l2pk, cpu=True):
    """Config 3's frame as the metric's second half: the 1080p perspective march (0.5
    voxel, 16^3 macrocells, ET 0.99, K 8) of a 512^3 blob volume through a T2^21 FP16
    network trained with config 2's recipe (2000 steps of 2^18 points).  Median device
    time of `frames` frames (the frame's input, the network and the volume already in
    HBM); per-kernel times from the same frames with events around each kernel; the
    rooflines of the gather (k_encode_tiles) and the tensor-core MLP (k_mlp_tc) in
    inference; the raw-volume march of the same frame on the same GPU; image PSNR of
    the neural frame against it; and the FP64 oracle's ms per frame from a 192x108
    subsample of the rays on the host cores."""
    cfg = CF.CFG3
    c = cfg["net"]
    D = cfg["volume"]
    vt = I.blob_volume_torch(D, cfg["volume_seed"], "cuda")
    lut, mu, opts = _render_setup(nv, I, torch, cfg, vt)
    W, H = cfg["image"]
    cam = I.perspective_camera(W, H, cfg["vfov"], cfg["eye"], cfg["target"])
    mc = (mu, cfg["cell"], vt.shape)
    r = nv.Renderer(W * H, K=cfg["K"])
    raw, raw_ms = _time_render(r, torch, max(3, frames), cam=cam, lut=lut, opts=opts, raw=vt, mc=mc)
    raw = raw.clone()
    raw_it, raw_ns = r.stats()
    net = nv.NeuralVolume(prec="fp16", **c.kwargs())
    net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims))
    for i in range(cfg["train_steps"]):
        net.train_step(n=cfg["batch"], vol=vt, seed=11)
    torch.cuda.synchronize()
    img, ms = _time_render(r, torch, frames, cam=cam, lut=lut, opts=opts, net=net, mc=mc)
    it, ns = r.stats()
    psnr = _psnr(nv.image_mse(img, raw).item())
    # the same frame by in-shader inference (Sec. 5.1, App. A): one megakernel
    sam = torch.zeros(1, dtype=torch.int64, device="cuda")
    is_img = torch.empty_like(img)
    is_img, is_ms = _median_frame_ms(
        torch, frames, lambda: nv.render_inshader(net, cam, lut, opts, mc=mc, out=is_img, samples=sam))
    inshader = {"frame_ms": is_ms, "samples_per_frame": int(sam.item()),
                "decoded_samples_per_s": int(sam.item()) / (is_ms / 1e3),
                "max_abs_diff_vs_streaming": float((is_img - img).abs().max().item())}
    # per-kernel device times over the same frames, read after every frame (the
    # library keeps at most 8192 timed launches between reads; a frame has ~800)
    net.profile(True)
    classes = ("encode", "mlp", "other", "render")
    for k in classes:
        net.profile_read(k)
    kt = {k: [0.0, 0] for k in classes}
    for f in range(frames):
        r.render(cam, lut, opts, net=net, mc=mc, out=img)
        for k in classes:
            t, n = net.profile_read(k)
            kt[k][0] += t
            kt[k][1] += n
    net.profile(False)
    per = {"k_encode_tiles": kt["encode"][0] / frames, "k_mlp_tc": kt["mlp"][0] / frames,
           "k_coords": kt["other"][0] / frames, "k_composite": kt["render"][0] / frames}
    launches = {k: v[1] // frames for k, v in kt.items()}
    L, F, D0 = c.L, c.F, c.dims[0]
    roof = gather_roofline(ns, per["k_encode_tiles"], L, F, D0, pk, pk_kind, l2pk)
    roof["launches_per_frame"] = launches["encode"]
    roof["traffic"] = None
    roof["traffic_note"] = "see profiles/cfg3_render_launches.md (launch list; no DRAM counters in this line)"
    m_ms = per["k_mlp_tc"]
    flops = ns * 2 * (D0 * 64 + 64 * 64 + 64)
    peak_t = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    out = {"workload": "cfg3: 512^3 blob volume, L16 F2 T2^21 FP16 network (2000 training steps), 1920x1080 "
                       "perspective, step 0.5 voxel, 16^3 macrocells, ET 0.99, K 8",
           "frame_ms": ms, "frames": frames, "iterations": it, "samples_per_frame": ns,
           "decoded_samples_per_s": ns / (ms / 1e3), "image_psnr_db_vs_raw": psnr,
           "path": "sample streaming (nv_render); the same image in-shader (nv_render_inshader) below",
           "inshader": inshader,
           "best_frame_ms": min(ms, is_ms), "best_path": "in-shader" if is_ms < ms else "sample streaming",
           "raw_volume_frame_ms": raw_ms, "raw_iterations": raw_it, "raw_samples_per_frame": raw_ns,
           "kernels_ms_per_frame": per, "launches_per_frame": launches,
           "roofline": roof,
           "mlp_tensor": {"kernel": "k_mlp_tc", "achieved": flops / (m_ms / 1e3) / 1e12, "peak": peak_t,
                          "unit": "TFLOP/s", "frac": flops / (m_ms / 1e3) / 1e12 / peak_t,
                          "algorithmic_flops_per_frame": flops, "ms_per_frame": m_ms,
                          "peak_kind": pk_kind + " (bf16 sustained; the FP16 dense rate is the same)"}}
    if cpu:
        params = net.get_params().cpu().numpy()
        o_ms, threads, secs, rays = oracle_render_rate(net, params, cam, lut.cpu().numpy(),
                                                       dict(opts, mc_cell=cfg["cell"]), mu.cpu().numpy(),
                                                       tuple(vt.shape))
        out["cpu_baseline"] = {"value": o_ms, "unit": "ms/frame", "cores": threads, "kind": "oracle",
                               "sample": f"FP64 oracle march of {rays} rays (every 10th pixel of every 10th row) "
                                         f"through the same trained network, per-ray cost extrapolated to "
                                         f"{W}x{H}", "seconds": secs}
    net.close()
    r.close()
    del vt
    torch.cuda.empty_cache()
    return out


def extra_cfg4_inloop(nv, I, CF, torch, pk, pk_kind, l2pk, frames=None):
    """Config 4: 1024^3 volume in HBM; each frame one 2^18-point training step and a
    1024x1024 render of the current FP16 network; ms/frame and the PSNR of the
    last frame against the raw-volume render.  The loop runs twice on fresh
    networks: rendering by sample streaming (the reported figures) and by the
    in-shader megakernel (inshader_loop)."""
    cfg = CF.CFG4
    c = cfg["net"]
    D = cfg["volume"]
    frames = frames or cfg["frames"]
    vt = I.blob_volume_torch(D, cfg["volume_seed"], "cuda")
    lut, mu, opts = _render_setup(nv, I, torch, cfg, vt)
    W, H = cfg["image"]
    cam = I.perspective_camera(W, H, 40.0, (0.5, 0.5, -1.0), (0.5, 0.5, 0.5))
    mc = (mu, cfg["cell"], vt.shape)
    r = nv.Renderer(W * H, K=cfg["K"])
    raw, raw_ms = _time_render(r, torch, 2, cam=cam, lut=lut, opts=opts, raw=vt, mc=mc)
    raw = raw.clone()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    img = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    cell = cfg["cell"]

    def in_loop(render):
        """frames x (one training step, mu_max from the online ranges, one render) of a
        fresh network; returns the network, its online macrocells and the timings."""
        net = nv.NeuralVolume(prec="fp16", **c.kwargs())
        net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims))
        psnr_curve = []
        # online macrocells (Sec. 5.3): the training samples grow the value ranges,
        # mu_max is refreshed from them before each frame's render
        mm_on = nv.online_macrocells(vt.shape, cell)
        mu_on = torch.zeros_like(mu)
        net.set_online_macrocells(mm_on, vt.shape, cell)
        mc_on = (mu_on, cell, vt.shape)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        split = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(frames)]
        e0.record()
        for f in range(frames):
            split[f][0].record()
            net.train_step(n=cfg["batch"], vol=vt, seed=21, loss_out=loss)
            nv.macrocells_mu(mm_on, vt.shape, cell, lut, out=mu_on)
            split[f][1].record()
            render(net, mc_on)
            split[f][2].record()
            if f % 100 == 99:
                psnr_curve.append((f + 1, nv.image_mse(img, raw)))
        e1.record()
        torch.cuda.synchronize()
        t = {"ms_per_frame": e0.elapsed_time(e1) / frames,
             "train_ms_per_frame": statistics.median(a.elapsed_time(b) for a, b, _ in split),
             "render_ms_per_frame": statistics.median(b.elapsed_time(c2) for _, b, c2 in split),
             "psnr_db_by_frame": [(f, _psnr(m.item())) for f, m in psnr_curve]}
        t["final_psnr_db"] = t["psnr_db_by_frame"][-1][1] if psnr_curve else None
        return net, mu_on, mc_on, t

    # the same loop with the in-shader megakernel (Sec. 5.1) as the renderer
    net, _, _, t_is = in_loop(lambda n, m: nv.render_inshader(n, cam, lut, opts, mc=m, out=img))
    net.close()
    net, mu_on, mc_on, t_ss = in_loop(lambda n, m: r.render(cam, lut, opts, net=n, mc=m, out=img))
    ms, train_ms, render_ms = t_ss["ms_per_frame"], t_ss["train_ms_per_frame"], t_ss["render_ms_per_frame"]
    curve = t_ss["psnr_db_by_frame"]
    # per-kernel times of the two halves, each profiled on its own over a few more frames
    net.profile(True)
    for k in ("encode", "mlp", "scatter", "adam", "other", "render"):
        net.profile_read(k)
    nprof = 5
    for f in range(nprof):
        net.train_step(n=cfg["batch"], vol=vt, seed=21, loss_out=loss)
    torch.cuda.synchronize()
    kt_train = {k: net.profile_read(k) for k in ("encode", "mlp", "scatter", "adam")}
    kt_render = {k: [0.0, 0] for k in ("encode", "mlp", "other", "render")}
    for f in range(nprof):  # read after every frame: at most 8192 timed launches are kept between reads
        r.render(cam, lut, opts, net=net, mc=mc_on, out=img)
        for k in kt_render:
            t, n = net.profile_read(k)
            kt_render[k][0] += t
            kt_render[k][1] += n
    net.profile(False)
    it, ns = r.stats()  # the last profiled frame's (the network no longer trains between them)
    avg = {k: v[0] / v[1] for k, v in kt_train.items() if v[1]}
    n_visit = net.adam_span()
    train_roof = {k: roofline_of(k, avg, "fp16", pk, pk_kind, cfg["batch"], n_visit, net.n_table, c.dims, c.L,
                                 c.F, l2pk) for k in ("encode", "mlp", "adam") if k in avg}
    render_roof = gather_roofline(ns, kt_render["encode"][0] / nprof, c.L, c.F, c.dims[0], pk, pk_kind, l2pk)
    # the last network rendered with ranges precomputed from the voxels instead
    img_pre = r.render(cam, lut, opts, net=net, mc=mc)
    psnr_pre = _psnr(nv.image_mse(img_pre, raw).item())
    cells_on = int((mu_on > 0).sum().item())
    cells_pre = int((mu > 0).sum().item())
    out = {"frames": frames, "ms_per_frame": ms, "train_ms_per_frame": train_ms, "render_ms_per_frame": render_ms,
           "train_kernels_ms": {k: v[0] / nprof for k, v in kt_train.items()},
           "render_kernels_ms": {k: v[0] / nprof for k, v in kt_render.items()},
           "train_rooflines": train_roof, "render_roofline": render_roof,
           "render_samples_per_frame": ns, "render_iterations": it,
           "raw_ms": raw_ms, "psnr_db_by_frame": curve,
           "final_psnr_db": curve[-1][1] if curve else None, "n_params": net.n_params,
           "macrocells": "online (training samples)", "final_psnr_db_precomputed_macrocells": psnr_pre,
           "nonempty_cells_online": cells_on, "nonempty_cells_precomputed": cells_pre,
           "inshader_loop": t_is}
    net.close()
    r.close()
    del vt
    torch.cuda.empty_cache()
    return out


def host_link_peak(torch, nbytes=1 << 30):
    """GB/s of a pinned host -> device copy of nbytes (median of 5, CUDA events)."""
    h = torch.empty(nbytes // 4, dtype=torch.float32).pin_memory()
    d = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    d.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        d.copy_(h, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    del h, d
    return nbytes / (statistics.median(ts) / 1e3) / 1e9


def extra_cfg5_ooc(nv, I, CF, torch, steps=200, warm=10):
    """Config 5: 2048^3 volume (32 GiB) held in pinned host memory as 64^3 bricks with
    a ghost layer; a device ring of 4096 bricks, 256 refreshed per step on a side
    stream; 2^19 BF16 training points per step from the resident bricks.  The
    device copy of the volume is freed before training; the final PSNR is taken
    on a 256^3 subsample (every 8th voxel) kept on the device."""
    cfg = CF.CFG5
    c = cfg["net"]
    D, B = cfg["volume"], cfg["brick"]
    t0 = time.perf_counter()
    vt = I.blob_volume_torch(D, cfg["volume_seed"], "cuda")
    sub = vt[4::8, 4::8, 4::8].contiguous().reshape(-1)
    ax = (torch.arange(4, D, 8, device="cuda", dtype=torch.float32) + 0.5) / D
    zz, yy, xx = torch.meshgrid(ax, ax, ax, indexing="ij")
    pts = torch.stack([xx, yy, zz], -1).reshape(-1, 3).contiguous()
    del zz, yy, xx
    host = I.host_bricks_from_device(vt, B)
    del vt
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    prep_s = time.perf_counter() - t0
    link_peak = host_link_peak(torch)
    ring = nv.BrickRing(host, (D, D, D), B, cfg["ring"], seed=1)
    net = nv.NeuralVolume(prec="bf16", **c.kwargs())
    net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims))
    n = cfg["batch"]
    xyz = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    tgt = torch.empty(n, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def step(s):
        ring.sample(n, seed=17, step=s, xyz=xyz, target=tgt)
        ring.refresh(cfg["refresh"], seed=1000 + s)  # overlaps the training step below
        net.train_step(xyz, tgt, loss_out=loss)

    for s in range(warm):
        step(s)
    torch.cuda.synchronize()
    b0, c0 = ring.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in range(warm, warm + steps):
        step(s)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    b1, c1 = ring.stats()
    y = net.infer(pts)
    psnr = _psnr(nv.mse(y, sub).item())
    out = {"steps": steps, "ms_per_step": ms, "steps_per_s": 1e3 / ms, "samples_per_s": n * 1e3 / ms,
           "bytes_per_step": (b1 - b0) / steps, "host_link_gbs": (b1 - b0) / (c1 - c0) / 1e6 if c1 > c0 else None,
           "sustained_host_gbs": (b1 - b0) / (steps * ms) / 1e6, "final_loss": loss.item(),
           "psnr_db_256cube_subsample": psnr, "host_bytes": host.numel() * 4, "prep_s": prep_s,
           "ring_bricks": cfg["ring"], "refresh_per_step": cfg["refresh"], "n_params": net.n_params,
           "host_link_copy_peak_gbs": link_peak,
           "host_link_peak_kind": "measured: 1 GiB pinned host -> device cudaMemcpyAsync, median of 5"}
    if out["host_link_gbs"]:
        out["host_link_frac"] = out["host_link_gbs"] / link_peak
    out["sustained_host_frac"] = out["sustained_host_gbs"] / link_peak
    net.close()
    ring.close()
    del host, pts, sub
    torch.cuda.empty_cache()
    return out


def run_extras(args, pk, pk_kind, l2pk):
    import functools

    import torch
    from paper_2207_11620_gb300 import configs as CF
    from paper_2207_11620_gb300 import inputs as I
    from paper_2207_11620_gb300 import nv
    out = {}
    cfg4 = functools.partial(extra_cfg4_inloop, pk=pk, pk_kind=pk_kind, l2pk=l2pk)
    cfg2 = functools.partial(extra_cfg2_quality, pk=pk)
    for name, fn in (("cfg2_quality", cfg2), ("cfg3_render", extra_cfg3_render),
                     ("cfg4_inloop", cfg4), ("cfg5_ooc", extra_cfg5_ooc)):
        if name not in args.extras:
            continue
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        try:
            out[name] = fn(nv, I, CF, torch)
        except Exception as e:  # report and keep the main line
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
        out[name]["clocks"] = clocks.stop()
    return out


def run_case(args):
    """Profiling cases (for ncu captures); each prints one JSON line.

    train_cfg2    args.warmup + args.steps config-2 training steps (2^18 sampled points; FP16, or
                  the precision --prec names)
    render1080p   the config-3 1080p frame of a trained FP16 network: 2000 training steps, one
                  frame, then args.steps frames (and the timing helper's first call) in the NVTX
                  range "frame"
    The train case's last args.steps steps sit in the NVTX range "steps"."""
    import torch
    from paper_2207_11620_gb300 import build as B
    from paper_2207_11620_gb300 import configs as CF
    from paper_2207_11620_gb300 import inputs as I
    from paper_2207_11620_gb300 import nv
    B.build()
    if args.case == "train_cfg2":
        cfg = CF.CFG2
        c = cfg["net"]
        net = nv.NeuralVolume(prec="fp16" if args.prec == "auto" else args.prec, **c.kwargs())
        net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims))
        vol = torch.from_numpy(I.blob_volume(cfg["volume"], seed=cfg["volume_seed"])).cuda()
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        for i in range(args.warmup):
            net.train_step(n=cfg["batch"], vol=vol, seed=1000, loss_out=loss)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("steps")  # the launches a profiler capture selects
        for i in range(args.steps):
            net.train_step(n=cfg["batch"], vol=vol, seed=1000, loss_out=loss)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"case": args.case, "steps": args.warmup + args.steps, "loss": loss.item()}), flush=True)
        return 0
    cfg = CF.CFG3
    c = cfg["net"]
    D = cfg["volume"]
    vt = I.blob_volume_torch(D, cfg["volume_seed"], "cuda")
    lut, mu, opts = _render_setup(nv, I, torch, cfg, vt)
    net = nv.NeuralVolume(prec="fp16", **c.kwargs())
    net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims))
    for i in range(cfg["train_steps"]):
        net.train_step(n=cfg["batch"], vol=vt, seed=11)
    torch.cuda.synchronize()
    W, H = cfg["image"]
    cam = I.perspective_camera(W, H, cfg["vfov"], cfg["eye"], cfg["target"])
    r = nv.Renderer(W * H, K=cfg["K"])
    mc = (mu, cfg["cell"], vt.shape)
    r.render(cam, lut, opts, net=net, mc=mc)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("frame")  # the launches a profiler capture selects
    img, ms = _median_frame_ms(torch, max(1, args.steps), lambda: r.render(cam, lut, opts, net=net, mc=mc))
    torch.cuda.nvtx.range_pop()
    it, ns = r.stats()
    print(json.dumps({"case": args.case, "frame_ms": ms, "iterations": it, "samples": ns,
                      "mean_alpha": float(img[..., 3].mean())}), flush=True)
    return 0


def main():
    args = parse()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
