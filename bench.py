"""Throughput benchmark: decoded information Gbit/s of the CI-schedule decoders
on one GB300, next to flooding BP at equal FER and the CPU oracle.

Workload (default): the WiFi-like rate-1/2 QC code (12x24 protograph, Z=96,
n=2304, E=7776, k=1152), BPSK/AWGN at Eb/N0 = 1.5 dB, FP32 sum-product,
ME-LMD-CIRBP (Algorithm 6) with N_P = 64, N_G = 16, budget 3 iteration
equivalents (3E committed messages: the I_max = 3 regime of Sec. 5, where the
frame error rate is above zero), syndrome checked after every step.
One step = channel kernel (Philox AWGN LLRs) + decode of one batch of 65,536
frames; LLR inputs (604 MB) exceed L2.  The end-to-end figure (`e2e`) decodes
batches copied from pinned host memory each step and reads the decisions back.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SM_COUNT_NOMINAL = 152
SMEM_BYTES_PER_CLK_PER_SM = 128  # 32 banks x 4 B


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--schedule", default="me-lmd-cirbp")
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--ebn0", type=float, default=1.5)
    ap.add_argument("--budget-iters", type=float, default=3.0)
    ap.add_argument("--n-p", type=int, default=64)
    ap.add_argument("--n-g", type=int, default=16)
    ap.add_argument("--arith", default="fp32")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--decode-only", action="store_true",
                    help="generate one batch with the channel kernel and time --reps decode launches "
                         "(the command the ncu captures under profiles/ use)")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--queue-frames", type=int, default=6144,
                    help="frames of the mixed-lifting BG2-shaped queue comparison (extras)")
    ap.add_argument("--queue-stream", type=int, default=0,
                    help="stream this many mixed-lifting frames through one persistent queue launch and print "
                         "its JSON (config 3 at its stated size: 1000000)")
    ap.add_argument("--queue-only", action="store_true",
                    help="run only the mixed-lifting queue comparison and print its JSON")
    ap.add_argument("--large-frames", type=int, default=304,
                    help="frames per point of the 26,112-bit BG1-shaped comparison (extras)")
    ap.add_argument("--wbp-only", action="store_true",
                    help="run only the weighted-BP forward/adjoint timing and print its JSON")
    ap.add_argument("--large-only", action="store_true",
                    help="run only the BG1-shaped cluster / global-memory comparison and print its JSON")
    ap.add_argument("--no-sweep", action="store_true",
                    help="leave out the Eb/N0 x N_P x budget sweep and the gamma sweep (extras)")
    ap.add_argument("--sweep-only", action="store_true",
                    help="run only the Eb/N0 x N_P x budget sweep and the gamma sweep and print their JSON")
    return ap.parse_args()


def workload(args):
    from paper_2102_11089_gb300 import workloads as wl
    d = wl.wifi_like(2, 96)
    return d, 96


def config_dict(args, code):
    return {"workload": "wifi-like-qc-n2304-rate1/2", "code": "12x24 protograph, Z=96",
            "n": code.N, "k": code.K, "edges": code.E, "ebn0_db": args.ebn0,
            "schedule": args.schedule, "n_p": args.n_p, "n_g": args.n_g,
            "budget_updates": int(args.budget_iters * code.E), "batch_frames": args.batch,
            "arith": args.arith, "l2": "inputs larger than L2 (LLR batch %.0f MB)" %
            (args.batch * code.N * 4 / 1e6), "parallelism": f"frames sharded, dp{args.gpus}"}


# ---------------------------------------------------------------------------
# clocks sampling


class Clocks:
    """nvidia-smi clock / throttle samples every 200 ms.  start() returns once the
    first sample arrived: on a freshly booted box nvidia-smi's start-up takes
    seconds and stalled the GPU work submitted meanwhile."""

    def __init__(self):
        self.samples = []
        self.proc = None
        self.ready = threading.Event()

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
            self.ready.wait(timeout=60)
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])
            self.ready.set()
        self.ready.set()

    def mark(self):
        """Keep only the samples taken from now on (the timed region)."""
        self.samples = []

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [s for s in self.samples if len(s) >= 9 and s[0] == str(gpu_index)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# algorithmic work model (per committed update, FP32 state in shared memory)


def bytes_per_update(code, arith):
    """Algorithmic shared-memory bytes of one committed C2V update (FP32 state,
    V2C derived as L_j - L^C), from the per-update work of Table I with the
    code's average degrees (dv, dc):
      CN selection   8 dv       (L~^C and L^C of the dv edges into n*)
      commit         16         (read L~^C, write L^C, read/write L_n*)
      refresh        (dv-1) [8 dc + 8 (dc-1)]   (V2C inputs L_j, L^C; old/new L~^C)
      CI update      (dv-1)(dc-1) 12            (read/write L~_j, write D_j)
    with m = 4-byte messages and l = 4-byte LLRs / metrics; 6-bit mode: m = 1,
    l = 2 in the same terms."""
    dv = code.E / code.N
    dc = code.E / code.M
    m, l = (4, 4) if arith == "fp32" else (1, 2)
    return (2 * m * dv + (2 * m + 2 * l) + (dv - 1) * ((l + m) * dc + 2 * m * (dc - 1))
            + (dv - 1) * (dc - 1) * 3 * l)


def kernel_digest():
    import hashlib
    h = hashlib.sha1()
    for f in ["decode_me.cu", "device_math.cuh", "graph.cuh"]:
        with open(os.path.join(ROOT, "paper_2102_11089_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_traffic(args, batch):
    """DRAM bytes per decode launch from the committed ncu summary of this kernel
    and workload, scaled by frames; None unless the kernel sources still match
    the digest recorded with the capture (and the workload is the bench default)."""
    import re
    path = os.path.join(ROOT, "profiles", "me_decode_kernel_wifi_n2304_fp32.md")
    if not os.path.exists(path) or args.schedule != "me-lmd-cirbp" or args.arith != "fp32" or \
            args.n_p != 64 or args.n_g != 16 or args.ebn0 != 1.5 or args.budget_iters != 3.0:
        return None, None
    text = open(path).read()
    m = re.search(r"digest \(decode_me.cu,\s+device_math.cuh, graph.cuh\): ([0-9a-f]{12})", text)
    t = re.search(r"DRAM traffic per full bench launch \(65,536 frames, scaled by frames\): ([0-9.]+) MB", text)
    i = re.search(r"\| issue active \| ([0-9.]+) % \|", text)
    if not m or not t or m.group(1) != kernel_digest():
        return None, None
    return float(t.group(1)) * 1e6 * batch / 65536, (float(i.group(1)) if i else None)


def measured_smem_peak(L, device, stream):
    """Shared-memory read bandwidth (GB/s) of the ldpc_smem_stream kernel: best of
    a few launch shapes (CTAs per SM x threads), each timed with CUDA events on
    the launching stream after a warm-up launch."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    best = 0.0
    shapes = []
    for per_sm, threads in ((2, 1024), (4, 512), (8, 256)):
        blocks = sms * per_sm
        sink = torch.empty(blocks * threads, dtype=torch.int32, device=device)
        iters = 4096
        L.smem_stream(blocks, threads, iters, sink, stream=stream)
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            nbytes = L.smem_stream(blocks, threads, iters, sink, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        gbs = nbytes / (min(ts) * 1e-3) / 1e9
        shapes.append({"ctas_per_sm": per_sm, "threads": threads, "gb_s": gbs, "ms": min(ts)})
        best = max(best, gbs)
    return best, shapes


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# distributed plumbing


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def dist_max(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)


def cpu_baseline(args, design, Z, seconds):
    import oracle
    from paper_2102_11089_gb300 import workloads as wl
    base = design.shifts(Z)
    chk, var = oracle.qc_lift(base, Z)
    M, N = base.shape[0] * Z, base.shape[1] * Z
    K = design.info_cols * Z
    E = len(chk)
    cores = os.cpu_count() or 1
    sch = args.schedule
    budget = int(args.budget_iters * E)
    frames = 0
    t0 = time.perf_counter()
    el = 0.0
    batch = cores
    seed = 90000
    while el < seconds and frames < 4096:
        lam = oracle.awgn_llr(N, K / N, np.full(batch, args.ebn0), seed=seed, frame_offset=frames)
        if args.arith == "int6":
            q = oracle.quantize(lam.astype(np.float32), 0.5)
            oracle.decode(chk, var, M, N, qllr=q, schedule=sch, max_updates=budget, n_p=args.n_p,
                          n_g=args.n_g, threads=cores)
        else:
            oracle.decode(chk, var, M, N, llr=lam, schedule=sch, max_updates=budget, n_p=args.n_p,
                          n_g=args.n_g, threads=cores)
        frames += batch
        el = time.perf_counter() - t0
    return {"value": frames * K / el / 1e9, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
            "sample": f"{frames} frames of the same workload ({sch}, FP64 oracle, one frame per "
                      f"thread), {el:.1f} s"}


def run_reference(args):
    world, rank, local = dist_setup(args)
    try:
        if rank == 0:
            _reference_rank0(args, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


def _reference_rank0(args, world):
    from paper_2102_11089_gb300 import workloads as wl
    import oracle
    oracle.build()
    design, Z = workload(args)

    class _C:
        pass
    code = _C()
    sz = design.sizes(Z)
    code.N, code.K, code.E, code.M = sz["N"], sz["K"], sz["E"], sz["M"]
    per_step = min(args.cpu_seconds, max(2.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(args, design, Z, per_step / 4)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(args, design, Z, per_step))
    el = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    line = {"metric": "decoded info Gbit/s on 1 GB300 at fixed FER & update budget; vs flooding BP",
            "value": v, "unit": "Gbit/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, code), "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "Gbit/s", "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# our arm


def fer_of(out):
    hard = out["hard"]
    return float((hard.sum(1) > 0).float().mean().item())


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2102_11089_gb300 as L

    design, Z = workload(args)
    code = L.Code.from_protograph(design.shifts(Z), Z, design.info_cols * Z, design.punct_cols)
    B, N, K, E = args.batch, code.N, code.K, code.E
    budget = int(args.budget_iters * E)
    params = L.make_params(args.schedule, args.arith, gamma=0.1, n_p=args.n_p, n_g=args.n_g,
                           max_updates=budget, check_interval=1, seed=1234)
    stream = torch.cuda.current_stream()
    eb = torch.full((B,), args.ebn0, dtype=torch.float32, device=device)
    llr = torch.empty((B, N), dtype=torch.float32, device=device)
    qllr = torch.empty((B, N), dtype=torch.int8, device=device) if args.arith == "int6" else None
    out = dict(hard=torch.empty((B, N), dtype=torch.uint8, device=device),
               updates=torch.empty(B, dtype=torch.int64, device=device),
               converged=torch.empty(B, dtype=torch.uint8, device=device))
    frame_base = rank * (10 ** 9)
    dec_ev = []

    ch_ev = []

    def step(i, record=False):
        off = frame_base + i * B
        if record:
            c0 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
        L.awgn_llr(code, eb, seed=2021, frame_offset=off, out=llr, qout=qllr,
                   quantize=qllr is not None, stream=stream)
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ch_ev.append((c0, e0))
        L.decode(code, qllr if qllr is not None else llr, params, out=out, stream=stream)
        if record:
            e1.record(stream)
            dec_ev.append((e0, e1))

    clocks = Clocks()  # sampler started before the warm-up: its start-up must not overlap timing
    clocks.start()
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    L.sync(stream)
    upd_total = 0
    barrier(world, device)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    upd_hist = torch.empty((args.steps, B), dtype=torch.int64, device=device)
    upd_hist[0].copy_(out["updates"])  # first use of the copy path outside the timed region
    torch.cuda.synchronize()
    clocks.mark()
    t0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i, record=True)
        upd_hist[i].copy_(out["updates"])  # device-to-device copy; summed after timing
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world, device)
    ms = t0.elapsed_time(t1)
    clk = clocks.stop(local)
    upd_total = int(upd_hist.sum().item())
    fer = fer_of(out)
    conv = float((out["converged"] & 1).float().mean().item())
    mean_upd = float(out["updates"].float().mean().item())
    ms_max = dist_max(ms, world, device)
    value = world * B * args.steps * K / (ms_max * 1e-3) / 1e9
    dec_ms = [a.elapsed_time(b) for a, b in dec_ev]
    dec_avg = float(np.mean(dec_ms))
    ch_avg = float(np.mean([a.elapsed_time(b) for a, b in ch_ev]))
    # time of the timed region not inside a channel or decode launch (host enqueue
    # stalls, bookkeeping reductions); near zero when the stream stays busy
    gap_ms = ms / args.steps - dec_avg - ch_avg

    # ---- roofline of the decode kernel: algorithmic shared-memory bytes / time
    peaks, peaks_kind = measured_peaks()
    bpu = bytes_per_update(code, args.arith)
    alg_bytes = bpu * upd_total / args.steps
    achieved = alg_bytes / (dec_avg * 1e-3) / 1e9
    props = torch.cuda.get_device_properties(device)
    sm_count = props.multi_processor_count
    clk_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    smem_derived = sm_count * SMEM_BYTES_PER_CLK_PER_SM * clk_mhz * 1e6 / 1e9
    smem_peak, smem_shapes = measured_smem_peak(L, device, stream)
    traffic, issue_pct = profiled_traffic(args, B)
    roofline = {"bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
                "frac": achieved / smem_peak, "traffic": traffic,
                "traffic_note": "DRAM bytes per launch (ncu, 16,384-frame capture scaled by frames); "
                                "the bound is shared memory, DRAM carries only LLRs in and decisions out",
                "peak_source": "measured: ldpc_smem_stream (conflict-free 128-bit ld.shared over every SM, "
                               "CUDA events, best launch shape); shared memory is not in MEASURED_PEAKS",
                "peak_shapes": smem_shapes,
                "peak_derived_gbs": smem_derived,
                "peak_derived_note": f"{sm_count} SMs x 128 B/clk x median SM clock {clk_mhz:.0f} MHz",
                "kernel": f"me_decode_kernel ({args.schedule}, {args.arith})",
                "bytes_per_update": bpu, "updates_per_launch": upd_total / args.steps,
                "launch_ms": dec_avg, "hbm_peak_gbs": peaks.get("hbm_gbs"), "peaks": peaks_kind,
                "issue_active_pct": issue_pct,
                "binder": "instruction issue and the barriers between the phases of a step (ncu issue-active "
                          "share of the same kernel source, profiles/me_decode_kernel_wifi_n2304_fp32.md)"}

    # ---- end to end through host buffers: each step's LLR batch comes from pinned
    #      host memory and its decisions and counters go back to pinned host memory,
    #      copies inside the timed region.  Double-buffered: a copy stream brings in
    #      batch i+1 and takes out the results of batch i while batch i+1 decodes.
    #      The batches are made beforehand by the channel kernel (two alternate).
    x_dev = qllr if qllr is not None else llr
    e_steps = max(1, min(args.steps, 5))
    x_host = [torch.empty(tuple(x_dev.shape), dtype=x_dev.dtype, pin_memory=True) for _ in range(2)]
    for i in range(2):
        L.awgn_llr(code, eb, seed=2021, frame_offset=frame_base + (args.warmup + args.steps + i) * B, out=llr,
                   qout=qllr, quantize=qllr is not None, stream=stream)
        x_host[i].copy_(x_dev)
    xd = [x_dev, torch.empty_like(x_dev)]
    outs = [out, {k: torch.empty_like(v) for k, v in out.items()}]
    host_out = [{k: torch.empty(tuple(v.shape), dtype=v.dtype, pin_memory=True) for k, v in out.items()}
                for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=device)
    ev = lambda: torch.cuda.Event()  # noqa: E731
    torch.cuda.synchronize()
    barrier(world, device)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    copy_stream.wait_stream(stream)
    ev_in, ev_dec, ev_out = [ev() for _ in range(e_steps)], [ev() for _ in range(e_steps)], [ev() for _ in range(e_steps)]
    with torch.cuda.stream(copy_stream):
        xd[0].copy_(x_host[0], non_blocking=True)
    ev_in[0].record(copy_stream)
    for i in range(e_steps):
        b = i % 2
        stream.wait_event(ev_in[i])
        if i >= 2:
            stream.wait_event(ev_out[i - 2])  # outputs of step i-2 read back before they are reused
        L.decode(code, xd[b], params, out=outs[b], stream=stream)
        ev_dec[i].record(stream)
        if i + 1 < e_steps:
            if i >= 1:
                copy_stream.wait_event(ev_dec[i - 1])  # the other input buffer is free again
            with torch.cuda.stream(copy_stream):
                xd[1 - b].copy_(x_host[(i + 1) % 2], non_blocking=True)
            ev_in[i + 1].record(copy_stream)
        copy_stream.wait_event(ev_dec[i])
        with torch.cuda.stream(copy_stream):
            for k in ("hard", "updates", "converged"):
                host_out[b][k].copy_(outs[b][k], non_blocking=True)
        ev_out[i].record(copy_stream)
    stream.wait_stream(copy_stream)
    s1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = dist_max(s0.elapsed_time(s1), world, device)
    e2e = {"value": world * B * e_steps * K / (e2e_ms * 1e-3) / 1e9, "unit": "Gbit/s",
           "h2d_bytes_per_step": x_dev.numel() * x_dev.element_size(), "d2h_bytes_per_step": B * N + B * 8 + B,
           "steps": e_steps,
           "api": "ldpc_decode on one stream; LLR batches from pinned host memory and decisions and counters "
                  "to pinned host memory on a second stream, double-buffered"}
    del x_host, xd, outs, host_out

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(args, L, code, device, stream, fer, budget, value)

    # launches in the timed region: channel + decode per step
    launches = 2 * args.steps
    cpu = None
    if rank == 0 and world == 1:
        cpu = cpu_baseline(args, design, Z, args.cpu_seconds)
    if rank == 0:
        line = {"metric": "decoded info Gbit/s on 1 GB300 at fixed FER & update budget; vs flooding BP",
                "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.arith == "fp32" else "int8",
                "data": "synthetic (seeded Philox AWGN, all-zero codeword, seeded stand-in code)",
                "config": config_dict(args, code), "fer": fer, "frames_converged": conv,
                "mean_updates_per_frame": mean_upd, "decode_ms_per_launch": dec_avg,
                "channel_ms_per_launch": ch_avg, "other_ms_per_step": gap_ms,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, **extras}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def time_decode(L, code, x, params, reps=3):
    import torch
    out = L.decode(code, x, params)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = L.decode(code, x, params, out=out)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts)), out


def run_extras(args, L, code, device, stream, fer_ci, budget, value):
    """Flooding at equal FER and the single-edge LMD-CIRBP on a sub-batch."""
    import torch
    B2 = min(args.batch, 8192)
    eb = torch.full((B2,), args.ebn0, dtype=torch.float32, device=device)
    llr, q = L.awgn_llr(code, eb, seed=2021, frame_offset=0, quantize=args.arith == "int6")
    x = q if args.arith == "int6" else llr
    res = {}
    p_ci = L.make_params(args.schedule, args.arith, gamma=0.1, n_p=args.n_p, n_g=args.n_g,
                         max_updates=budget, check_interval=1, seed=1234)
    ms_ci, o_ci = time_decode(L, code, x, p_ci, reps=1)
    f_ci = fer_of(o_ci)
    flood = None
    for it in list(range(1, 21)) + [25, 30, 40, 50]:
        p = L.make_params("flooding", args.arith, max_updates=it * code.E, check_interval=code.E)
        ms, o = time_decode(L, code, x, p, reps=1)
        f = fer_of(o)
        if f <= f_ci:
            ms, o = time_decode(L, code, x, p, reps=3)
            flood = {"iterations": it, "fer": f, "ms": ms,
                     "gbit_s": B2 * code.K / (ms * 1e-3) / 1e9}
            break
    res["flooding_equal_fer"] = flood if flood else {"reached": False, "fer_ci": f_ci}
    res["ci_subbatch"] = {"frames": B2, "fer": f_ci, "ms": ms_ci,
                          "gbit_s": B2 * code.K / (ms_ci * 1e-3) / 1e9}
    B3 = min(B2, 2048)
    p_se = L.make_params("lmd-cirbp", args.arith, gamma=0.1, max_updates=budget, check_interval=1)
    ms_se, o_se = time_decode(L, code, x[:B3].contiguous(), p_se, reps=1)
    res["single_edge_lmd_cirbp"] = {"frames": B3, "fer": fer_of(o_se), "ms": ms_se,
                                    "gbit_s": B3 * code.K / (ms_se * 1e-3) / 1e9}
    res["single_edge_forms"] = run_se_forms(args, L, code, device)
    if not args.no_sweep:
        res["sweep_config2"] = run_sweep(args, L, code, device)
        res["gamma_sweep_cirbp"] = run_gamma_sweep(args, L, code, device)
    if args.queue_frames > 0:
        res["queue_mixed_bg2"] = run_queue_mixed(args, L, device)
    if args.large_frames > 0:
        res["large_bg1_z384"] = run_large_bg1(args, L, device)
        res["large_bg1_ebn0_sweep"] = run_large_sweep(args, L, device)
    res["weighted_bp_config4"] = run_wbp_config4(args, L, device)
    # Properties 1 and 2 (Sec. 3.A) on flooding: empirical J(gamma), F(gamma) at
    # gamma = 0, 0.1, ..., 0.9 for iterations 0-2 (analogue of the paper's Fig. 1b)
    from paper_2102_11089_gb300.ci_stats import flooding_counts, j_and_f
    cnt = flooding_counts(code, llr, 3, n_bins=10)
    J, F = j_and_f(cnt)
    clean = lambda a: [None if not np.isfinite(v) else float(v) for v in a]  # noqa: E731
    res["ci_properties_flooding"] = {"frames": int(llr.shape[0]), "gamma": [b / 10 for b in range(10)],
                                     "J": [clean(J[k]) for k in range(3)], "F": [clean(F[k]) for k in range(3)],
                                     "incorrect_per_iteration": [int(cnt[k][:, 1].sum()) for k in range(3)]}
    return res


def clopper_pearson(k, n, alpha=0.05):
    from scipy import stats
    lo = 0.0 if k == 0 else float(stats.beta.ppf(alpha / 2, k, n - k + 1))
    hi = 1.0 if k == n else float(stats.beta.ppf(1 - alpha / 2, k + 1, n - k))
    return lo, hi


def frame_errors(out):
    return int((out["hard"].sum(1) > 0).sum().item())


def run_sweep(args, L, code, device, ebn0s=(1.0, 1.25, 1.5, 1.75, 2.0, 2.25, 2.5), nps=(4, 16, 64),
              budgets=(1, 2, 3, 5, 10), frames=65536, frames_np4=16384):
    """The WiFi-like code over Eb/N0 x N_P x budget (ME-LMD-CIRBP, FP32), each
    point against flooding BP at equal FER on the same frames.

    Flooding's FER after I iterations follows from one run of 50 iterations
    that stops each frame at its first zero syndrome: a frame is decoded
    correctly within I iterations iff it stopped by iteration I on the all-zero
    word (its run up to then is the same at any budget >= I).  The equal-FER
    iteration count I* is the smallest I whose FER is at most the CI FER; its
    throughput is timed by a run at budget I*E.  Also reported: flooding's FER
    at the CI budget itself (the same number of committed messages)."""
    import torch
    E, K = code.E, code.K
    rows = []
    variants = []
    flood_ms_cache = {}
    t_start = time.perf_counter()
    for eb in ebn0s:
        B = frames
        ebt = torch.full((B,), eb, dtype=torch.float32, device=device)
        llr, _ = L.awgn_llr(code, ebt, seed=4242, frame_offset=0)
        pf = L.make_params("flooding", "fp32", max_updates=50 * E, check_interval=E)
        of = L.decode(code, llr, pf)
        torch.cuda.synchronize()
        it_used = (of["updates"] // E).cpu().numpy()
        ok = ((of["hard"].sum(1) == 0) & ((of["converged"] & 1) == 1)).cpu().numpy()
        flood_fer = [1.0 - float(np.mean(ok & (it_used <= i))) for i in range(0, 51)]
        for n_p in nps:
            Bn = frames_np4 if n_p <= 4 else frames
            x = llr[:Bn]
            for bi in budgets:
                p = L.make_params("me-lmd-cirbp", "fp32", gamma=0.1, n_p=n_p, n_g=16, max_updates=bi * E,
                                  check_interval=1, seed=1234)
                ms, o = time_decode(L, code, x, p, reps=1)
                errs = frame_errors(o)
                fer = errs / Bn
                lo, hi = clopper_pearson(errs, Bn)
                fsub = [1.0 - float(np.mean((ok & (it_used <= i))[:Bn])) for i in range(0, 51)]
                istar = next((i for i in range(1, 51) if fsub[i] <= fer), None)
                row = {"ebn0_db": eb, "n_p": n_p, "budget_iters": bi, "frames": Bn, "ci_fer": fer,
                       "ci_fer_ci95": [lo, hi], "ci_ms": ms, "ci_gbit_s": Bn * K / (ms * 1e-3) / 1e9,
                       "ci_mean_updates": float(o["updates"].float().mean().item()),
                       "flood_fer_same_budget": fsub[bi]}
                if istar is None:
                    row["flood_equal_fer"] = {"reached": False, "flood_fer_50": fsub[50]}
                else:
                    key = (eb, Bn, istar)
                    if key not in flood_ms_cache:
                        pfi = L.make_params("flooding", "fp32", max_updates=istar * E, check_interval=E)
                        flood_ms_cache[key] = time_decode(L, code, x, pfi, reps=1)[0]
                    fms = flood_ms_cache[key]
                    fg = Bn * K / (fms * 1e-3) / 1e9
                    row["flood_equal_fer"] = {"iterations": istar, "fer": fsub[istar], "ms": fms, "gbit_s": fg}
                    row["ci_over_flood"] = row["ci_gbit_s"] / fg
                rows.append(row)
        if eb == 1.5:  # the other multi-edge settings of the config at the headline point
            for sch, n_p, n_g in (("me-cirbp", 64, 16), ("me-lmd-cirbp", 64, 4), ("me-lmd-cirbp", 64, 8)):
                p = L.make_params(sch, "fp32", gamma=0.1, n_p=n_p, n_g=n_g, max_updates=3 * E, check_interval=1,
                                  seed=1234)
                ms, o = time_decode(L, code, llr, p, reps=1)
                errs = frame_errors(o)
                variants.append({"schedule": sch, "n_p": n_p, "n_g": n_g, "ebn0_db": eb, "budget_iters": 3,
                                 "frames": B, "fer": errs / B, "fer_ci95": list(clopper_pearson(errs, B)),
                                 "ms": ms, "gbit_s": B * K / (ms * 1e-3) / 1e9,
                                 "mean_updates": float(o["updates"].float().mean().item())})
        del llr, of
    return {"workload": "wifi-like n2304, ME-LMD-CIRBP FP32, N_G 16, Eb/N0 x N_P x budget; flooding at equal "
                        "FER on the same frames", "points": rows, "variants": variants,
            "seconds": time.perf_counter() - t_start}


def run_se_forms(args, L, code, device, frames=8192, ebn0=1.5, budget_iters=3):
    """The single-edge schedules (Algorithms 1 and 3, RBP) on the WiFi-like code in
    their three execution forms: frame state in shared memory (two FP32 frames per
    SM), in global memory (32 warps per SM), and split (VN and check arrays in
    shared memory, edge arrays in global memory).  Results are identical in every
    form (checked)."""
    import torch
    E, K = code.E, code.K
    ebt = torch.full((frames,), ebn0, dtype=torch.float32, device=device)
    llr, _ = L.awgn_llr(code, ebt, seed=7171, frame_offset=0)
    rows = []
    for sch in ("lmd-cirbp", "cirbp", "rbp"):
        row = {"schedule": sch}
        ref = None
        for name, form in (("smem", L.FORM_SMEM), ("global", L.FORM_GLOBAL), ("split", L.FORM_SPLIT),
                           ("auto", L.FORM_AUTO)):
            p = L.make_params(sch, "fp32", gamma=0.1, max_updates=budget_iters * E, check_interval=1, form=form)
            ms, o = time_decode(L, code, llr, p, reps=1)
            if ref is None:
                ref = o
                row["fer"] = fer_of(o)
            row[name] = {"ms": ms, "gbit_s": frames * K / (ms * 1e-3) / 1e9,
                         "identical": all(torch.equal(ref[k], o[k]) for k in ref)}
        rows.append(row)
    return {"workload": f"wifi-like n2304, FP32, Eb/N0 {ebn0} dB, budget {budget_iters}E", "frames": frames,
            "points": rows}


def run_gamma_sweep(args, L, code, device, gammas=(0.0, 0.05, 0.1, 0.15, 0.2, 0.25, 0.3), frames=8192,
                    ebn0=1.5, budget_iters=3):
    """CIRBP (Algorithm 1) over the CI threshold gamma on the WiFi-like code:
    FER and kappa = Pr(D_{n*} < gamma), the share of updates whose edge came
    from the residual fallback (Sec. 5.A), with the decode throughput."""
    import torch
    E, K = code.E, code.K
    ebt = torch.full((frames,), ebn0, dtype=torch.float32, device=device)
    llr, _ = L.awgn_llr(code, ebt, seed=5151, frame_offset=0)
    rows = []
    for gmm in gammas:
        p = L.make_params("cirbp", "fp32", gamma=gmm, max_updates=budget_iters * E, check_interval=1)
        L.decode(code, llr, p)  # warm-up
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        o = L.decode(code, llr, p, want_fallbacks=True)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        errs = frame_errors(o)
        upd = int(o["updates"].sum().item())
        fb = int(o["fallbacks"].sum().item())
        rows.append({"gamma": gmm, "fer": errs / frames, "fer_ci95": list(clopper_pearson(errs, frames)),
                     "kappa": fb / max(1, upd), "mean_updates": upd / frames, "ms": ms,
                     "gbit_s": frames * K / (ms * 1e-3) / 1e9})
    return {"workload": f"wifi-like n2304, CIRBP FP32, Eb/N0 {ebn0} dB, budget {budget_iters}E",
            "frames": frames, "points": rows}


QUEUE_ZS = (16, 32, 64, 128, 256, 384)


def mixed_bg2(L, device, frames, arith="fp32", seed=3):
    """Frames of the BG2-shaped code (42x52 protograph, 2 punctured columns) at
    lifting sizes drawn uniformly from 16..384, Eb/N0 ~ U[0.5, 3.0] dB and an
    update budget ~ U{2..20} x E per frame.  Frames are stored grouped by
    (Z, budget), so per-batch launches read contiguous blocks; frame ids run in
    that order (channel counter and Algorithm 4 keys)."""
    import torch
    from paper_2102_11089_gb300 import workloads as wl
    design = wl.bg2_like(3)
    rng = np.random.default_rng(seed)
    zi = rng.integers(0, len(QUEUE_ZS), frames)
    ebn0 = rng.uniform(0.5, 3.0, frames).astype(np.float32)
    bud = rng.integers(2, 21, frames)
    order = np.lexsort((bud, zi))
    zi, ebn0, bud = zi[order], ebn0[order], bud[order]
    codes = [L.Code.from_protograph(design.shifts(Z), Z, design.info_cols * Z, design.punct_cols)
             for Z in QUEUE_ZS]
    Ns = np.array([c.N for c in codes])
    Es = np.array([c.E for c in codes])
    Ks = np.array([c.K for c in codes])
    n_of = Ns[zi]
    off = np.concatenate([[0], np.cumsum(n_of)[:-1]]).astype(np.int64)
    total = int(n_of.sum())
    dt = torch.int8 if arith == "int6" else torch.float32
    llr = torch.empty(total, dtype=dt, device=device)
    groups = []  # (code index, budget, first frame, count, offset)
    for ci, c in enumerate(codes):
        idx = np.nonzero(zi == ci)[0]
        if len(idx) == 0:
            continue
        f0, B = int(idx[0]), len(idx)
        eb = torch.from_numpy(ebn0[idx]).to(device)
        lam, q = L.awgn_llr(c, eb, seed=2021, frame_offset=f0, quantize=arith == "int6")
        x = q if arith == "int6" else lam
        llr[off[f0]:off[f0] + B * c.N].copy_(x.reshape(-1))
        for b in np.unique(bud[idx]):
            sub = idx[bud[idx] == b]
            groups.append((ci, int(b) * c.E, int(sub[0]), len(sub), int(off[sub[0]])))
    budget = bud * Es[zi]
    return dict(codes=codes, zi=zi, budget=budget, off=off, total=total, llr=llr, groups=groups,
                info_bits=int(Ks[zi].sum()), Es=Es, frames=frames)


def run_queue_mixed(args, L, device, frames=None, reps=2):
    """Persistent work queue (one launch, items in decreasing-cost order, launch
    shape from the autotuner) against per-batch launches of the same frames:
    ldpc_decode per (Z, budget) group, and the queue kernel in static mode per
    Z group.  Every form computes the same results (checked)."""
    import tempfile
    import torch
    from paper_2102_11089_gb300 import autotune as at
    frames = frames or args.queue_frames
    arith = "fp32"
    w = mixed_bg2(L, device, frames, arith)
    codes, zi, F = w["codes"], w["zi"], frames
    p = L.make_params("me-lmd-cirbp", arith, gamma=0.1, n_p=args.n_p, n_g=args.n_g, check_interval=1, seed=1234)
    cost = w["budget"].astype(np.float64)
    lpt = np.argsort(-cost, kind="stable")
    items = L.make_items(zi[lpt], w["off"][lpt], w["off"][lpt], w["budget"][lpt], lpt, device=device)
    hard = torch.empty(w["total"], dtype=torch.uint8, device=device)
    upd = torch.empty(F, dtype=torch.int64, device=device)
    conv = torch.empty(F, dtype=torch.uint8, device=device)

    def ev_time(fn, n):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(n):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.min(ts))

    # autotune the queue launch on a calibration queue (the costliest quarter of the items)
    nc = max(1, F // 4)
    cal = L.make_items(zi[lpt[:nc]], w["off"][lpt[:nc]], w["off"][lpt[:nc]], w["budget"][lpt[:nc]],
                       lpt[:nc], device=device)
    with tempfile.TemporaryDirectory() as d:
        cache = at.TuneCache(os.path.join(d, "tune.json"))
        tune = at.tune_queue(codes, cal, nc, w["llr"], p, hard=hard, updates=upd, converged=conv,
                             cache=cache, repeats=1)
        tune_ms = json.load(open(cache.path))
    tune_ms = next(iter(tune_ms.values()))["ms"]
    p.tune = tune

    def persistent():
        L.decode_queue(codes, items, F, w["llr"], p, hard=hard, updates=upd, converged=conv,
                       mode=L.QUEUE_PERSISTENT)

    ms_q = ev_time(persistent, reps)
    inv = torch.from_numpy(np.argsort(lpt)).to(device)
    upd_q, conv_q = upd[inv].clone(), conv[inv].clone()  # item order -> frame id

    # per-batch launches: ldpc_decode per (Z, budget) group
    p_b = L.make_params("me-lmd-cirbp", arith, gamma=0.1, n_p=args.n_p, n_g=args.n_g, check_interval=1,
                        seed=1234)
    hard_b = torch.empty_like(hard)
    upd_b = torch.empty(F, dtype=torch.int64, device=device)
    conv_b = torch.empty(F, dtype=torch.uint8, device=device)
    views = []
    for ci, budget, f0, B, o in w["groups"]:
        c = codes[ci]
        x = w["llr"][o:o + B * c.N].view(B, c.N)
        out = dict(hard=hard_b[o:o + B * c.N].view(B, c.N), updates=upd_b[f0:f0 + B],
                   converged=conv_b[f0:f0 + B])
        pg = L.make_params("me-lmd-cirbp", arith, gamma=0.1, n_p=args.n_p, n_g=args.n_g,
                           check_interval=1, seed=1234, max_updates=budget, frame_offset=f0)
        views.append((c, x, pg, out))

    def per_batch():
        for c, x, pg, out in views:
            L.decode(c, x, pg, out=out)

    ms_b = ev_time(per_batch, reps)

    # queue kernel in static mode (one CTA per item), one launch per Z group
    zitems = []
    for ci in range(len(codes)):
        idx = np.nonzero(zi == ci)[0]
        if len(idx):
            zitems.append((L.make_items(zi[idx], w["off"][idx], w["off"][idx], w["budget"][idx], idx,
                                        device=device), len(idx)))
    hard_s = torch.empty_like(hard)
    upd_s = torch.empty(F, dtype=torch.int64, device=device)
    conv_s = torch.empty(F, dtype=torch.uint8, device=device)

    def static_per_z():
        pos = 0
        for it, n in zitems:
            L.decode_queue(codes, it, n, w["llr"], p_b, hard=hard_s, updates=upd_s[pos:pos + n],
                           converged=conv_s[pos:pos + n], mode=L.QUEUE_STATIC)
            pos += n

    ms_s = ev_time(static_per_z, reps)
    torch.cuda.synchronize()
    L.sync()
    same = bool(torch.equal(hard, hard_b) and torch.equal(upd_q, upd_b) and torch.equal(conv_q, conv_b)
                and torch.equal(hard, hard_s) and torch.equal(upd_s, upd_b) and torch.equal(conv_s, conv_b))
    # frame errors: any decided bit of a frame set (all-zero codeword)
    errs = 0
    hb = hard.cpu().numpy()
    for f in range(F):
        n = codes[zi[f]].N
        o = w["off"][f]
        errs += int(hb[o:o + n].any())
    gbit = lambda ms: w["info_bits"] / (ms * 1e-3) / 1e9  # noqa: E731
    return {"workload": "bg2-like 42x52, Z~U{16..384}, Eb/N0~U[0.5,3] dB, budget~U{2..20}E per frame",
            "frames": F, "schedule": "me-lmd-cirbp", "arith": arith, "n_p": args.n_p,
            "fer": errs / F, "mean_updates_per_frame": float(upd_b.float().mean().item()),
            "identical_results": same,
            "persistent": {"ms": ms_q, "gbit_s": gbit(ms_q), "launches": 1, "tune": tune,
                           "tune_shape": at.describe(tune), "tune_search_ms": tune_ms,
                           "order": "decreasing budget"},
            "per_batch_decode": {"ms": ms_b, "gbit_s": gbit(ms_b), "launches": len(views),
                                 "grouping": "(Z, budget)"},
            "static_queue_per_z": {"ms": ms_s, "gbit_s": gbit(ms_s), "launches": len(zitems)},
            "speedup_vs_per_batch": ms_b / ms_q, "speedup_vs_static_per_z": ms_s / ms_q}


def run_large_bg1(args, L, device, frames=None, reps=2, points=None):
    """The BG1-shaped code (46x68 protograph, Z=384: n=26,112, about 120k edges),
    ME-LMD-CIRBP at Eb/N0 = 1.2 dB with budget 5E: frame state spread over a
    thread-block cluster's shared memory against global-memory slots, FP32 and
    6-bit, N_P = 64 and 256.  Both forms give identical results (checked)."""
    import torch
    from paper_2102_11089_gb300 import workloads as wl
    frames = frames or args.large_frames
    d = wl.bg1_like(5)
    code = L.Code.from_protograph(d.shifts(384), 384, d.info_cols * 384, d.punct_cols)
    eb = torch.full((frames,), 1.2, dtype=torch.float32, device=device)
    res = {"workload": "bg1-like 46x68, Z=384, n=26112, Eb/N0 1.2 dB, budget 5E", "frames": frames,
           "n": code.N, "edges": code.E, "k": code.K, "points": []}
    for arith, n_p in (points or [("fp32", 64), ("fp32", 256), ("int6", 256)]):
        lam, q = L.awgn_llr(code, eb, seed=2021, frame_offset=0, quantize=arith == "int6")
        x = q if arith == "int6" else lam
        row = {"arith": arith, "n_p": n_p}
        outs = {}
        for name, form in (("cluster", L.FORM_CLUSTER), ("global", L.FORM_GLOBAL)):
            p = L.make_params("me-lmd-cirbp", arith, gamma=0.1, n_p=n_p, n_g=16, max_updates=5 * code.E,
                              check_interval=1, seed=1234, form=form)
            try:
                ms, o = time_decode(L, code, x, p, reps=reps)
            except L.LdpcError as e:
                row[name] = {"unavailable": str(e)}
                continue
            outs[name] = o
            row[name] = {"ms": ms, "gbit_s": frames * code.K / (ms * 1e-3) / 1e9, "fer": fer_of(o),
                         "mean_updates": float(o["updates"].float().mean().item())}
        if len(outs) == 2:
            row["identical_results"] = all(torch.equal(outs["cluster"][k], outs["global"][k]) for k in outs["global"])
            row["speedup_cluster_vs_global"] = row["global"]["ms"] / row["cluster"]["ms"]
        res["points"].append(row)
    return res


def run_large_sweep(args, L, device, frames=1216, ebn0s=(0.8, 1.0, 1.2, 1.4, 1.6)):
    """The 26,112-bit BG1-shaped code over Eb/N0 0.8-1.6 dB (ME-LMD-CIRBP, budget
    5E, FP32 at N_P = 64 and 256, 6-bit at N_P = 256; default form): FER and
    decoded Gbit/s on a bounded batch per point (four waves of the global-memory
    form) in place of the HBM-sized batch."""
    import torch
    from paper_2102_11089_gb300 import workloads as wl
    d = wl.bg1_like(5)
    code = L.Code.from_protograph(d.shifts(384), 384, d.info_cols * 384, d.punct_cols)
    rows = []
    for eb in ebn0s:
        ebt = torch.full((frames,), eb, dtype=torch.float32, device=device)
        lam, q = L.awgn_llr(code, ebt, seed=3131, frame_offset=0, quantize=True)
        for arith, n_p in (("fp32", 64), ("fp32", 256), ("int6", 256)):
            x = q if arith == "int6" else lam
            p = L.make_params("me-lmd-cirbp", arith, gamma=0.1, n_p=n_p, n_g=16, max_updates=5 * code.E,
                              check_interval=1, seed=1234)
            ms, o = time_decode(L, code, x, p, reps=1)
            errs = frame_errors(o)
            rows.append({"ebn0_db": eb, "arith": arith, "n_p": n_p, "fer": errs / frames,
                         "fer_ci95": list(clopper_pearson(errs, frames)), "ms": ms,
                         "gbit_s": frames * code.K / (ms * 1e-3) / 1e9,
                         "mean_updates": float(o["updates"].float().mean().item())})
        del lam, q
    return {"workload": "bg1-like 46x68, Z=384, n=26112, budget 5E, ME-LMD-CIRBP", "frames_per_point": frames,
            "points": rows}


def run_queue_stream(args, L, device, frames):
    """Config 3 at its stated size: `frames` mixed-lifting BG2-shaped frames (Z
    uniform over 16..384, Eb/N0 ~ U[0.5, 3.0] dB, budget ~ U{2..20}E per frame)
    streamed through one persistent queue launch (items in decreasing-budget
    order, autotuned launch shape); FER and decoded Gbit/s."""
    import tempfile
    import torch
    from paper_2102_11089_gb300 import autotune as at
    w = mixed_bg2(L, device, frames, "fp32")
    codes, zi = w["codes"], w["zi"]
    p = L.make_params("me-lmd-cirbp", "fp32", gamma=0.1, n_p=args.n_p, n_g=args.n_g, check_interval=1, seed=1234)
    lpt = np.argsort(-w["budget"].astype(np.float64), kind="stable")
    items = L.make_items(zi[lpt], w["off"][lpt], w["off"][lpt], w["budget"][lpt], lpt, device=device)
    hard = torch.empty(w["total"], dtype=torch.uint8, device=device)
    upd = torch.empty(frames, dtype=torch.int64, device=device)
    conv = torch.empty(frames, dtype=torch.uint8, device=device)
    nc = min(frames, 4096)
    cal = L.make_items(zi[lpt[:nc]], w["off"][lpt[:nc]], w["off"][lpt[:nc]], w["budget"][lpt[:nc]], lpt[:nc],
                       device=device)
    with tempfile.TemporaryDirectory() as dd:
        p.tune = at.tune_queue(codes, cal, nc, w["llr"], p, hard=hard, updates=upd, converged=conv,
                               cache=at.TuneCache(os.path.join(dd, "tune.json")), repeats=1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    L.decode_queue(codes, items, frames, w["llr"], p, hard=hard, updates=upd, converged=conv,
                   mode=L.QUEUE_PERSISTENT)
    b.record()
    torch.cuda.synchronize()
    L.sync()
    ms = a.elapsed_time(b)
    # frame errors: any decided bit of a frame set (all-zero codeword), per Z block
    errs = 0
    hb = hard.cpu().numpy()
    Ns = np.array([c.N for c in codes])
    for ci in range(len(codes)):
        idx = np.nonzero(zi == ci)[0]
        if len(idx) == 0:
            continue
        o0 = int(w["off"][idx[0]])
        errs += int(hb[o0:o0 + len(idx) * Ns[ci]].reshape(len(idx), Ns[ci]).any(axis=1).sum())
    return {"workload": "bg2-like 42x52, Z~U{16..384}, Eb/N0~U[0.5,3] dB, budget~U{2..20}E per frame",
            "frames": frames, "launches": 1, "ms": ms, "gbit_s": w["info_bits"] / (ms * 1e-3) / 1e9,
            "fer": errs / frames, "fer_ci95": list(clopper_pearson(errs, frames)),
            "mean_updates_per_frame": float(upd.float().mean().item()), "tune": at.describe(p.tune),
            "llr_gb": w["total"] * 4 / 1e9}


def run_wbp_config4(args, L, device, frames=4096, reps=2):
    """Weighted BP and its adjoint (12x24 protograph, Z=24: n=576), T = 8E
    updates of an LMD-CIRBP schedule recorded at 2.0 dB, 4,096 frames: time of
    the forward replay and of the adjoint (CUDA events), BCE loss."""
    import torch
    from paper_2102_11089_gb300 import workloads as wl
    from paper_2102_11089_gb300.wbp import bce_all_zero, record_schedule, weighted_bp
    d = wl.wifi_like(2, 24)
    code = L.Code.from_protograph(d.shifts(24), 24, d.info_cols * 24, d.punct_cols)
    eb = torch.full((frames,), 2.0, dtype=torch.float32, device=device)
    llr, _ = L.awgn_llr(code, eb, seed=2021)
    T = 8 * code.E
    trace, _ = record_schedule(code, llr, T)
    w = torch.ones(T, device=device, requires_grad=True)
    x = llr.requires_grad_(False)

    def fwd():
        return weighted_bp(code, x, trace, w)

    out = fwd()
    loss = bce_all_zero(out)
    loss.backward()
    torch.cuda.synchronize()
    tf, tb = [], []
    for _ in range(reps):
        w.grad = None
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        out = fwd()
        b.record()
        loss = bce_all_zero(out)
        loss.backward()
        c.record()
        torch.cuda.synchronize()
        tf.append(a.elapsed_time(b))
        tb.append(b.elapsed_time(c))
    upd = frames * T
    return {"workload": "wifi-like 12x24, Z=24 (n=576), T=8E LMD-CIRBP schedule, 2.0 dB", "frames": frames,
            "T": T, "forward_ms": min(tf), "backward_ms": min(tb), "loss": float(loss.detach()),
            "forward_updates_per_s": upd / (min(tf) * 1e-3), "backward_updates_per_s": upd / (min(tb) * 1e-3),
            "grad_norm": float(w.grad.norm())}


def run_decode_only(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2102_11089_gb300 as L
    design, Z = workload(args)
    code = L.Code.from_protograph(design.shifts(Z), Z, design.info_cols * Z, design.punct_cols)
    eb = torch.full((args.batch,), args.ebn0, dtype=torch.float32, device="cuda")
    llr, q = L.awgn_llr(code, eb, seed=2021, quantize=args.arith == "int6")
    x = q if args.arith == "int6" else llr
    p = L.make_params(args.schedule, args.arith, gamma=0.1, n_p=args.n_p, n_g=args.n_g,
                      max_updates=int(args.budget_iters * code.E), check_interval=1, seed=1234)
    for _ in range(args.reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = L.decode(code, x, p)
        b.record()
        torch.cuda.synchronize()
        print(json.dumps({"schedule": args.schedule, "arith": args.arith, "batch": args.batch,
                          "ms": a.elapsed_time(b), "mean_updates": out["updates"].float().mean().item(),
                          "fer": fer_of(out)}))


def main():
    args = parse()
    if args.queue_stream > 0:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_2102_11089_gb300 as L
        print(json.dumps(run_queue_stream(args, L, torch.device("cuda", 0), args.queue_stream)))
        return
    if args.queue_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_2102_11089_gb300 as L
        print(json.dumps(run_queue_mixed(args, L, torch.device("cuda", 0), reps=args.reps)))
        return
    if args.wbp_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_2102_11089_gb300 as L
        print(json.dumps(run_wbp_config4(args, L, torch.device("cuda", 0), reps=args.reps)))
        return
    if args.large_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_2102_11089_gb300 as L
        print(json.dumps(run_large_bg1(args, L, torch.device("cuda", 0), reps=args.reps)))
        return
    if args.decode_only:
        run_decode_only(args)
        return
    if args.sweep_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_2102_11089_gb300 as L
        design, Z = workload(args)
        code = L.Code.from_protograph(design.shifts(Z), Z, design.info_cols * Z, design.punct_cols)
        dev = torch.device("cuda", 0)
        print(json.dumps({"sweep_config2": run_sweep(args, L, code, dev),
                          "gamma_sweep_cirbp": run_gamma_sweep(args, L, code, dev)}))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
