"""Benchmark of the GCDF hot path: value + df/dq for every (waypoint, point)
pair of a synthetic scene, fused with the per-waypoint soft-min collision cost.

Workload (one step): the single-trajectory box scene — 9-DOF net (4 x 256 SiLU,
He-uniform seed 0), 128 waypoints, 16,384 points on the surfaces of 20 seeded
boxes in a 10 x 10 x 2 m room, soft-min temperature 0.02 — i.e. 2,097,152
value+gradient pairs reduced to 128 costs and gradients.  Inputs are synthetic
(`synth`); the paper's benchmark maps are not available.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the same workload
    python bench.py --serve                 # served-planning latency (see run_serve)
    python bench.py --plan [--plan-problems P]   # batched trajectory optimisation (see run_plan)
    python bench.py --aux                   # partition, Jacobian scatter, projection kernels
    python bench.py --fit                   # differentiable-fit training step (see run_fit)

Multi-GPU: one process per GPU (torchrun); every rank runs its own replica of
the workload (weak scaling, no collective on the data path); the time is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def flops_per_pair(shape: synth.NetShape) -> int:
    """Algorithmic FLOPs of one value + df/dq pair (multiply-add = 2 FLOPs):
    forward (L-1) H x H layers, the output dot product and the outer-sum add of
    the split first layer; reverse (L-1) H x H layers and the d_q x H input
    Jacobian."""
    H, L, dq = shape.hidden, shape.n_layers, shape.d_q
    fwd = (L - 1) * 2 * H * H + 2 * H + H
    rev = (L - 1) * 2 * H * H + 2 * dq * H
    return fwd + rev


def job_throughput(local_seconds: float, units_per_rank: float, dist=None, device=None):
    """Whole-job rate for replicas that each process `units_per_rank` units:
    the slowest rank's time (maximum over ranks) bounds the job.  Returns
    (max_seconds, units_per_second over all ranks)."""
    world = 1
    t = local_seconds
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        buf = torch.tensor([local_seconds], dtype=torch.float64, device=device)
        dist.all_reduce(buf, op=dist.ReduceOp.MAX)
        t = float(buf.item())
    return t, world * units_per_rank / t


def measured_traffic(precision: str, workload: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    or None when that summary is for another workload or a source file of the
    kernel has changed since the counters were taken (sha1 over the files in
    order)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh).get(precision)
    if not rec or not workload.startswith(rec["workload"]):
        return None
    if "sources" not in rec:
        return None
    h = hashlib.sha1()
    for src in rec["sources"]:
        with open(os.path.join(ROOT, src), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != rec["sha1"]:
        return None
    return rec["dram_bytes_per_launch"]


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return dict(PEAKS_FALLBACK, sm_max_mhz=2070.0), "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None, interval_ms: int = 200):
        self.uuid = uuid
        self.interval_ms = int(interval_ms)
        self.proc = None
        self.path = os.path.join("/tmp", f"gcdf_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", str(self.interval_ms)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and parts[1] != self.uuid:
                    continue
                try:
                    sm.append(float(parts[2]))
                    smax.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[6:10]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:  # a record field only
        return None


WAYPOINTS, POINTS = 128, 16384


def make_workload():
    return synth.box_scene(n_waypoints=WAYPOINTS, n_points=POINTS)


# ---------------------------------------------------------------------------
# CPU oracle leg (the only place this script runs oracle/)
# ---------------------------------------------------------------------------

def host_cpu() -> dict:
    """The host's logical CPU count and model (for the CPU baseline's record)."""
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part"):
                    model = f"{platform.machine()} {line.split(':', 1)[1].strip()}"
                    break
    except Exception:  # a record field only: never fail the benchmark over it
        pass
    return {"nproc": os.cpu_count(), "model": model}


def cpu_oracle_leg(wl, budget_s: float = 12.0, gpu_result=None):
    """Time the FP64 oracle on a bounded sample of the workload: whole waypoints
    (all 16,384 points each, evenly spread over the trajectory) until about
    `budget_s` seconds have elapsed (at least one waypoint)."""
    from oracle import metrics, reduce as red
    s = wl.shape
    N, M = wl.q.shape[0], wl.p.shape[0]
    order = [int(i) for i in np.argsort(np.arange(N) * 0.61803398875 % 1.0)]
    done, costs, grads = [], [], []
    t0 = time.perf_counter()
    for i in order:
        c, g, _ = red.collision_cost(s.n_dof, s.hidden, s.n_layers, wl.weights, wl.q, wl.p,
                                     wl.reduction, wl.param, waypoints=[i])
        done.append(i)
        costs.append(c[0])
        grads.append(g[0])
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    pairs = len(done) * M
    try:
        import threadpoolctl
        cores = max([d.get("num_threads", 1) for d in threadpoolctl.threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    out = {"value": pairs / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
           "sample": f"{len(done)} of {N} waypoints x {M} points ({pairs} pairs), FP64 NumPy, {dt:.1f} s",
           "pairs": pairs, "seconds": dt, "host": host_cpu()}
    if gpu_result is not None:
        c_gpu, g_gpu = gpu_result
        out["sample_err_cost_max"] = float(metrics.rel_err_scalar(c_gpu[done], np.array(costs)).max())
        out["sample_err_grad_max"] = float(metrics.rel_err_vector(g_gpu[done], np.array(grads)).max())
    return out


_SINGLE_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                      "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")


def cpu_oracle_single_thread(budget_s: float = 6.0):
    """The same oracle leg in a fresh interpreter with every BLAS / OpenMP pool
    limited to one thread (the limits must be set before NumPy loads)."""
    env = dict(os.environ)
    for k in _SINGLE_THREAD_ENV:
        env[k] = "1"
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "r = bench.cpu_oracle_leg(bench.make_workload(), budget_s=%r); r['cores'] = 1; "
            "print(json.dumps(r))") % (ROOT, float(budget_s))
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=budget_s * 10 + 120)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # a record field only: never fail the benchmark over it
        return {"error": f"{type(e).__name__}: {e}"}


def run_reference(args):
    """The oracle as it stands, timed on this host's cores, one bounded sample
    per step; only rank 0 works."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = make_workload()
    per_step = min(args.ref_budget, 150.0 / (args.steps + args.warmup))
    rs = [cpu_oracle_leg(wl, budget_s=per_step) for _ in range(args.warmup + args.steps)][args.warmup:]
    pairs = sum(r["pairs"] for r in rs)
    secs = sum(r["seconds"] for r in rs)
    value = pairs / secs
    line = {
        "impl": "reference", "metric": "GCDF value+grad pairs/s (soft-min collision cost)", "value": value,
        "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / len(rs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name + "_softmin_T0.02", "n_waypoints": wl.q.shape[0],
                   "n_points": wl.p.shape[0], "net": "9-DOF 4x256 SiLU",
                   "sample": "whole waypoints, bounded time per step"},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": rs[-1]["cores"], "kind": "oracle",
                         "sample": rs[-1]["sample"], "host": rs[-1]["host"]},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch
    import paper_2601_18548_gb300 as g
    import __graft_entry__
    __graft_entry__.build()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    wl = make_workload()
    s = wl.shape
    P = wl.n_pairs
    net = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, args.precision)
    q = torch.from_numpy(wl.q).to(dev)
    p = torch.from_numpy(wl.p).to(dev)
    out = (torch.empty(q.shape[0], device=dev), torch.empty(q.shape[0], s.n_dof, device=dev),
           torch.empty(q.shape[0], device=dev, dtype=torch.int32))
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)  # 256 MiB > 129 MB L2
    stream = torch.cuda.current_stream()

    def step():
        g.collision_cost(net, q, p, wl.reduction, wl.param, out=out)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()

    k_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_stop = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    s_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    s_stop = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for ev in k_start + k_stop:
        ev.record(stream)  # creates the CUDA event (PyTorch creates it on first record)
    torch.cuda.synchronize()
    clocks = ClockSampler(_uuid(torch, dev), interval_ms=50)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.fill_(float(k))  # evict the previous step's lines from L2 (not timed)
        g.set_profile_events(net, k_start[k], k_stop[k])
        s_start[k].record(stream)
        step()
        s_stop[k].record(stream)
    torch.cuda.synchronize()
    g.set_profile_events(net)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(s_start, s_stop)]
    kern_ms = [a.elapsed_time(b) for a, b in zip(k_start, k_stop)]
    total_s, value = job_throughput(sum(step_ms) / 1e3, P * args.steps, dist, dev)
    if dist:
        dist.barrier()

    # end to end through the public API with host buffers (pinned), copies timed:
    # q and p packed in one pinned buffer (one host-to-device copy per step), the
    # cost, gradient and argmin carved from one device buffer (one copy back);
    # each piece starts on a 256-byte boundary
    def r64(x):
        return (x + 63) // 64 * 64
    N, n, M = q.shape[0], s.n_dof, p.shape[0]
    o_p = r64(N * n)
    in_h = torch.zeros(o_p + r64(M * 3)).pin_memory()
    in_h[:N * n].copy_(torch.from_numpy(wl.q).reshape(-1))
    in_h[o_p:o_p + M * 3].copy_(torch.from_numpy(wl.p).reshape(-1))
    in_d = torch.empty_like(in_h, device=dev)
    q_e, p_e = in_d[:N * n].view(N, n), in_d[o_p:o_p + M * 3].view(M, 3)
    o_g, o_a = r64(N), r64(N) + r64(N * n)
    out_d = torch.empty(o_a + r64(N), device=dev)
    out_e = (out_d[:N], out_d[o_g:o_g + N * n].view(N, n), out_d[o_a:o_a + N].view(torch.int32))
    out_h = torch.empty(out_d.numel()).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        in_d.copy_(in_h, non_blocking=True)
        g.collision_cost(net, q_e, p_e, wl.reduction, wl.param, out=out_e)
        out_h.copy_(out_d, non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_s, e2e_value = job_throughput(sum(e2e_ms) / 1e3, P * args.steps, dist, dev)
    # the host copies hold the same bits as the device-timed run's outputs
    e2e_same = bool(torch.equal(out_h[:N], out[0].cpu()) and torch.equal(out_h[o_g:o_g + N * n].view(N, n), out[1].cpu())
                    and torch.equal(out_h[o_a:o_a + N].view(torch.int32), out[2].cpu()))

    if rank != 0:
        dist.destroy_process_group()
        return 0

    peaks, peak_src = load_peaks()
    fpp = flops_per_pair(s)
    kern_avg_s = statistics.mean(kern_ms) / 1e3
    achieved_tflops = fpp * P / kern_avg_s / 1e12
    if args.precision in ("bf16", "fp16"):
        peak = float(peaks["bf16_tflops"])
        bound, punit = "tensor", "TFLOP/s"
        peak_note = f"bf16 dense burst, {peak_src} (fp16 dense rate is the same)"
    elif args.precision == "fp8":
        peak = 2.0 * float(peaks["bf16_tflops"])
        bound, punit = "tensor", "TFLOP/s"
        peak_note = f"fp8 dense = 2 x bf16 dense burst {peak_src} (nominal ratio 4.5 / 2.25 PFLOP/s)"
    else:
        fma = measure_fp32_fma_peak(g, torch)
        peak = fma["tflops"]
        bound, punit = "alu", "TFLOP/s"
        peak_note = "measured FP32 FMA loop (gcdf_diag_fp32_fma): " + fma["launch"]
    extras = {}
    if world == 1 and not args.no_extras:
        extras = gpu_extras(g, torch, dev, wl, net, args, peaks)
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_oracle_leg(wl, budget_s=args.ref_budget,
                            gpu_result=(out[0].cpu().numpy(), out[1].cpu().numpy()))
        cb["single_thread"] = cpu_oracle_single_thread(min(6.0, args.ref_budget))
    line = {
        "metric": "GCDF value+grad pairs/s (soft-min collision cost)",
        "value": value,
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp16": "f16", "fp8": "e4m3", "fp32": "f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": wl.name + "_softmin_T0.02", "n_waypoints": int(q.shape[0]),
                   "n_points": int(p.shape[0]), "pairs_per_step": P, "net": "9-DOF 4x256 SiLU",
                   "precision": args.precision, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": bound, "achieved": achieved_tflops, "peak": peak, "unit": punit,
                     "frac": achieved_tflops / peak,
                     "traffic": args.traffic if args.traffic is not None else measured_traffic(args.precision, wl.name),
                     "peak_source": peak_note,
                     "kernel_ms": 1e3 * kern_avg_s, "flops_per_pair": fpp},
        "cpu_baseline": cb,
        "e2e": {"value": e2e_value, "unit": "pairs/s",
                "h2d_bytes_per_step": int(in_h.numel() * 4),
                "d2h_bytes_per_step": int(out_h.numel() * 4), "outputs_match_device_run": e2e_same},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        **extras,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def measure_fp32_fma_peak(g, torch, reps=7):
    """Measured FP32 FMA rate (TFLOP/s) of the library's FMA loop: 4 blocks of
    256 threads per SM, 8 independent chains per thread, median of `reps`
    launches timed with CUDA events after one warm-up launch."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, threads, iters = 4 * sms, 256, 20000
    sink = torch.empty(blocks * threads, device="cuda")
    flops = g.diag_fp32_fma(blocks, threads, iters, sink)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.diag_fp32_fma(blocks, threads, iters, sink)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    return {"tflops": flops / (ms / 1e3) / 1e12, "ms": ms, "flops_per_launch": flops,
            "launch": f"{blocks} x {threads} threads, 8 FMA chains x {4 * iters} steps each"}


def _kernel_ms(g, torch, net, fn, reps, flush=None):
    """Median duration (ms) of the fused kernel inside fn(), from the library's
    profile events on the current stream."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()  # PyTorch creates the CUDA event on its first record
        b.record()
        g.set_profile_events(net, a, b)
        fn()
        torch.cuda.synchronize()
        g.set_profile_events(net)
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def gpu_extras(g, torch, dev, wl, net, args, peaks):
    """Measurements reported beside the headline (after its timed region):
      fp32_path   the FP32 CUDA-core kernel on the same workload against the
                  measured FP32 FMA rate;
      sweep       the BF16 kernel at larger scenes (128-2048 waypoints x
                  16,384-65,536 points) against the BF16 dense peak;
      sustained   the step back to back for ~2 s (no flush) with its own clock
                  record: the steady-state rate against the sustained peak."""
    s = wl.shape
    fpp = flops_per_pair(s)
    out = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    fma = measure_fp32_fma_peak(g, torch)
    q = torch.from_numpy(wl.q).to(dev)
    p = torch.from_numpy(wl.p).to(dev)
    net32 = g.create_net(s.n_dof, s.hidden, s.n_layers, wl.weights, "fp32")
    ms32 = _kernel_ms(g, torch, net32, lambda: g.collision_cost(net32, q, p, wl.reduction, wl.param), 5, flush)
    del net32
    out["fp32_path"] = {"kernel_ms": ms32, "pairs_per_s": wl.n_pairs / (ms32 / 1e3),
                        "achieved_tflops": fpp * wl.n_pairs / (ms32 / 1e3) / 1e12,
                        "peak_tflops": fma["tflops"], "frac": fpp * wl.n_pairs / (ms32 / 1e3) / 1e12 / fma["tflops"],
                        "peak_source": "measured FP32 FMA loop (gcdf_diag_fp32_fma): " + fma["launch"],
                        "bound": "alu"}
    peak = float(peaks["bf16_tflops"])
    # value-only query (forward layers alone: the first pass of the HINGE / MIN active sets)
    if args.precision in ("bf16", "fp16"):
        fbuf = torch.empty(wl.n_pairs, device=dev)
        msv = _kernel_ms(g, torch, net, lambda: g.query(net, q, p, with_grad=False, out=(fbuf, None)), 5, flush)
        H, L = s.hidden, s.n_layers
        fwd_fpp = (L - 1) * 2 * H * H + 2 * H + H
        out["value_only_query"] = {"kernel_ms": msv, "pairs_per_s": wl.n_pairs / (msv / 1e3),
                                   "flops_per_pair": fwd_fpp,
                                   "achieved_tflops": fwd_fpp * wl.n_pairs / (msv / 1e3) / 1e12,
                                   "frac": fwd_fpp * wl.n_pairs / (msv / 1e3) / 1e12 / peak,
                                   "note": "f only (no reverse sweep), per-pair f written to HBM"}
        del fbuf
    sweep = []
    if args.precision in ("bf16", "fp16"):
        for (N, M) in ((128, 65536), (512, 16384), (512, 65536), (2048, 16384), (2048, 65536)):
            sc = synth.box_scene(n_waypoints=N, n_points=M)
            qs = torch.from_numpy(sc.q).to(dev)
            ps = torch.from_numpy(sc.p).to(dev)
            ms = _kernel_ms(g, torch, net, lambda: g.collision_cost(net, qs, ps, wl.reduction, wl.param), 3)
            P = N * M
            sweep.append({"n_waypoints": N, "n_points": M, "pairs": P, "kernel_ms": ms,
                          "pairs_per_s": P / (ms / 1e3), "achieved_tflops": fpp * P / (ms / 1e3) / 1e12,
                          "frac": fpp * P / (ms / 1e3) / 1e12 / peak})
            del qs, ps
        out["sweep"] = {"precision": args.precision, "peak_tflops": peak, "points": sweep}
    # steady state: back-to-back steps for about two seconds
    outb = (torch.empty(q.shape[0], device=dev), torch.empty(q.shape[0], s.n_dof, device=dev),
            torch.empty(q.shape[0], device=dev, dtype=torch.int32))
    one = _kernel_ms(g, torch, net, lambda: g.collision_cost(net, q, p, wl.reduction, wl.param, out=outb), 3)
    n_rep = max(10, int(2000.0 / max(one, 1e-3)))
    clocks = ClockSampler(_uuid(torch, dev), interval_ms=50)
    clocks.start()
    time.sleep(0.2)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(n_rep):
        g.collision_cost(net, q, p, wl.reduction, wl.param, out=outb)
    b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = a.elapsed_time(b) / 1e3
    sus_peak = float(peaks.get("bf16_tflops_sustained", peak))
    if args.precision in ("bf16", "fp16"):
        out["sustained"] = {"steps": n_rep, "seconds": sec, "pairs_per_s": wl.n_pairs * n_rep / sec,
                            "achieved_tflops": fpp * wl.n_pairs * n_rep / sec / 1e12, "peak_tflops": sus_peak,
                            "frac": fpp * wl.n_pairs * n_rep / sec / 1e12 / sus_peak,
                            "peak_source": "bf16 dense sustained (seconds-long loop under the power cap)",
                            "clocks": clk}
    return out


def _serve_requests(rng, pools, rate, duration, h_rng, m_rng):
    """Poisson arrivals over `duration` seconds: (arrival, n_dof, N, points, q_start, q_goal)."""
    out, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration:
            return out
        n = 9 if rng.random() < 0.5 else 10
        pts = pools[n][int(rng.integers(len(pools[n])))]
        N = int(rng.integers(h_rng[0], h_rng[1] + 1))
        M = int(rng.integers(m_rng[0], m_rng[1] + 1))
        sm = synth.SplitMix64(int(rng.integers(1 << 62)))
        qs = synth.random_config(sm, n, -5.0, 5.0).astype(np.float32)
        qg = synth.random_config(sm, n, -5.0, 5.0).astype(np.float32)
        out.append((t, n, N, pts[:M], qs, qg))


def _lat(lat, span, done, rejected):
    lat = np.asarray(lat)
    return {"completed": int(done), "rejected": int(rejected),
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "throughput_rps": float(done / span) if span > 0 else None}


def _run_server(g, nets, params, reqs, budget, max_active, max_queued):
    """Replay the arrivals against a planning server; latency = done - submit (server clock)."""
    srv = g.Server(budget, max_active, max_queued, params)
    pending, lat, rejected, first, last = {}, [], 0, None, 0.0
    t0 = time.perf_counter()
    i = 0
    try:
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i][0] <= now:
                _, n, N, pts, qs, qg = reqs[i]
                try:
                    pending[srv.submit(nets[n], N, qs, qg, pts)] = True
                except g.GcdfError as e:
                    if e.code != 5:  # GCDF_EAGAIN: shed
                        raise
                    rejected += 1
                i += 1
            for tk in list(pending):
                r = srv.poll(tk)
                if r is not None:
                    del pending[tk]
                    lat.append(r["done_s"] - r["submit_s"])
                    first = r["submit_s"] if first is None else min(first, r["submit_s"])
                    last = max(last, r["done_s"])
            time.sleep(0.0005)
        st = srv.stats()
    finally:
        srv.close()
    out = _lat(lat, last - (first or 0.0), len(lat), rejected)
    if st["steps"]:
        k = st["steps"]
        out["worker_loop"] = {
            "steps": k, "mean_batch": st["active_sum"] / k,
            "step_device_ms": 1e3 * st["step_device_s"] / k,
            "step_host_ms": 1e3 * st["step_host_s"] / k,
            "pass_ms": 1e3 * st["pass_s"] / k,
            "host_overhead_ms_per_step": 1e3 * (st["pass_s"] - st["step_device_s"]) / k,
            "host_overhead_frac": (st["pass_s"] - st["step_device_s"]) / st["pass_s"] if st["pass_s"] > 0 else None}
    return out


def _run_sequential(g, torch, nets, params, reqs):
    """The plain per-request path: one gcdf_plan_solve at a time in arrival
    order (FIFO); each request's service time is measured, its latency is
    its completion minus its arrival."""
    clock, lat = 0.0, []
    for (t, n, N, pts, qs, qg) in reqs:
        prob = {"n_waypoints": N, "q_start": torch.from_numpy(qs).cuda(), "q_goal": torch.from_numpy(qg).cuda(),
                "points": torch.from_numpy(np.ascontiguousarray(pts)).cuda()}
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        g.plan_solve(nets[n], [prob], params, history=False)
        torch.cuda.synchronize()
        svc = time.perf_counter() - s0
        clock = max(clock, t) + svc
        lat.append(clock - t)
    return _lat(lat, clock - reqs[0][0], len(reqs), 0)


def run_serve(args):
    """Served planning: Poisson arrivals of trajectory-optimisation requests of
    uneven horizon and point-cloud size, 9- and 10-DOF robots, 50 optimiser
    steps each.  (A) a mix both paths can finish, the continuously batched
    BF16 server against the plain FP32 (and BF16) per-request paths; (C) many
    small requests, where one request at a time is bound by its launches; (B) the
    offered load of 2,000 requests/s at the full request sizes, which no path
    sustains on one GPU: served with a bounded queue, shed requests counted."""
    import torch
    import paper_2601_18548_gb300 as g
    params = g.PlanParams(iterations=50)
    nets = {p: {} for p in ("bf16", "fp32")}
    for n in (9, 10):
        shape = synth.NetShape(n, 256, 4)
        w = synth.he_uniform_weights(shape, seed=0)
        for p in nets:
            nets[p][n] = g.create_net(n, 256, 4, w, p)
    pools = {n: [synth.box_scene(n_waypoints=2, n_points=65536, seed_scene=300 + k, n_dof=n).p.astype(np.float32)
                 for k in range(4)] for n in (9, 10)}
    rng = np.random.default_rng(7)
    reqs_a = _serve_requests(rng, pools, rate=args.serve_rate, duration=args.serve_seconds,
                             h_rng=(32, 128), m_rng=(1000, 8000))
    # warm-up: one request through each path
    _run_sequential(g, torch, nets["bf16"], params, reqs_a[:1])
    _run_sequential(g, torch, nets["fp32"], params, reqs_a[:1])
    budget = 120 << 30
    served = _run_server(g, nets["bf16"], params, reqs_a, budget, 64, 256)
    fp32_seq = _run_sequential(g, torch, nets["fp32"], params, reqs_a)
    bf16_seq = _run_sequential(g, torch, nets["bf16"], params, reqs_a)
    # (C) many small requests: the per-request path is bound by its launches
    reqs_c = _serve_requests(np.random.default_rng(9), pools, rate=150.0, duration=1.0,
                             h_rng=(32, 64), m_rng=(500, 2000))
    served_c = _run_server(g, nets["bf16"], params, reqs_c, budget, 64, 1024)
    bf16_seq_c = _run_sequential(g, torch, nets["bf16"], params, reqs_c)
    fp32_seq_c = _run_sequential(g, torch, nets["fp32"], params, reqs_c)
    reqs_b = _serve_requests(np.random.default_rng(8), pools, rate=2000.0, duration=args.overload_seconds,
                             h_rng=(32, 256), m_rng=(1000, 65536))
    overload = _run_server(g, nets["bf16"], params, reqs_b, budget, 64, 64)
    overload["offered"] = len(reqs_b)
    # the same offered load with the partitions of Sec. IV-A: every waypoint
    # only considers the points within 1.5 m (planar) of its reference base
    params_p = g.PlanParams(iterations=50, partition_radius=1.5)
    overload_p = _run_server(g, nets["bf16"], params_p, reqs_b, budget, 64, 64)
    overload_p["offered"] = len(reqs_b)
    line = {
        "metric": "served plan p50/p99 latency and throughput", "unit": "s / requests per s",
        "n_gpus": 1, "data": "synthetic",
        "summary": {"mix": "A", "served_p50_s": served["p50_s"], "served_p99_s": served["p99_s"],
                    "served_rps": served["throughput_rps"], "fp32_per_request_p50_s": fp32_seq["p50_s"],
                    "fp32_per_request_p99_s": fp32_seq["p99_s"],
                    "fp32_per_request_rps": fp32_seq["throughput_rps"],
                    "served_beats_fp32_per_request": bool(served["throughput_rps"] >= fp32_seq["throughput_rps"]
                                                          and served["p99_s"] <= fp32_seq["p99_s"])},
        "config": {"arrivals": "Poisson", "steps_per_request": 50, "robots": "9- and 10-DOF, 4 x 256 SiLU",
                   "budget_bytes": budget,
                   "mix_A": {"rate_rps": args.serve_rate, "seconds": args.serve_seconds, "requests": len(reqs_a),
                             "horizon": [32, 128], "points": [1000, 8000]},
                   "small_C": {"rate_rps": 150.0, "seconds": 1.0, "requests": len(reqs_c), "horizon": [32, 64],
                               "points": [500, 2000]},
                   "overload_B": {"rate_rps": 2000.0, "seconds": args.overload_seconds, "horizon": [32, 256],
                                  "points": [1000, 65536], "max_active": 64, "max_queued": 64}},
        "A_served_bf16_continuous_batching": served,
        "A_per_request_fp32": fp32_seq,
        "A_per_request_bf16": bf16_seq,
        "C_served_bf16_continuous_batching": served_c,
        "C_per_request_bf16": bf16_seq_c,
        "C_per_request_fp32": fp32_seq_c,
        "B_served_bf16_overload": overload,
        "B_served_bf16_overload_partition_1.5m": overload_p,
    }
    print(json.dumps(line))
    return 0


def run_plan(args):
    """Batched trajectory optimisation: `--plan-problems` problems with horizons
    uniform in [32, 256] and point clouds uniform in [1k, 64k] from seeded box
    scenes, half 9-DOF and half 10-DOF robots (one gcdf_plan_solve per net),
    50 steps each (51 HINGE collision passes).  Timed with CUDA events around
    the two calls; inputs resident on the device."""
    import torch
    import paper_2601_18548_gb300 as g
    params = g.PlanParams(iterations=50)
    rng = np.random.default_rng(11)
    batches, pairs = [], 0
    for n in (9, 10):
        shape = synth.NetShape(n, 256, 4)
        net = g.create_net(n, 256, 4, synth.he_uniform_weights(shape, seed=0), args.precision)
        pool = [synth.box_scene(n_waypoints=2, n_points=65536, seed_scene=400 + k, n_dof=n).p.astype(np.float32)
                for k in range(4)]
        probs = []
        for _ in range(args.plan_problems // 2):
            N = int(rng.integers(32, 257))
            M = int(rng.integers(1000, 65537))
            sm = synth.SplitMix64(int(rng.integers(1 << 62)))
            qs = torch.from_numpy(synth.random_config(sm, n, -5.0, 5.0).astype(np.float32)).cuda()
            qg = torch.from_numpy(synth.random_config(sm, n, -5.0, 5.0).astype(np.float32)).cuda()
            pts = torch.from_numpy(np.ascontiguousarray(pool[int(rng.integers(4))][:M])).cuda()
            probs.append({"n_waypoints": N, "q_start": qs, "q_goal": qg, "points": pts})
            pairs += N * M
        batches.append((net, probs))
    warm = g.PlanParams(iterations=1)
    for net, probs in batches:
        g.plan_solve(net, probs[:2], warm, history=False)
    torch.cuda.synchronize()

    def timed(active):
        for net, _ in batches:
            g.set_active_set(net, active)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for net, probs in batches:
            g.plan_solve(net, probs, params)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3
    sec_one_pass = timed(False)
    sec = timed(True)
    evals = params.iterations + 1
    n_prob = sum(len(p) for _, p in batches)
    fpp = flops_per_pair(synth.NetShape(9, 256, 4))
    line = {"metric": "batched trajectory optimisation", "unit": "problems/s",
            "value": n_prob / sec, "n_gpus": 1, "dtype": args.precision, "data": "synthetic",
            "config": {"problems": n_prob, "horizon": [32, 256], "points": [1000, 65536], "robots": "9/10-DOF",
                       "steps": params.iterations, "evaluations": evals},
            "seconds": sec, "pairs_per_evaluation": pairs, "pairs_per_s": pairs * evals / sec,
            "tflops_collision_equivalent": pairs * evals * fpp / sec / 1e12,
            "one_pass": {"seconds": sec_one_pass, "problems_per_s": n_prob / sec_one_pass,
                         "pairs_per_s": pairs * evals / sec_one_pass,
                         "tflops_collision": pairs * evals * fpp / sec_one_pass / 1e12},
            "active_set_speedup": sec_one_pass / sec,
            "note": "HINGE collision passes with active sets (value-only pass, then gradients of the pairs "
                    "with f < delta); one_pass: value and gradient of every pair"}
    print(json.dumps(line))
    return 0


def _time_events(fn, reps=20, flush=None):
    """Median device time (ms) of fn() over reps calls, CUDA events on the
    current stream, optional L2 flush between calls."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def run_aux(args):
    """Constraint-structure kernels at the largest sizes of the request mix:
    the spatial partition (256 waypoints x 65,536 points), the dense->sparse
    Jacobian (2,097,152 rows x 9) and the single-step projection of the box
    scene (128 x 16,384 pairs, BF16 field).  L2 flushed between calls; the
    bound of each is HBM or L2 traffic, reported against the measured copy
    bandwidth."""
    import torch
    import paper_2601_18548_gb300 as g
    from paper_2601_18548_gb300 import _lib
    peaks, src = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    flush = torch.empty(64 << 20, device="cuda", dtype=torch.float32)
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    out = {}
    # partition: every waypoint reads the (x, y) of every point (the cloud stays in L2)
    N, M, R = 256, 65536, 1.5
    r = synth.SplitMix64(71)
    base = torch.from_numpy(np.ascontiguousarray(synth.uniform_points(r, N, [-5, -5, 0], [5, 5, 0])[:, :2]
                                                 .astype(np.float32))).cuda()
    pts = torch.from_numpy(synth.box_scene(n_waypoints=2, n_points=M, seed_scene=72).p.astype(np.float32)).cuda()
    off = torch.empty(N + 1, device="cuda", dtype=torch.int32)
    lib.gcdf_partition_offsets(base.data_ptr(), N, pts.data_ptr(), M, R, off.data_ptr(), stream)
    torch.cuda.synchronize()
    total = int(off[-1].item())
    idx = torch.empty(max(total, 4), device="cuda", dtype=torch.int32)

    def part():
        lib.gcdf_partition_offsets(base.data_ptr(), N, pts.data_ptr(), M, R, off.data_ptr(), stream)
        lib.gcdf_partition_indices(base.data_ptr(), N, pts.data_ptr(), M, R, off.data_ptr(), idx.data_ptr(), stream)
    ms = _time_events(part, flush=flush)
    out["partition"] = {"waypoints": N, "points": M, "radius_m": R, "listed_pairs": total, "ms": ms,
                        "tests_per_s": 2 * N * M / (ms / 1e3),
                        "note": "two passes (count, fill) over N x M planar distance tests; the 786 KB cloud is "
                                "read from L2 by every waypoint, DRAM sees it once"}
    # Jacobian scatter: read grad (P n 4 B), write values (P n 4 B), col_idx (P n 4 B), row_ptr (8 B per row)
    P, n = 128 * 16384, 9
    grad = torch.randn(P, n, device="cuda")
    rp = torch.empty(P + 1, device="cuda", dtype=torch.int64)
    col = torch.empty(P * n, device="cuda", dtype=torch.int32)
    val = torch.empty(P * n, device="cuda", dtype=torch.float32)
    ms = _time_events(lambda: lib.gcdf_jacobian_scatter(grad.data_ptr(), 128, n, None, 16384, P, rp.data_ptr(),
                                                        col.data_ptr(), val.data_ptr(), stream), flush=flush)
    byts = P * n * 12 + (P + 1) * 8
    out["jacobian_scatter"] = {"rows": P, "n": n, "ms": ms, "bytes": byts, "achieved_gbs": byts / ms / 1e6,
                               "peak_gbs": hbm, "frac": byts / ms / 1e6 / hbm, "bound": "hbm"}
    # projection of the scene: the fused query plus the in-place q - f M^-1 g pass
    wl = synth.box_scene()
    s_ = wl.shape
    net = g.create_net(s_.n_dof, s_.hidden, s_.n_layers, wl.weights, "bf16")
    q = torch.from_numpy(wl.q).cuda()
    p = torch.from_numpy(wl.p).cuda()
    qz = torch.empty(wl.n_pairs, s_.n_dof, device="cuda")
    fbuf = torch.empty(wl.n_pairs, device="cuda")
    ms_q = _time_events(lambda: g.query(net, q, p, out=(fbuf, qz)), flush=flush)
    ms_p = _time_events(lambda: g.project(net, q, p, out=qz), flush=flush)
    # the projection pass alone: read f (4 B) and g (4 n B), write q_z (4 n B) per pair
    byts = wl.n_pairs * (4 + 8 * s_.n_dof)
    extra = max(ms_p - ms_q, 1e-6)
    out["projection"] = {"pairs": wl.n_pairs, "ms_query": ms_q, "ms_project": ms_p,
                         "pairs_per_s": wl.n_pairs / (ms_p / 1e3), "projection_pass_ms": ms_p - ms_q,
                         "projection_pass_gbs": byts / extra / 1e6, "peak_gbs": hbm,
                         "frac": byts / extra / 1e6 / hbm, "bound": "hbm"}
    print(json.dumps({"metric": "constraint-structure kernels", "peaks": src, "n_gpus": 1,
                      "data": "synthetic", "l2": "flushed between calls (256 MiB write)", **out}))
    return 0


def run_fit(args):
    """One training step of the differentiable fit (distance loss of Table I):
    forward of every sample, the loss gradient, and the vector-Jacobian
    product with respect to the flat FP32 weights — 10-DOF net, 5 hidden
    layers of 512, SiLU, batch 65,536 (the differentiable-fit configuration),
    synthetic samples and targets.  Timed with CUDA events; inputs resident.
    --precision bf16 (the default) runs every matrix product on the tensor
    cores with BF16 operands and FP32 accumulation and master weights;
    --precision fp32 the SIMT FP32 GEMMs."""
    import torch
    import paper_2601_18548_gb300 as g
    if args.precision not in ("bf16", "fp32"):
        raise SystemExit("--fit runs in bf16 or fp32")
    prec = args.precision
    n, H, L, B = 10, 512, 5, args.fit_batch
    shape = synth.NetShape(n, H, L)
    w = torch.from_numpy(synth.he_uniform_weights(shape, seed=0)).cuda()
    r = synth.SplitMix64(91)
    q = torch.from_numpy(np.stack([synth.random_config(r, n, -3.0, 3.0) for _ in range(B)]).astype(np.float32)).cuda()
    p = torch.from_numpy(synth.uniform_points(r, B, [-3, -3, 0], [3, 3, 2]).astype(np.float32)).cuda()
    target = torch.zeros(B, device="cuda")

    def step():
        if prec == "bf16":
            # the forward keeps its tape; the VJP runs the reverse sweep from it
            f, tape = g.fit_forward_tape((n, H, L), w, q, p, precision=prec)
            gf = (2.0 / B) * (f - target)
            return g.fit_vjp_tape((n, H, L), w, q, p, gf, tape, want_dq=False, precision=prec)
        f = g.fit_forward((n, H, L), w, q, p, precision=prec)
        gf = (2.0 / B) * (f - target)
        return g.fit_vjp((n, H, L), w, q, p, gf, want_dq=False, precision=prec)
    ms = _time_events(step, reps=args.steps if args.steps < 20 else 10)
    d_in = 3 + 2 + 2 * (n - 2)
    # GEMM FLOPs: forward (d_in H + (L-1) H^2 + H) x 2 per sample (twice with
    # FP32, whose VJP recomputes the forward), weight gradients the same
    # again, back-products (L-1) H^2 x 2
    fwd = 2 * (d_in * H + (L - 1) * H * H + H)
    flops = B * ((1 if prec == "bf16" else 2) * fwd + fwd + 2 * (L - 1) * H * H)
    if prec == "fp32":
        fma = measure_fp32_fma_peak(g, torch)
        peak, bound = fma["tflops"], "alu"
        src = "measured FP32 FMA loop (gcdf_diag_fp32_fma): " + fma["launch"]
    else:
        peaks, psrc = load_peaks()
        peak, bound = float(peaks["bf16_tflops"]), "tensor"
        src = f"bf16 dense burst, {psrc}"
    assert g.fit_device_status() == 0, "a tensor-core wait of the fit gave up"
    line = {"metric": "differentiable fit training step", "unit": "samples/s", "value": B / (ms / 1e3),
            "n_gpus": 1, "dtype": "bf16" if prec == "bf16" else "f32", "data": "synthetic",
            "config": {"net": "10-DOF 5 x 512 SiLU", "batch": B, "loss": "distance (Table I)",
                       "operands": "BF16, FP32 accumulation and master weights" if prec == "bf16" else "FP32",
                       "backward": ("from the forward's tape (gcdf_fit_forward_tape / gcdf_fit_vjp_tape)"
                                    if prec == "bf16" else "recomputes the forward (gcdf_fit_vjp)")},
            "ms_per_step": ms,
            "roofline": {"bound": bound, "achieved": flops / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (ms / 1e3) / 1e12 / peak, "peak_source": src,
                         "note": "matrix-product FLOPs of the whole step over its time"}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp16", "fp8", "fp32"])
    ap.add_argument("--ref-budget", type=float, default=12.0, help="seconds of oracle work per sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP32-path, scene-sweep and sustained measurements after the timed region")
    ap.add_argument("--traffic", type=float, default=None, help="DRAM bytes per launch from ncu")
    ap.add_argument("--waypoints", type=int, default=128, help="smaller scenes for profiling only")
    ap.add_argument("--points", type=int, default=16384, help="smaller scenes for profiling only")
    ap.add_argument("--serve", action="store_true", help="served-planning latency benchmark instead")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--overload-seconds", type=float, default=10.0)
    ap.add_argument("--plan", action="store_true", help="batched trajectory-optimisation benchmark instead")
    ap.add_argument("--plan-problems", type=int, default=64)
    ap.add_argument("--aux", action="store_true", help="partition / Jacobian / projection kernels instead")
    ap.add_argument("--fit", action="store_true", help="differentiable-fit training step instead")
    ap.add_argument("--fit-batch", type=int, default=65536)
    args = ap.parse_args()
    global WAYPOINTS, POINTS
    WAYPOINTS, POINTS = args.waypoints, args.points
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.serve:
        return run_serve(args)
    if args.plan:
        return run_plan(args)
    if args.aux:
        return run_aux(args)
    if args.fit:
        return run_fit(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
