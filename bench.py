#!/usr/bin/env python
"""Joint-MM beta-NMF benchmark on one GB300 (replicas on N GPUs).

Default workload: dense quadratic-loss NMF (beta = 2) shaped like a face-image
collection, F = 361 (19 x 19 pixels), N = 2429 images, K = 49; synthetic data
(paper_2106_15214_gb300.inputs.dense_quadratic_faces). One step is one outer
JMM iteration (Algorithm 2, L = 1): the product at the iterate, both factor
updates, the objective at the iterate and the normalisation. The metric is
JMM iterations/s; beside it: the dominant kernel's roofline, the host-buffer
end-to-end rate, the CPU oracle's rate, and the time to the paper's stopping
tolerance of JMM against alternating MU (BMM) on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "joint-MM iters/s"
L2_FLUSH_BYTES = 512 << 20

WORKLOADS = {
    "faces": dict(gen="dense_quadratic_faces", beta=2.0, desc="dense quadratic (beta=2) faces F=361 N=2429 K=49"),
    "spectrogram": dict(gen="dense_is_spectrogram", beta=0.0, desc="dense Itakura-Saito (beta=0) F=513 N=20000 K=20"),
    # V = 410 MB, well above the 129 MB L2: every sweep streams V from HBM
    "spectrogram_large": dict(gen="dense_is_spectrogram", kw={"N": 200000}, beta=0.0,
                              desc="dense Itakura-Saito (beta=0) F=513 N=200000 K=20"),
    "kl_small": dict(gen="dense_kl_small", beta=1.0, desc="dense KL (beta=1) F=200 N=500 K=10"),
}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of each kernel as it now stands, keyed by (workload, precision,
# order, kernel name as in `kernels`); ncu flushes caches before each captured
# launch. Sources and commands: the traffic summaries under profiles/. An
# entry is removed when its kernel changes.
NCU_TRAFFIC = {
    ("faces", "tf32", "W", "tc_row_sweep"): 4920320,
    ("faces", "tf32", "W", "rows_epilogue"): 5478912,
    ("faces", "tf32", "W", "tc_col_sweep"): 4515840,
    ("faces", "tf32", "W", "cols_epilogue"): 6276864,
    ("spectrogram", "tf32", "W", "tc_row_sweep"): 46302976,
    ("spectrogram", "tf32", "W", "rows_epilogue"): 2534400,
    ("spectrogram", "tf32", "W", "tc_col_sweep"): 43898112,
    ("spectrogram", "tf32", "W", "cols_epilogue"): 7789056,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="faces", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, help="tf32 (default) | fp32 | fp64")
    ap.add_argument("--order", default="W")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-ttt", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--max-ttt-iters", type=int, default=10000)
    ap.add_argument("--no-kernel-timing", action="store_true",
                    help="skip the per-kernel timing pass (no roofline, no launch count)")
    return ap.parse_args()


def problem(name):
    from paper_2106_15214_gb300 import inputs
    wl = WORKLOADS[name]
    return getattr(inputs, wl["gen"])(**wl.get("kw", {})), wl


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def time_oracle(p, beta, seconds, max_iters=None, warmup=1):
    """Oracle JMM iterations (as written, no tuning) on the host cores."""
    import oracle as O
    W, H = p.W0.copy(), p.H0.copy()
    for _ in range(warmup):
        W, H = O.jmm_iteration(p.V, W, H, beta)
        W, H = O.normalize(W, H)
    n, t0 = 0, time.perf_counter()
    while True:
        _ = O.D_beta(p.V, W @ H, beta)
        W, H = O.jmm_iteration(p.V, W, H, beta)
        W, H = O.normalize(W, H)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_iters and n >= max_iters):
            return n, el


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []          # (arrival time, csv line)
        self.window = None       # (t0, t1) of the timed region, time.monotonic()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: wait (bounded) for its first sample
            t_end = time.monotonic() + 5.0
            while not self.lines and time.monotonic() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def begin(self):
        self.window = (time.monotonic(), None)

    def end(self):
        self.window = (self.window[0], time.monotonic())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if self.window and self.window[1] is not None:
            # samples taken during the timed region (plus one sampling period, the line's delivery delay)
            inside = [ln for t, ln in lines if self.window[0] <= t <= self.window[1] + 0.05]
            lines = inside or [ln for _, ln in lines]
        else:
            lines = [ln for _, ln in lines]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world, device="cuda"):
    """Max of a host scalar over the ranks (the NCCL group's device, or "cpu"
    under a gloo group)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, steps, max_seconds):
    """Whole-job throughput: every rank runs `steps` steps of its own replica;
    the job takes the slowest rank's time."""
    return world * steps / max_seconds


def algorithmic_bytes(kernel, F, N, K, esize=4):
    """Minimal DRAM bytes one launch of `kernel` must move: V once, every
    factor-sized operand it reads once, what it writes once. Partial-sum
    slices from splitting the streamed dimension are not counted (they are
    the kernel's choice, not the algorithm's)."""
    V = F * N * esize
    FK, KN = F * K * esize, K * N * esize
    table = {
        # Vt tile operand (W~), the MMA1 operand (H~), the two contraction operands (H~ or chi(H)); P, Q out
        "row_sweep": V + FK + 3 * KN + 2 * FK,
        "tc_row_sweep": V + FK + 3 * KN + 2 * FK,
        # H~, W~, chi(W) twice; Hn, Hd out
        "col_sweep": V + 3 * FK + KN + 2 * KN,
        "tc_col_sweep": V + 3 * FK + KN + 2 * KN,
        # P, Q and W~ in; W, chi_1(W), chi_2(W) and their two tensor-core copies out
        "rows_epilogue": 8 * FK,
        # W first, the iteration's last kernel: Hn, Hd and H~ in; H, H~ and the
        # two tensor-core copies of H out; W in; W, W~ and W's two copies out
        "cols_epilogue": 7 * KN + 5 * FK,
        # W, H in; W~, H~ and two tensor-core copies of each out
        "begin_iteration": 4 * (FK + KN),
        "normalize": 2 * (FK + KN),
    }
    return table.get(kernel)


def run_reference(args):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    import oracle as O
    p, wl = problem(args.workload)
    beta = wl["beta"]
    W, H = p.W0.copy(), p.H0.copy()
    for _ in range(args.warmup):
        W, H = O.jmm_iteration(p.V, W, H, beta)
        W, H = O.normalize(W, H)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _ = O.D_beta(p.V, W @ H, beta)
        W, H = O.jmm_iteration(p.V, W, H, beta)
        W, H = O.normalize(W, H)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = args.steps / tot
    F, N, K = p.shape
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "F": F, "N": N, "K": K, "beta": beta,
                   "step": "one JMM outer iteration (L=1) with objective and normalisation"},
        "cpu_baseline": {"value": val, "unit": "iters/s", "cores": cpu_threads(), "kind": "oracle",
                         "sample": f"{args.steps} full JMM iterations of the workload (numpy FP64 oracle)"},
        "e2e": {"value": val, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def timing_records(m):
    import ctypes
    lib = m._lib
    recs, i = [], 0
    while True:
        name, n, ms = ctypes.c_char_p(), ctypes.c_int64(), ctypes.c_double()
        if lib.nmf_get_timing(m._ctx, i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms)) != 0:
            break
        recs.append((name.value.decode(), n.value, ms.value))
        i += 1
    name, n, ms = ctypes.c_char_p(), ctypes.c_int64(), ctypes.c_double()
    lib.nmf_get_timing(m._ctx, -1, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms))
    return recs, n.value


def time_to_tolerance(p, beta, precision, method, tol, max_iters, order="W"):
    import torch
    from paper_2106_15214_gb300.binding import NMF
    F, N, K = p.shape
    dt = torch.float64 if precision == "fp64" else torch.float32
    m = NMF(F, N, K, beta, precision=precision, order=order)
    V = torch.tensor(p.V, dtype=dt, device="cuda")
    W = torch.tensor(p.W0, dtype=dt, device="cuda")
    H = torch.tensor(p.H0, dtype=dt, device="cuda")
    m.set_dense(V)
    m.set_factors(W, H)
    step = m.step_joint if method == "jmm" else m.step_alternating
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prev = step(1)
    it = 1
    cur = prev
    while it < max_iters:
        cur = step(1)          # objective at the iterate entering this iteration
        it += 1
        if (prev - cur) / cur <= tol:
            break
        prev = cur
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    # objective of the returned factors, re-evaluated in FP64 on the GPU
    m64 = NMF(F, N, K, beta, precision="fp64")
    V64, W64, H64 = V.double(), W.double(), H.double()
    m64.set_dense(V64)
    m64.set_factors(W64, H64)
    return {"s": el, "iters": it, "D": m64.loss(), "stopped_by_tol": it < max_iters}


def run_ours(args):
    import torch
    from paper_2106_15214_gb300 import binding
    from paper_2106_15214_gb300.binding import NMF
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    binding.load()
    p, wl = problem(args.workload)
    beta = wl["beta"]
    F, N, K = p.shape
    precision = args.precision or "tf32"
    esize = 8 if precision == "fp64" else 4
    dt = torch.float64 if precision == "fp64" else torch.float32
    m = NMF(F, N, K, beta, precision=precision, order=args.order)
    V = torch.tensor(p.V, dtype=dt, device="cuda")
    W = torch.tensor(p.W0, dtype=dt, device="cuda")
    H = torch.tensor(p.H0, dtype=dt, device="cuda")
    m.set_dense(V)
    m.set_factors(W, H)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    loss_dev = torch.zeros(max(args.steps, args.warmup, 1), dtype=torch.float64, device="cuda")
    for i in range(args.warmup):
        m.step_joint_async(loss_dev[i:i + 1])
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # Timed region: K steps enqueued back to back. Each step computes the
    # objective into device memory (no host round trip inside the region);
    # the L2 flush runs between steps, outside the step's events. About 2 ms
    # of untimed flushes are queued first so the host runs ahead of the GPU
    # and a host-side pause cannot leave the GPU idle inside a step's events.
    # The clock sampler is started (and has delivered a sample) before it.
    import gc
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        gc.disable()
        clk.begin()
        for j in range(30):
            flush.fill_(float(-j))
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            m.step_joint_async(loss_dev[i:i + 1])
            ends[i].record(stream)
        torch.cuda.synchronize()
        clk.end()
        gc.enable()
        barrier(world)
    wall = time.perf_counter() - wall0
    st = m._lib.nmf_get_status(m._ctx)
    if st != 0:
        raise RuntimeError(f"device status {st} after the timed region")
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_s = sum(step_ms) / 1e3
    dev_s_max = reduce_max(dev_s, world)
    value = aggregate_rate(world, args.steps, dev_s_max)
    losses = loss_dev[:args.steps].cpu().tolist()
    # Kernel pass: the same steps with the library's per-kernel CUDA events on
    # the launching stream (they add a little time per launch, so the value
    # above comes from the untimed pass): per-kernel durations, launch counts.
    kt_steps = 0 if args.no_kernel_timing else min(args.steps, 50)
    recs, launches_per_step = [], None
    if kt_steps:
        m._lib.nmf_reset_timing(m._ctx)
        m._lib.nmf_set_timing(m._ctx, 1)
        for i in range(kt_steps):
            flush.fill_(float(i))
            m.step_joint_async(loss_dev[i:i + 1])
        torch.cuda.synchronize()
        recs, n_launch = timing_records(m)
        m._lib.nmf_set_timing(m._ctx, 0)
        launches_per_step = n_launch / kt_steps
    # dominant kernel of the step and its roofline
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    def roof_of(rec):
        name, n, ms = rec
        per_launch_s = ms / 1e3 / max(n, 1)
        ab = algorithmic_bytes(name, F, N, K, esize)
        if not ab:
            return None
        ach = ab / per_launch_s / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": NCU_TRAFFIC.get((args.workload, precision, args.order, name)),
                "algorithmic_bytes": ab,
                "avg_launch_us": per_launch_s * 1e6, "launches": n, "peak_source": peak_src,
                "share_of_step": ms / (sum(r[2] for r in recs) or 1.0)}

    dom = max(recs, key=lambda r: r[2]) if recs else None
    roof = roof_of(dom) if dom else None
    kernels = {}
    for r in recs:
        rf = roof_of(r)
        kernels[r[0]] = {"launches": r[1], "avg_us": round(1e3 * r[2] / max(r[1], 1), 2),
                         "GB/s": round(rf["achieved"], 1) if rf else None,
                         "frac": round(rf["frac"], 4) if rf else None}
    launches = round(launches_per_step * args.steps) if launches_per_step is not None else None
    # end to end through the host-buffer C-ABI call
    Vh = torch.tensor(p.V, dtype=dt).pin_memory()
    Wh = torch.tensor(p.W0, dtype=dt).pin_memory()
    Hh = torch.tensor(p.H0, dtype=dt).pin_memory()
    me = NMF(F, N, K, beta, precision=precision, order=args.order)
    for _ in range(3):
        me.step_joint_host(Vh, Wh, Hh, 1)
    torch.cuda.synchronize()
    e2e_steps = max(10, min(args.steps, 200))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        me.step_joint_host(Vh, Wh, Hh, 1)
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    e2e = {"value": world * e2e_steps / e2e_s, "unit": "iters/s",
           "h2d_bytes_per_step": (F * N + F * K + K * N) * esize,
           "d2h_bytes_per_step": (F * K + K * N) * esize + 8}
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "tf32": "tf32", "bf16": "bf16"}[precision],
        "data": "synthetic",
        "config": {"workload": wl["desc"], "F": F, "N": N, "K": K, "beta": beta, "precision": precision,
                   "order": args.order, "step": "one JMM outer iteration (L=1) with objective and normalisation",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write, outside the step events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof, "gpu_launches": launches, "kernels": kernels,
        "e2e": e2e, "wall_s": wall,
        "step_ms_median": statistics.median(step_ms),
        "objective": {"first": losses[0], "last": losses[-1]},
    }
    if rank == 0:
        if not args.no_cpu_baseline:
            n_it, el = time_oracle(p, beta, args.cpu_seconds)
            line["cpu_baseline"] = {"value": n_it / el, "unit": "iters/s", "cores": cpu_threads(), "kind": "oracle",
                                    "sample": f"{n_it} full JMM iterations of the workload ({el:.1f} s, numpy FP64)"}
        if not args.no_ttt:
            tol = 1e-5
            line["time_to_tolerance"] = {
                "tol": tol, "rule": "(D_prev - D)/D <= tol, max %d iterations" % args.max_ttt_iters,
                "jmm": time_to_tolerance(p, beta, precision, "jmm", tol, args.max_ttt_iters, args.order),
                "bmm_same_precision": time_to_tolerance(p, beta, precision, "bmm", tol,
                                                        args.max_ttt_iters, args.order),
                "bmm_fp64": time_to_tolerance(p, beta, "fp64", "bmm", tol, args.max_ttt_iters, args.order),
            }
    clocks = clk.summary()
    line["clocks"] = clocks
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
