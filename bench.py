#!/usr/bin/env python
"""Joint-MM beta-NMF benchmark on one GB300 (replicas on N GPUs).

Default workload: dense Itakura-Saito NMF (beta = 0) shaped like an audio
power spectrogram, F = 513 frequency bins, N = 20000 frames, K = 20;
synthetic data (paper_2106_15214_gb300.inputs.dense_is_spectrogram). One step
is one outer JMM iteration (Algorithm 2, L = 1, H first): the product at the
iterate, both factor updates, the objective at the iterate and the
normalisation, on the fused single-read path (TF32 product, bf16
contractions). The metric is JMM iterations/s; beside it: the dominant
kernel's and the whole step's HBM roofline, the host-buffer end-to-end rate,
the CPU oracle's rate, the time to fixed objective targets D* and to the
paper's stopping rule of JMM against alternating MU (BMM) on the same GPU,
and extra workloads (the same problem at N = 200000, the TF32 two-sweep
form, the adjoint, sparse KL count data, 512 batched problems).

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
    "spectrogram": dict(gen="dense_is_spectrogram", beta=0.0, precision="bf16", order="H",
                        desc="dense Itakura-Saito (beta=0) F=513 N=20000 K=20"),
    # V = 410 MB, well above the 129 MB L2: every read of V comes from HBM
    "spectrogram_large": dict(gen="dense_is_spectrogram", kw={"N": 200000}, beta=0.0, precision="bf16", order="H",
                              desc="dense Itakura-Saito (beta=0) F=513 N=200000 K=20"),
    "faces": dict(gen="dense_quadratic_faces", beta=2.0, precision="tf32", order="W",
                  desc="dense quadratic (beta=2) faces F=361 N=2429 K=49"),
    "kl_small": dict(gen="dense_kl_small", beta=1.0, precision="fp64", order="W",
                     desc="dense KL (beta=1) F=200 N=500 K=10"),
}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of each kernel as it now stands, keyed by (workload, precision,
# order, kernel name as in `kernels`); ncu flushes caches before each captured
# launch. Sources and commands: the traffic summaries under profiles/. An
# entry is removed when its kernel changes.
NCU_TRAFFIC = {
    ("spectrogram", "bf16", "H", "tc_fused"): 45_574_144,     # profiles/tc_fused_spectrogram_ncu.md
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="spectrogram", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, help="bf16 | tf32 | fp32 | fp64 (default: the workload's)")
    ap.add_argument("--order", default=None, help="W | H (default: the workload's)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-target and stopping-rule runs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the extra workloads")
    ap.add_argument("--max-ttt-iters", type=int, default=6000)
    ap.add_argument("--no-kernel-timing", action="store_true",
                    help="skip the per-kernel timing pass (no roofline, no launch count)")
    ap.add_argument("--extra", default=None, choices=["sparse_kl", "batched"],
                    help="run only this extra workload (--steps timed steps) and print its JSON object")
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


def time_oracle(p, beta, seconds, order="H", warmup=1):
    """Oracle JMM iterations (as written, no tuning) of the whole workload on
    the host cores, for about `seconds`; returns (iterations, seconds)."""
    import oracle as O
    W, H = p.W0.copy(), p.H0.copy()
    for _ in range(warmup):
        W, H = O.normalize(*O.jmm_iteration(p.V, W, H, beta, order=order))
    n, t0 = 0, time.perf_counter()
    while True:
        _ = O.D_beta(p.V, W @ H, beta)
        W, H = O.normalize(*O.jmm_iteration(p.V, W, H, beta, order=order))
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
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


def algorithmic_bytes(kernel, F, N, K, esize=4, order="W"):
    """Minimal DRAM bytes one launch of `kernel` must move: V once, every
    distinct factor-sized operand it reads once (H~ counts once although the
    tensor-core kernels read it in two layouts; the tensor-core copies of a
    factor are not separate operands), what it writes once. Partial-sum
    slices from splitting the streamed dimension are not counted (they are
    the kernel's choice)."""
    V = F * N * esize
    FK, KN = F * K * esize, K * N * esize
    wfirst = order != "H"
    first_row = V + FK + KN + 2 * FK               # W half first: V, W~, H~ in; P, Q out
    second_col = V + FK + KN + 2 * FK + 2 * KN     # then: V, W~, H~, chi_1(W), chi_2(W) in; Hn, Hd out
    first_col = V + FK + KN + 2 * KN               # H half first: V, W~, H~ in; Hn, Hd out
    second_row = V + FK + KN + 2 * KN + 2 * FK     # then: V, W~, H~, chi_1(H), chi_2(H) in; P, Q out
    table = {
        "row_sweep": first_row if wfirst else second_row,
        "tc_row_sweep": first_row if wfirst else second_row,
        "col_sweep": second_col if wfirst else first_col,
        "tc_col_sweep": second_col if wfirst else first_col,
        # one read of V: V, W~ rows, H~ in; H out; P, Q out once
        "tc_fused": V + FK + KN + KN + 2 * FK,
        # P, Q and W~ in, W out; W first also chi_1(W), chi_2(W) out
        "rows_epilogue": 6 * FK if wfirst else 4 * FK,
        # W first, the iteration's last kernel: Hn, Hd and H~ in; H out; W in;
        # W and W~ out (normalisation)
        "cols_epilogue": 4 * KN + 3 * FK,
        # W, H in; W~, H~ out
        "begin_iteration": 2 * (FK + KN),
        "normalize": 2 * (FK + KN),
        # W, H in; W, H (normalised) out; the next iteration's W~, H~ are the same values
        "normalize_next": 2 * (FK + KN),
        # the W half after the fused sweep, then the normalisation: P, Q and
        # W~ in, W out; W, H in, W, H (normalised) out
        "fused_post": 4 * FK + 2 * (FK + KN),
    }
    return table.get(kernel)


def step_bytes(F, N, K, esize=4):
    """Algorithmic bytes of one JMM iteration: V read once, both factors read
    and written once."""
    return esize * (F * N + 2 * (F + N) * K)


def run_reference(args):
    """The oracle on the host cores, each step one JMM iteration on a sample of
    the workload's columns sized so that the K + W steps take about a minute;
    the rate is scaled to whole-workload iterations (the work is linear in N)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    p, wl = problem(args.workload)
    beta = wl["beta"]
    order = args.order or wl["order"]
    F, N, K = p.shape
    t0 = time.perf_counter()
    O.normalize(*O.jmm_iteration(p.V, p.W0, p.H0, beta, order=order))
    t_full = time.perf_counter() - t0
    budget = 60.0 / max(1, args.steps + args.warmup)
    Ns = int(max(32, min(N, round(N * budget / max(t_full, 1e-9)))))
    V, W, H = p.V[:, :Ns], p.W0.copy(), p.H0[:, :Ns].copy()
    for _ in range(args.warmup):
        W, H = O.normalize(*O.jmm_iteration(V, W, H, beta, order=order))
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _ = O.D_beta(V, W @ H, beta)
        W, H = O.normalize(*O.jmm_iteration(V, W, H, beta, order=order))
        times.append(time.perf_counter() - t0)
    val = (Ns / N) * args.steps / sum(times)
    sample = (f"{args.steps} JMM iterations (objective, both updates, normalisation; numpy FP64 oracle) on the "
              f"first {Ns} of the {N} columns, rate scaled by {Ns}/{N} to whole-workload iterations")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / val,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "F": F, "N": N, "K": K, "beta": beta, "order": order,
                   "step": "one JMM outer iteration (L=1) with objective and normalisation"},
        "cpu_baseline": {"value": val, "unit": "iters/s", "cores": cpu_threads(), "kind": "oracle", "sample": sample},
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


def fp64_objective(p, beta, W, H):
    """D_beta(V | WH) of (W, H) evaluated by the FP64 path on the GPU."""
    import torch
    from paper_2106_15214_gb300.binding import NMF
    F, N, K = p.shape
    m = NMF(F, N, K, beta, precision="fp64")
    V64 = torch.tensor(p.V, dtype=torch.float64, device="cuda")
    W64, H64 = W.double().contiguous(), H.double().contiguous()
    m.set_dense(V64)
    m.set_factors(W64, H64)
    d = m.loss()
    m.close()
    return d


def dense_context(p, beta, precision, order):
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
    return m, V, W, H


def time_to_target(p, beta, precision, method, order, targets, max_iters, chunk=25):
    """Iterations and GPU time until the FP64 objective of the iterate falls
    to each target D* (targets: label -> value). A search pass (untimed)
    steps in chunks, evaluates the FP64 objective after each chunk and
    resolves a crossing by re-running the chunk one iteration at a time from
    its saved start; the kernels are deterministic, so a second, timed pass
    from the initial factors runs the same trajectory: the largest count
    needed, back to back on the stream, with a CUDA event after each target's
    count."""
    import torch
    m, V, W, H = dense_context(p, beta, precision, order)
    step = m.step_joint_async if method == "jmm" else m.step_alternating_async
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    need, it = {}, 0
    d_last = fp64_objective(p, beta, W, H)
    while it < max_iters and len(need) < len(targets):
        W0c, H0c = W.clone(), H.clone()
        n = min(chunk, max_iters - it)
        step(ld, iters=n)
        d = fp64_objective(p, beta, W, H)
        crossed = [lb for lb, t in targets.items() if lb not in need and d <= t]
        if crossed:
            W.copy_(W0c)
            H.copy_(H0c)
            for k in range(1, n + 1):
                step(ld, iters=1)
                dk = fp64_objective(p, beta, W, H)
                for lb in crossed:
                    if lb not in need and dk <= targets[lb]:
                        need[lb] = it + k
                if all(lb in need for lb in crossed):
                    W.copy_(W0c)
                    H.copy_(H0c)
                    step(ld, iters=n)
                    break
        it += n
        d_last = d
    m.close()
    out = {"precision": precision, "method": method, "order": order, "iters_searched": it,
           "D_fp64_search_end": d_last}
    times = {}
    if need:
        m, V, W, H = dense_context(p, beta, precision, order)
        step = m.step_joint_async if method == "jmm" else m.step_alternating_async
        counts = sorted(set(need.values()))
        ld = torch.zeros(counts[-1], dtype=torch.float64, device="cuda")
        step(ld[:1], iters=1)          # graph capture and first-launch work outside the timing
        W.copy_(torch.tensor(p.W0, dtype=W.dtype, device="cuda"))
        H.copy_(torch.tensor(p.H0, dtype=H.dtype, device="cuda"))
        stream = torch.cuda.current_stream()
        ev0 = torch.cuda.Event(enable_timing=True)
        evs = {c: torch.cuda.Event(enable_timing=True) for c in counts}
        torch.cuda.synchronize()
        ev0.record(stream)
        done = 0
        for c in counts:
            for k in range(done, c):
                step(ld[k:k + 1], iters=1)
            evs[c].record(stream)
            done = c
        torch.cuda.synchronize()
        out["D_fp64_timed_end"] = fp64_objective(p, beta, W, H)
        times = {c: ev0.elapsed_time(e) / 1e3 for c, e in evs.items()}
        m.close()
    for lb in targets:
        out[lb] = ({"reached": True, "iters": need[lb], "s": times[need[lb]]} if lb in need
                   else {"reached": False})
    return out


def time_to_tolerance(p, beta, precision, method, tol, max_iters, order="W"):
    """The paper's stopping rule (Sec. 4.1.2): iterate until the relative
    decrease of the objective over one iteration falls to `tol`; wall time
    including the per-iteration objective read-back the rule needs. The final
    objective is re-evaluated in FP64."""
    import torch
    m, V, W, H = dense_context(p, beta, precision, order)
    step = m.step_joint if method == "jmm" else m.step_alternating
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prev = step(1)
    it = 1
    while it < max_iters:
        cur = step(1)          # objective at the iterate entering this iteration
        it += 1
        if (prev - cur) / cur <= tol:
            break
        prev = cur
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    d = fp64_objective(p, beta, W, H)
    m.close()
    return {"precision": precision, "s": el, "iters": it, "D_fp64": d, "stopped_by_tol": it < max_iters}


def ttt_block(args, p, beta, precision, order):
    """Time to the fixed targets D* = D_best x (1 + 1e-4) and x (1 + 1e-3)
    (D_best: the best long-run FP64-oracle objective, tests/golden/dstar_*.txt)
    of JMM at the workload's precision, JMM in TF32, BMM in TF32 and BMM in
    FP64 on the same GPU, every objective evaluated in FP64."""
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    from make_dstar import read_dstar
    d = read_dstar(args.workload)
    if not d or not isinstance(d.get("D_best"), float) or d["D_best"] != d["D_best"]:
        return {"unavailable": f"no stored D_best for {args.workload}"}
    best = d["D_best"]
    targets = {"D*(1e-4)": best * (1 + 1e-4), "D*(1e-3)": best * (1 + 1e-3)}
    out = {"D_best_oracle": best, "oracle_iterations": d.get("iterations"), "targets": targets}
    runs = [("jmm_" + precision, precision, "jmm")]
    if precision != "tf32":
        runs.append(("jmm_tf32", "tf32", "jmm"))
    runs += [("bmm_tf32", "tf32", "bmm"), ("bmm_fp64", "fp64", "bmm")]
    for name, prec, method in runs:
        out[name] = time_to_target(p, beta, prec, method, order, targets, args.max_ttt_iters)
    return out


def load_peaks():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    if "hbm_gbs" in peaks:
        return float(peaks["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def timed_steps(step, steps, flush, stream):
    """Per-step CUDA-event times (ms) of `steps` calls of step(i), the L2
    flushed between steps outside the events; about 2 ms of untimed flushes
    are queued first so the host runs ahead of the GPU."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for j in range(30):
        flush.fill_(float(-j))
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        step(i)
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def kernel_pass(m, step, steps, flush):
    """The library's per-kernel CUDA events (on the launching stream) over
    `steps` steps: [(kernel, launches, total ms)], launches per step."""
    import torch
    m._lib.nmf_reset_timing(m._ctx)
    m._lib.nmf_set_timing(m._ctx, 1)
    for i in range(steps):
        flush.fill_(float(i))
        step(i)
    torch.cuda.synchronize()
    recs, n_launch = timing_records(m)
    m._lib.nmf_set_timing(m._ctx, 0)
    return recs, n_launch / max(steps, 1)


def roofline_of(rec, recs, F, N, K, esize, order, peak, peak_src, key):
    name, n, ms = rec
    per_launch_s = ms / 1e3 / max(n, 1)
    ab = algorithmic_bytes(name, F, N, K, esize, order)
    if not ab:
        return None
    ach = ab / per_launch_s / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "traffic": NCU_TRAFFIC.get(key + (name,)),
            "algorithmic_bytes": ab, "avg_launch_us": per_launch_s * 1e6, "launches": n,
            "peak_source": peak_src, "share_of_step": ms / (sum(r[2] for r in recs) or 1.0)}


def kernel_table(recs, F, N, K, esize, order, peak, peak_src, key):
    out = {}
    for r in recs:
        rf = roofline_of(r, recs, F, N, K, esize, order, peak, peak_src, key)
        out[r[0]] = {"launches": r[1], "avg_us": round(1e3 * r[2] / max(r[1], 1), 2),
                     "GB/s": round(rf["achieved"], 1) if rf else None,
                     "frac": round(rf["frac"], 4) if rf else None}
    return out


def step_roofline(F, N, K, esize, ms_per_step, peak, peak_src):
    sb = step_bytes(F, N, K, esize)
    ach = sb / (ms_per_step / 1e3) / 1e9
    return {"bytes": sb, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_source": peak_src, "definition": "V read once + both factors read and written once, per iteration"}


def dense_extra(p, beta, precision, order, steps, flush, stream, peak, peak_src, name):
    """iters/s, the step-level and the dominant kernel's HBM fractions of one
    extra dense workload."""
    import torch
    F, N, K = p.shape
    esize = 8 if precision == "fp64" else 4
    m, V, W, H = dense_context(p, beta, precision, order)
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    step = lambda i: m.step_joint_async(ld)  # noqa: E731
    for _ in range(3):
        step(0)
    ms = timed_steps(step, steps, flush, stream)
    per = sum(ms) / len(ms)
    recs, lps = kernel_pass(m, step, min(steps, 20), flush)
    dom = max(recs, key=lambda r: r[2]) if recs else None
    key = (name, precision, order)
    out = {"workload": WORKLOADS[name]["desc"] if name in WORKLOADS else name, "F": F, "N": N, "K": K, "beta": beta,
           "precision": precision, "order": order, "iters_per_s": 1e3 / per, "ms_per_step": per,
           "step_ms_median": statistics.median(ms), "steps": steps,
           "step_roofline": step_roofline(F, N, K, esize, per, peak, peak_src),
           "roofline": roofline_of(dom, recs, F, N, K, esize, order, peak, peak_src, key) if dom else None,
           "kernels": kernel_table(recs, F, N, K, esize, order, peak, peak_src, key),
           "launches_per_step": lps, "objective": float(ld.item())}
    m.close()
    return out


def grad_extra(p, beta, steps, flush, stream, peak, peak_src):
    """The adjoint (a10): nmf_grad on the workload (both gradients at the
    current factors and the objective) on a BF16 context (the fused sweep's
    adjoint mode: one read of V) and on an FP32 context (the SIMT sweeps: two
    reads of V): time per call and the HBM fraction against V once + W, H
    read + both gradients written; the FP64 oracle's gradient on a column
    sample beside it."""
    import torch
    import oracle as O
    F, N, K = p.shape
    ab = 4 * (F * N + 2 * (F * K + K * N))
    out = {"workload": f"nmf_grad, F={F} N={N} K={K} beta={beta}", "algorithmic_bytes": ab,
           "note": "each call synchronises (the objective is read back), as a training step would"}
    for prec, order in (("bf16", "H"), ("fp32", "W")):
        m, V, W, H = dense_context(p, beta, prec, order)
        gW, gH = torch.empty_like(W), torch.empty_like(H)
        for _ in range(3):
            m.grad(gW, gH, want_loss=True)
        torch.cuda.synchronize()
        ms = timed_steps(lambda i: m.grad(gW, gH, want_loss=True), steps, flush, stream)
        per = sum(ms) / len(ms)
        m.close()
        out[prec] = {"ms_per_call": per, "calls_per_s": 1e3 / per, "achieved_GBs": ab / (per / 1e3) / 1e9,
                     "frac": ab / (per / 1e3) / 1e9 / peak}
    Ns = min(N, 2000)
    t0 = time.perf_counter()
    O.gradients(p.V[:, :Ns], p.W0, p.H0[:, :Ns], beta)
    out["oracle_s_per_call"] = (time.perf_counter() - t0) * N / Ns
    out["oracle_sample"] = f"first {Ns} of {N} columns, scaled to the full N"
    out["peak_source"] = peak_src
    return out


def sparse_extra(steps, flush, stream, peak, peak_src, tol_iters=2000):
    """Sparse KL (Sec. 4.4 stand-in, 20000 x 100000, 0.1 %, K = 50, CSR FP32):
    nnz/s of JMM and BMM and the HBM fraction against an iteration's
    algorithmic bytes: the nonzeros' values and column indices once, both
    factors read and written once (the kernels read the values twice, in
    the CSR and in the CSC layout, one per half). Beside it the time of each
    method to the paper's stopping rule (Sec. 4.1.2, 1e-5, at most tol_iters
    iterations): a long-run FP64 oracle target is out of reach at this size
    (about 7 s per oracle iteration)."""
    import torch
    from paper_2106_15214_gb300 import inputs
    from paper_2106_15214_gb300.binding import NMF
    p = inputs.sparse_counts()
    K = p.W0.shape[1]
    nnz = int(p.val.size)
    ab = 8 * nnz + 4 * 2 * (p.F + p.N) * K
    out = {"workload": f"sparse KL (beta=1) F={p.F} N={p.N} nnz={nnz} K={K} CSR fp32", "nnz": nnz,
           "algorithmic_bytes_per_iter": ab}
    for method in ("jmm", "bmm"):
        m = NMF(p.F, p.N, K, 1.0, precision="fp32", order="W")
        rp = torch.tensor(p.rowptr, dtype=torch.int32, device="cuda")
        cl = torch.tensor(p.col, dtype=torch.int32, device="cuda")
        vl = torch.tensor(p.val, dtype=torch.float32, device="cuda")
        m.set_csr(rp, cl, vl)
        W = torch.tensor(p.W0, dtype=torch.float32, device="cuda")
        H = torch.tensor(p.H0, dtype=torch.float32, device="cuda")
        m.set_factors(W, H)
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        fn = m.step_joint_async if method == "jmm" else m.step_alternating_async
        step = lambda i: fn(ld)  # noqa: E731
        for _ in range(3):
            step(0)
        ms = timed_steps(step, steps, flush, stream)
        per = sum(ms) / len(ms)
        recs, lps = kernel_pass(m, step, min(steps, 10), flush)
        out[method] = {"ms_per_iter": per, "iters_per_s": 1e3 / per, "nnz_per_s": nnz / (per / 1e3),
                       "achieved_GBs": ab / (per / 1e3) / 1e9, "frac": ab / (per / 1e3) / 1e9 / peak,
                       "kernels": {r[0]: {"launches": r[1], "avg_us": round(1e3 * r[2] / max(r[1], 1), 2)}
                                   for r in recs},
                       "launches_per_iter": lps, "objective": float(ld.item())}
        if tol_iters:
            # the paper's stopping rule from the initial factors (objective read back every iteration)
            W.copy_(torch.tensor(p.W0, dtype=torch.float32, device="cuda"))
            H.copy_(torch.tensor(p.H0, dtype=torch.float32, device="cuda"))
            m.set_factors(W, H)
            sfn = m.step_joint if method == "jmm" else m.step_alternating
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            prev, it = sfn(1), 1
            cur = prev
            while it < tol_iters:
                cur = sfn(1)
                it += 1
                if (prev - cur) / cur <= 1e-5:
                    break
                prev = cur
            torch.cuda.synchronize()
            out[method]["stopping_rule"] = {"tol": 1e-5, "s": time.perf_counter() - t0, "iters": it, "D": cur,
                                            "stopped_by_tol": it < tol_iters}
        m.close()
        del rp, cl, vl, W, H
    out["peak"], out["peak_source"] = peak, peak_src
    return out


def batched_extra(steps, flush, stream, peak, peak_src):
    """512 batched beta = 1.5 problems (Sec. 4.5 stand-in): time per JMM and
    per BMM step of the whole batch (one launch per half-sweep over all
    instances), and the HBM fraction against one read of every V plus the
    factors read and written once (the floor of a single-read iteration; the
    batched sweeps read each V once per half)."""
    import numpy as np
    import torch
    from paper_2106_15214_gb300 import inputs
    from paper_2106_15214_gb300.binding import BatchedNMF
    probs = inputs.batched_hyperspectral()
    shapes = [q.shape for q in probs]
    Vp = torch.tensor(np.concatenate([q.V.ravel() for q in probs]), dtype=torch.float32, device="cuda")
    Wi = np.concatenate([q.W0.ravel() for q in probs])
    Hi = np.concatenate([q.H0.ravel() for q in probs])
    fn_ = sum(F * N for F, N, K in shapes)
    fk = sum((F + N) * K for F, N, K in shapes)
    one_read = 4 * fn_ + 8 * fk
    out = {"workload": f"{len(shapes)} batched beta=1.5 problems, F in [64,256], N in [256,8192], K in [4,32]",
           "sum_FN": fn_, "bytes_one_read_of_V_plus_factors": one_read}
    # JMM on the fused single-read path (one launch over all problems' work
    # items; bf16 contractions, H first), then JMM and BMM on the FP32 SIMT sweeps
    for method, prec, order in (("jmm_bf16", "bf16", "H"), ("jmm", "fp32", "W"), ("bmm", "fp32", "W")):
        b = BatchedNMF(shapes, 1.5, precision=prec, order=order)
        Wd = torch.tensor(Wi, dtype=torch.float32, device="cuda")
        Hd = torch.tensor(Hi, dtype=torch.float32, device="cuda")
        b.set_packed(Vp, Wd, Hd)
        cap = b.autotune(3)
        fn = b.step_alternating if method == "bmm" else b.step_joint
        for _ in range(3):
            fn(1, want_loss=False)
        ms = timed_steps(lambda i: fn(1, want_loss=False), steps, flush, stream)
        per = sum(ms) / len(ms)
        out[method] = {"precision": prec, "order": order, "ms_per_step": per, "steps_per_s": 1e3 / per,
                       "autotuned_chunk_cap": cap,
                       "achieved_GBs_one_read": one_read / (per / 1e3) / 1e9,
                       "frac_one_read": one_read / (per / 1e3) / 1e9 / peak}
        b.close()
    out["peak"], out["peak_source"] = peak, peak_src
    return out


def run_ours(args):
    import gc

    import torch
    from paper_2106_15214_gb300 import binding
    from paper_2106_15214_gb300.binding import NMF
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    binding.load()
    p, wl = problem(args.workload)
    beta = wl["beta"]
    F, N, K = p.shape
    precision = args.precision or wl["precision"]
    order = args.order or wl["order"]
    esize = 8 if precision == "fp64" else 4
    dt = torch.float64 if precision == "fp64" else torch.float32
    m, V, W, H = dense_context(p, beta, precision, order)
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
    dev_s_max = reduce_max(sum(step_ms) / 1e3, world)
    value = aggregate_rate(world, args.steps, dev_s_max)
    losses = loss_dev[:args.steps].cpu().tolist()
    ms_per_step = 1e3 * dev_s_max / args.steps
    peak, peak_src = load_peaks()
    key = (args.workload, precision, order)
    # Kernel pass: the same steps with the library's per-kernel CUDA events on
    # the launching stream (they add a little time per launch, so the value
    # above comes from the untimed pass): per-kernel durations, launch counts.
    recs, launches_per_step = [], None
    if not args.no_kernel_timing:
        recs, launches_per_step = kernel_pass(m, lambda i: m.step_joint_async(loss_dev[i:i + 1]),
                                              min(args.steps, 50), flush)
    dom = max(recs, key=lambda r: r[2]) if recs else None
    roof = roofline_of(dom, recs, F, N, K, esize, order, peak, peak_src, key) if dom else None
    kernels = kernel_table(recs, F, N, K, esize, order, peak, peak_src, key)
    launches = round(launches_per_step * args.steps) if launches_per_step is not None else None
    m.close()
    del V, W, H
    # end to end through the host-buffer C-ABI call
    Vh = torch.tensor(p.V, dtype=dt).pin_memory()
    Wh = torch.tensor(p.W0, dtype=dt).pin_memory()
    Hh = torch.tensor(p.H0, dtype=dt).pin_memory()
    me = NMF(F, N, K, beta, precision=precision, order=order)
    for _ in range(3):
        me.step_joint_host(Vh, Wh, Hh, 1)
    torch.cuda.synchronize()
    e2e_steps = max(10, min(args.steps, 200))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        me.step_joint_host(Vh, Wh, Hh, 1)
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    me.close()
    e2e = {"value": world * e2e_steps / e2e_s, "unit": "iters/s",
           "h2d_bytes_per_step": (F * N + F * K + K * N) * esize,
           "d2h_bytes_per_step": (F * K + K * N) * esize + 8}
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "tf32": "tf32", "bf16": "bf16"}[precision],
        "data": "synthetic",
        "config": {"workload": wl["desc"], "F": F, "N": N, "K": K, "beta": beta, "precision": precision,
                   "order": order, "step": "one JMM outer iteration (L=1) with objective and normalisation",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write, outside the step events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof, "step_roofline": step_roofline(F, N, K, esize, ms_per_step, peak, peak_src),
        "gpu_launches": launches, "kernels": kernels, "e2e": e2e, "wall_s": wall,
        "step_ms_median": statistics.median(step_ms),
        "objective": {"first": losses[0], "last": losses[-1]},
    }
    if rank == 0:
        if not args.no_cpu_baseline:
            n_it, el = time_oracle(p, beta, args.cpu_seconds, order=order)
            line["cpu_baseline"] = {"value": n_it / el, "unit": "iters/s", "cores": cpu_threads(), "kind": "oracle",
                                    "sample": f"{n_it} full JMM iterations of the workload ({el:.1f} s, numpy FP64)"}
        if not args.no_ttt:
            line["time_to_target"] = ttt_block(args, p, beta, precision, order)
            tol = 1e-5
            line["time_to_tolerance"] = {
                "tol": tol, "rule": "(D_prev - D)/D <= tol (Sec. 4.1.2), max %d iterations" % args.max_ttt_iters,
                "jmm": time_to_tolerance(p, beta, precision, "jmm", tol, args.max_ttt_iters, order),
                "bmm_tf32": time_to_tolerance(p, beta, "tf32", "bmm", tol, args.max_ttt_iters, order),
                "bmm_fp64": time_to_tolerance(p, beta, "fp64", "bmm", tol, args.max_ttt_iters, order),
            }
        if not args.no_extras:
            extras = {}
            if args.workload == "spectrogram":
                extras["tf32_two_sweeps"] = dense_extra(p, beta, "tf32", "W", 200, flush, stream, peak, peak_src,
                                                        "spectrogram")
                extras["adjoint"] = grad_extra(p, beta, 50, flush, stream, peak, peak_src)
                big, _ = problem("spectrogram_large")
                extras["spectrogram_large"] = dense_extra(big, beta, precision, order, 100, flush, stream, peak,
                                                          peak_src, "spectrogram_large")
                del big
            extras["sparse_kl"] = sparse_extra(20, flush, stream, peak, peak_src)
            extras["batched"] = batched_extra(20, flush, stream, peak, peak_src)
            line["extras"] = extras
    line["clocks"] = clk.summary()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_extra(args):
    import torch
    from paper_2106_15214_gb300 import binding
    binding.load()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    peak, peak_src = load_peaks()
    fn = sparse_extra if args.extra == "sparse_kl" else batched_extra
    print(json.dumps(fn(args.steps, flush, torch.cuda.current_stream(), peak, peak_src)), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.extra:
        return run_extra(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
