"""bench.py on the CPU: the reference arm's JSON line (the oracle timed on the
host cores) and the host-side helpers the GPU arm relies on."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "iters/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["vs_baseline"] is None and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert "Itakura-Saito" in d["config"]["workload"] and d["config"]["N"] == 20000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_algorithmic_bytes():
    """V once, each distinct factor-sized operand once (no tensor-core copies),
    outputs once; the fused sweep reads V once per iteration."""
    F, N, K, s = 513, 20000, 20, 4
    V, FK, KN = F * N * s, F * K * s, K * N * s
    assert bench.algorithmic_bytes("tc_row_sweep", F, N, K, order="W") == V + FK + KN + 2 * FK
    assert bench.algorithmic_bytes("tc_col_sweep", F, N, K, order="W") == V + 3 * FK + KN + 2 * KN
    assert bench.algorithmic_bytes("tc_col_sweep", F, N, K, order="H") == V + FK + KN + 2 * KN
    assert bench.algorithmic_bytes("tc_row_sweep", F, N, K, order="H") == V + 3 * KN + FK + 2 * FK
    assert bench.algorithmic_bytes("tc_fused", F, N, K, order="H") == V + 3 * FK + 2 * KN
    assert bench.algorithmic_bytes("cols_epilogue", F, N, K) == 4 * KN + 3 * FK
    assert bench.algorithmic_bytes("nope", F, N, K) is None
    assert bench.step_bytes(F, N, K) == V + 2 * (FK + KN)


def test_clock_sampler_keeps_samples_inside_the_timed_region():
    c = bench.ClockSampler(0)
    t = time.monotonic()
    fields = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {cap}"
    c.lines = [(t - 1.0, fields.format(sm=600, hw="Not Active", cap="Not Active")),        # before: ignored
               (t + 0.01, fields.format(sm=2070, hw="Not Active", cap="Active")),
               (t + 0.02, fields.format(sm=2055, hw="Not Active", cap="Not Active")),
               (t + 5.0, fields.format(sm=300, hw="Active", cap="Not Active"))]           # after: ignored
    c.window = (t, t + 0.03)
    s = c.summary()
    assert s["samples"] == 2 and s["sm_max_mhz"] == 2070.0
    assert s["sm_mhz"] == (2070 + 2055) / 2
    assert s["reasons"] == ["sw_power_cap"]


def _two_rank_worker(rank, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        bench.barrier(2)
        m = bench.reduce_max(1.5 + rank, 2, device="cpu")
        rate = bench.aggregate_rate(2, 100, m)
        with open(os.path.join(out_dir, f"r{rank}"), "w") as f:
            f.write(f"{m} {rate}")
    finally:
        dist.destroy_process_group()


def test_replica_helpers_on_two_gloo_ranks(tmp_path):
    """The N > 1 helpers (barrier, max over ranks, whole-job rate) on two CPU
    ranks: both see the slower rank's time and the same aggregate."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_two_rank_worker, args=(port, str(tmp_path)), nprocs=2, join=True)
    for r in (0, 1):
        m, rate = map(float, open(tmp_path / f"r{r}").read().split())
        assert m == 2.5 and rate == 2 * 100 / 2.5


def test_reference_arm_under_torchrun_prints_once():
    """Launched as two ranks, only rank 0 runs the oracle and prints its line."""
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
                          "--master-addr", "127.0.0.1", "--master-port", "0", os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and json.loads(lines[0])["impl"] == "reference"
