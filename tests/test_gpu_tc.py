"""Tensor-core (tcgen05 kind::tf32) path against the FP64 oracle.

TF32 tolerance: the factor operands of the three products are rounded to a
10-bit mantissa (u = 2^-11) and the A/B tiles truncated to it by the tensor
core (< 2u); each product term then errs by at most ~2u-3u relative and sums
of nonnegative terms keep that bound, the elementwise powers scale the error
of Vt by |beta - 2|, and the MU ratio, gamma and chi compound a few such
factors: 1e-2 relative on W, H after one iteration bounds it; the objective
at the iterate is within 2e-3.
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_15214_gb300 import inputs

pytestmark = pytest.mark.gpu

BETAS = [-1.0, 0.0, 0.5, 1.0, 1.5, 2.0, 3.0]
TF32_RTOL = 1e-2
TF32_LOSS_RTOL = 2e-3


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def problem(F, N, K, seed=0):
    rng = np.random.default_rng(seed)
    V = rng.gamma(1.0, 1.0, (F, K)) @ rng.gamma(1.0, 1.0, (K, N)) + 0.05
    V = V * rng.uniform(0.5, 1.5, (F, N))
    W0, H0 = inputs.uniform_init(F, N, K, seed=seed + 7)
    return V, W0, H0


def run_tc(V, W0, H0, beta, method="jmm", iters=1, order="W", L=1, kappa=0.0, prec="tf32", floor=None):
    from paper_2106_15214_gb300.binding import NMF
    F, N = V.shape
    K = W0.shape[1]
    m = NMF(F, N, K, beta, precision=prec, order=order, L=L, kappa=kappa, floor=floor)
    Vd, Wd, Hd = dev(V), dev(W0), dev(H0)
    m.set_dense(Vd)
    m.set_factors(Wd, Hd)
    loss = m.step_joint(iters) if method == "jmm" else m.step_alternating(iters)
    return Wd.double().cpu().numpy(), Hd.double().cpu().numpy(), loss, m


def maxrel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("beta", BETAS)
@pytest.mark.parametrize("method,order", [("jmm", "W"), ("jmm", "H"), ("bmm", "W"), ("bmm", "H")])
def test_tf32_one_iteration_matches_oracle(lib, beta, method, order):
    V, W0, H0 = problem(200, 300, 20, seed=1)     # 2 row tiles of 128, 3 column tiles, ragged
    W, H, loss, m = run_tc(V, W0, H0, beta, method, 1, order)
    Wo, Ho, lo = O.run(V, W0, H0, beta, method=method, iters=1, order=order)
    assert maxrel(W, Wo) < TF32_RTOL
    assert maxrel(H, Ho) < TF32_RTOL
    assert loss == pytest.approx(lo[0], rel=TF32_LOSS_RTOL)


@pytest.mark.parametrize("K", [1, 7, 16, 33, 64, 100, 128])
def test_tf32_ranks(lib, K):
    V, W0, H0 = problem(150, 170, K, seed=2)
    for beta in (0.0, 1.5):
        W, H, loss, _ = run_tc(V, W0, H0, beta, "jmm", 1, "W")
        Wo, Ho, lo = O.run(V, W0, H0, beta, iters=1)
        assert maxrel(W, Wo) < TF32_RTOL, K
        assert maxrel(H, Ho) < TF32_RTOL, K


@pytest.mark.parametrize("order", ["W", "H"])
def test_tf32_subiterations_and_kappa(lib, order):
    V, W0, H0 = problem(140, 260, 12, seed=3)
    for beta in (0.0, 1.0, 2.5):
        W, H, _, _ = run_tc(V, W0, H0, beta, "jmm", 1, order, L=2, kappa=0.01)
        Wo, Ho, _ = O.run(V, W0, H0, beta, iters=1, order=order, L=2, kappa=0.01)
        assert maxrel(W, Wo) < TF32_RTOL
        assert maxrel(H, Ho) < TF32_RTOL


def test_tf32_agrees_with_fp32_path(lib):
    V, W0, H0 = problem(300, 400, 24, seed=4)
    W, H, l, _ = run_tc(V, W0, H0, 0.0, "jmm", 5, "H")
    W2, H2, l2, _ = run_tc(V, W0, H0, 0.0, "jmm", 5, "H", prec="fp32")
    assert maxrel(W, W2) < 3e-2 and maxrel(H, H2) < 3e-2
    assert l == pytest.approx(l2, rel=5e-3)


def test_tf32_descends(lib):
    V, W0, H0 = problem(256, 384, 16, seed=5)
    from paper_2106_15214_gb300.binding import NMF
    m = NMF(256, 384, 16, 1.0, precision="tf32")
    Vd, Wd, Hd = dev(V), dev(W0), dev(H0)
    m.set_dense(Vd)
    m.set_factors(Wd, Hd)
    losses = [m.step_joint(1) for _ in range(60)]
    d = np.diff(losses)
    assert losses[-1] < 0.5 * losses[0]
    assert np.all(d <= 1e-3 * np.abs(np.array(losses[1:])))


def test_tf32_faces_full_size(lib):
    p = inputs.dense_quadratic_faces()
    W, H, loss, _ = run_tc(p.V, p.W0, p.H0, 2.0, "jmm", 1, "W")
    Wo, Ho, lo = O.run(p.V, p.W0, p.H0, 2.0, iters=1)
    assert maxrel(W, Wo) < TF32_RTOL
    assert maxrel(H, Ho) < TF32_RTOL
    assert loss == pytest.approx(lo[0], rel=TF32_LOSS_RTOL)


def test_tf32_spectrogram_full_size(lib):
    p = inputs.dense_is_spectrogram()
    W, H, loss, _ = run_tc(p.V, p.W0, p.H0, 0.0, "jmm", 1, "H")
    Wo, Ho, lo = O.run(p.V, p.W0, p.H0, 0.0, iters=1, order="H")
    assert maxrel(W, Wo) < TF32_RTOL
    assert maxrel(H, Ho) < TF32_RTOL
    assert loss == pytest.approx(lo[0], rel=TF32_LOSS_RTOL)


@pytest.mark.parametrize("cluster,K,method,order", [(2, 40, "jmm", "W"), (4, 64, "jmm", "H"), (8, 20, "jmm", "W"),
                                                    (8, 33, "bmm", "H")])
def test_tf32_cluster_reduction(lib, monkeypatch, cluster, K, method, order):
    """Blocks of a tile in clusters of 2/4/8 combined through distributed
    shared memory (padding blocks included) give the oracle's iterate."""
    monkeypatch.setenv("NMF_TC_CLUSTER", str(cluster))
    V, W0, H0 = problem(300, 2100, K, seed=3)
    W, H, loss, _ = run_tc(V, W0, H0, 1.0, method, 2, order)
    Wo, Ho, lo = O.run(V, W0, H0, 1.0, method=method, iters=2, order=order)
    assert maxrel(W, Wo) < TF32_RTOL
    assert maxrel(H, Ho) < TF32_RTOL
    assert loss == pytest.approx(lo[1], rel=TF32_LOSS_RTOL)
    monkeypatch.delenv("NMF_TC_CLUSTER")
    W1, H1, _, _ = run_tc(V, W0, H0, 1.0, method, 2, order)
    assert maxrel(W, W1) < 1e-3 and maxrel(H, H1) < 1e-3


@pytest.mark.parametrize("prec,method", [("tf32", "jmm"), ("fp32", "bmm"), ("fp64", "jmm")])
def test_async_step_matches_sync(lib, prec, method):
    """nmf_step_*_async computes the same iterates and objective as the
    synchronous call (bitwise: same kernels, same order), leaving the loss in
    device memory; nmf_get_status then reports OK."""
    import torch
    from paper_2106_15214_gb300.binding import NMF
    V, W0, H0 = problem(257, 331, 20, seed=8)
    dt = torch.float64 if prec == "fp64" else torch.float32
    outs = []
    for mode in ("sync", "async"):
        m = NMF(257, 331, 20, 1.0, precision=prec, order="H")
        Vd = torch.tensor(V, dtype=dt, device="cuda")
        Wd = torch.tensor(W0, dtype=dt, device="cuda")
        Hd = torch.tensor(H0, dtype=dt, device="cuda")
        m.set_dense(Vd)
        m.set_factors(Wd, Hd)
        losses = []
        if mode == "sync":
            for _ in range(4):
                losses.append(m.step_joint(1) if method == "jmm" else m.step_alternating(1))
        else:
            buf = torch.zeros(4, dtype=torch.float64, device="cuda")
            for i in range(4):
                if method == "jmm":
                    m.step_joint_async(buf[i:i + 1])
                else:
                    m.step_alternating_async(buf[i:i + 1])
            assert lib.nmf_get_status(m._ctx) == 0
            losses = buf.cpu().tolist()
        outs.append((Wd.cpu().numpy(), Hd.cpu().numpy(), losses))
    (W1, H1, l1), (W2, H2, l2) = outs
    assert np.array_equal(W1, W2) and np.array_equal(H1, H2)
    assert l1 == l2


@pytest.mark.parametrize("order,beta,K,F,N", [("W", 2.0, 49, 300, 4100), ("H", 0.0, 20, 300, 4100),
                                               ("H", 1.0, 8, 200, 20000), ("W", 1.5, 64, 300, 4100)])
def test_tf32_persistent_step_kernel(lib, monkeypatch, order, beta, K, F, N):
    """NMF_TC_STEP=1: the whole JMM iteration in one cooperative launch (grid
    barriers between the phases, several units per block when the sweeps have
    more units than SMs) gives the oracle's iterates and objective, and
    agrees with the per-kernel sequence."""
    monkeypatch.setenv("NMF_TC_STEP", "1")
    V, W0, H0 = problem(F, N, K, seed=21)         # N = 20000: more column-sweep units than SMs
    W, H, loss, _ = run_tc(V, W0, H0, beta, "jmm", 3, order)
    Wo, Ho, lo = O.run(V, W0, H0, beta, iters=3, order=order)
    assert maxrel(W, Wo) < TF32_RTOL
    assert maxrel(H, Ho) < TF32_RTOL
    assert loss == pytest.approx(lo[2], rel=TF32_LOSS_RTOL)
    monkeypatch.delenv("NMF_TC_STEP")
    W1, H1, loss1, _ = run_tc(V, W0, H0, beta, "jmm", 3, order)
    assert maxrel(W, W1) < 1e-3 and maxrel(H, H1) < 1e-3
    assert loss == pytest.approx(loss1, rel=1e-4)


@pytest.mark.parametrize("order,method,K", [("H", "jmm", 20), ("W", "jmm", 33), ("H", "bmm", 16)])
def test_tf32_stream_k_column_sweep(lib, monkeypatch, order, method, K):
    """157 column tiles on 152 SMs: the column sweep is split stream-K (block
    ranges cross column tiles, per-tile slice counts in the H epilogue) and
    matches the oracle and the uniform split (NMF_TC_SK=0)."""
    V, W0, H0 = problem(300, 20000, K, seed=23)
    W, H, loss, _ = run_tc(V, W0, H0, 1.0, method, 2, order)
    Wo, Ho, lo = O.run(V, W0, H0, 1.0, method=method, iters=2, order=order)
    assert maxrel(W, Wo) < TF32_RTOL
    assert maxrel(H, Ho) < TF32_RTOL
    assert loss == pytest.approx(lo[1], rel=TF32_LOSS_RTOL)
    monkeypatch.setenv("NMF_TC_SK", "0")
    W1, H1, loss1, _ = run_tc(V, W0, H0, 1.0, method, 2, order)
    assert maxrel(W, W1) < 1e-3 and maxrel(H, H1) < 1e-3
    assert loss == pytest.approx(loss1, rel=1e-4)


@pytest.mark.parametrize("order", ["W", "H"])
@pytest.mark.parametrize("K", [20, 49])
@pytest.mark.parametrize("N", [300, 20000])
def test_tf32_floor_matches_oracle(lib, order, K, N):
    """The floor in the tensor-core path's epilogues (the 16-byte vector H
    epilogue and the stream-K column sweep at N = 20000): one JMM iteration
    with eps at the median of the raw first update."""
    V, W0, H0 = problem(200, N, K, seed=13)
    W1, H1 = O.jmm_iteration(V, W0, H0, 0.0, order=order)
    eps = float(np.median(W1 if order == "W" else H1))
    W, H, _, _ = run_tc(V, W0, H0, 0.0, "jmm", 1, order, floor=eps)
    Wo, Ho, _ = O.run(V, W0, H0, 0.0, iters=1, order=order, eps=eps)
    assert maxrel(W, Wo) < TF32_RTOL
    assert maxrel(H, Ho) < TF32_RTOL


@pytest.mark.parametrize("prec", ["tf32", "fp32"])
def test_long_itakura_saito_run_stays_finite(lib, prec):
    """Itakura-Saito JMM on spectrogram-shaped data drives entries of H toward
    zero geometrically (about 1e-40 after 700 iterations in FP32 at N = 1000);
    without a floor they underflow and chi's ratio becomes 0 / 0. The default
    single-precision floor (1e-30) keeps 1200 iterations finite and descending."""
    from paper_2106_15214_gb300.binding import NMF
    p = inputs.dense_is_spectrogram(N=1000)
    F, N, K = p.shape
    m = NMF(F, N, K, 0.0, precision=prec, order="H")
    Vd, Wd, Hd = dev(p.V), dev(p.W0), dev(p.H0)
    m.set_dense(Vd)
    m.set_factors(Wd, Hd)
    losses = [m.step_joint(100) for _ in range(12)]
    assert all(np.isfinite(losses))
    assert all(b <= a * (1 + 1e-4) for a, b in zip(losses, losses[1:]))
    W, H = Wd.double().cpu().numpy(), Hd.double().cpu().numpy()
    assert np.isfinite(W).all() and np.isfinite(H).all()
    assert H.min() < 1e-20          # the run did reach the regime where FP32 would underflow


@pytest.mark.parametrize("F,N,K", [(200, 300, 20), (361, 2429, 49), (150, 1030, 33), (513, 20000, 20)])
@pytest.mark.parametrize("beta", [0.0, 1.0, 2.0])
def test_fused_next_copies_match_the_copies_kernel(lib, monkeypatch, F, N, K, beta):
    """W first: the iteration's last kernel also makes the next iteration's
    operand copies, and the next step (or iteration) skips the copies kernel.
    Bitwise the same iterates and objectives as with the separate copies
    kernel (NMF_TC_FUSE_COPIES=0), across calls (graph capture and replay from
    the third call on) and within a multi-iteration call."""
    V, W0, H0 = problem(F, N, K, seed=21)

    from paper_2106_15214_gb300.binding import NMF
    out = []
    for fuse in ("1", "0"):
        monkeypatch.setenv("NMF_TC_FUSE_COPIES", fuse)
        m = NMF(F, N, K, beta, precision="tf32", order="W")
        Vd, Wd, Hd = dev(V), dev(W0), dev(H0)
        m.set_dense(Vd)
        m.set_factors(Wd, Hd)
        losses = [m.step_joint(1) for _ in range(5)] + [m.step_joint(3)]
        out.append((Wd.cpu().numpy(), Hd.cpu().numpy(), losses))
    (Wa, Ha, la), (Wb, Hb, lb) = out
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    assert la == lb


def test_fused_copies_are_dropped_by_set_factors_and_other_calls(lib):
    """After an in-place write of W followed by nmf_set_factors, and around
    nmf_loss and alternating steps, a context with fused copies gives the same
    iterates as a fresh context started from the same W, H."""
    from paper_2106_15214_gb300.binding import NMF
    import torch
    V, W0, H0 = problem(240, 700, 24, seed=22)
    m = NMF(240, 700, 24, 1.0, precision="tf32", order="W")
    Vd, Wd, Hd = dev(V), dev(W0), dev(H0)
    m.set_dense(Vd)
    m.set_factors(Wd, Hd)
    for _ in range(3):
        m.step_joint(1)
    Wd.mul_(1.5)                                 # in-place change of W ...
    m.set_factors(Wd, Hd)                        # ... announced to the context
    W1, H1 = Wd.clone(), Hd.clone()
    m.step_joint(1)
    m.loss()
    m.step_joint(1)
    m.step_alternating(1)
    m.step_joint(2)
    f = NMF(240, 700, 24, 1.0, precision="tf32", order="W")
    W2, H2 = W1.clone(), H1.clone()
    f.set_dense(Vd)
    f.set_factors(W2, H2)
    f.step_joint(1)
    f.loss()
    f.step_joint(1)
    f.step_alternating(1)
    f.step_joint(2)
    torch.cuda.synchronize()
    assert torch.equal(Wd, W2) and torch.equal(Hd, H2)


@pytest.mark.parametrize("F,N,K,order", [(361, 2429, 49, "W"), (513, 20000, 20, "W"), (513, 20000, 20, "H"),
                                         (200, 300, 20, "H")])
def test_early_second_sweep_matches_waiting_one(lib, monkeypatch, F, N, K, order):
    """The second sweep of a joint iteration reads W~, H~ and V before the
    epilogue ahead of it has finished; bitwise the same iterates and
    objectives as with the sweep waiting for it at entry (NMF_TC_EARLY=0)."""
    from paper_2106_15214_gb300.binding import NMF
    V, W0, H0 = problem(F, N, K, seed=41)
    out = []
    for early in ("1", "0"):
        monkeypatch.setenv("NMF_TC_EARLY", early)
        m = NMF(F, N, K, 0.5, precision="tf32", order=order)
        Vd, Wd, Hd = dev(V), dev(W0), dev(H0)
        m.set_dense(Vd)
        m.set_factors(Wd, Hd)
        losses = [m.step_joint(1) for _ in range(4)] + [m.step_joint(3)]
        out.append((Wd.cpu().numpy(), Hd.cpu().numpy(), losses))
    (Wa, Ha, la), (Wb, Hb, lb) = out
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    assert la == lb


def test_tf32_spectrogram_large_matches_oracle(lib):
    """513 x 200000 (V = 410 MB, above L2): one JMM iteration with W first
    through the stream-K column sweep (about 175 tile steps per block) and the
    fused copies; every entry of W and H against the FP64 oracle."""
    p = inputs.dense_is_spectrogram(N=200000)
    W, H, loss, _ = run_tc(p.V, p.W0, p.H0, 0.0, "jmm", 1, "W")
    Wo, Ho, lo = O.run(p.V, p.W0, p.H0, 0.0, iters=1)
    assert maxrel(W, Wo) < TF32_RTOL
    assert maxrel(H, Ho) < TF32_RTOL
    assert loss == pytest.approx(lo[0], rel=TF32_LOSS_RTOL)
