"""The fused single-read JMM iteration (NMF_BF16, tc_fused.cu) against the
FP64 oracle.

One launch per iteration reads V once: the product in TF32, A and B once,
both contractions from on-chip bf16 copies of A and B (H first, L = 1; the
inverted update order of Sec. 4.1.1), the H partials exchanged inside a
cluster of ceil(F / 128) blocks. Tolerances (derived in the design notes):
3e-2 relative on W and H after one iteration (bf16 operands, u = 2^-9, in
both contractions and the MU ratio), 5e-3 on the objective at the iterate
(its terms use the TF32 product, as on the TF32 path).
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_15214_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_WH, TOL_D = 3e-2, 5e-3


def problem(F, N, K, seed):
    rng = np.random.default_rng(seed)
    V = rng.gamma(1.0, 1.0, (F, K)) @ rng.gamma(1.0, 1.0, (K, N)) + 0.05
    V = V * rng.uniform(0.5, 1.5, (F, N))
    W0, H0 = inputs.uniform_init(F, N, K, seed=seed + 7)
    return V, W0, H0


def run_bf16(V, W0, H0, beta, iters=1, order="H", want_loss=True):
    import torch
    from paper_2106_15214_gb300.binding import NMF
    F, N = V.shape
    K = W0.shape[1]
    m = NMF(F, N, K, beta, precision="bf16", order=order)
    Vd = torch.tensor(V, dtype=torch.float32, device="cuda")
    W = torch.tensor(W0, dtype=torch.float32, device="cuda")
    H = torch.tensor(H0, dtype=torch.float32, device="cuda")
    m.set_dense(Vd)
    m.set_factors(W, H)
    loss = m.step_joint(iters, want_loss=want_loss)
    out = (W.double().cpu().numpy(), H.double().cpu().numpy(), loss)
    m.close()
    return out


def oracle_h_first(V, W0, H0, beta, iters=1):
    W, H, losses = O.run(V, W0, H0, beta, iters=iters, order="H", eps=1e-30)
    return W, H, losses


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("shape", [(100, 300, 4), (200, 333, 20), (361, 517, 32), (513, 1000, 20), (129, 260, 8),
                                   (257, 700, 32)])
@pytest.mark.parametrize("beta", [0.0, 1.0, 1.5, 2.0])
def test_one_iteration_matches_oracle(lib, shape, beta):
    """Clusters of 1, 2, 3 and 4 blocks; ragged rows (F % 128) and columns (N %
    128); F = 513, 129 and 257 put their last row on the last block's
    tail-row warp (clusters of 4, 1 and 2 blocks)."""
    F, N, K = shape
    V, W0, H0 = problem(F, N, K, seed=F + N)
    W, H, loss = run_bf16(V, W0, H0, beta)
    Wo, Ho, lo = oracle_h_first(V, W0, H0, beta)
    assert np.all(np.isfinite(W)) and np.all(np.isfinite(H))
    assert rel(W, Wo) < TOL_WH
    assert rel(H, Ho) < TOL_WH
    assert loss == pytest.approx(lo[0], rel=TOL_D)


@pytest.mark.parametrize("shape,beta", [((101, 301, 5), 1.0), ((130, 40000, 8), 0.0), ((1024, 700, 32), 1.5)])
def test_w_half_launch_shapes(lib, shape, beta):
    """The launch after the fused sweep (every cluster sums all the partial
    slices; column norms combined over distributed shared memory; W and H
    normalised with their next copies) on F K not a multiple of 4 (no 16-byte
    loads), more columns of H per block than one pass through shared memory,
    and the largest F and K: two iterations (the second from the copies the
    first left) against the oracle; one iteration against the separate W
    epilogue and normalisation kernels (NMF_FU_POST=0), which differ only in
    the order of the slice sums (the objective, from the same sweep, equal)."""
    import os
    F, N, K = shape
    V, W0, H0 = problem(F, N, K, seed=F * 3 + K)
    W, H, loss = run_bf16(V, W0, H0, beta, iters=2)
    Wo, Ho, lo = oracle_h_first(V, W0, H0, beta, iters=2)
    assert rel(W, Wo) < 2 * TOL_WH and rel(H, Ho) < 2 * TOL_WH
    assert loss == pytest.approx(lo[1], rel=TOL_D)
    W1, H1, loss1 = run_bf16(V, W0, H0, beta)
    os.environ["NMF_FU_POST"] = "0"
    try:
        W2, H2, loss2 = run_bf16(V, W0, H0, beta)
    finally:
        del os.environ["NMF_FU_POST"]
    assert rel(W1, W2) < 1e-5 and rel(H1, H2) < 1e-5
    assert loss1 == loss2


@pytest.mark.parametrize("shape,beta", [((513, 2000, 20), 0.0), ((385, 900, 12), 1.5)])
def test_tail_rows_against_full_blocks(lib, shape, beta):
    """The tail row (F = 128 c + 1 on the last block's warp 0, in FP32)
    and the plain layout (NMF_FU_TAIL=0: one more block per cluster) both
    match the oracle over three iterations, and each other to the bf16
    tolerance."""
    import os
    F, N, K = shape
    V, W0, H0 = problem(F, N, K, seed=F + 11)
    W, H, loss = run_bf16(V, W0, H0, beta, iters=3)
    os.environ["NMF_FU_TAIL"] = "0"
    try:
        W2, H2, loss2 = run_bf16(V, W0, H0, beta, iters=3)
    finally:
        del os.environ["NMF_FU_TAIL"]
    Wo, Ho, lo = oracle_h_first(V, W0, H0, beta, iters=3)
    for Wx, Hx, lx in ((W, H, loss), (W2, H2, loss2)):
        assert rel(Wx, Wo) < 3 * TOL_WH and rel(Hx, Ho) < 3 * TOL_WH
        assert lx == pytest.approx(lo[2], rel=TOL_D)
    assert rel(W, W2) < 3 * TOL_WH and rel(H, H2) < 3 * TOL_WH


@pytest.mark.parametrize("beta", [-1.0, 0.5, 3.0])
def test_general_beta(lib, beta):
    V, W0, H0 = problem(300, 400, 16, seed=5)
    W, H, loss = run_bf16(V, W0, H0, beta)
    Wo, Ho, lo = oracle_h_first(V, W0, H0, beta)
    assert rel(W, Wo) < TOL_WH and rel(H, Ho) < TOL_WH
    assert loss == pytest.approx(lo[0], rel=TOL_D)


def test_many_iterations_follow_the_oracle(lib):
    """20 iterations on a spectrogram-shaped problem: the objective stays within
    5e-3 of the oracle's (the iterates follow a nearby trajectory)."""
    p = inputs.dense_is_spectrogram(N=2000)
    W, H, loss = run_bf16(p.V, p.W0, p.H0, 0.0, iters=20)
    Wo, Ho, lo = oracle_h_first(p.V, p.W0, p.H0, 0.0, iters=20)
    assert loss == pytest.approx(lo[19], rel=TOL_D)
    D_gpu = O.D_beta(p.V, W @ H, 0.0)
    assert D_gpu == pytest.approx(lo[20], rel=TOL_D)


def test_full_size_spectrogram(lib):
    """The spectrogram workload at full size (F = 513, N = 20000, K = 20): one
    iteration, element-wise against the oracle."""
    p = inputs.dense_is_spectrogram()
    W, H, loss = run_bf16(p.V, p.W0, p.H0, 0.0)
    Wo, Ho, lo = oracle_h_first(p.V, p.W0, p.H0, 0.0)
    assert rel(W, Wo) < TOL_WH and rel(H, Ho) < TOL_WH
    assert loss == pytest.approx(lo[0], rel=TOL_D)


@pytest.mark.parametrize("shape,ncl", [((513, 2560, 20), 2), ((200, 5000, 32), 3), ((100, 3000, 4), 1)])
def test_many_batches_per_cluster(lib, shape, ncl):
    """NMF_FU_CLUSTERS caps the clusters, so each one runs many 128-column
    batches through the double-buffered pipeline and the cluster handshakes."""
    import os
    F, N, K = shape
    V, W0, H0 = problem(F, N, K, seed=N)
    os.environ["NMF_FU_CLUSTERS"] = str(ncl)
    try:
        W, H, loss = run_bf16(V, W0, H0, 0.0)
    finally:
        del os.environ["NMF_FU_CLUSTERS"]
    Wo, Ho, lo = oracle_h_first(V, W0, H0, 0.0)
    assert rel(W, Wo) < TOL_WH and rel(H, Ho) < TOL_WH
    assert loss == pytest.approx(lo[0], rel=TOL_D)


def test_deterministic_and_async_equals_sync(lib):
    import torch
    from paper_2106_15214_gb300.binding import NMF
    V, W0, H0 = problem(513, 1500, 20, seed=9)
    outs = []
    for mode in ("sync", "sync", "async"):
        m = NMF(513, 1500, 20, 0.0, precision="bf16", order="H")
        Vd = torch.tensor(V, dtype=torch.float32, device="cuda")
        W = torch.tensor(W0, dtype=torch.float32, device="cuda")
        H = torch.tensor(H0, dtype=torch.float32, device="cuda")
        m.set_dense(Vd)
        m.set_factors(W, H)
        if mode == "sync":
            loss = m.step_joint(3)
        else:
            ld = torch.zeros(1, dtype=torch.float64, device="cuda")
            m.step_joint_async(ld, iters=3)
            torch.cuda.synchronize()
            loss = float(ld.item())
        outs.append((W.cpu().numpy(), H.cpu().numpy(), loss))
        m.close()
    for W, H, loss in outs[1:]:
        assert np.array_equal(W, outs[0][0]) and np.array_equal(H, outs[0][1]) and loss == outs[0][2]


def test_unsupported_forms_are_rejected(lib):
    import torch
    from paper_2106_15214_gb300.binding import NMF, NMF_EUNSUPPORTED, NMFError
    V, W0, H0 = problem(64, 96, 4, seed=1)
    for kw, call in ((dict(order="W"), "joint"), (dict(order="H"), "alternating"), (dict(order="H", L=2), "joint")):
        m = NMF(64, 96, 4, 1.0, precision="bf16", **kw)
        m.set_dense(torch.tensor(V, dtype=torch.float32, device="cuda"))
        m.set_factors(torch.tensor(W0, dtype=torch.float32, device="cuda"),
                      torch.tensor(H0, dtype=torch.float32, device="cuda"))
        with pytest.raises(NMFError) as e:
            (m.step_joint if call == "joint" else m.step_alternating)(1)
        assert e.value.code == NMF_EUNSUPPORTED
        m.close()
    m = NMF(64, 96, 40, 1.0, precision="bf16", order="H")       # K > 32
    Wb, Hb = inputs.uniform_init(64, 96, 40, seed=2)
    m.set_dense(torch.tensor(V, dtype=torch.float32, device="cuda"))
    m.set_factors(torch.tensor(Wb, dtype=torch.float32, device="cuda"),
                  torch.tensor(Hb, dtype=torch.float32, device="cuda"))
    with pytest.raises(NMFError) as e:
        m.step_joint(1)
    assert e.value.code == NMF_EUNSUPPORTED
    m.close()


@pytest.mark.parametrize("F", [200, 257])
def test_cluster_wait_timeout_returns_etimeout(lib, F):
    """The cluster exchange's waits expect one arrival more than there are
    blocks (nmf_set_barrier_test): every such wait runs out after 2 ms, the
    step returns NMF_ETIMEOUT with W and H restored, and the context then
    computes the oracle's iterate with the defaults back. F = 257: the tail
    row's warp (which polls its loads while it waits) gives up too."""
    import torch
    from paper_2106_15214_gb300.binding import NMF, NMF_ETIMEOUT, NMFError, check
    V, W0, H0 = problem(F, 333, 20, seed=3)
    m = NMF(F, 333, 20, 1.0, precision="bf16", order="H")
    Vd = torch.tensor(V, dtype=torch.float32, device="cuda")
    W = torch.tensor(W0, dtype=torch.float32, device="cuda")
    H = torch.tensor(H0, dtype=torch.float32, device="cuda")
    W1, H1 = W.clone(), H.clone()
    m.set_dense(Vd)
    m.set_factors(W, H)
    check(lib.nmf_set_barrier_test(m._ctx, 2_000_000, 1), "nmf_set_barrier_test")
    with pytest.raises(NMFError) as e:
        m.step_joint(1)
    assert e.value.code == NMF_ETIMEOUT
    torch.cuda.synchronize()
    assert torch.equal(W, W1) and torch.equal(H, H1)
    check(lib.nmf_set_barrier_test(m._ctx, 1_000_000_000, 0), "nmf_set_barrier_test")
    m.set_factors(W, H)
    m.step_joint(1)
    Wo, Ho, _ = oracle_h_first(V, W0, H0, 1.0)
    assert rel(W.double().cpu().numpy(), Wo) < TOL_WH and rel(H.double().cpu().numpy(), Ho) < TOL_WH
    m.close()


@pytest.mark.parametrize("F", [300, 257])
@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_kappa_and_no_normalisation(lib, beta, F):
    """kappa > 0 (Sec. 4.1.3: added to V and to every product) and the step
    without the normalisation (the last kernel then only makes the next
    iteration's copies), three iterations in one call; F = 257 with the tail
    row on the last block's warp 0."""
    import torch
    from paper_2106_15214_gb300.binding import NMF
    V, W0, H0 = problem(F, 700, 20, seed=21)
    for kappa, normalize in ((0.05, True), (0.0, False), (0.05, False)):
        m = NMF(F, 700, 20, beta, precision="bf16", order="H", kappa=kappa, normalize=normalize)
        W = torch.tensor(W0, dtype=torch.float32, device="cuda")
        H = torch.tensor(H0, dtype=torch.float32, device="cuda")
        m.set_dense(torch.tensor(V, dtype=torch.float32, device="cuda"))
        m.set_factors(W, H)
        loss = m.step_joint(3)
        Wo, Ho, lo = O.run(V, W0, H0, beta, iters=3, order="H", kappa=kappa, do_normalize=normalize, eps=1e-30)
        assert rel(W.double().cpu().numpy(), Wo) < 2 * TOL_WH, (kappa, normalize)
        assert rel(H.double().cpu().numpy(), Ho) < 2 * TOL_WH, (kappa, normalize)
        assert loss == pytest.approx(lo[2], rel=TOL_D), (kappa, normalize)
        m.close()


def test_floor_matches_the_constrained_update(lib):
    """nmf_set_floor(eps): every update clamped to eps (the constraint of eqs.
    Wll / Hll), here with eps inside the range of the first update."""
    import torch
    from paper_2106_15214_gb300.binding import NMF
    V, W0, H0 = problem(200, 400, 12, seed=22)
    W1, H1, _ = O.run(V, W0, H0, 0.0, iters=1, order="H", eps=0.0)
    eps = float(np.quantile(np.concatenate([W1.ravel(), H1.ravel()]), 0.2))
    m = NMF(200, 400, 12, 0.0, precision="bf16", order="H", floor=eps)
    W = torch.tensor(W0, dtype=torch.float32, device="cuda")
    H = torch.tensor(H0, dtype=torch.float32, device="cuda")
    m.set_dense(torch.tensor(V, dtype=torch.float32, device="cuda"))
    m.set_factors(W, H)
    m.step_joint(2)
    Wo, Ho, _ = O.run(V, W0, H0, 0.0, iters=2, order="H", eps=eps)
    Wg, Hg = W.double().cpu().numpy(), H.double().cpu().numpy()
    assert rel(Wg, Wo) < 2 * TOL_WH and rel(Hg, Ho) < 2 * TOL_WH
    m.close()


@pytest.mark.parametrize("beta,shape", [(0.0, (300, 700, 20)), (1.5, (200, 333, 12)), (1.0, (129, 500, 32))])
def test_fused_adjoint_matches_oracle(lib, beta, shape):
    """nmf_grad on a BF16 context: the fused sweep's adjoint mode (grad_H =
    W^T (B - A), grad_W = (B - A) H^T from one read of V) against the oracle's
    gradient; each gradient is a difference of two bf16 contractions, so the
    bar is 3e-2 of the larger of the two terms' scale, taken as max |grad| of
    the oracle plus the mean absolute MU numerator (P or Hn) of the oracle."""
    import torch
    from paper_2106_15214_gb300.binding import NMF
    F, N, K = shape
    V, W0, H0 = problem(F, N, K, seed=F + K)
    m = NMF(F, N, K, beta, precision="bf16", order="H")
    W = torch.tensor(W0, dtype=torch.float32, device="cuda")
    H = torch.tensor(H0, dtype=torch.float32, device="cuda")
    m.set_dense(torch.tensor(V, dtype=torch.float32, device="cuda"))
    m.set_factors(W, H)
    gW, gH = torch.empty_like(W), torch.empty_like(H)
    loss = m.grad(gW, gH, want_loss=True)
    oW, oH = O.gradients(V, W0, H0, beta)
    Vt = W0 @ H0
    A = V * Vt ** (beta - 2.0)
    for g, o, num in ((gW, oW, A @ H0.T), (gH, oH, W0.T @ A)):
        scale = np.max(np.abs(o)) + np.mean(np.abs(num))
        assert np.max(np.abs(g.double().cpu().numpy() - o)) < 3e-2 * scale
    assert loss == pytest.approx(O.D_beta(V, Vt, beta), rel=TOL_D)
    assert torch.equal(W, torch.tensor(W0, dtype=torch.float32, device="cuda"))    # factors untouched
    assert torch.equal(H, torch.tensor(H0, dtype=torch.float32, device="cuda"))
    # a step after the gradient (the copies it left are of the same W, H)
    m.step_joint(1)
    Wo, Ho, _ = oracle_h_first(V, W0, H0, beta)
    assert rel(W.double().cpu().numpy(), Wo) < TOL_WH and rel(H.double().cpu().numpy(), Ho) < TOL_WH
    m.close()


def test_autograd_fused_adjoint(lib):
    """binding.beta_divergence(..., fused=True): backward runs the fused sweep's
    adjoint mode on a cached BF16 context; the scaled gradients meet the same
    bar as nmf_grad on BF16 against the oracle's gradient, and the value is
    the objective at W, H."""
    import torch
    from paper_2106_15214_gb300.binding import beta_divergence
    F, N, K, beta = 300, 700, 20, 0.0
    V, W0, H0 = problem(F, N, K, seed=77)
    Vd = torch.tensor(V, dtype=torch.float32, device="cuda")
    W = torch.tensor(W0, dtype=torch.float32, device="cuda").requires_grad_()
    H = torch.tensor(H0, dtype=torch.float32, device="cuda").requires_grad_()
    D = beta_divergence(Vd, W, H, beta, fused=True)
    (0.5 * D).backward()
    Vt = W0 @ H0
    assert D.item() == pytest.approx(O.D_beta(V, Vt, beta), rel=1e-5)
    oW, oH = O.gradients(V, W0, H0, beta)
    A = V * Vt ** (beta - 2.0)
    for g, o, num in ((W.grad, oW, A @ H0.T), (H.grad, oH, W0.T @ A)):
        scale = np.max(np.abs(o)) + np.mean(np.abs(num))
        assert np.max(np.abs(g.double().cpu().numpy() - 0.5 * o)) < 0.5 * 3e-2 * scale
