"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  FP64: 1e-12 relative on W, H after one iteration; 1e-8 relative on the
        objective after 200 iterations (small dense KL case).
  FP32: every sum here has nonnegative terms, so recursive summation of n
        terms errs by at most (n-1)u relative (u = 2^-24); with K-term
        products, chunked reductions of at most ~2k terms and a few ulps from
        powers, one iteration stays within 2e-4 relative (bound), observed
        ~1e-6.
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_15214_gb300 import inputs

pytestmark = pytest.mark.gpu

BETAS = [-1.0, 0.0, 0.5, 1.0, 1.5, 2.0, 3.0]
RTOL = {"fp64": 1e-12, "fp32": 2e-4}


def torch_mod():
    import torch
    return torch


def to_dev(a, prec):
    torch = torch_mod()
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def gpu_run(lib, V, W0, H0, beta, prec="fp64", method="jmm", iters=1, order="W", L=1, kappa=0.0,
            normalize=True, floor=None):
    from paper_2106_15214_gb300.binding import NMF
    F, N = V.shape
    K = W0.shape[1]
    m = NMF(F, N, K, beta, precision=prec, order=order, normalize=normalize, kappa=kappa, L=L, floor=floor)
    Vd, Wd, Hd = to_dev(V, prec), to_dev(W0, prec), to_dev(H0, prec)
    m.set_dense(Vd)
    m.set_factors(Wd, Hd)
    loss = m.step_joint(iters) if method == "jmm" else m.step_alternating(iters)
    out = (Wd.double().cpu().numpy(), Hd.double().cpu().numpy(), loss, m)
    return out


def oracle_run(V, W0, H0, beta, method="jmm", iters=1, order="W", L=1, kappa=0.0, normalize=True, eps=0.0):
    W, H, losses = O.run(V, W0, H0, beta, method=method, iters=iters, order=order, L=L, kappa=kappa,
                         do_normalize=normalize, eps=eps)
    return W, H, losses


def assert_close(got, want, rtol, what):
    err = np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-300))
    assert err <= rtol, f"{what}: max relative error {err:.3e} > {rtol:.1e}"


def problem(F, N, K, seed=0, offset=0.05):
    rng = np.random.default_rng(seed)
    V = rng.gamma(1.0, 1.0, (F, K)) @ rng.gamma(1.0, 1.0, (K, N)) + offset
    V = V * rng.uniform(0.5, 1.5, (F, N))
    W0, H0 = inputs.uniform_init(F, N, K, seed=seed + 7)
    return V, W0, H0


# ---------------------------------------------------------------------------
# The paper's algorithms on every beta regime, both orders, both methods
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("beta", BETAS)
@pytest.mark.parametrize("method,order", [("jmm", "W"), ("jmm", "H"), ("bmm", "W"), ("bmm", "H")])
def test_one_iteration_matches_oracle(lib, prec, beta, method, order):
    V, W0, H0 = problem(70, 101, 6, seed=1)       # 3 x 4 tiles, ragged edges
    W, H, loss, _ = gpu_run(lib, V, W0, H0, beta, prec, method, 1, order)
    Wo, Ho, lo = oracle_run(V, W0, H0, beta, method, 1, order)
    assert_close(W, Wo, RTOL[prec], "W")
    assert_close(H, Ho, RTOL[prec], "H")
    assert loss == pytest.approx(lo[0], rel=RTOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 2), (33, 31, 33), (64, 64, 64), (40, 97, 100),
                                   (257, 45, 128)])
def test_shapes_and_ranks(lib, prec, shape):
    F, N, K = shape
    V, W0, H0 = problem(F, N, K, seed=2)
    for beta in (0.0, 1.5):
        W, H, loss, _ = gpu_run(lib, V, W0, H0, beta, prec, "jmm", 1, "W")
        Wo, Ho, lo = oracle_run(V, W0, H0, beta, "jmm", 1, "W")
        tol = RTOL[prec] * (5 if prec == "fp32" and K > 64 else 1)
        assert_close(W, Wo, tol, f"W {shape}")
        assert_close(H, Ho, tol, f"H {shape}")


@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("order", ["W", "H"])
def test_subiterations(lib, L, order):
    V, W0, H0 = problem(45, 66, 4, seed=3)
    for beta in (0.0, 1.0, 2.5):
        for method in ("jmm", "bmm"):
            W, H, _, _ = gpu_run(lib, V, W0, H0, beta, "fp64", method, 1, order, L=L)
            Wo, Ho, _ = oracle_run(V, W0, H0, beta, method, 1, order, L=L)
            assert_close(W, Wo, 1e-12, f"W L={L}")
            assert_close(H, Ho, 1e-12, f"H L={L}")


def test_kappa_and_zeros(lib):
    V, W0, H0 = problem(50, 60, 5, seed=4)
    V[::4, ::3] = 0.0
    for beta in (0.0, 0.5, 1.0):
        W, H, loss, _ = gpu_run(lib, V, W0, H0, beta, "fp64", "jmm", 3, "W", kappa=0.05)
        Wo, Ho, lo = oracle_run(V, W0, H0, beta, "jmm", 3, "W", kappa=0.05)
        assert_close(W, Wo, 1e-11, "W")
        assert_close(H, Ho, 1e-11, "H")
        assert loss == pytest.approx(lo[2], rel=1e-11)


def test_no_normalisation(lib):
    V, W0, H0 = problem(30, 40, 3, seed=5)
    W, H, _, _ = gpu_run(lib, V, W0, H0, 1.5, "fp64", "jmm", 5, "W", normalize=False)
    Wo, Ho, _ = oracle_run(V, W0, H0, 1.5, "jmm", 5, "W", normalize=False)
    assert_close(W, Wo, 1e-11, "W")
    assert_close(H, Ho, 1e-11, "H")


# ---------------------------------------------------------------------------
# The small dense KL case (F=200, N=500, K=10): 1e-12 after 1, 1e-8 after 200
# ---------------------------------------------------------------------------

def test_dense_kl_fp64_acceptance(lib):
    p = inputs.dense_kl_small()
    W1, H1, l1, _ = gpu_run(lib, p.V, p.W0, p.H0, 1.0, "fp64", "jmm", 1, "W")
    Wo, Ho, lo = oracle_run(p.V, p.W0, p.H0, 1.0, "jmm", 1, "W")
    assert_close(W1, Wo, 1e-12, "W after 1")
    assert_close(H1, Ho, 1e-12, "H after 1")
    W, H, l200, m = gpu_run(lib, p.V, p.W0, p.H0, 1.0, "fp64", "jmm", 200, "W")
    Wo, Ho, lo = oracle_run(p.V, p.W0, p.H0, 1.0, "jmm", 200, "W")
    assert l200 == pytest.approx(lo[199], rel=1e-8)
    assert m.loss() == pytest.approx(lo[200], rel=1e-8)
    assert np.all(np.diff(lo) <= 0)


# ---------------------------------------------------------------------------
# Loss, gradient, KKT
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("beta", BETAS)
def test_loss_and_gradient(lib, prec, beta):
    torch = torch_mod()
    from paper_2106_15214_gb300.binding import NMF
    V, W0, H0 = problem(61, 83, 7, seed=6)
    m = NMF(61, 83, 7, beta, precision=prec, kappa=0.01)
    Vd, Wd, Hd = to_dev(V, prec), to_dev(W0, prec), to_dev(H0, prec)
    m.set_dense(Vd)
    m.set_factors(Wd, Hd)
    D = O.D_beta(V + 0.01, W0 @ H0 + 0.01, beta)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert m.loss() == pytest.approx(D, rel=tol)
    gW = torch.empty_like(Wd)
    gH = torch.empty_like(Hd)
    l = m.grad(gW, gH, want_loss=True)
    assert l == pytest.approx(D, rel=tol)
    oW, oH = O.gradients(V, W0, H0, beta, kappa=0.01)
    gtol = 1e-11 if prec == "fp64" else 5e-4
    scaleW, scaleH = np.abs(oW).max(), np.abs(oH).max()
    assert np.max(np.abs(gW.double().cpu().numpy() - oW)) <= gtol * scaleW
    assert np.max(np.abs(gH.double().cpu().numpy() - oH)) <= gtol * scaleH
    rw, rh = m.kkt()
    ow, oh = O.kkt_residuals(V, W0, H0, beta, kappa=0.01)
    assert rw == pytest.approx(ow, rel=1e-10 if prec == "fp64" else 1e-3)
    assert rh == pytest.approx(oh, rel=1e-10 if prec == "fp64" else 1e-3)


# ---------------------------------------------------------------------------
# Failure detection: a non-finite input is reported and the factors restored
# ---------------------------------------------------------------------------

def test_nonfinite_is_reported_and_factors_restored(lib):
    from paper_2106_15214_gb300.binding import NMF, NMFError, NMF_ENONFINITE
    V, W0, H0 = problem(40, 50, 3, seed=8)
    V[5, 7] = np.nan                                   # planted on the host
    m = NMF(40, 50, 3, 1.0, precision="fp64")
    Vd, Wd, Hd = to_dev(V, "fp64"), to_dev(W0, "fp64"), to_dev(H0, "fp64")
    m.set_dense(Vd)
    m.set_factors(Wd, Hd)
    with pytest.raises(NMFError) as ei:
        m.step_joint(3)
    assert ei.value.code == NMF_ENONFINITE
    assert np.array_equal(Wd.cpu().numpy(), W0) and np.array_equal(Hd.cpu().numpy(), H0)
    Vd[5, 7] = 1.0                                     # repaired data, status cleared by set_factors
    m.set_factors(Wd, Hd)
    assert np.isfinite(m.step_joint(1))


# ---------------------------------------------------------------------------
# Full-size dense configurations, in the launch configuration of the benchmark
# ---------------------------------------------------------------------------

def test_dense_quadratic_faces_full_size_fp32(lib):
    p = inputs.dense_quadratic_faces()
    W, H, loss, _ = gpu_run(lib, p.V, p.W0, p.H0, 2.0, "fp32", "jmm", 1, "W")
    Wo, Ho, lo = oracle_run(p.V, p.W0, p.H0, 2.0, "jmm", 1, "W")
    assert_close(W, Wo, 2e-4, "W")
    assert_close(H, Ho, 2e-4, "H")
    assert loss == pytest.approx(lo[0], rel=1e-5)


def test_dense_is_full_size_fp32(lib):
    p = inputs.dense_is_spectrogram()
    W, H, loss, _ = gpu_run(lib, p.V, p.W0, p.H0, 0.0, "fp32", "jmm", 1, "H")
    Wo, Ho, lo = oracle_run(p.V, p.W0, p.H0, 0.0, "jmm", 1, "H")
    assert_close(W, Wo, 2e-4, "W")
    assert_close(H, Ho, 2e-4, "H")
    assert loss == pytest.approx(lo[0], rel=1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32"])
def test_graph_replay_matches_eager_bitwise(lib, prec):
    """Repeated step calls are captured into a CUDA graph from the second call
    on; replays run the same kernels in the same order, so the iterates equal
    a fresh context's eager run bit for bit (timing on or off)."""
    from paper_2106_15214_gb300.binding import NMF
    V, W0, H0 = problem(90, 130, 8, seed=12)
    outs = []
    for timing in (0, 1):
        m = NMF(90, 130, 8, 0.0, precision=prec)
        Vd, Wd, Hd = to_dev(V, prec), to_dev(W0, prec), to_dev(H0, prec)
        m.set_dense(Vd)
        m.set_factors(Wd, Hd)
        m._lib.nmf_set_timing(m._ctx, timing)
        losses = [m.step_joint(1) for _ in range(6)]            # calls 2..6 replay a graph
        outs.append((Wd.cpu().numpy(), Hd.cpu().numpy(), losses))
    ref = NMF(90, 130, 8, 0.0, precision=prec)
    Vd, Wd, Hd = to_dev(V, prec), to_dev(W0, prec), to_dev(H0, prec)
    ref.set_dense(Vd)
    ref.set_factors(Wd, Hd)
    for i in range(6):
        ref.set_factors(Wd, Hd)                                  # resets the graph cache: always eager
        l = ref.step_joint(1)
        for W, H, losses in outs:
            assert losses[i] == l
    for W, H, _ in outs:
        assert np.array_equal(W, Wd.cpu().numpy()) and np.array_equal(H, Hd.cpu().numpy())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("method", ["jmm", "bmm"])
@pytest.mark.parametrize("order", ["W", "H"])
@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_floor_matches_oracle(lib, prec, method, order, beta):
    """nmf_set_floor: every update is clamped to eps (the constraint W, H >= eps
    of eqs. Wll, Hll). eps is the median of the first raw update of the block
    updated first, so about half of it is clamped; 10 iterations."""
    V, W0, H0 = problem(90, 130, 6, seed=11)
    it = O.jmm_iteration if method == "jmm" else O.bmm_iteration
    W1, H1 = it(V, W0, H0, beta, order=order)
    eps = float(np.median(W1 if order == "W" else H1))
    W, H, loss, _ = gpu_run(lib, V, W0, H0, beta, prec, method, iters=10, order=order, floor=eps)
    Wo, Ho, lo = oracle_run(V, W0, H0, beta, method, iters=10, order=order, eps=eps)
    rtol = 1e-11 if prec == "fp64" else 2e-3
    assert_close(W, Wo, rtol, "W")
    assert_close(H, Ho, rtol, "H")
    assert loss == pytest.approx(lo[9], rel=1e-11 if prec == "fp64" else 1e-5)


def test_floor_defaults_and_errors(lib):
    """Default floor: 0 in FP64 (the unconstrained method), 1e-30 in single
    precision; eps < 0 restores the default; NaN / Inf are rejected."""
    from paper_2106_15214_gb300.binding import NMF, NMFError
    V, W0, H0 = problem(30, 40, 3, seed=12)
    m = NMF(30, 40, 3, 1.0, precision="fp64")
    for bad in (float("nan"), float("inf")):
        with pytest.raises(NMFError):
            m.set_floor(bad)
    m.set_floor(0.5)
    m.set_floor(-1.0)
    Vd, Wd, Hd = to_dev(V, "fp64"), to_dev(W0, "fp64"), to_dev(H0, "fp64")
    m.set_dense(Vd)
    m.set_factors(Wd, Hd)
    m.step_joint(3)
    Wo, Ho, _ = oracle_run(V, W0, H0, 1.0, iters=3)
    assert_close(Wd.cpu().numpy(), Wo, 1e-12, "W (default floor, FP64)")


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32"])
@pytest.mark.parametrize("shape", [(90, 130, 6), (361, 2429, 49)])
def test_host_buffer_step_matches_device_step(lib, prec, shape):
    """nmf_step_joint_host (host V, W, H copied in, W, H and the objective
    copied out, one synchronisation) gives the device step's iterates and
    objectives bitwise, call after call (graph replay from the third)."""
    import torch
    from paper_2106_15214_gb300.binding import NMF
    F, N, K = shape
    V, W0, H0 = problem(F, N, K, seed=31)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Vh = torch.tensor(V, dtype=dt).pin_memory()
    Wh = torch.tensor(W0, dtype=dt).pin_memory()
    Hh = torch.tensor(H0, dtype=dt).pin_memory()
    mh = NMF(F, N, K, 1.5, precision=prec)
    lh = [mh.step_joint_host(Vh, Wh, Hh, 1) for _ in range(4)]
    md = NMF(F, N, K, 1.5, precision=prec)
    Vd, Wd, Hd = to_dev(V, prec), to_dev(W0, prec), to_dev(H0, prec)
    md.set_dense(Vd)
    ld = []
    for _ in range(4):
        md.set_factors(Wd, Hd)          # each host step starts from W, H copied in
        ld.append(md.step_joint(1))
    assert lh == ld
    assert torch.equal(Wh, Wd.cpu()) and torch.equal(Hh, Hd.cpu())


def test_host_buffer_step_nonfinite_restores_the_factors(lib):
    """A NaN in host V: NMF_ENONFINITE, and the host W, H come back as they went in."""
    import torch
    from paper_2106_15214_gb300.binding import NMF, NMFError
    V, W0, H0 = problem(60, 80, 4, seed=32)
    V[3, 5] = np.nan
    Vh = torch.tensor(V, dtype=torch.float32).pin_memory()
    Wh = torch.tensor(W0, dtype=torch.float32).pin_memory()
    Hh = torch.tensor(H0, dtype=torch.float32).pin_memory()
    m = NMF(60, 80, 4, 1.0, precision="fp32")
    with pytest.raises(NMFError) as e:
        m.step_joint_host(Vh, Wh, Hh, 1)
    assert e.value.code == 4
    assert torch.equal(Wh, torch.tensor(W0, dtype=torch.float32))
    assert torch.equal(Hh, torch.tensor(H0, dtype=torch.float32))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("beta", [0.0, 1.0, 1.5, 2.0, 3.0])
def test_autograd_beta_divergence(lib, prec, beta):
    """binding.beta_divergence (a torch.autograd.Function over nmf_grad): the
    value is D_beta, backward scales the library's one-pass gradient by the
    incoming gradient, matching the oracle's gradient and central finite
    differences of the forward value."""
    import torch
    from paper_2106_15214_gb300.binding import beta_divergence
    V, W0, H0 = problem(40, 55, 4, seed=51)
    Vd = to_dev(V, prec)
    W = to_dev(W0, prec).requires_grad_()
    H = to_dev(H0, prec).requires_grad_()
    D = beta_divergence(Vd, W, H, beta)
    (2.5 * D).backward()
    rtol = 1e-10 if prec == "fp64" else 2e-4
    assert D.item() == pytest.approx(O.D_beta(V, W0 @ H0, beta), rel=1e-12 if prec == "fp64" else 1e-5)
    gWo, gHo = O.gradients(V, W0, H0, beta)
    for got, want in ((W.grad, gWo), (H.grad, gHo)):
        got = got.double().cpu().numpy()
        assert np.allclose(got, 2.5 * want, rtol=rtol, atol=rtol * np.abs(want).max() * 2.5)
    if prec == "fp64":
        h = 1e-6
        for (i, j) in ((0, 0), (7, 2), (39, 3)):
            Wp, Wm = W.detach().clone(), W.detach().clone()
            Wp[i, j] += h
            Wm[i, j] -= h
            fd = (beta_divergence(Vd, Wp, H.detach(), beta).item() - beta_divergence(Vd, Wm, H.detach(), beta).item()) / (2 * h)
            assert fd * 2.5 == pytest.approx(W.grad[i, j].item(), rel=1e-6, abs=1e-8)


def test_autograd_reuses_contexts(lib):
    """Forward alone allocates no context (the objective goes to device memory
    through nmf_loss_noalloc); repeated backward passes of one shape share one
    cached context; the values stay those of the oracle."""
    import torch
    from paper_2106_15214_gb300 import binding
    binding._grad_contexts.clear()
    V, W0, H0 = problem(40, 55, 4, seed=52)
    Vd = to_dev(V, "fp64")
    for _ in range(3):
        D = binding.beta_divergence(Vd, to_dev(W0, "fp64"), to_dev(H0, "fp64"), 0.5)
    assert len(binding._grad_contexts) == 0
    assert D.item() == pytest.approx(O.D_beta(V, W0 @ H0, 0.5), rel=1e-12)
    gWo, _ = O.gradients(V, W0, H0, 0.5)
    for _ in range(3):
        W = to_dev(W0, "fp64").requires_grad_()
        binding.beta_divergence(Vd, W, to_dev(H0, "fp64"), 0.5).backward()
        assert np.allclose(W.grad.cpu().numpy(), gWo, rtol=1e-10, atol=1e-12 * np.abs(gWo).max())
    assert len(binding._grad_contexts) == 1


@pytest.mark.parametrize("prec", ["fp32", "tf32", "fp64"])
@pytest.mark.parametrize("beta", [0.0, 1.0, 0.5, -1.0])
def test_objective_with_tiny_ratios(lib, prec, beta):
    """Entries of V far below WH (x / y ~ 1e-9, below single precision's
    resolution of 1 - x / y): every term stays finite and the objective
    matches the oracle (single-precision bars as elsewhere)."""
    from paper_2106_15214_gb300.binding import NMF
    V, W0, H0 = problem(60, 90, 4, seed=61)
    V[::7, ::5] = 1e-8
    m = NMF(60, 90, 4, beta, precision=prec)
    Vd, Wd, Hd = to_dev(V, prec), to_dev(W0, prec), to_dev(H0, prec)
    m.set_dense(Vd)
    m.set_factors(Wd, Hd)
    want = O.D_beta(V, W0 @ H0, beta)
    got = m.loss()
    assert np.isfinite(got)
    assert got == pytest.approx(want, rel=1e-12 if prec == "fp64" else 1e-5)
    step = m.step_joint(1)                       # the sweep's own objective at the same iterate
    assert np.isfinite(step)
    assert step == pytest.approx(want, rel=1e-12 if prec == "fp64" else (2e-3 if prec == "tf32" else 1e-5))
