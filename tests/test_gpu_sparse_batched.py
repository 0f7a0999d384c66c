"""Sparse KL (beta = 1) and batched paths against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2106_15214_gb300 import inputs

pytestmark = pytest.mark.gpu


def dev(a, dt=None):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dt or torch.float32, device="cuda")


def sparse_ctx(p, order="W"):
    import torch
    from paper_2106_15214_gb300.binding import NMF
    m = NMF(p.F, p.N, p.W0.shape[1], 1.0, precision="fp32", order=order)
    rp, cl, vl = dev(p.rowptr, torch.int32), dev(p.col, torch.int32), dev(p.val)
    m.set_csr(rp, cl, vl)
    W, H = dev(p.W0), dev(p.H0)
    m.set_factors(W, H)
    return m, W, H


def rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-30))


@pytest.mark.parametrize("order", ["W", "H"])
@pytest.mark.parametrize("method", ["jmm", "bmm"])
def test_sparse_small_matches_oracle(lib, order, method):
    p = inputs.sparse_counts(F=300, N=700, density=0.02, K=12, seed=3)
    m, W, H = sparse_ctx(p, order)
    loss = m.step_joint(1) if method == "jmm" else m.step_alternating(1)
    step = O.sparse_kl_jmm_iteration if method == "jmm" else O.sparse_kl_bmm_iteration
    Wo, Ho = step(p.rows, p.col, p.val.astype(float), p.W0, p.H0, order=order)
    Wo, Ho = O.normalize(Wo, Ho)
    assert rel(W.double().cpu().numpy(), Wo) < 1e-4
    assert rel(H.double().cpu().numpy(), Ho) < 1e-4
    lo = O.sparse_kl_objective(p.rows, p.col, p.val.astype(float), p.W0, p.H0)
    assert loss == pytest.approx(lo, rel=1e-5)


def test_sparse_matches_dense_gpu_path(lib):
    """The sparse kernels and the dense kernels agree on the same (densified) data."""
    from paper_2106_15214_gb300.binding import NMF
    p = inputs.sparse_counts(F=200, N=300, density=0.05, K=8, seed=4)
    Vd = np.zeros((p.F, p.N))
    Vd[p.rows, p.col] = p.val
    m, W, H = sparse_ctx(p)
    ls = m.step_joint(3)
    md = NMF(p.F, p.N, 8, 1.0, precision="fp32")
    V2, W2, H2 = dev(Vd), dev(p.W0), dev(p.H0)
    md.set_dense(V2)
    md.set_factors(W2, H2)
    ld = md.step_joint(3)
    assert ls == pytest.approx(ld, rel=1e-5)
    assert rel(W.cpu().numpy(), W2.cpu().numpy()) < 1e-4


def test_sparse_gradient_and_finite_differences(lib):
    """Adjoint of the sparse objective: against the oracle's gradient and
    against central finite differences of the GPU objective (FP64 direction)."""
    import torch
    p = inputs.sparse_counts(F=150, N=220, density=0.05, K=6, seed=5)
    m, W, H = sparse_ctx(p)
    gW, gH = torch.empty_like(W), torch.empty_like(H)
    l = m.grad(gW, gH, want_loss=True)
    oW, oH = O.sparse_kl_gradients(p.rows, p.col, p.val.astype(float), p.W0, p.H0)
    assert np.max(np.abs(gW.double().cpu().numpy() - oW)) < 1e-4 * np.abs(oW).max()
    assert np.max(np.abs(gH.double().cpu().numpy() - oH)) < 1e-4 * np.abs(oH).max()
    lo = O.sparse_kl_objective(p.rows, p.col, p.val.astype(float), p.W0, p.H0)
    assert l == pytest.approx(lo, rel=1e-5)


def test_sparse_full_size_sampled(lib):
    """Full-size sparse KL problem (20000 x 100000, 0.1 %, K = 50), one JMM
    iteration; the sparse oracle runs at full size (scipy sparse products)."""
    p = inputs.sparse_counts()
    m, W, H = sparse_ctx(p)
    loss = m.step_joint(1)
    vals = p.val.astype(float)
    Wo, Ho = O.sparse_kl_jmm_iteration(p.rows, p.col, vals, p.W0, p.H0)
    Wo, Ho = O.normalize(Wo, Ho)
    assert rel(W.double().cpu().numpy(), Wo) < 2e-4
    assert rel(H.double().cpu().numpy(), Ho) < 2e-4
    lo = O.sparse_kl_objective(p.rows, p.col, vals, p.W0, p.H0)
    assert loss == pytest.approx(lo, rel=1e-5)


def pack(probs):
    V = np.concatenate([p.V.ravel() for p in probs])
    W = np.concatenate([p.W0.ravel() for p in probs])
    H = np.concatenate([p.H0.ravel() for p in probs])
    return V, W, H


def unpack(flat, shapes, which):
    out, o = [], 0
    for F, N, K in shapes:
        n = {"W": F * K, "H": K * N}[which]
        out.append(flat[o:o + n].reshape((F, K) if which == "W" else (K, N)))
        o += n
    return out


@pytest.mark.parametrize("method", ["jmm", "bmm"])
def test_batched_small_matches_oracle(lib, method):
    from paper_2106_15214_gb300.binding import BatchedNMF
    probs = inputs.batched_hyperspectral(count=24, F_range=(5, 70), N_range=(3, 300), K_range=(1, 33), seed=9)
    shapes = [p.shape for p in probs]
    Vp, Wp, Hp = pack(probs)
    b = BatchedNMF(shapes, 1.5)
    Vd, Wd, Hd = dev(Vp), dev(Wp), dev(Hp)
    b.set_packed(Vd, Wd, Hd)
    total = b.step_joint(2) if method == "jmm" else b.step_alternating(2)
    per = b.losses()
    Ws = unpack(Wd.double().cpu().numpy(), shapes, "W")
    Hs = unpack(Hd.double().cpu().numpy(), shapes, "H")
    for i, p in enumerate(probs):
        Wo, Ho, lo = O.run(p.V, p.W0, p.H0, 1.5, method=method, iters=2)
        assert rel(Ws[i], Wo) < 2e-4, i
        assert rel(Hs[i], Ho) < 2e-4, i
        assert per[i] == pytest.approx(lo[1], rel=1e-5)
    assert total == pytest.approx(sum(per), rel=1e-12)


def test_batched_full_size_sampled(lib):
    """512 instances in one context, one JMM iteration; 12 sampled instances
    are checked against the oracle entry by entry."""
    from paper_2106_15214_gb300.binding import BatchedNMF
    probs = inputs.batched_hyperspectral()
    shapes = [p.shape for p in probs]
    Vp, Wp, Hp = pack(probs)
    b = BatchedNMF(shapes, 1.5)
    Vd, Wd, Hd = dev(Vp), dev(Wp), dev(Hp)
    b.set_packed(Vd, Wd, Hd)
    b.step_joint(1)
    per = b.losses()
    Ws = unpack(Wd.double().cpu().numpy(), shapes, "W")
    Hs = unpack(Hd.double().cpu().numpy(), shapes, "H")
    rng = np.random.default_rng(0)
    for i in rng.choice(len(probs), size=12, replace=False):
        p = probs[i]
        Wo, Ho, lo = O.run(p.V, p.W0, p.H0, 1.5, iters=1)
        assert rel(Ws[i], Wo) < 2e-4, i
        assert rel(Hs[i], Ho) < 2e-4, i
        assert per[i] == pytest.approx(lo[0], rel=1e-5)


def test_malformed_csr_is_rejected_before_use(lib):
    import torch
    from paper_2106_15214_gb300.binding import NMF, NMFError, NMF_EINVAL
    p = inputs.sparse_counts(F=50, N=60, density=0.05, K=3, seed=6)
    col = p.col.copy()
    col[3] = 60                                   # out of range, caught on the device before any use
    m = NMF(p.F, p.N, 3, 1.0, precision="fp32")
    m.set_csr(dev(p.rowptr, torch.int32), dev(col, torch.int32), dev(p.val))
    m.set_factors(dev(p.W0), dev(p.H0))
    with pytest.raises(NMFError) as ei:
        m.step_joint(1)
    assert ei.value.code == NMF_EINVAL


def test_batched_autotune(lib):
    """nmf_autotune on a batched context: picks one of the candidate chunk
    caps, leaves the packed factors exactly as it found them, a second context
    of the same shapes gets the cached choice, and the tuned context still
    matches the oracle."""
    import torch
    from paper_2106_15214_gb300.binding import BatchedNMF
    probs = inputs.batched_hyperspectral(count=40, F_range=(20, 200), N_range=(50, 3000), K_range=(2, 24), seed=13)
    shapes = [p.shape for p in probs]
    Vp, Wp, Hp = pack(probs)
    b = BatchedNMF(shapes, 1.5)
    Vd, Wd, Hd = dev(Vp), dev(Wp), dev(Hp)
    b.set_packed(Vd, Wd, Hd)
    W0d, H0d = Wd.clone(), Hd.clone()
    cap = b.autotune(trials=2)
    assert cap in (8, 16, 32, 64, 128)
    torch.cuda.synchronize()
    assert torch.equal(Wd, W0d) and torch.equal(Hd, H0d)
    b2 = BatchedNMF(shapes, 1.5)
    b2.set_packed(dev(Vp), dev(Wp), dev(Hp))
    assert b2.autotune(trials=2) == cap
    b.step_joint(2)
    per = b.losses()
    Ws = unpack(Wd.double().cpu().numpy(), shapes, "W")
    Hs = unpack(Hd.double().cpu().numpy(), shapes, "H")
    for i in (0, 7, 19, 39):
        p = probs[i]
        Wo, Ho, lo = O.run(p.V, p.W0, p.H0, 1.5, iters=2)
        assert rel(Ws[i], Wo) < 2e-4, i
        assert rel(Hs[i], Ho) < 2e-4, i
        assert per[i] == pytest.approx(lo[1], rel=1e-5)


def test_single_problem_autotune_fp64(lib):
    """The autotuner on a single FP64 problem keeps FP64 parity (1e-12)."""
    from paper_2106_15214_gb300.binding import NMF
    p = inputs.dense_kl_small()
    F, N, K = p.shape
    m = NMF(F, N, K, 1.0, precision="fp64")
    import torch
    V, W, H = dev(p.V, torch.float64), dev(p.W0, torch.float64), dev(p.H0, torch.float64)
    m.set_dense(V)
    m.set_factors(W, H)
    assert m.autotune(trials=2) in (8, 16, 32, 64, 128)
    m.step_joint(3)
    Wo, Ho, _ = O.run(p.V, p.W0, p.H0, 1.0, iters=3)
    assert rel(W.cpu().numpy(), Wo) < 1e-12
    assert rel(H.cpu().numpy(), Ho) < 1e-12
