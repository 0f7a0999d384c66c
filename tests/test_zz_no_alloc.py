"""nmf_loss_noalloc: the objective computed with the library's static scratch
instead of a device allocation, for callers that cannot call cudaMalloc (code
running under stream capture, hosts with a fixed memory budget or their own
pool, latency-critical loops).

Its result must match the FP64 oracle's D_beta within the tolerances the
other parity tests use, on two calls in a row (the second call reuses the
shared scratch the first one left behind), and it must agree with the
context-based nmf_loss. Collected last, so that a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import oracle as O
from paper_2106_15214_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_loss_noalloc_matches_oracle_twice(lib, prec, tol):
    import torch
    from paper_2106_15214_gb300.binding import NMF, loss_noalloc
    dt = torch.float64 if prec == "fp64" else torch.float32
    p = inputs.random_dense(150, 230, 9, seed=11)
    V = torch.tensor(p.V, dtype=dt, device="cuda")
    for beta, kappa, scale in ((1.0, 0.0, 1.0), (0.5, 0.01, 1.7), (0.0, 0.0, 0.9)):
        Wn, Hn = p.W0 * scale, p.H0
        W = torch.tensor(Wn, dtype=dt, device="cuda")
        H = torch.tensor(Hn, dtype=dt, device="cuda")
        # the oracle sees exactly the values the GPU sees (rounded to dt)
        Vo, Wo, Ho = (t.double().cpu().numpy() for t in (V, W, H))
        want = O.D_beta(Vo + kappa, Wo @ Ho + kappa, beta)
        for _ in range(2):
            got = loss_noalloc(V, W, H, beta, kappa)
            torch.cuda.synchronize()
            assert float(got.item()) == pytest.approx(want, rel=tol)
        m = NMF(150, 230, 9, beta, precision=prec, kappa=kappa)
        m.set_dense(V)
        m.set_factors(W, H)
        assert m.loss() == pytest.approx(float(got.item()), rel=tol)
        m.close()


def test_loss_noalloc_rejects_sizes_beyond_its_scratch(lib):
    """ceil(F/32) * ceil(N/32) = 257 * 256 > 65536 tiles: NMF_EINVAL before
    any launch. The buffers are real device allocations of the stated sizes,
    so even a regressed size check could not read outside them."""
    import torch
    from paper_2106_15214_gb300.binding import NMF_EINVAL, NMFError, loss_noalloc
    F, N, K = 257 * 32, 256 * 32, 4
    V = torch.ones((F, N), dtype=torch.float32, device="cuda")
    W = torch.ones((F, K), dtype=torch.float32, device="cuda")
    H = torch.ones((K, N), dtype=torch.float32, device="cuda")
    with pytest.raises(NMFError) as e:
        loss_noalloc(V, W, H, 1.0)
    assert e.value.code == NMF_EINVAL
    # one row fewer fits (256 * 256 tiles) and gives d_1(1 | K) per entry
    got = loss_noalloc(V[:F - 32], W[:F - 32], H, 1.0)
    torch.cuda.synchronize()
    want = (F - 32) * N * float(O.beta_divergence(1.0, float(K), 1.0))
    assert float(got.item()) == pytest.approx(want, rel=1e-6)
