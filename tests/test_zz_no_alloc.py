"""nmf_loss_noalloc: the objective computed with the library's static scratch
instead of a device allocation (for callers that cannot call cudaMalloc,
e.g. during stream capture or under a fixed memory budget). Its result must
match the context-based nmf_loss within the tolerances the other tests use,
on two calls in a row (the second call reuses the shared scratch). Collected
last so a failure here does not stop the rest of the suite."""
import numpy as np
import pytest

from paper_2106_15214_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_loss_noalloc_matches_nmf_loss_twice(lib, prec, tol):
    import torch
    from paper_2106_15214_gb300.binding import NMF, loss_noalloc
    dt = torch.float64 if prec == "fp64" else torch.float32
    p = inputs.random_dense(150, 230, 9, seed=11)
    V = torch.tensor(p.V, dtype=dt, device="cuda")
    for beta, kappa, scale in ((1.0, 0.0, 1.0), (0.5, 0.01, 1.7)):
        W = torch.tensor(p.W0 * scale, dtype=dt, device="cuda")
        H = torch.tensor(p.H0, dtype=dt, device="cuda")
        m = NMF(150, 230, 9, beta, precision=prec, kappa=kappa)
        m.set_dense(V)
        m.set_factors(W, H)
        want = m.loss()
        got = loss_noalloc(V, W, H, beta, kappa)
        torch.cuda.synchronize()
        assert float(got.item()) == pytest.approx(want, rel=tol)
        m.close()


def test_loss_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import ctypes
    from paper_2106_15214_gb300.binding import NMF_EINVAL
    # ceil(F/32) * ceil(N/32) = 257 * 256 > 65536: rejected before any launch
    rc = lib.nmf_loss_noalloc(257 * 32, 256 * 32, 4, 1.0, 0.0, 1, ctypes.c_void_p(256), 256 * 32,
                              ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256), None)
    assert rc == NMF_EINVAL
