"""The bounded-wait timeout path on the GPU, without a fault or a hang.

The persistent step kernel (one cooperative launch per JMM iteration, opted
into with NMF_TC_STEP=1) separates its phases by grid barriers whose waits
give up after a bound. nmf_set_barrier_test shortens that bound to a few
milliseconds and makes the barriers expect one arrival more than there are
blocks, a flag nothing sets: every wait then runs out, the kernel records
NMF_ETIMEOUT and runs to its end without further work, and the step returns
NMF_ETIMEOUT with W and H restored. Afterwards the same context, with the
defaults back and the status cleared, computes the oracle's iterate.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2106_15214_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_grid_barrier_timeout_returns_etimeout_and_restores(lib):
    import torch
    from paper_2106_15214_gb300.binding import NMF, NMF_ETIMEOUT, NMFError, check
    q = inputs.random_dense(200, 300, 20, seed=4)
    os.environ["NMF_TC_STEP"] = "1"
    try:
        m = NMF(200, 300, 20, 1.0, precision="tf32", order="W")
        V = torch.tensor(q.V, dtype=torch.float32, device="cuda")
        W = torch.tensor(q.W0, dtype=torch.float32, device="cuda")
        H = torch.tensor(q.H0, dtype=torch.float32, device="cuda")
        W0, H0 = W.clone(), H.clone()
        m.set_dense(V)
        m.set_factors(W, H)
        check(lib.nmf_set_barrier_test(m._ctx, 2_000_000, 1), "nmf_set_barrier_test")
        with pytest.raises(NMFError) as e:
            m.step_joint(1)
        assert e.value.code == NMF_ETIMEOUT
        torch.cuda.synchronize()
        assert torch.equal(W, W0) and torch.equal(H, H0)
        # defaults back, status cleared: the context works again
        check(lib.nmf_set_barrier_test(m._ctx, 1_000_000_000, 0), "nmf_set_barrier_test")
        m.set_factors(W, H)
        m.step_joint(1)
        Wo, Ho = O.normalize(*O.jmm_iteration(q.V, q.W0, q.H0, 1.0))
        assert np.max(np.abs(W.double().cpu().numpy() - Wo) / Wo) < 1e-2
        assert np.max(np.abs(H.double().cpu().numpy() - Ho) / Ho) < 1e-2
        m.close()
    finally:
        del os.environ["NMF_TC_STEP"]
