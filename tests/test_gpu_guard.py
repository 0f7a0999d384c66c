"""The small-Vt guard of the single-precision paths (FP32 SIMT and TF32
tensor cores) against the FP64 oracle.

One row of W and one column of H are scaled down so that the product at their
crossing is tiny, while A = V Vt^(beta-2) and B = Vt^(beta-1) there still fit
in float. In float the power Vt^(beta-2) itself overflows at that entry
(checked below with numpy's float32), so without the guard the updates of
that row and column turn into Inf / NaN; with it they match the oracle within
the paths' usual tolerances. Handling of small values: Sec. 4.1.3.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

F, N, K = 64, 96, 4
F0, N0 = 5, 17


def planted(beta, s, seed=31):
    rng = np.random.default_rng(seed)
    W = rng.uniform(0.5, 1.5, size=(F, K))
    H = rng.uniform(0.5, 1.5, size=(K, N))
    W[F0, :] *= s
    H[:, N0] *= s
    # V near the product, so that A and B are of the order of Vt^(beta-1)
    V = (W @ H) * rng.uniform(0.8, 1.2, size=(F, N))
    return V, W, H


CASES = [
    # beta, scale s; the crossing's product is about K s^2
    (0.5, 1e-14),    # Vt ~ 4e-28 < 2^-80: Vt^-1.5 ~ 1e41 overflows float, A, B ~ 5e13 fit
    (-1.0, 5e-9),    # Vt ~ 1e-16 < 2^-40: Vt^-3 ~ 1e48 overflows, A, B ~ 1e32 fit
    (0.0, 1e-13),    # Itakura-Saito, Vt ~ 4e-26 < 2^-60: guarded branch, no float overflow either way
]


@pytest.mark.parametrize("beta,s", CASES)
# the objective is dominated by the planted entries, so on the tensor cores
# their TF32 product error (~1e-3 relative, squared-error-like terms near an
# exact fit) is not averaged away: 3e-2 on D there instead of the usual 2e-3
@pytest.mark.parametrize("prec,tol,tol_d", [("fp32", 2e-4, 1e-5), ("tf32", 1e-2, 3e-2)])
@pytest.mark.parametrize("order", ["W", "H"])
def test_tiny_products_match_oracle(lib, beta, s, prec, tol, tol_d, order):
    import torch
    from paper_2106_15214_gb300.binding import NMF
    V, W0, H0 = planted(beta, s)
    vt_min = float((W0 @ H0)[F0, N0])
    if beta < 0.5 + 1e-9 and beta != 0.0:
        with np.errstate(over="ignore"):
            assert np.isinf(np.float32(vt_min) ** np.float32(beta - 2.0))
    Vt = torch.tensor(V, dtype=torch.float32, device="cuda")
    Wt = torch.tensor(W0, dtype=torch.float32, device="cuda")
    Ht = torch.tensor(H0, dtype=torch.float32, device="cuda")
    Vo, Wo0, Ho0 = (t.double().cpu().numpy() for t in (Vt, Wt, Ht))
    m = NMF(F, N, K, beta, precision=prec, order=order)
    m.set_dense(Vt)
    m.set_factors(Wt, Ht)
    loss = m.step_joint(1)
    Wo, Ho = O.normalize(*O.jmm_iteration(Vo, Wo0, Ho0, beta, order=order, eps=1e-30))
    Wg, Hg = Wt.double().cpu().numpy(), Ht.double().cpu().numpy()
    assert np.all(np.isfinite(Wg)) and np.all(np.isfinite(Hg))
    assert np.max(np.abs(Wg - Wo) / Wo) < tol
    assert np.max(np.abs(Hg - Ho) / Ho) < tol
    D0 = O.D_beta(Vo, Wo0 @ Ho0, beta)
    assert loss == pytest.approx(D0, rel=tol_d)
    m.close()
