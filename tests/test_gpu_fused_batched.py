"""Many problems in one fused single-read launch (batched contexts, NMF_BF16)
against the FP64 oracle, problem by problem.

The batched fused sweep runs every problem's 128-column batches as work items
on clusters of ceil(max F / 128) blocks (one launch per iteration), reading
each problem's V, W~ and H~^T through its own tensor maps. Same bars as the
single-problem fused path: 3e-2 relative on W and H after one iteration,
5e-3 on the objective (bf16 contractions, TF32 product).
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_15214_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_WH, TOL_D = 3e-2, 5e-3


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def pack(probs):
    return (np.concatenate([p.V.ravel() for p in probs]), np.concatenate([p.W0.ravel() for p in probs]),
            np.concatenate([p.H0.ravel() for p in probs]))


def unpack(flat, shapes, which):
    out, o = [], 0
    for F, N, K in shapes:
        n = {"W": F * K, "H": K * N}[which]
        out.append(flat[o:o + n].reshape((F, K) if which == "W" else (K, N)))
        o += n
    return out


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def run_batched(probs, beta, iters=1):
    from paper_2106_15214_gb300.binding import BatchedNMF
    shapes = [p.shape for p in probs]
    Vp, Wp, Hp = pack(probs)
    b = BatchedNMF(shapes, beta, precision="bf16", order="H")
    Vd, Wd, Hd = dev(Vp), dev(Wp), dev(Hp)
    b.set_packed(Vd, Wd, Hd)
    total = b.step_joint(iters)
    per = b.losses()
    Ws = unpack(Wd.double().cpu().numpy(), shapes, "W")
    Hs = unpack(Hd.double().cpu().numpy(), shapes, "H")
    b.close()
    return Ws, Hs, per, total


@pytest.mark.parametrize("beta", [1.5, 0.0, 1.0])
def test_batched_fused_matches_oracle(lib, beta):
    """24 problems, F in [5, 250] (clusters of 2 blocks; some problems use one
    row tile), N in [3, 700] (ragged, rows not 16-byte aligned: the padded
    copy of V), K in [1, 32]."""
    probs = inputs.batched_hyperspectral(count=24, F_range=(5, 250), N_range=(3, 700), K_range=(1, 32), seed=11)
    Ws, Hs, per, total = run_batched(probs, beta)
    for i, p in enumerate(probs):
        Wo, Ho, lo = O.run(p.V, p.W0, p.H0, beta, iters=1, order="H", eps=1e-30)
        assert np.all(np.isfinite(Ws[i])) and np.all(np.isfinite(Hs[i])), i
        assert rel(Ws[i], Wo) < TOL_WH, i
        assert rel(Hs[i], Ho) < TOL_WH, i
        assert per[i] == pytest.approx(lo[0], rel=TOL_D), i
    assert total == pytest.approx(sum(per), rel=1e-12)


def test_batched_fused_several_iterations(lib):
    probs = inputs.batched_hyperspectral(count=10, F_range=(100, 200), N_range=(200, 1500), K_range=(4, 20), seed=3)
    Ws, Hs, per, _ = run_batched(probs, 1.5, iters=5)
    for i, p in enumerate(probs):
        _, _, lo = O.run(p.V, p.W0, p.H0, 1.5, iters=5, order="H", eps=1e-30)
        assert per[i] == pytest.approx(lo[4], rel=TOL_D), i
        assert O.D_beta(p.V, Ws[i] @ Hs[i], 1.5) == pytest.approx(lo[5], rel=TOL_D), i


def test_batched_fused_full_size_sampled(lib):
    """The 512-problem workload, one iteration; 12 sampled problems against
    the oracle entry by entry."""
    probs = inputs.batched_hyperspectral()
    Ws, Hs, per, _ = run_batched(probs, 1.5)
    rng = np.random.default_rng(1)
    for i in rng.choice(len(probs), size=12, replace=False):
        p = probs[i]
        Wo, Ho, lo = O.run(p.V, p.W0, p.H0, 1.5, iters=1, order="H", eps=1e-30)
        assert rel(Ws[i], Wo) < TOL_WH, i
        assert rel(Hs[i], Ho) < TOL_WH, i
        assert per[i] == pytest.approx(lo[0], rel=TOL_D), i


def test_batched_fused_autotune_and_determinism(lib):
    """nmf_autotune picks the batches per work item; the result of a step does
    not depend on the choice beyond rounding (the slices differ) and repeated
    steps from the same start are bitwise equal."""
    from paper_2106_15214_gb300.binding import BatchedNMF
    probs = inputs.batched_hyperspectral(count=16, F_range=(64, 256), N_range=(256, 3000), K_range=(4, 32), seed=5)
    shapes = [p.shape for p in probs]
    Vp, Wp, Hp = pack(probs)
    outs = []
    for tune in (False, True, True):
        b = BatchedNMF(shapes, 1.5, precision="bf16", order="H")
        Vd, Wd, Hd = dev(Vp), dev(Wp), dev(Hp)
        b.set_packed(Vd, Wd, Hd)
        if tune:
            assert b.autotune(2) in (8, 16, 32, 64, 128)
        b.step_joint(1)
        outs.append((Wd.cpu().numpy(), Hd.cpu().numpy(), b.losses()))
        b.close()
    assert np.array_equal(outs[1][0], outs[2][0]) and np.array_equal(outs[1][1], outs[2][1])
    Ws = unpack(outs[1][0].astype(np.float64), shapes, "W")
    for i, p in enumerate(probs):
        Wo, Ho, lo = O.run(p.V, p.W0, p.H0, 1.5, iters=1, order="H", eps=1e-30)
        assert rel(Ws[i], Wo) < TOL_WH, i


def test_batched_fused_rejects_other_forms(lib):
    from paper_2106_15214_gb300.binding import BatchedNMF, NMF_EUNSUPPORTED, NMFError
    probs = inputs.batched_hyperspectral(count=3, F_range=(20, 40), N_range=(50, 90), K_range=(2, 5), seed=2)
    shapes = [p.shape for p in probs]
    Vp, Wp, Hp = pack(probs)
    for kw, call in ((dict(order="W"), "joint"), (dict(order="H"), "alternating")):
        b = BatchedNMF(shapes, 1.0, precision="bf16", **kw)
        b.set_packed(dev(Vp), dev(Wp), dev(Hp))
        with pytest.raises(NMFError) as e:
            (b.step_joint if call == "joint" else b.step_alternating)(1)
        assert e.value.code == NMF_EUNSUPPORTED
        b.close()
    big = [(30, 60, 40)]                             # K > 32
    b = BatchedNMF(big, 1.0, precision="bf16", order="H")
    W, H = inputs.uniform_init(30, 60, 40, seed=1)
    b.set_packed(dev(np.ones(30 * 60)), dev(W), dev(H))
    with pytest.raises(NMFError) as e:
        b.step_joint(1)
    assert e.value.code == NMF_EUNSUPPORTED
    b.close()


def test_padded_v_is_rebuilt_with_the_plan(lib):
    """A context whose V rows are not 16-byte aligned streams a padded copy of
    V; a precision change rebuilds every buffer of the context, the padded
    copy included, and the next steps read the new one (one problem, TF32 ->
    FP32 -> TF32, and the fused BF16 path)."""
    from paper_2106_15214_gb300.binding import NMF, PRECISIONS
    q = inputs.random_dense(200, 333, 20, seed=8, beta=1.0)           # N % 4 == 1
    for prec, order in (("tf32", "W"), ("bf16", "H")):
        m = NMF(200, 333, 20, 1.0, precision=prec, order=order)
        V = dev(q.V)
        W, H = dev(q.W0), dev(q.H0)
        m.set_dense(V)
        m.set_factors(W, H)
        m.step_joint(1)
        for p in ("fp32", prec):                                       # two rebuilds of the plan
            m.precision = PRECISIONS[p]
            m.set_options()
            W.copy_(dev(q.W0))
            H.copy_(dev(q.H0))
            m.set_factors(W, H)
            m.step_joint(1)
        Wo, Ho, _ = O.run(q.V, q.W0, q.H0, 1.0, iters=1, order=order, eps=1e-30)
        assert rel(W.double().cpu().numpy(), Wo) < TOL_WH
        assert rel(H.double().cpu().numpy(), Ho) < TOL_WH
        m.close()


def test_batched_cluster_wait_timeout_returns_etimeout(lib):
    """The many-problem launch shares the single-problem kernel's bounded
    cluster waits: with one arrival too many expected and a 2 ms limit every
    such wait gives up, the step returns NMF_ETIMEOUT with W and H restored,
    and with the defaults back the same context computes the oracle's iterate."""
    import torch
    from paper_2106_15214_gb300.binding import BatchedNMF, NMF_ETIMEOUT, NMFError, check
    probs = inputs.batched_hyperspectral(count=6, F_range=(100, 250), N_range=(300, 900), K_range=(4, 24), seed=7)
    shapes = [p.shape for p in probs]
    Vp, Wp, Hp = pack(probs)
    b = BatchedNMF(shapes, 1.5, precision="bf16", order="H")
    Vd, Wd, Hd = dev(Vp), dev(Wp), dev(Hp)
    W1, H1 = Wd.clone(), Hd.clone()
    b.set_packed(Vd, Wd, Hd)
    check(lib.nmf_set_barrier_test(b._ctx, 2_000_000, 1), "nmf_set_barrier_test")
    with pytest.raises(NMFError) as e:
        b.step_joint(1)
    assert e.value.code == NMF_ETIMEOUT
    torch.cuda.synchronize()
    assert torch.equal(Wd, W1) and torch.equal(Hd, H1)
    check(lib.nmf_set_barrier_test(b._ctx, 1_000_000_000, 0), "nmf_set_barrier_test")
    b.set_packed(Vd, Wd, Hd)
    b.step_joint(1)
    Ws = unpack(Wd.double().cpu().numpy(), shapes, "W")
    Hs = unpack(Hd.double().cpu().numpy(), shapes, "H")
    b.close()
    for i, p in enumerate(probs):
        Wo, Ho, _ = O.run(p.V, p.W0, p.H0, 1.5, iters=1, order="H", eps=1e-30)
        assert rel(Ws[i], Wo) < TOL_WH and rel(Hs[i], Ho) < TOL_WH, i
