"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: hand-derived closed
forms, textbook/library routines, the majorisation properties of G (Sec. 3.1),
the argmin property of every half-update found by an independent 1-D root
search on the numerical derivative of G (Sec. 3.2), fixed points, symmetry,
monotone descent (eq. desc_lemm), Table 2's simplified forms and finite
differences. A plausible mistake in the oracle (a wrong exponent, a swapped
chi, a transposed product, a dropped kappa) fails at least one of them.
"""
import os

import numpy as np
import pytest
from scipy import optimize, special

import oracle as O
from paper_2106_15214_gb300 import inputs

BETAS = [-1.0, 0.0, 0.5, 1.0, 1.5, 2.0, 3.0]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(seed=0, F=3, N=4, K=2):
    rng = np.random.default_rng(seed)
    V = rng.uniform(0.2, 2.0, size=(F, N))
    Wt = rng.uniform(0.2, 1.5, size=(F, K))
    Ht = rng.uniform(0.2, 1.5, size=(K, N))
    return V, Wt, Ht


# --------------------------------------------------------------------------
# d_beta and gamma
# --------------------------------------------------------------------------

def test_beta_divergence_golden_values():
    """Hand-derived values of eq. beta-div (tests/golden/beta_divergence_values.txt)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "beta_divergence_values.txt"), comments="#")
    assert rows.shape[0] >= 10
    for beta, x, y, val in rows:
        got = O.beta_divergence(x, y, beta)
        assert got == pytest.approx(val, rel=1e-14, abs=1e-15), (beta, x, y)


@pytest.mark.parametrize("beta", BETAS)
def test_beta_divergence_is_a_divergence(beta):
    rng = np.random.default_rng(1)
    x = rng.uniform(0.05, 5, 1000)
    y = rng.uniform(0.05, 5, 1000)
    assert np.all(O.beta_divergence(x, y, beta) >= -1e-12)
    assert np.allclose(O.beta_divergence(x, x, beta), 0.0, atol=1e-12)


def test_beta_divergence_special_cases_match_textbook():
    rng = np.random.default_rng(2)
    x = rng.uniform(0.05, 5, 500)
    y = rng.uniform(0.05, 5, 500)
    # quadratic loss (beta = 2) is half the squared error
    assert np.allclose(O.beta_divergence(x, y, 2.0), 0.5 * (x - y) ** 2, rtol=1e-12)
    # generalised KL (beta = 1) is scipy's kl_div
    assert np.allclose(O.beta_divergence(x, y, 1.0), special.kl_div(x, y), rtol=1e-12)
    # the general formula tends to KL and IS at beta -> 1 and beta -> 0
    for b0 in (0.0, 1.0):
        for eps in (1e-6, -1e-6):
            assert np.allclose(O.beta_divergence(x, y, b0 + eps), O.beta_divergence(x, y, b0),
                               rtol=2e-5, atol=1e-8)


def test_gamma_values():
    assert O.gamma(0.0) == 0.5 and O.gamma(-1.0) == pytest.approx(1 / 3)
    assert O.gamma(0.5) == pytest.approx(2 / 3)
    assert O.gamma(1.0) == O.gamma(1.5) == O.gamma(2.0) == 1.0
    assert O.gamma(3.0) == 0.5 and O.gamma(5.0) == 0.25


def test_objective_is_sum_of_elementwise():
    V, W, H = tiny()
    WH = W @ H
    brute = sum(float(O.beta_divergence(V[f, n], WH[f, n], 0.5))
                for f in range(3) for n in range(4))
    assert O.D_beta(V, WH, 0.5) == pytest.approx(brute, rel=1e-14)


# --------------------------------------------------------------------------
# Table 1 and the joint majoriser G (Sec. 3.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("beta", BETAS)
def test_table1_decomposition(beta):
    rng = np.random.default_rng(3)
    v = rng.uniform(0.1, 4, 400)
    y = rng.uniform(0.1, 4, 400)
    conv, conc, const = O.divergence_parts(v, y, beta)
    assert np.allclose(conv + conc + const, O.beta_divergence(v, y, beta), rtol=1e-11, atol=1e-12)
    h = 1e-3
    c2 = lambda part: (O.divergence_parts(v, y + h, beta)[part] - 2 * O.divergence_parts(v, y, beta)[part]
                       + O.divergence_parts(v, y - h, beta)[part]) / h ** 2
    assert np.all(c2(0) >= -1e-6), "convex part must be convex in y"
    assert np.all(c2(1) <= 1e-6), "concave part must be concave in y"
    # the tangent slope is the derivative of the concave part
    fd = (O.divergence_parts(v, y + 1e-6, beta)[1] - O.divergence_parts(v, y - 1e-6, beta)[1]) / 2e-6
    assert np.allclose(O.divergence_parts_dy(v, y, beta), fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("beta", BETAS)
def test_G_is_a_tight_majoriser(beta):
    V, Wt, Ht = tiny(4)
    D0 = O.D_beta(V, Wt @ Ht, beta)
    assert O.auxiliary_G(V, Wt, Ht, Wt, Ht, beta) == pytest.approx(D0, rel=1e-12)
    rng = np.random.default_rng(5)
    for _ in range(300):
        W = Wt * np.exp(rng.normal(0, 0.7, Wt.shape))
        H = Ht * np.exp(rng.normal(0, 0.7, Ht.shape))
        G = O.auxiliary_G(V, W, H, Wt, Ht, beta)
        D = O.D_beta(V, W @ H, beta)
        assert G >= D - 1e-10 * max(1.0, abs(D))


# --------------------------------------------------------------------------
# Every half-update is the exact per-entry argmin of G (Sec. 3.2)
# --------------------------------------------------------------------------

def _argmin_entry(fun, x0):
    """Root of the numerical derivative of a 1-D convex function, searched in log space."""
    def dfun(t):
        w = np.exp(t)
        h = 1e-6 * w
        return (fun(w + h) - fun(w - h)) / (2 * h)
    lo, hi = np.log(x0) - 12, np.log(x0) + 12
    return float(np.exp(optimize.brentq(dfun, lo, hi, xtol=1e-13, rtol=1e-13)))


def argmin_W(V, H, Wt, Ht, beta):
    W = Wt.copy()
    out = np.empty_like(Wt)
    for f in range(W.shape[0]):
        for k in range(W.shape[1]):
            def g(w):
                Wm = W.copy()
                Wm[f, k] = w
                return O.auxiliary_G(V, Wm, H, Wt, Ht, beta)
            out[f, k] = _argmin_entry(g, Wt[f, k])
    return out


def argmin_H(V, W, Wt, Ht, beta):
    H = Ht.copy()
    out = np.empty_like(Ht)
    for k in range(H.shape[0]):
        for n in range(H.shape[1]):
            def g(h):
                Hm = H.copy()
                Hm[k, n] = h
                return O.auxiliary_G(V, W, Hm, Wt, Ht, beta)
            out[k, n] = _argmin_entry(g, Ht[k, n])
    return out


@pytest.mark.parametrize("beta", BETAS)
def test_jmm_updates_are_argmins_of_G(beta):
    V, Wt, Ht = tiny(6)
    # W first (Algorithm 2, L = 1): W = argmin G(., Ht | Wt, Ht), then H = argmin G(W, . | Wt, Ht)
    W, H = O.jmm_iteration(V, Wt, Ht, beta, L=1, order="W")
    Wb = argmin_W(V, Ht, Wt, Ht, beta)
    assert np.allclose(W, Wb, rtol=1e-7)
    Hb = argmin_H(V, W, Wt, Ht, beta)
    assert np.allclose(H, Hb, rtol=1e-7)
    # H first (inverted order)
    W2, H2 = O.jmm_iteration(V, Wt, Ht, beta, L=1, order="H")
    Hb2 = argmin_H(V, Wt, Wt, Ht, beta)
    assert np.allclose(H2, Hb2, rtol=1e-7)
    Wb2 = argmin_W(V, H2, Wt, Ht, beta)
    assert np.allclose(W2, Wb2, rtol=1e-7)


@pytest.mark.parametrize("beta", [0.0, 1.0, 1.5, 3.0])
def test_jmm_subiterations_are_argmins_of_G(beta):
    """L = 2: the second inner pass minimises the SAME G (tilde point fixed)."""
    V, Wt, Ht = tiny(7)
    W, H = O.jmm_iteration(V, Wt, Ht, beta, L=2, order="W")
    W1 = argmin_W(V, Ht, Wt, Ht, beta)
    H1 = argmin_H(V, W1, Wt, Ht, beta)
    W2 = argmin_W(V, H1, Wt, Ht, beta)
    H2 = argmin_H(V, W2, Wt, Ht, beta)
    assert np.allclose(W, W2, rtol=1e-7)
    assert np.allclose(H, H2, rtol=1e-7)


@pytest.mark.parametrize("beta", BETAS)
def test_bmm_updates_are_argmins_of_block_majorisers(beta):
    """BMM's W update minimises G(., H | W, H); its H update minimises
    G(W_new, . | W_new, H) (the majoriser rebuilt at the new W, eqs. Wll, Hll)."""
    V, W0, H0 = tiny(8)
    W, H = O.bmm_iteration(V, W0, H0, beta, order="W")
    assert np.allclose(W, argmin_W(V, H0, W0, H0, beta), rtol=1e-7)
    assert np.allclose(H, argmin_H(V, W, W, H0, beta), rtol=1e-7)


def _argmin_entry_above(fun, x0, eps):
    """Minimiser over [eps, inf) of a 1-D convex function: eps when the
    numerical derivative there is >= 0, else the root of the derivative
    above eps (searched in log space)."""
    def dfun(t):
        w = np.exp(t)
        h = 1e-6 * w
        return (fun(w + h) - fun(w - h)) / (2 * h)
    if dfun(np.log(eps)) >= 0:
        return eps
    return float(np.exp(optimize.brentq(dfun, np.log(eps), np.log(x0) + 12, xtol=1e-13, rtol=1e-13)))


@pytest.mark.parametrize("beta", [0.0, 1.0, 1.5, 3.0])
@pytest.mark.parametrize("order", ["W", "H"])
def test_jmm_with_floor_is_the_constrained_argmin(beta, order):
    """With eps > 0 each half-update is the argmin of G over entries >= eps
    (the positivity constraint of eqs. Wll, Hll), and the second half uses the
    constrained first half. eps is set inside the range of the first
    unconstrained update so that part of it is clamped."""
    V, Wt, Ht = tiny(9)
    W0, H0 = O.jmm_iteration(V, Wt, Ht, beta, order=order)
    eps = float(np.median(W0 if order == "W" else H0))
    W, H = O.jmm_iteration(V, Wt, Ht, beta, order=order, eps=eps)

    def constrained_W(Hfix):
        out = np.empty_like(Wt)
        for f in range(Wt.shape[0]):
            for k in range(Wt.shape[1]):
                def g(w):
                    Wm = Wt.copy()
                    Wm[f, k] = w
                    return O.auxiliary_G(V, Wm, Hfix, Wt, Ht, beta)
                out[f, k] = _argmin_entry_above(g, Wt[f, k], eps)
        return out

    def constrained_H(Wfix):
        out = np.empty_like(Ht)
        for k in range(Ht.shape[0]):
            for n in range(Ht.shape[1]):
                def g(h):
                    Hm = Ht.copy()
                    Hm[k, n] = h
                    return O.auxiliary_G(V, Wfix, Hm, Wt, Ht, beta)
                out[k, n] = _argmin_entry_above(g, Ht[k, n], eps)
        return out

    if order == "W":
        Wb = constrained_W(Ht)
        assert (Wb == eps).sum() >= Wt.size // 3          # the constraint is active
        assert np.allclose(W, Wb, rtol=1e-7)
        assert np.allclose(H, constrained_H(W), rtol=1e-7)
    else:
        Hb = constrained_H(Wt)
        assert (Hb == eps).sum() >= Ht.size // 3
        assert np.allclose(H, Hb, rtol=1e-7)
        assert np.allclose(W, constrained_W(H), rtol=1e-7)
    # monotone descent survives the constraint while the iterate stays
    # feasible (no normalisation, which could rescale entries below eps)
    D = O.run(V, np.maximum(Wt, eps), np.maximum(Ht, eps), beta, iters=30, order=order, eps=eps,
              do_normalize=False)[2]
    assert np.all(np.diff(D) <= 1e-12 * D[:-1])


def test_jmm_with_kappa_is_jmm_on_shifted_problem():
    """kappa acts as a (K+1)-th constant component (Sec. 4.1.3): JMM on
    (V + kappa) with W augmented by a column of kappa and H by a row of ones,
    whose added entries are held fixed, gives the same update of W and H."""
    V, Wt, Ht = tiny(9)
    kappa = 0.3
    for beta in BETAS:
        W, H = O.jmm_iteration(V, Wt, Ht, beta, kappa=kappa)
        Vt = Wt @ Ht + kappa
        A = (V + kappa) / Vt ** (2 - beta)
        B = Vt ** (beta - 1)
        g = O.gamma(beta)
        Wk = Wt * ((A @ Ht.T) / (B @ Ht.T)) ** g           # chi(Ht, Ht) = Ht
        assert np.allclose(W, Wk, rtol=1e-12)
        # and the unaugmented argmin of the kappa-shifted G: same as above via the
        # augmented factors (the extra column is kappa, the extra row ones)
        Wa = np.hstack([Wt, np.full((3, 1), kappa)])
        Ha = np.vstack([Ht, np.ones((1, 4))])
        Wa_new = argmin_W(V + kappa, Ha, Wa, Ha, beta)
        assert np.allclose(W, Wa_new[:, :2], rtol=1e-7)


# --------------------------------------------------------------------------
# Relations between JMM and BMM, fixed points, symmetry, Table 2
# --------------------------------------------------------------------------

@pytest.mark.parametrize("beta", BETAS)
def test_first_half_of_jmm_equals_bmm(beta):
    """At L = 1 the W updates of JMM and BMM coincide (Sec. 4.1.1)."""
    V, W0, H0 = tiny(10)
    Wj, _ = O.jmm_iteration(V, W0, H0, beta)
    Wb, _ = O.bmm_iteration(V, W0, H0, beta)
    assert np.allclose(Wj, Wb, rtol=1e-13)


@pytest.mark.parametrize("beta", BETAS)
@pytest.mark.parametrize("method", ["jmm", "bmm"])
def test_exact_fixed_point(beta, method):
    rng = np.random.default_rng(11)
    W0 = rng.uniform(0.2, 1.5, (6, 3))
    H0 = rng.uniform(0.2, 1.5, (3, 7))
    V = W0 @ H0
    step = O.jmm_iteration if method == "jmm" else O.bmm_iteration
    for order in ("W", "H"):
        W, H = step(V, W0, H0, beta, order=order)
        assert np.allclose(W, W0, rtol=1e-13) and np.allclose(H, H0, rtol=1e-13)


@pytest.mark.parametrize("beta", BETAS)
def test_transpose_symmetry(beta):
    """H-first on V is W-first on V^T with (W, H) -> (H^T, W^T)."""
    V, Wt, Ht = tiny(12, F=5, N=6, K=3)
    W1, H1 = O.jmm_iteration(V, Wt, Ht, beta, order="H")
    Ht2, Wt2 = O.jmm_iteration(V.T, Ht.T, Wt.T, beta, order="W")
    assert np.allclose(W1, Wt2.T, rtol=1e-13) and np.allclose(H1, Ht2.T, rtol=1e-13)


def test_table2_simplified_forms():
    """Table 2: the H updates of BMM and JMM at beta = 0, 1, 2 (W updated first)."""
    V, Wt, Ht = tiny(13, F=5, N=7, K=3)
    ones = np.ones_like(V)
    Vt = Wt @ Ht
    # JMM
    W, H = O.jmm_iteration(V, Wt, Ht, 0.0)
    assert np.allclose(H, Ht * (((Wt ** 2 / W).T @ (V / Vt ** 2)) / (W.T @ (1 / Vt))) ** 0.5, rtol=1e-12)
    W, H = O.jmm_iteration(V, Wt, Ht, 1.0)
    assert np.allclose(H, Ht * (Wt.T @ (V / Vt)) / (W.T @ ones), rtol=1e-12)
    W, H = O.jmm_iteration(V, Wt, Ht, 2.0)
    assert np.allclose(H, Ht * (W.T @ V) / ((W ** 2 / Wt).T @ Vt), rtol=1e-12)
    # BMM (H's update uses the new W and the current H)
    W, H = O.bmm_iteration(V, Wt, Ht, 0.0)
    WH = W @ Ht
    assert np.allclose(H, Ht * ((W.T @ (V / WH ** 2)) / (W.T @ (1 / WH))) ** 0.5, rtol=1e-12)
    W, H = O.bmm_iteration(V, Wt, Ht, 1.0)
    assert np.allclose(H, Ht * (W.T @ (V / (W @ Ht))) / (W.T @ ones), rtol=1e-12)
    W, H = O.bmm_iteration(V, Wt, Ht, 2.0)
    assert np.allclose(H, Ht * (W.T @ V) / (W.T @ W @ Ht), rtol=1e-12)


def test_brute_force_scalar_loops():
    """Eq. jnt_update written entry by entry with scalar loops on 3 x 4 x 2."""
    V, Wt, Ht = tiny(14)
    F, N, K = 3, 4, 2
    for beta in BETAS:
        g = O.gamma(beta)
        vt = [[sum(Wt[f, k] * Ht[k, n] for k in range(K)) for n in range(N)] for f in range(F)]
        W = np.zeros((F, K))
        for f in range(F):
            for k in range(K):
                num = sum(V[f, n] * vt[f][n] ** (beta - 2) * Ht[k, n] for n in range(N))
                den = sum(vt[f][n] ** (beta - 1) * Ht[k, n] for n in range(N))
                W[f, k] = Wt[f, k] * (num / den) ** g
        def c1(w, wt):
            return wt ** (2 - beta) / w ** (1 - beta) if beta <= 2 else w
        def c2(w, wt):
            return w if beta < 1 else w ** beta / wt ** (beta - 1)
        H = np.zeros((K, N))
        for k in range(K):
            for n in range(N):
                num = sum(c1(W[f, k], Wt[f, k]) * V[f, n] * vt[f][n] ** (beta - 2) for f in range(F))
                den = sum(c2(W[f, k], Wt[f, k]) * vt[f][n] ** (beta - 1) for f in range(F))
                H[k, n] = Ht[k, n] * (num / den) ** g
        Wo, Ho = O.jmm_iteration(V, Wt, Ht, beta)
        assert np.allclose(Wo, W, rtol=1e-13) and np.allclose(Ho, H, rtol=1e-13)


# --------------------------------------------------------------------------
# Descent, normalisation, stopping rule (eq. desc_lemm, Sec. 4.1.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("beta", BETAS)
@pytest.mark.parametrize("method,L,order", [("jmm", 1, "W"), ("jmm", 1, "H"), ("jmm", 3, "W"),
                                            ("bmm", 1, "W"), ("bmm", 2, "H")])
def test_monotone_descent(beta, method, L, order):
    p = inputs.random_dense(10, 14, 3, seed=15)
    _, _, losses = O.run(p.V, p.W0, p.H0, beta, method=method, iters=150, L=L, order=order)
    assert np.all(np.diff(losses) <= 1e-12 * np.abs(losses[1:]))
    assert losses[-1] < losses[0]


def test_monotone_descent_with_kappa_and_zeros():
    p = inputs.random_dense(10, 14, 3, seed=16)
    V = p.V.copy()
    V[::3, ::2] = 0.0
    for beta in (0.0, 0.5, 1.0):
        _, _, losses = O.run(V, p.W0, p.H0, beta, iters=100, kappa=1e-3)
        assert np.all(np.isfinite(losses))
        assert np.all(np.diff(losses) <= 1e-12 * np.abs(losses[1:]))


@pytest.mark.parametrize("method", ["jmm", "bmm"])
def test_normalisation_leaves_the_product_trajectory_unchanged(method):
    """The updates are equivariant to W -> W D^-1, H -> D H (chi is homogeneous
    of degree 1), so normalising every iteration changes no product WH."""
    p = inputs.random_dense(8, 11, 3, seed=17)
    for beta in (0.0, 1.0, 1.5, 3.0):
        W1, H1, l1 = O.run(p.V, p.W0, p.H0, beta, method=method, iters=40, do_normalize=True)
        W2, H2, l2 = O.run(p.V, p.W0, p.H0, beta, method=method, iters=40, do_normalize=False)
        assert np.allclose(W1 @ H1, W2 @ H2, rtol=1e-10)
        assert np.allclose(l1, l2, rtol=1e-10)
        assert np.allclose(np.linalg.norm(W1, axis=0), 1.0, rtol=1e-13)


def test_stopping_rule_stops_at_first_iteration_meeting_it():
    p = inputs.random_dense(8, 11, 3, seed=18)
    tol = 1e-4
    _, _, losses = O.run(p.V, p.W0, p.H0, 1.0, iters=10000, tol=tol)
    rel = (losses[:-1] - losses[1:]) / losses[1:]
    assert rel[-1] <= tol and np.all(rel[:-1] > tol)


# --------------------------------------------------------------------------
# Gradient and KKT (Sec. 4.1.5)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("beta", BETAS)
@pytest.mark.parametrize("kappa", [0.0, 0.2])
def test_gradient_matches_finite_differences(beta, kappa):
    V, W, H = tiny(19, F=4, N=5, K=2)
    gW, gH = O.gradients(V, W, H, beta, kappa)
    rng = np.random.default_rng(20)
    for _ in range(5):
        dW = rng.normal(size=W.shape)
        dH = rng.normal(size=H.shape)
        eps = 1e-6
        Dp = O.D_beta(V + kappa, (W + eps * dW) @ (H + eps * dH) + kappa, beta)
        Dm = O.D_beta(V + kappa, (W - eps * dW) @ (H - eps * dH) + kappa, beta)
        fd = (Dp - Dm) / (2 * eps)
        an = np.sum(gW * dW) + np.sum(gH * dH)
        assert fd == pytest.approx(an, rel=1e-6, abs=1e-8)


def test_kkt_residual_vanishes_at_exact_fit_and_not_elsewhere():
    rng = np.random.default_rng(21)
    W0 = rng.uniform(0.2, 1.5, (6, 3))
    H0 = rng.uniform(0.2, 1.5, (3, 7))
    V = W0 @ H0
    for beta in BETAS:
        rW, rH = O.kkt_residuals(V, W0, H0, beta)
        assert rW < 1e-13 and rH < 1e-13
        rW, rH = O.kkt_residuals(V, W0 * 1.3, H0, beta)
        assert rW > 1e-3 or rH > 1e-3


def test_mu_ratio_is_the_gradient_split():
    """grad = (B - A) H^T: the MU denominator minus its numerator (BMM, L = 1)."""
    V, W, H = tiny(22)
    for beta in BETAS:
        WH = W @ H
        A = V * WH ** (beta - 2)
        B = WH ** (beta - 1)
        gW, gH = O.gradients(V, W, H, beta)
        assert np.allclose(gW, B @ H.T - A @ H.T, rtol=1e-12, atol=1e-13)
        assert np.allclose(gH, W.T @ B - W.T @ A, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------------------
# Sparse beta = 1 oracle against the dense oracle; batching
# --------------------------------------------------------------------------

def _small_sparse(seed=23, F=30, N=40, K=4, density=0.2):
    rng = np.random.default_rng(seed)
    mask = rng.uniform(size=(F, N)) < density
    V = np.where(mask, rng.geometric(0.3, size=(F, N)).astype(float), 0.0)
    rows, cols = np.nonzero(V)
    W, H = inputs.uniform_init(F, N, K, seed=seed)
    return V, rows, cols, V[rows, cols], W, H


@pytest.mark.parametrize("order", ["W", "H"])
def test_sparse_kl_matches_dense_oracle(order):
    V, rows, cols, vals, W, H = _small_sparse()
    Wd, Hd = O.jmm_iteration(V, W, H, 1.0, order=order)
    Ws, Hs = O.sparse_kl_jmm_iteration(rows, cols, vals, W, H, order=order)
    assert np.allclose(Ws, Wd, rtol=1e-12) and np.allclose(Hs, Hd, rtol=1e-12)
    Wd, Hd = O.bmm_iteration(V, W, H, 1.0, order=order)
    Ws, Hs = O.sparse_kl_bmm_iteration(rows, cols, vals, W, H, order=order)
    assert np.allclose(Ws, Wd, rtol=1e-12) and np.allclose(Hs, Hd, rtol=1e-12)
    assert O.sparse_kl_objective(rows, cols, vals, W, H) == pytest.approx(
        O.D_beta(V, W @ H, 1.0), rel=1e-12)
    gW, gH = O.gradients(V, W, H, 1.0)
    sW, sH = O.sparse_kl_gradients(rows, cols, vals, W, H)
    assert np.allclose(sW, gW, rtol=1e-11, atol=1e-12) and np.allclose(sH, gH, rtol=1e-11, atol=1e-12)


def test_sparse_generator_structure():
    p = inputs.sparse_counts(F=300, N=500, density=0.01, K=5)
    assert p.rowptr[-1] == p.col.size == round(0.01 * 300 * 500)
    lin = p.rows * p.N + p.col
    assert np.unique(lin).size == lin.size                     # no repeated position
    assert np.all(p.val >= 1) and np.all(p.val == np.round(p.val))


def test_batched_is_independent_runs():
    probs = inputs.batched_hyperspectral(count=3, N_range=(20, 40), F_range=(8, 12), K_range=(2, 4))
    outs = O.batched_run([(p.V, p.W0, p.H0) for p in probs], 1.5, iters=3)
    for p, (W, H, losses) in zip(probs, outs):
        W2, H2, l2 = O.run(p.V, p.W0, p.H0, 1.5, iters=3)
        assert np.array_equal(W, W2) and np.array_equal(l2, losses)


# --------------------------------------------------------------------------
# Observations of Sec. 4 on synthetic data (loose)
# --------------------------------------------------------------------------

def _separable_problem(seed=24, F=24, N=40, K=3):
    rng = np.random.default_rng(seed)
    W0 = np.zeros((F, K))
    for k in range(K):                                  # disjoint supports: unique NMF
        W0[k * (F // K):(k + 1) * (F // K), k] = rng.uniform(0.5, 1.5, F // K)
    H0 = rng.uniform(0.1, 1.0, (K, N))
    H0[:, :K] = np.eye(K)
    return W0 @ H0 + 1e-3, W0


def test_jmm_and_bmm_reach_the_same_solution_up_to_permutation():
    V, W0 = _separable_problem()
    W, H = inputs.uniform_init(V.shape[0], V.shape[1], 3, seed=2)
    Wj, Hj, lj = O.run(V, W, H, 1.0, method="jmm", iters=3000, tol=1e-10)
    Wb, Hb, lb = O.run(V, W, H, 1.0, method="bmm", iters=3000, tol=1e-10)
    C = (Wj / np.linalg.norm(Wj, axis=0)).T @ (Wb / np.linalg.norm(Wb, axis=0))
    assert np.all(C.max(axis=1) > 0.99)
    assert lj[-1] == pytest.approx(lb[-1], rel=2e-2, abs=1e-6)


def test_update_order_does_not_change_the_solution():
    V, _ = _separable_problem(25)
    W, H = inputs.uniform_init(V.shape[0], V.shape[1], 3, seed=3)
    _, _, lw = O.run(V, W, H, 0.0, order="W", iters=3000, tol=1e-10)
    _, _, lh = O.run(V, W, H, 0.0, order="H", iters=3000, tol=1e-10)
    assert lw[-1] == pytest.approx(lh[-1], rel=2e-2, abs=1e-6)
